"""GPU k-mers and minimizers (Sec. 2.4) against the oracle, bit for bit, through the C ABI."""

import numpy as np
import pytest
import torch

import oracle
from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import synth
from gpu_common import random_nblocks, require_gpu, to_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


# ---------------------------------------------------------------------------------------------
# k-mers
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 5, 15, 16, 17, 19, 31, 32])
@pytest.mark.parametrize("n", [1, 16, 17, 4095, 4096 + 40, 100_003])
def test_kmers_match_oracle(k, n):
    seq = synth.acgt_uniform_packed(n, seed=n + k)
    sd = seq.cuda()
    for kind in ("fwd", "rc", "canonical", "hash"):
        got = B.kmers(sd, n, k, kind)
        torch.cuda.synchronize()
        ref = oracle.kmers(seq, n, k, kind)
        assert got.shape[0] == ref.shape[0]
        g = to_u64(got)
        bad = np.nonzero(g != ref)[0]
        assert bad.size == 0, (kind, bad[:5], g[bad[:5]], ref[bad[:5]])


# ---------------------------------------------------------------------------------------------
# minimizers
# ---------------------------------------------------------------------------------------------

def check_minimizers(seq_cpu, n, k, w, mode="hash", nblocks=None):
    nb_t = None if nblocks is None or len(nblocks) == 0 else torch.from_numpy(nblocks).cuda()
    h, p = B.minimizers(seq_cpu.cuda(), n, k, w, mode, nblocks=nb_t)
    rh, rp = oracle.minimizers(seq_cpu, n, k, w, mode, nblocks=nblocks)
    gh, gp = to_u64(h), p.cpu().numpy().view(np.uint32)
    assert gh.shape == rh.shape, (n, k, w, mode, gh.shape, rh.shape)
    bad = np.nonzero((gh != rh) | (gp != rp))[0]
    assert bad.size == 0, (n, k, w, mode, bad[:5], gp[bad[:5]], rp[bad[:5]])
    return gh, gp


def test_minimizers_plain_workload():
    """1,000,000 uniform i.i.d. bases (seed 42), k=15, w=10, hashed canonical k-mers."""
    n = 1_000_000
    seq = synth.acgt_uniform_packed(n, seed=42)
    gh, gp = check_minimizers(seq, n, 15, 10)
    dens = gh.size / (n - 14)
    assert abs(dens - 2 / 11) < 0.01


@pytest.mark.parametrize("k,w", [(1, 1), (3, 3), (5, 4), (15, 10), (16, 10), (17, 10), (19, 10), (15, 50),
                                 (31, 2), (32, 7), (11, 257), (15, 1000), (9, 4000)])
@pytest.mark.parametrize("mode", ["hash", "canonical", "fwd"])
def test_minimizers_random(k, w, mode):
    rng = np.random.default_rng(k * 1000 + w)
    for n in (1, k + w - 2, k + w - 1, k + w, 4032 + k + w, 3 * 4096 + 7, 40_000):
        seq = synth.acgt_uniform_packed(n, seed=int(rng.integers(1 << 30)))
        check_minimizers(seq, n, k, w, mode)


@pytest.mark.parametrize("k,w", [(15, 10), (19, 10), (5, 3), (15, 50)])
def test_minimizers_with_nblocks(k, w):
    rng = np.random.default_rng(5 + k + w)
    for n, count, maxlen in ((5000, 3, 40), (60_000, 30, 3000), (200_000, 400, 50), (30_000, 300, 5)):
        seq = synth.acgt_uniform_packed(n, seed=int(rng.integers(1 << 30)))
        iv = random_nblocks(n, rng, count, maxlen)
        check_minimizers(seq, n, k, w, "hash", iv)


def test_minimizers_low_complexity_ties_staged():
    """A repetitive sequence long enough for the staged kernel (more than 4 tiles per SM), with
    N-blocks: equal keys everywhere, the leftmost must win."""
    unit = synth.codes_from_string("ACGTTGCAACGGA")
    codes = unit.repeat(200_000)
    codes[12345] = 3
    seq = synth.pack_codes(codes)
    n = codes.numel()
    rng = np.random.default_rng(8)
    for k, w, mode in ((15, 10, "hash"), (5, 4, "fwd"), (9, 16, "canonical")):
        check_minimizers(seq, n, k, w, mode)
        check_minimizers(seq, n, k, w, mode, random_nblocks(n, rng, 300, 40))


def test_minimizers_low_complexity_ties():
    """A repetitive sequence makes many equal keys: the leftmost must win everywhere."""
    unit = synth.codes_from_string("ACGTTGCAAC")
    codes = unit.repeat(5000)
    codes[777] = 3
    seq = synth.pack_codes(codes)
    n = codes.numel()
    for k, w in ((5, 10), (15, 10), (3, 20)):
        for mode in ("hash", "fwd"):
            check_minimizers(seq, n, k, w, mode)


def test_minimizers_capacity_overflow():
    n = 50_000
    seq = synth.acgt_uniform_packed(n, seed=9)
    rh, rp = oracle.minimizers(seq, n, 15, 10)
    cap = rh.size // 2
    h, p, cnt = B.minimizers(seq.cuda(), n, 15, 10, capacity=cap, sync=False)
    torch.cuda.synchronize()
    assert int(cnt.item()) == rh.size
    assert (to_u64(h[:cap]) == rh[:cap]).all() and (p[:cap].cpu().numpy().view(np.uint32) == rp[:cap]).all()
    with pytest.raises(B.SwsError, match="CAPACITY"):
        B.minimizers(seq.cuda(), n, 15, 10, capacity=cap)


def test_minimizers_from_keys():
    rng = np.random.default_rng(3)
    for m, w, hi in ((1, 1, 10), (100, 4, 5), (4096 * 3 + 11, 17, 1 << 30), (100_000, 10, 50), (50_000, 1000, 1 << 20)):
        keys = rng.integers(0, hi, size=m, dtype=np.int64).astype(np.uint32)
        kd = torch.from_numpy(keys.view(np.int32)).cuda()
        h, p = B.minimizers_from_keys(kd, w)
        rh, rp = oracle.minimizers_from_keys(keys.astype(np.uint64), w)
        assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all(), (m, w)


def test_minimizers_batch_matches_per_read_oracle():
    rng = np.random.default_rng(11)
    lens = np.concatenate([rng.integers(0, 30, size=50), rng.integers(100, 251, size=400),
                           rng.integers(1000, 20000, size=12), [0, 0, 5000]])
    rng.shuffle(lens)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(offs[-1])
    seq = synth.acgt_uniform_packed(total, seed=77)
    for k, w, mode in ((15, 10, "hash"), (19, 10, "hash"), (5, 3, "fwd")):
        h, p, po = B.minimizers_batch(seq.cuda(), torch.from_numpy(offs).cuda(), total, k, w, mode)
        rh, rp, rpo = oracle.minimizers_batch(seq, offs, k, w, mode)
        assert (po.cpu().numpy().view(np.uint64) == rpo).all()
        assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all()


# Every window length of the kernel specialized on w (4..16; 32-bit key values for 2k <= 32 and
# 64-bit ones above).  The API
# takes that (staged) path once an input fills the GPU, more than (256 * floor(16/w) - 2) * w
# windows per SM; 640 tiles plus a ragged tail exceed it on a 152-SM GB300, and a 3-tile input
# takes the single-kernel look-back path.
@pytest.mark.parametrize("w", list(range(4, 17)))
def test_specialized_window_lengths(w):
    rng = np.random.default_rng(1000 + w)
    tw = (256 * (16 // w) - 2) * w
    for k, mode in ((15, "hash"), (16, "fwd"), (5, "canonical"), (19, "hash"), (32, "canonical"), (17, "fwd")):
        for ntiles in (640, 3):
            n = ntiles * tw + int(rng.integers(1, tw))
            seq = synth.acgt_uniform_packed(n, seed=int(rng.integers(1 << 30)))
            check_minimizers(seq, n, k, w, mode)
            iv = random_nblocks(n, rng, 6 + ntiles // 4, 3 * w)
            check_minimizers(seq, n, k, w, mode, iv)
    keys = rng.integers(0, 1000, size=640 * tw + 17, dtype=np.int64).astype(np.uint32)
    h, p = B.minimizers_from_keys(torch.from_numpy(keys.view(np.int32)).cuda(), w)
    rh, rp = oracle.minimizers_from_keys(keys.astype(np.uint64), w)
    assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all()
    lens = rng.integers(0, 3 * w + 40, size=300)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    bseq = synth.acgt_uniform_packed(int(offs[-1]), seed=w)
    bh, bp, bpo = B.minimizers_batch(bseq.cuda(), torch.from_numpy(offs).cuda(), int(offs[-1]), 15, w)
    rh, rp, rpo = oracle.minimizers_batch(bseq, offs, 15, w)
    assert (bpo.cpu().numpy().view(np.uint64) == rpo).all()
    assert (to_u64(bh) == rh).all() and (bp.cpu().numpy().view(np.uint32) == rp).all()


# Edge cases of the values-only pick rule (a new pick iff the previous window's first key was its
# minimum, or the entering key is strictly smaller), on both paths: inputs of a few tiles take the
# look-back kernel, inputs of 700 tiles the staged kernel.
@pytest.mark.parametrize("w", [4, 5, 7, 8, 10, 13, 16])
def test_key_minimizers_edge_cases(w):
    rng = np.random.default_rng(77 + w)
    tw = (256 * (16 // w) - 2) * w
    cases = {
        "short": rng.integers(0, 1 << 30, size=w, dtype=np.int64),
        "w+1": rng.integers(0, 1 << 30, size=w + 1, dtype=np.int64),
        "tile-1": rng.integers(0, 1 << 30, size=tw + w - 2, dtype=np.int64),
        "tile+1": rng.integers(0, 1 << 30, size=tw + w, dtype=np.int64),
        "increasing": np.arange(5 * tw + 3, dtype=np.int64),            # every pick leaves by expiry
        "decreasing": np.arange(5 * tw + 3, 0, -1, dtype=np.int64),     # every entering key is smaller
        "few values": rng.integers(0, 3, size=7 * tw + 11, dtype=np.int64),  # ties everywhere
        "constant": np.full(3 * tw + 5, 12345, dtype=np.int64),
        "full range": rng.integers(0, 1 << 32, size=50 * tw + 7, dtype=np.int64),
        "increasing, staged": np.arange(700 * tw + 3, dtype=np.int64),
        "decreasing, staged": np.arange(700 * tw + 3, 0, -1, dtype=np.int64),
        "few values, staged": rng.integers(0, 3, size=700 * tw + 11, dtype=np.int64),
        "sawtooth, staged": np.arange(700 * tw + 5, dtype=np.int64) % (3 * w + 1),
    }
    for name, k64 in cases.items():
        keys = k64.astype(np.uint32)
        kd = torch.from_numpy(keys.view(np.int32)).cuda()
        for view in ("aligned", "offset"):
            kv = kd if view == "aligned" else torch.cat([kd[:1], kd])[1:]  # 4-byte aligned only
            h, p = B.minimizers_from_keys(kv, w)
            rh, rp = oracle.minimizers_from_keys(keys.astype(np.uint64), w)
            assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all(), (w, name, view)


def test_key_minimizers_full_size_sampled():
    """2^28 uniform 30-bit keys, w = 10 (the benchmark's configuration): the picks whose key lies
    at least w keys inside a segment depend only on that segment."""
    m, w = 1 << 28, 10
    keys = synth.uint32_hashes(m, device="cuda")
    h, p, cnt = B.minimizers_from_keys(keys, w, capacity=m // 4, sync=False)
    count = int(cnt.item())
    assert abs(count / m - 2 / (w + 1)) < 0.01
    pos = p[:count].to(torch.int64) & 0xFFFFFFFF
    assert bool((pos[1:] > pos[:-1]).all())
    rng = np.random.default_rng(9)
    for a in np.concatenate([[0, m - 30_000], rng.integers(0, m - 30_000, size=40)]):
        a = int(a)
        b = min(a + 30_000, m)
        lo = a + w if a > 0 else 0
        hi = b - w if b < m else m
        seg = keys[a:b].cpu().numpy().view(np.uint32).astype(np.uint64)
        rh, rp = oracle.minimizers_from_keys(seg, w)
        rp = rp.astype(np.int64) + a
        sel = (rp >= lo) & (rp < hi)
        i0, i1 = torch.searchsorted(pos, torch.tensor([lo, hi], device=pos.device)).tolist()
        assert (pos[i0:i1].cpu().numpy() == rp[sel]).all() and (to_u64(h[i0:i1]) == rh[sel]).all(), a


@pytest.mark.parametrize("k", [5, 6, 15, 19, 32])
def test_minimizer_strands(k):
    """Strand of canonical picks (0 forward / palindrome, 1 reverse complement) against the oracle,
    for one sequence and for a read batch."""
    n = 300_000
    seq = synth.acgt_uniform_packed(n, seed=k)
    h, p = B.minimizers(seq.cuda(), n, k, 10, "canonical")
    got = B.minimizer_strands(seq.cuda(), n, k, p).cpu().numpy()
    ref = oracle.strands(seq, n, k, p.cpu().numpy().view(np.uint32))
    assert (got == ref).all() and set(np.unique(ref).tolist()) <= {0, 1}
    if k % 2 == 1:
        assert 0.4 < ref.mean() < 0.6  # both strands equally likely for random sequence
    rng = np.random.default_rng(k)
    lens = rng.integers(0, 300, size=500)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    bseq = synth.acgt_uniform_packed(int(offs[-1]), seed=k + 1)
    od = torch.from_numpy(offs).cuda()
    bh, bp, bpo = B.minimizers_batch(bseq.cuda(), od, int(offs[-1]), k, 10, "canonical")
    got = B.minimizer_strands(bseq.cuda(), int(offs[-1]), k, bp, od, bpo).cpu().numpy()
    ref = oracle.strands(bseq, int(offs[-1]), k, bp.cpu().numpy().view(np.uint32), offs,
                         bpo.cpu().numpy().view(np.uint64))
    assert (got == ref).all()
    # positions outside the sequence
    bad = torch.tensor([n - k + 1, n], dtype=torch.int32, device="cuda")
    assert B.minimizer_strands(seq.cuda(), n, k, bad).tolist() == [255, 255]


# Window lengths 17..256 of the staged kernel's chunked form (w at run time; a window is the
# suffix of its first 16-k-mer chunk, whole chunks, and a prefix of its last chunk).  Inputs of
# 700 tiles take the staged path, more than 4 tiles per SM on a 152-SM GB300.
CHUNK_WS = [17, 18, 31, 32, 33, 47, 48, 49, 50, 63, 64, 65, 100, 128, 200, 255, 256]


@pytest.mark.parametrize("w", CHUNK_WS)
def test_chunked_window_lengths(w):
    rng = np.random.default_rng(5000 + w)
    tw = (4096 - 2 * w + 1) // 16 * 16
    combos = [(15, "hash"), (19, "hash"), (32, "canonical"), (5, "fwd"), (16, "canonical"), (17, "fwd")]
    for k, mode in combos[w % 2::2]:
        n = 700 * tw + int(rng.integers(1, tw))
        seq = synth.acgt_uniform_packed(n, seed=int(rng.integers(1 << 30)))
        check_minimizers(seq, n, k, w, mode)
        iv = random_nblocks(n, rng, 300, 3 * w)
        check_minimizers(seq, n, k, w, mode, iv)
    m = 700 * tw + 13
    for name, k64 in (("few values", rng.integers(0, 3, size=m, dtype=np.int64)),
                      ("sawtooth", np.arange(m, dtype=np.int64) % (3 * w + 1)),
                      ("decreasing", np.arange(m, 0, -1, dtype=np.int64)),
                      ("full range", rng.integers(0, 1 << 32, size=m, dtype=np.int64))):
        keys = k64.astype(np.uint32)
        h, p = B.minimizers_from_keys(torch.from_numpy(keys.view(np.int32)).cuda(), w)
        rh, rp = oracle.minimizers_from_keys(keys.astype(np.uint64), w)
        assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all(), (w, name)
    lens = rng.integers(0, 6 * w + 200, size=3_000_000 // (3 * w + 100))
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    bseq = synth.acgt_uniform_packed(int(offs[-1]), seed=w)
    bh, bp, bpo = B.minimizers_batch(bseq.cuda(), torch.from_numpy(offs).cuda(), int(offs[-1]), 15, w)
    rh, rp, rpo = oracle.minimizers_batch(bseq, offs, 15, w)
    assert (bpo.cpu().numpy().view(np.uint64) == rpo).all()
    assert (to_u64(bh) == rh).all() and (bp.cpu().numpy().view(np.uint32) == rp).all()


@pytest.mark.parametrize("k,w", [(15, 17), (15, 50), (19, 50), (12, 257), (15, 1000)])
def test_generic_staged_path(k, w):
    """Window lengths beyond the w <= 16 kernel, inputs large enough (more than 4 tiles per SM)
    for the staged path: the chunked form of the staged kernel up to w = 256, the generic kernel
    (per-tile slots, then a scan and a gather) beyond.  One sequence with and without N-blocks,
    and a read batch."""
    rng = np.random.default_rng(k * 1000 + w)
    n = 3_000_000 + int(rng.integers(1, 5000))
    seq = synth.acgt_uniform_packed(n, seed=k + w)
    h, p = B.minimizers(seq.cuda(), n, k, w)
    rh, rp = oracle.minimizers(seq, n, k, w, deque=True)
    assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all()
    iv = random_nblocks(n, rng, 400, 5 * w)
    nb = torch.from_numpy(iv).cuda()
    h, p = B.minimizers(seq.cuda(), n, k, w, nblocks=nb)
    rh, rp = oracle.minimizers(seq, n, k, w, nblocks=iv, deque=True)
    assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all()
    lens = rng.integers(0, 6 * w + 200, size=max(3_000_000 // (3 * w + 100), 10))
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    bseq = synth.acgt_uniform_packed(int(offs[-1]), seed=w)
    bh, bp, bpo = B.minimizers_batch(bseq.cuda(), torch.from_numpy(offs).cuda(), int(offs[-1]), k, w)
    rh, rp, rpo = oracle.minimizers_batch(bseq, offs, k, w)
    assert (bpo.cpu().numpy().view(np.uint64) == rpo).all()
    assert (to_u64(bh) == rh).all() and (bp.cpu().numpy().view(np.uint32) == rp).all()


# The single-pass kernel on packed bases (hashed k-mers, k <= 29, 4 <= w <= 17, the sequence
# 4-byte aligned): each thread hashes 16 k-mers; a warp's halo k-mers are hashed by its first w-1
# lanes and its previous k-mer by lane 31.  Lengths around tiles of 4096 windows, ties from
# low-complexity sequences, and an unaligned view that takes the staged path instead.
@pytest.mark.parametrize("w", list(range(4, 18)))
def test_dna_single_pass_kernel(w):
    rng = np.random.default_rng(3000 + w)
    # 32-bit keys up to k = 16; 64-bit above, with tile position codes up to k = 25 (the hash's
    # high word at most 14 bits up to k = 23, 26 bits above) and thread-frame codes from k = 26
    for k in (1, 2, 7, 15, 16, 17, 19, 23, 25, 27, 29):
        span = k + w - 1
        for n in (k + 32, span + 4095, span + 4096, span + 4097, span + 3 * 4096 + 1, 2_000_003):
            seq = synth.acgt_uniform_packed(n, seed=int(rng.integers(1 << 30)))
            check_minimizers(seq, n, k, w, "hash")
    n = 300_001
    for name, codes in (("constant", np.zeros(n, np.uint8)),
                        ("period 3", np.tile(np.array([0, 1, 3], np.uint8), n // 3 + 1)[:n]),
                        ("two letters", rng.integers(0, 2, size=n).astype(np.uint8))):
        seq = synth.pack_codes(torch.from_numpy(codes))
        for k in (5, 16, 19):
            check_minimizers(seq, n, k, w, "hash")
    # a view starting one byte in (bases 4 .. n+3): not 4-byte aligned, so the staged kernel runs
    n = 50_000
    full = synth.acgt_uniform_packed(n + 8, seed=w)
    fd = full.cuda()
    h, p = B.minimizers(fd[1:], n, 15, w)
    rh, rp = oracle.minimizers(full[1:].clone(), n, 15, w)
    assert (to_u64(h) == rh).all() and (p.cpu().numpy().view(np.uint32) == rp).all()


def check_batch_single_pass(seq, offs, k, w):
    total = int(offs[-1])
    h, p, po = B.minimizers_batch(seq.cuda(), torch.from_numpy(offs).cuda(), total, k, w, "hash")
    rh, rp, rpo = oracle.minimizers_batch(seq, offs, k, w, "hash")
    assert (po.cpu().numpy().view(np.uint64) == rpo).all(), (k, w, offs.size)
    gh, gp = to_u64(h), p.cpu().numpy().view(np.uint32)
    assert gh.shape == rh.shape, (k, w, gh.shape, rh.shape)
    bad = np.nonzero((gh != rh) | (gp != rp))[0]
    assert bad.size == 0, (k, w, bad[:5], gp[bad[:5]], rp[bad[:5]])


# Read batches on the single-pass kernel (hashed k-mers, k <= 16, 4 <= w <= 17): read starts act
# as window barriers, positions are read-local, each read's first pick gives its pick offset.
@pytest.mark.parametrize("k,w", [(15, 10), (16, 17), (5, 4), (11, 13), (19, 10), (29, 4), (17, 17)])
def test_batch_single_pass_kernel(k, w):
    rng = np.random.default_rng(k * 100 + w)
    span = k + w - 1
    cases = [
        rng.integers(100, 251, size=3000),                      # short reads
        rng.integers(0, 3 * span, size=4000),                   # tiny and empty reads: > 128 starts a tile
        np.array([4096 * 3 + span - 1]),                        # one read, 3 tiles exactly
        np.array([span - 1, span, span + 1, 0, 5000, 1, 4095 + span, 4097]),
        rng.integers(5_000, 60_000, size=40),                   # long reads across tiles
    ]
    for lens in cases:
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        if offs[-1] < k + 32:
            continue
        seq = synth.acgt_uniform_packed(int(offs[-1]), seed=int(rng.integers(1 << 30)))
        check_batch_single_pass(seq, offs, k, w)
    # low complexity: ties inside reads and across read starts
    lens = rng.integers(20, 400, size=2000)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    codes = np.tile(np.array([0, 0, 1, 0, 0, 1, 2], np.uint8), int(offs[-1]) // 7 + 1)[: int(offs[-1])]
    check_batch_single_pass(synth.pack_codes(torch.from_numpy(codes)), offs, k, w)


# The same kernel with N-blocks (windows touching one dropped, the first window after one stores).
@pytest.mark.parametrize("w", [4, 10, 17])
def test_nblocks_single_pass_kernel(w):
    rng = np.random.default_rng(500 + w)
    for n, count, maxlen in ((300_000, 3000, 30), (200_000, 50, 20_000), (100_000, 600, 3)):
        seq = synth.acgt_uniform_packed(n, seed=int(rng.integers(1 << 30)))
        iv = random_nblocks(n, rng, count, maxlen)
        check_minimizers(seq, n, 15, w, "hash", iv)
        check_minimizers(seq, n, 19, w, "hash", iv)
