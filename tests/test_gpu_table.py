"""GPU seed table (Sec. 2.4, Fig. 1) against the oracle: sorted hits and bucket pointers."""

import numpy as np
import pytest
import torch

import oracle
from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import synth
from gpu_common import require_gpu, to_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def run_table(h: np.ndarray, p: np.ndarray, hash_bits: int, bucket_bits: int):
    if hash_bits <= 32:
        hd = torch.from_numpy(h.astype(np.uint32).view(np.int32)).cuda()
    else:
        hd = torch.from_numpy(h.astype(np.uint64).view(np.int64)).cuda()
    pd = torch.from_numpy(p.astype(np.uint32).view(np.int32)).cuda()
    sh, sp, off = B.kmer_table(hd, pd, hash_bits, bucket_bits)
    torch.cuda.synchronize()
    return to_u64(sh), sp.cpu().numpy().view(np.uint32), off.cpu().numpy().view(np.uint64)


def check(h, p, hash_bits, bucket_bits):
    gh, gp, go = run_table(h, p, hash_bits, bucket_bits)
    rh, rp, ro = oracle.kmer_table(h, p, hash_bits, bucket_bits)
    assert (gh == rh).all() and (gp == rp).all(), (hash_bits, bucket_bits, h.size)
    bad = np.nonzero(go != ro)[0]
    assert bad.size == 0, (hash_bits, bucket_bits, bad[:5], go[bad[:5]], ro[bad[:5]])


@pytest.mark.parametrize("hash_bits,bucket_bits", [(1, 1), (8, 0), (8, 8), (20, 12), (30, 20), (32, 16), (32, 24),
                                                   (38, 18), (64, 10)])
@pytest.mark.parametrize("m", [0, 1, 4095, 4096, 4097, 100_003])
def test_table_random_hits(hash_bits, bucket_bits, m):
    rng = np.random.default_rng(hash_bits * 31 + m)
    hi = 1 << hash_bits
    h = rng.integers(0, hi, size=m, dtype=np.uint64) if hash_bits < 64 else rng.integers(0, 1 << 63, size=m, dtype=np.uint64) * 2 + 1
    if m > 10:
        h[rng.integers(0, m, size=m // 5)] = h[0]  # repeated seeds: stability matters
    p = np.sort(rng.choice(1 << 31, size=m, replace=False)).astype(np.uint32) if m else np.zeros(0, np.uint32)
    check(h, p, hash_bits, bucket_bits)


@pytest.mark.parametrize("k,w,bucket_bits", [(15, 10, 20), (19, 10, 16), (15, 50, 30)])
def test_table_from_minimizers(k, w, bucket_bits):
    n = 600_000
    seq = synth.acgt_uniform_packed(n, seed=k + w)
    rh, rp = oracle.minimizers(seq, n, k, w)
    gh, gp = B.minimizers(seq.cuda(), n, k, w)
    hb = 2 * k
    sh, sp, off = B.kmer_table(gh, gp, hb, bucket_bits)
    torch.cuda.synchronize()
    oh, op, oo = oracle.kmer_table(rh, rp, hb, bucket_bits)
    assert (to_u64(sh) == oh).all() and (sp.cpu().numpy().view(np.uint32) == op).all()
    assert (off.cpu().numpy().view(np.uint64) == oo).all()
    # every hit is found through its bucket
    shift = hb - bucket_bits
    o = off.cpu().numpy()
    s = to_u64(sh)
    for i in np.random.default_rng(1).integers(0, s.size, size=200):
        b = int(s[i]) >> shift
        assert o[b] <= i < o[b + 1]


def test_table_invalid_arguments():
    x = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(B.SwsError, match="INVALID"):
        B.kmer_table(x, x, 8, 9)
    with pytest.raises(B.SwsError, match="INVALID"):
        B.kmer_table(x, x, 0, 0)


# The segmented sort (top 8 bits packed into 64-bit records, next 8 bits per segment, every one
# of the 65,536 buckets sorted in shared memory) serves 16 < hash_bits <= 40 from 2^16 hits on.
@pytest.mark.parametrize("hash_bits,bucket_bits", [(17, 17), (24, 12), (30, 24), (32, 20), (38, 24), (40, 16),
                                                   (38, 26), (28, 27), (30, 0)])
def test_segmented_sort_random_hits(hash_bits, bucket_bits):
    rng = np.random.default_rng(hash_bits)
    m = 2_000_003
    h = rng.integers(0, 1 << hash_bits, size=m, dtype=np.uint64)
    h[rng.integers(0, m, size=m // 50)] = h[7]  # a repeated seed across many buckets' worth of hits
    p = np.sort(rng.choice(1 << 31, size=m, replace=False)).astype(np.uint32)
    check(h, p, hash_bits, bucket_bits)


def test_segmented_sort_oversize_buckets():
    """Heavy repeats: a few hashes with hundreds of thousands of hits each (buckets far beyond
    shared memory), and a bucket whose hits crowd a few sub-bins: both take the stable path in
    global memory; positions must stay ascending within every hash."""
    rng = np.random.default_rng(3)
    m = 1_500_000
    h = rng.integers(0, 1 << 38, size=m, dtype=np.uint64)
    h[: m // 3] = 12345 << 10  # one hash, 500k hits
    h[m // 3: m // 2] = (12345 << 10) + rng.integers(0, 3, size=m // 2 - m // 3)  # same bucket, 3 hashes
    h[m // 2: m // 2 + 20_000] = (999 << 22) + rng.integers(0, 40, size=20_000)  # crowded sub-bins
    rng.shuffle(h)
    p = np.sort(rng.choice(1 << 31, size=m, replace=False)).astype(np.uint32)
    check(h, p, 38, 20)
    check(h & np.uint64((1 << 30) - 1), p, 30, 16)


@pytest.mark.parametrize("k,w,bucket_bits", [(15, 10, 24), (19, 10, 24)])
def test_segmented_sort_table_from_genome_minimizers(k, w, bucket_bits):
    n = 6_000_000
    seq, iv = synth.genome_packed(n)
    nb = torch.from_numpy(iv).cuda()
    gh, gp = B.minimizers(seq.cuda(), n, k, w, nblocks=nb)
    assert gh.shape[0] >= (1 << 16)
    sh, sp, off = B.kmer_table(gh, gp, 2 * k, bucket_bits)
    torch.cuda.synchronize()
    rh, rp, ro = oracle.kmer_table(to_u64(gh), gp.cpu().numpy().view(np.uint32), 2 * k, bucket_bits)
    assert np.array_equal(to_u64(sh), rh) and np.array_equal(sp.cpu().numpy().view(np.uint32), rp)
    assert np.array_equal(off.cpu().numpy().view(np.uint64), ro)


@pytest.mark.parametrize("hash_bits,m", [(30, 300_000), (38, 300_000), (38, 3000), (24, 2_000_000)])
def test_table_is_stable_for_any_position_order(hash_bits, m):
    """Positions in no particular order (read-local positions of a batch, say): equal hashes keep
    their input order, through either sort and through every bucket path (heavy repeats included)."""
    rng = np.random.default_rng(hash_bits + m)
    h = rng.integers(0, 1 << hash_bits, size=m, dtype=np.uint64)
    h[rng.integers(0, m, size=m // 4)] = h[1]
    h[rng.integers(0, m, size=m // 20)] = rng.integers(0, 50, size=m // 20, dtype=np.uint64)
    p = rng.integers(0, 1 << 32, size=m, dtype=np.uint64).astype(np.uint32)
    gh, gp, _ = run_table(h, p, hash_bits, hash_bits // 2)
    order = np.argsort(h, kind="stable")
    assert np.array_equal(gh, h[order]) and np.array_equal(gp, p[order])


@pytest.mark.parametrize("hash_bits,bucket_bits", [(38, 24), (30, 20), (34, 26), (38, 18)])
def test_segmented_sort_pieces(hash_bits, bucket_bits):
    """Buckets (top 16 hash bits) far above the average: sorted by one CTA with an SM's shared
    memory to itself when the hits spread over the bucket (12289 .. 52224 hits), by the global LSD
    path when larger, or when the hits crowd a few sub-bins."""
    rng = np.random.default_rng(hash_bits * 7 + bucket_bits)
    rb = hash_bits - 16
    parts = [rng.integers(0, 1 << hash_bits, size=400_000, dtype=np.uint64)]
    for prefix, size in ((5, 9216), (6, 9217), (77, 20_000), (300, 41_000), (301, 60_000), (9000, 65_535),
                         (9001, 70_000)):
        parts.append((np.uint64(prefix) << np.uint64(rb)) + rng.integers(0, 1 << rb, size=size, dtype=np.uint64))
    # 30k hits in the lowest quarter of one bucket's range
    parts.append((np.uint64(12345) << np.uint64(rb)) + rng.integers(0, 1 << (rb - 2), size=30_000, dtype=np.uint64))
    # hits in the lower half only
    parts.append((np.uint64(400) << np.uint64(rb)) + rng.integers(0, 1 << (rb - 1), size=18_432, dtype=np.uint64))
    h = np.concatenate(parts)
    rng.shuffle(h)
    p = np.sort(rng.choice(1 << 31, size=h.size, replace=False)).astype(np.uint32)
    check(h, p, hash_bits, bucket_bits)
