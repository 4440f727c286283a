"""Seeding (Sec. 2.3) through the seed table (Sec. 2.4): GPU lookup + hit expansion against the
oracle's seed hits, computed from the unsorted (hash, position) seeds of the reference."""

import numpy as np
import pytest
import torch

import oracle
import paper_1811_10074_gb300 as P
from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import synth
from gpu_common import require_gpu, to_u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def run_gpu(h, p, q, hash_bits, bucket_bits, max_occ):
    dtype = np.uint64 if hash_bits > 32 else np.uint32
    hd = torch.from_numpy(h.astype(dtype).view(np.int64 if hash_bits > 32 else np.int32)).cuda()
    pd = torch.from_numpy(p.astype(np.uint32).view(np.int32)).cuda()
    qd = torch.from_numpy(q.astype(dtype).view(np.int64 if hash_bits > 32 else np.int32)).cuda()
    sh, sp, off = P.kmer_table(hd, pd, hash_bits, bucket_bits)
    first, count = P.seed_lookup(sh, off, hash_bits, bucket_bits, qd)
    hq, hp = P.seed_hits(first, count, sp, max_occ)
    torch.cuda.synchronize()
    return sh, sp, first, count, hq, hp


@pytest.mark.parametrize("hash_bits,bucket_bits", [(30, 16), (38, 20), (20, 20), (8, 4), (64, 24)])
@pytest.mark.parametrize("max_occ", [0, 3, 40])
def test_seed_hits_match_oracle(hash_bits, bucket_bits, max_occ):
    rng = np.random.default_rng(hash_bits * 100 + max_occ)
    for m, nq, hi in ((0, 10, 1 << hash_bits), (1, 1, 1), (5000, 2000, min(1 << hash_bits, 4000)),
                      (100_000, 30_000, 1 << min(hash_bits, 40)), (20_000, 5000, 50)):
        h = rng.integers(0, min(hi, 1 << 63), size=m, dtype=np.uint64) if m else np.zeros(0, np.uint64)
        p = np.sort(rng.permutation(1 << 24)[:m]).astype(np.uint32)  # positions ascending, as minimizers give them
        q = rng.integers(0, min(hi, 1 << 63), size=nq, dtype=np.uint64)
        if m:
            q[::2] = h[rng.integers(0, m, size=q[::2].size)]
        cnt, eq, ep = oracle.seed_hits(h, p, q, max_occ)
        sh, sp, first, count, hq, hp = run_gpu(h, p, q, hash_bits, bucket_bits, max_occ)
        assert (count.cpu().numpy().view(np.uint32) == cnt).all()
        assert (hq.cpu().numpy().view(np.uint32) == eq).all() and (hp.cpu().numpy().view(np.uint32) == ep).all()
        # every run holds exactly its query's hash
        f = first.cpu().numpy()
        c = count.cpu().numpy()
        shn = to_u64(sh)
        for i in rng.integers(0, nq, size=min(nq, 50)):
            assert (shn[f[i]:f[i] + c[i]] == q[i]).all()


def test_seed_hits_capacity_and_empty():
    h = np.arange(100, dtype=np.uint64) % 7
    p = np.arange(100, dtype=np.uint32)
    q = np.array([3, 3, 9], dtype=np.uint64)
    cnt, eq, ep = oracle.seed_hits(h, p, q, 0)
    sh, sp, first, count, _, _ = run_gpu(h, p, q, 30, 10, 0)
    with pytest.raises(B.SwsError, match="CAPACITY"):
        P.seed_hits(first, count, sp, 0, capacity=5)
    hq, hp, c = P.seed_hits(first, count, sp, 0, capacity=5, sync=False)
    torch.cuda.synchronize()
    assert int(c.item()) == eq.size and (hp[:5].cpu().numpy().view(np.uint32) == ep[:5]).all()
    hq, hp = P.seed_hits(first[:0], count[:0], sp, 0)
    assert hq.numel() == 0


def test_reads_against_genome_table():
    """Reads cut from a synthetic genome, their minimizers looked up in the genome's seed table."""
    n = 2_000_000
    seq, iv = synth.genome_packed(n, lmin=1000, lmax=20_000, device=torch.device("cuda"))
    k, w = 19, 10
    gh, gp = P.minimizers(seq, n, k, w, nblocks=torch.from_numpy(iv).cuda())
    rng = np.random.default_rng(3)
    starts = np.sort(rng.integers(0, n // 4 - 100, size=400)) * 4
    lens = rng.integers(25, 60, size=400) * 4
    codes = synth.unpack_codes(seq.cpu(), n)
    rcodes = torch.cat([codes[s:s + L] for s, L in zip(starts, lens)])
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    rseq = synth.pack_codes(rcodes)
    qh, qp, po = P.minimizers_batch(rseq.cuda(), torch.from_numpy(offs).cuda(), int(offs[-1]), k, w)
    sh, sp, off = P.kmer_table(gh, gp, 2 * k, 20)
    first, count = P.seed_lookup(sh, off, 2 * k, 20, qh)
    hq, hp = P.seed_hits(first, count, sp, 100)
    cnt, eq, ep = oracle.seed_hits(to_u64(gh), gp.cpu().numpy().view(np.uint32), to_u64(qh), 100)
    assert (hq.cpu().numpy().view(np.uint32) == eq).all() and (hp.cpu().numpy().view(np.uint32) == ep).all()
    # reads come from the genome: most of their seeds hit (not all: windows cut short at a read's
    # ends can pick k-mers that no full genome window picks, and reads may cross N-blocks)
    assert (cnt > 0).mean() > 0.6
