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
