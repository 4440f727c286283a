"""The capacity query and the one-call seed table of the C ABI (Sec. 2.4, Fig. 1) against the
oracle: sws_minimizers_count equals the number of the oracle's minimizers (with and without
N-blocks, on the single-kernel path and on the staged path of large inputs), and sws_build_table
equals the oracle's seed table of the oracle's minimizers."""

import ctypes

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


CASES = [  # (n, k, w, mode, nblocks (count, max length) or None)
    (0, 15, 10, "hash", None),
    (23, 15, 10, "hash", None),
    (24, 15, 10, "hash", None),
    (100_000, 15, 10, "hash", None),
    (250_001, 15, 10, "hash", (30, 4000)),
    (300_000, 19, 10, "hash", (20, 2000)),
    (200_000, 15, 50, "canonical", (10, 1000)),
    (150_000, 11, 300, "hash", None),
    (120_000, 3, 5, "fwd", None),
    (4_000_000, 15, 10, "hash", (50, 20_000)),   # staged path (fills the GPU)
    (3_000_000, 19, 12, "hash", None),           # staged path, 64-bit keys
    (2_500_000, 15, 40, "hash", (5, 100_000)),   # staged chunked kernel
    (1_500_000, 15, 300, "hash", None),          # generic kernel (look-back below 4 tiles per SM)
]


def inputs(n, k, w, nbspec, seed):
    seq = synth.acgt_uniform_packed(max(n, 1), seed=seed)
    nb = None
    if nbspec is not None:
        nb = random_nblocks(n, np.random.default_rng(seed), *nbspec)
    return seq, nb


@pytest.mark.parametrize("n,k,w,mode,nbspec", CASES)
def test_minimizers_count_equals_oracle(n, k, w, mode, nbspec):
    seq, nb = inputs(n, k, w, nbspec, n + k + w)
    want, _ = oracle.minimizers(seq, n, k, w, mode=mode, nblocks=nb)
    nbt = None if nb is None else torch.from_numpy(nb).cuda()
    seq_d = seq.cuda()
    got = B.minimizers_count(seq_d, n, k, w, mode=mode, nblocks=nbt)
    assert got == want.size, (n, k, w, mode)
    # the count sizes sws_minimizers exactly
    if n > 0:
        h, p = B.minimizers(seq_d, n, k, w, mode=mode, nblocks=nbt, capacity=got)
        assert h.shape[0] == got


@pytest.mark.parametrize("n,k,w,mode,nbspec,bucket_bits", [
    (0, 15, 10, "hash", None, 12),
    (100_000, 15, 10, "hash", None, 16),
    (250_001, 15, 10, "hash", (30, 4000), 20),
    (300_000, 19, 10, "hash", (20, 2000), 18),
    (200_000, 15, 50, "canonical", None, 30),
    (60_000, 4, 3, "fwd", None, 8),          # one radix pass: hits staged apart from the outputs
    (50_000, 5, 4, "hash", None, 0),
    (4_000_000, 15, 10, "hash", (50, 20_000), 24),
    (3_000_000, 19, 12, "hash", None, 24),
])
def test_build_table_equals_oracle(n, k, w, mode, nbspec, bucket_bits):
    seq, nb = inputs(n, k, w, nbspec, 7 * n + k)
    mh, mp = oracle.minimizers(seq, n, k, w, mode=mode, nblocks=nb)
    rh, rp, ro = oracle.kmer_table(mh, mp, 2 * k, bucket_bits)
    nbt = None if nb is None else torch.from_numpy(nb).cuda()
    sh, sp, off = B.build_table(seq.cuda(), n, k, w, bucket_bits, mode=mode, nblocks=nbt)
    torch.cuda.synchronize()
    assert sh.shape[0] == mh.size
    assert np.array_equal(to_u64(sh), rh)
    assert np.array_equal(sp.cpu().numpy().view(np.uint32), rp)
    assert np.array_equal(off.cpu().numpy().view(np.uint64), ro)


def test_build_table_capacity_error_reports_count():
    n, k, w = 100_000, 15, 10
    seq = synth.acgt_uniform_packed(n, seed=3).cuda()
    want = B.minimizers_count(seq, n, k, w)
    sh = torch.empty(want - 1, dtype=torch.int32, device="cuda")
    sp = torch.empty(want - 1, dtype=torch.int32, device="cuda")
    off = torch.empty((1 << 10) + 1, dtype=torch.int64, device="cuda")
    ctx = B.default_context(0)
    m = ctypes.c_uint64()
    st = B.load().sws_build_table(ctx.handle, B._ptr(seq), n, k, w, 0, ctypes.c_void_p(0), 0, 10, B._ptr(sh),
                                  B._ptr(sp), want - 1, B._ptr(off), ctypes.byref(m), B._stream(None))
    assert st == 3 and m.value == want  # SWS_ERR_CAPACITY with the exact count
    torch.cuda.synchronize()
