"""The allocation-free minimizer entry point, for callers that cannot allocate device memory.

sws_minimizers_noalloc keeps its scratch in a fixed array that the library declares in device
memory instead of a workspace grown with cudaMalloc.  These tests call it through the C ABI and
compare it with sws_minimizers (the context entry point) bit for bit, on calls made one after
another, so that a call that inherits the previous call's scratch contents is checked too.  The
file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import synth
from gpu_common import random_nblocks, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def noalloc_call(lib, seq, n, k, w, nblocks=None):
    cap = max(n - (w + k - 1) + 1, 1)
    h = torch.empty(cap, dtype=torch.int32 if 2 * k <= 32 else torch.int64, device="cuda")
    p = torch.empty(cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    nb = 0 if nblocks is None else nblocks.shape[0]
    st = lib.sws_minimizers_noalloc(ctypes.c_void_p(seq.data_ptr()), n, k, w, 0,
                                    ctypes.c_void_p(nblocks.data_ptr() if nb else 0), nb,
                                    ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(p.data_ptr()), cap,
                                    ctypes.c_void_p(cnt.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.sws_last_error()
    torch.cuda.synchronize()
    c = int(cnt.item())
    assert 0 <= c <= cap
    return h[:c], p[:c]


def test_noalloc_matches_context_entry_point_on_consecutive_calls():
    lib = B.load()
    rng = np.random.default_rng(21)
    cases = [(1_000_000, 15, 10, None), (300_001, 19, 10, None), (250_000, 15, 10, (40, 2000)),
             (77_777, 5, 3, None)]
    for i, (n, k, w, nbspec) in enumerate(cases):
        seq = synth.acgt_uniform_packed(n, seed=500 + i).cuda()
        nbt = None
        if nbspec is not None:
            nbt = torch.from_numpy(random_nblocks(n, rng, *nbspec)).cuda()
        ref_h, ref_p = B.minimizers(seq, n, k, w, nblocks=nbt)
        for _ in range(2):  # the same input twice in a row: leftover scratch must not matter
            h, p = noalloc_call(lib, seq, n, k, w, nbt)
            assert h.shape == ref_h.shape
            assert torch.equal(h, ref_h) and torch.equal(p, ref_p), (n, k, w)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    lib = B.load()
    seq = torch.zeros(16, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    n = (1 << 32) - 4096  # valid for sws_minimizers, too long for the fixed scratch
    st = lib.sws_minimizers_noalloc(ctypes.c_void_p(seq.data_ptr()), n, 15, 10, 0, ctypes.c_void_p(0), 0,
                                    ctypes.c_void_p(0), ctypes.c_void_p(0), 0, ctypes.c_void_p(cnt.data_ptr()),
                                    ctypes.c_void_p(0))
    assert st == 1 and b"fixed scratch" in lib.sws_last_error()
    assert int(cnt.item()) == 0  # nothing was queued
