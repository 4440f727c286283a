"""The allocation-free minimizer entry point, for callers that cannot allocate device memory.

sws_minimizers_noalloc keeps its scratch in a fixed array that the library declares in device
memory instead of a workspace grown with cudaMalloc.  These tests call it through the C ABI and
check it against the plain CPU oracle (``oracle.minimizers``) and against sws_minimizers (the
context entry point), on calls made one after another, so that a call that inherits the previous
call's scratch contents is checked too.  One case sits exactly at the scratch limit (the last
tile's status word is the last word before the per-tile barrier summaries), and one tile more
is rejected.  The file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import synth
from gpu_common import random_nblocks, require_gpu, to_u64

pytestmark = pytest.mark.gpu

# The fixed scratch: 4 MiB = a 256-byte header + 16 bytes per tile (status word + barrier summary).
MAX_TILES = ((4 << 20) - 256) // 16


def tile_windows(w: int) -> int:
    return (4096 - w) // 64 * 64


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def noalloc_call(lib, seq, n, k, w, nblocks=None, cap=None):
    if cap is None:
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


def test_noalloc_matches_oracle_on_consecutive_calls():
    lib = B.load()
    rng = np.random.default_rng(21)
    cases = [(1_000_000, 15, 10, None), (300_001, 19, 10, None), (250_000, 15, 10, (40, 2000)),
             (200_003, 19, 12, (25, 3000)), (77_777, 5, 3, None)]
    for i, (n, k, w, nbspec) in enumerate(cases):
        seq = synth.acgt_uniform_packed(n, seed=500 + i)
        nb = None if nbspec is None else random_nblocks(n, rng, *nbspec)
        want_h, want_p = oracle.minimizers(seq, n, k, w, nblocks=nb)
        seq_d = seq.cuda()
        nbt = None if nb is None else torch.from_numpy(nb).cuda()
        ref_h, ref_p = B.minimizers(seq_d, n, k, w, nblocks=nbt)
        for _ in range(2):  # the same input twice in a row: leftover scratch must not matter
            h, p = noalloc_call(lib, seq_d, n, k, w, nbt)
            assert np.array_equal(to_u64(h), want_h), (n, k, w, "keys vs oracle")
            assert np.array_equal(p.cpu().numpy().view(np.uint32), want_p), (n, k, w, "positions vs oracle")
            assert torch.equal(h, ref_h) and torch.equal(p, ref_p), (n, k, w)


def oracle_picks_in(seq_bytes: np.ndarray, n: int, k: int, w: int, nb: np.ndarray, a: int, b: int):
    """Picks of the whole sequence whose positions lie in [a + w - 1, b - w - k + 1], from the
    oracle run on bases [a, b) alone: every window of such a pick lies inside [a, b), and pick
    positions strictly increase, so the sub-range's picks there are exactly the full sequence's."""
    a4 = a // 4 * 4
    sub = seq_bytes[a4 // 4:(b + 3) // 4]
    m = b - a4
    nbs = nb.copy()
    nbs = nbs[(nbs[:, 1] > a4) & (nbs[:, 0] < b)] - a4
    nbs = np.clip(nbs, 0, m)
    h, p = oracle.minimizers(sub, m, k, w, nblocks=nbs)
    p = p.astype(np.int64) + a4
    lo, hi = a + w - 1, b - w - k + 1
    keep = (p >= lo) & (p <= hi)
    return h[keep], p[keep], lo, hi


def test_noalloc_at_the_scratch_limit_with_nblocks():
    lib = B.load()
    k, w = 15, 10
    span = w + k - 1
    n = MAX_TILES * tile_windows(w) + span - 1  # exactly MAX_TILES tiles
    rng = np.random.default_rng(5)
    seq_d = synth.acgt_uniform_packed(n, seed=77, device="cuda")
    nb = random_nblocks(n, rng, 400, 50_000)
    nb = np.concatenate([nb, [[n - 3000, n - 2000]]]).astype(np.int64)  # one in the last tile
    nbt = torch.from_numpy(nb).cuda()
    cap = int(n * 2.6 / (w + 1)) + 4096
    ref_h, ref_p, ref_c = B.minimizers(seq_d, n, k, w, nblocks=nbt, capacity=cap, sync=False)
    torch.cuda.synchronize()
    c = int(ref_c.item())
    ref_h, ref_p = ref_h[:c], ref_p[:c]
    h, p = noalloc_call(lib, seq_d, n, k, w, nbt, cap=cap)
    assert torch.equal(h, ref_h) and torch.equal(p, ref_p)
    # the oracle on two stretches: one in the first tiles, one that covers the last tiles
    seq_b = seq_d.cpu().numpy()
    pos = p.cpu().numpy().view(np.uint32).astype(np.int64)
    keys = to_u64(h)
    for a, b in ((0, 200_000), (n - 300_000, n)):
        wh, wp, lo, hi = oracle_picks_in(seq_b, n, k, w, nb, a, b)
        sel = (pos >= lo) & (pos <= hi)
        assert np.array_equal(pos[sel], wp), (a, b)
        assert np.array_equal(keys[sel], wh), (a, b)
    del seq_d, h, p, ref_h, ref_p
    torch.cuda.empty_cache()


def test_noalloc_rejects_inputs_beyond_its_scratch():
    lib = B.load()
    seq = torch.zeros(16, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    k, w = 15, 10
    over = MAX_TILES * tile_windows(w) + (w + k - 1) - 1 + 1  # one window more: MAX_TILES + 1 tiles
    for n in (over, (1 << 32) - 4096):
        st = lib.sws_minimizers_noalloc(ctypes.c_void_p(seq.data_ptr()), n, k, w, 0, ctypes.c_void_p(0), 0,
                                        ctypes.c_void_p(0), ctypes.c_void_p(0), 0, ctypes.c_void_p(cnt.data_ptr()),
                                        ctypes.c_void_p(0))
        assert st == 1 and b"fixed scratch" in lib.sws_last_error(), n
        torch.cuda.synchronize()
        assert int(cnt.item()) == 0  # nothing was queued
