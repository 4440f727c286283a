"""Failure detection without a GPU fault: each bounded device-side wait of the library is made to
run out on a flag that nothing sets; the host must see SWS_ERR_TIMEOUT from the next sync within
seconds, and the context must keep working afterwards."""

import time

import numpy as np
import pytest
import torch

from paper_1811_10074_gb300 import binding as B
from gpu_common import make_input, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("which", ["lookback", "mbarrier"])
def test_bounded_wait_reports_timeout_and_context_survives(which):
    ctx = B.Context(0)
    try:
        ctx.sync()  # a clean start
        t0 = time.perf_counter()
        B.selftest_wait_timeout(which, ctx=ctx)
        with pytest.raises(B.SwsError, match="TIMEOUT"):
            ctx.sync()
        assert time.perf_counter() - t0 < 30.0
        ctx.sync()  # the error word was cleared
        x = make_input("add_i32", 1 << 16, device="cuda")
        y = B.sliding_sum("add_i32", 16, x, ctx=ctx)
        ctx.sync()
        xs = x[:18].cpu().numpy().astype(np.int64)
        want = np.array([xs[i:i + 16].sum() & 0xFFFFFFFF for i in range(3)], dtype=np.uint64).astype(np.uint32)
        assert (y[:3].cpu().numpy().view(np.uint32) == want).all()
    finally:
        ctx.close()


def test_selftest_rejects_unknown_wait():
    ctx = B.Context(0)
    try:
        with pytest.raises(B.SwsError, match="INVALID"):
            B._check(B.load().sws_selftest_wait_timeout(ctx.handle, 7, None))
    finally:
        ctx.close()


def test_minimizer_copy_timeout_leaves_count_all_ones():
    """The look-back minimizer kernel (the path of small sws_minimizers calls and of
    sws_minimizers_noalloc) with its input copies withheld: each tile's bounded copy wait runs
    out, the tile publishes a failure instead of its count, and no tile writes the total."""
    ctx = B.Context(0)
    try:
        ctx.sync()
        t0 = time.perf_counter()
        cnt = B.selftest_minimizer_timeout(ctx=ctx)
        with pytest.raises(B.SwsError, match="TIMEOUT"):
            ctx.sync()
        assert time.perf_counter() - t0 < 30.0
        assert int(cnt.item()) == -1  # all ones: the ordered output was not completed
        ctx.sync()
        from paper_1811_10074_gb300 import synth
        import oracle
        n = 20_000
        seq = synth.acgt_uniform_packed(n, seed=3)
        h, p = B.minimizers(seq.cuda(), n, 15, 10, ctx=ctx)
        want_h, want_p = oracle.minimizers(seq, n, 15, 10)
        assert np.array_equal(p.cpu().numpy().view(np.uint32), want_p)
        assert np.array_equal(h.cpu().numpy().view(np.uint32).astype(np.uint64), want_h)
    finally:
        ctx.close()
