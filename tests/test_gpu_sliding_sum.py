"""GPU sliding window sum (Eq. 2) against the oracle, element by element, through the C ABI."""

import numpy as np
import pytest
import torch

import oracle
from paper_1811_10074_gb300 import binding as B
from gpu_common import assert_sampled, assert_sliding_equal, make_input, oracle_sliding, require_gpu, sample_indices

pytestmark = pytest.mark.gpu

OPS = ["add_i32", "min_i32", "max_i32", "xor_i32", "affine_u32", "add_f32"]
INT_OPS = ["add_i32", "min_i32", "max_i32", "xor_i32"]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def variants_for(op):
    v = ["block_combine", "doubling", "auto"]
    if op in ("add_i32", "xor_i32"):
        v.append("prefix_diff")
    return v


# (w, n) pairs: empty, exact, one tile, tile edges, several tiles with a ragged tail
# Dispatch coverage: w in {1,2,4,8} run fully in registers; multiples of the thread chunk take the
# aligned block-combine (blocks within a warp, or several whole warps: w = 512, 1024, 1536, 2048);
# everything else the general segmented block-combine.
CASES = [(1, 1), (1, 4097), (2, 1), (2, 2), (2, 33), (3, 10), (4, 4095), (4, 4096 + 3), (7, 9000), (8, 8),
         (8, 50_001), (16, 16), (16, 24593), (32, 20000), (33, 40000), (48, 20000), (64, 100_003), (255, 30000),
         (256, 70_001), (512, 40000), (1024, 1023), (1024, 1024), (1024, 50_000), (1025, 33333), (1536, 30000),
         (2048, 30000)]


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("w,n", CASES)
def test_sliding_sum_matches_oracle(op, w, n):
    x, ref = oracle_sliding(op, w, n, 7, op in INT_OPS)
    xd = x.cuda()
    for variant in variants_for(op):
        if variant == "doubling" and w > 1100 and op == "affine_u32":
            continue  # covered at smaller w; keeps the suite short
        y = B.sliding_sum(op, w, xd, variant=variant)
        torch.cuda.synchronize()
        assert y.shape[0] == max(n - w + 1, 0)
        if y.shape[0]:
            assert_sliding_equal(op, w, x, y, ref)


@pytest.mark.parametrize("op", OPS)
def test_unaligned_pointers(op):
    """Views that start one element into a buffer disable the 16-byte vector path."""
    n, w = 20011, 37
    x, _ = oracle_sliding(op, w, n + 1, 3, False)
    xd = x.cuda()[1:]
    ref = oracle.sliding_sum(op, w, x[1:])
    buf = torch.empty((n - w + 2,) + tuple(x.shape[1:]), dtype=x.dtype, device="cuda")
    y = B.sliding_sum(op, w, xd, out=buf[1:])
    torch.cuda.synchronize()
    assert_sliding_equal(op, w, x[1:], y, ref)


def test_n_smaller_than_w_writes_nothing():
    x = make_input("add_i32", 10).cuda()
    out = torch.full((4,), 12345, dtype=torch.int32, device="cuda")
    y = B.sliding_sum("add_i32", 11, x, out=out[:0])
    torch.cuda.synchronize()
    assert y.numel() == 0 and (out == 12345).all()


def test_invalid_arguments_are_rejected():
    x = make_input("add_i32", 100).cuda()
    with pytest.raises(B.SwsError, match="INVALID"):
        B.sliding_sum("add_i32", 0, x)
    with pytest.raises(B.SwsError, match="INVALID"):
        B.sliding_sum("min_i32", 4, x, variant="prefix_diff")
    with pytest.raises(B.SwsError, match="INVALID"):
        B.sliding_sum("add_i32", 4, x, out=x[:97])  # overlapping


# ---------------------------------------------------------------------------------------------
# the persistent TMA-fed block combine ("stream")
# ---------------------------------------------------------------------------------------------
def stream_ws(op):
    c = 8 if op == "affine_u32" else 16
    return [c, 2 * c, 4 * c, 16 * c, 32 * c, 64 * c, 128 * c]


@pytest.mark.parametrize("op", OPS)
def test_stream_variant_matches_oracle(op):
    """Every block shape (blocks inside a warp, whole warps), one tile to many, a ragged tail
    that ends inside a 128-byte row (those elements bypass the tensor copy)."""
    for w in stream_ws(op):
        for n in (w + 40, 4096 + 7, 3 * 8192 + 17, 100_003):
            if n < w:
                continue
            x, ref = oracle_sliding(op, w, n, 11, op in INT_OPS)
            y = B.sliding_sum(op, w, x.cuda(), variant="stream")
            torch.cuda.synchronize()
            assert_sliding_equal(op, w, x, y, ref)


@pytest.mark.parametrize("op", OPS)
def test_stream_variant_many_tiles_per_cta(op):
    """Enough tiles that every CTA cycles its two stages many times (mbarrier phases wrap)."""
    rng = np.random.default_rng(3)
    n = (1 << 23) + 13
    x = make_input(op, n, seed=5, device="cuda")
    for w in stream_ws(op)[::2]:
        y = B.sliding_sum(op, w, x, variant="stream")
        yb = B.sliding_sum(op, w, x, variant="block_combine")
        torch.cuda.synchronize()
        if op != "add_f32":
            assert torch.equal(y, yb), (op, w)
        assert_sampled(op, w, x, y, sample_indices(n - w + 1, rng, 4096))


@pytest.mark.parametrize("op", ["add_i32", "affine_u32"])
def test_stream_variant_unsupported_shapes(op):
    c = 8 if op == "affine_u32" else 16
    x = make_input(op, 1 << 23, device="cuda")
    with pytest.raises(B.SwsError, match="UNSUPPORTED"):
        B.sliding_sum(op, 3 * c, x, variant="stream")  # 3 chunks per block
    with pytest.raises(B.SwsError, match="UNSUPPORTED"):
        B.sliding_sum(op, 4 * c, x[1:], variant="stream")  # input not 16-byte aligned
    with pytest.raises(B.SwsError, match="UNSUPPORTED"):
        B.sliding_sum(op, c, x[: c + 4], variant="stream")  # less than one 128-byte row
    # the automatic choice falls back to the one-shot tiles for the unaligned view
    y = B.sliding_sum(op, 4 * c, x[1:])
    torch.cuda.synchronize()
    assert_sampled(op, 4 * c, x[1:], y, sample_indices(y.shape[0], np.random.default_rng(1)))


# ---------------------------------------------------------------------------------------------
# the warp-private streaming block combine ("warp"): blocks of G = 1..32 lanes
# ---------------------------------------------------------------------------------------------
def warp_ws(op):
    """Blocks of 1..32 lanes, and blocks of 2, 4 and 8 whole warp-tiles."""
    c = 8 if op == "affine_u32" else 16
    return [c, 2 * c, 4 * c, 8 * c, 16 * c, 32 * c, 64 * c, 128 * c, 256 * c]


@pytest.mark.parametrize("op", OPS)
def test_warp_variant_matches_oracle(op):
    """Runs shorter and longer than one warp's share, ragged tails inside a 128-byte row."""
    es = 8 if op == "affine_u32" else 4
    for w in warp_ws(op):
        for n in (w, w + 40, 2048 + 7, 3 * 8192 + 17, 100_003, 7 * w):
            x, ref = oracle_sliding(op, w, n, 13, op in INT_OPS)
            if n * es < 128:  # less than one 128-byte row: not for the tensor copies
                with pytest.raises(B.SwsError, match="UNSUPPORTED"):
                    B.sliding_sum(op, w, x.cuda(), variant="warp")
                continue
            y = B.sliding_sum(op, w, x.cuda(), variant="warp")
            torch.cuda.synchronize()
            assert_sliding_equal(op, w, x, y, ref)


@pytest.mark.parametrize("op", OPS)
def test_warp_variant_many_tiles_per_warp(op):
    """Long runs per warp (stage slots and mbarrier phases wrap many times), against the one-shot
    kernel bit for bit and the oracle on sampled outputs."""
    rng = np.random.default_rng(4)
    n = (1 << 23) + 29
    x = make_input(op, n, seed=6, device="cuda")
    for w in warp_ws(op):
        y = B.sliding_sum(op, w, x, variant="warp")
        yb = B.sliding_sum(op, w, x, variant="block_combine")
        torch.cuda.synchronize()
        if op != "add_f32":
            assert torch.equal(y, yb), (op, w)
        assert_sampled(op, w, x, y, sample_indices(n - w + 1, rng, 4096))


def test_warp_variant_unsupported_shapes():
    x = make_input("add_i32", 1 << 20, device="cuda")
    for w, xv in ((48, x), (96, x), (8192, x), (64, x[1:]), (16, x[:20])):
        with pytest.raises(B.SwsError, match="UNSUPPORTED"):
            B.sliding_sum("add_i32", w, xv, variant="warp")


# ---------------------------------------------------------------------------------------------
# the autotuner
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("op,w", [("add_i32", 64), ("min_i32", 1024), ("xor_i32", 5), ("affine_u32", 48),
                                  ("add_f32", 256)])
def test_tuner_picks_an_applicable_variant_and_auto_uses_it(op, w):
    ctx = B.Context(0)
    try:
        n = 1 << 22
        chosen, ms = B.tune_sliding_sum(op, w, n, ctx=ctx)
        assert chosen in ms and all(v > 0 for v in ms.values())
        if chosen != "auto":  # a tuned variant must beat the fixed rule ("auto") by 2%
            assert ms[chosen] == min(ms.values()) and ms[chosen] <= 0.98 * ms["auto"]
        assert "block_combine" in ms and "doubling" in ms
        assert ("prefix_diff" in ms) == (op in ("add_i32", "xor_i32"))
        x = make_input(op, n, seed=3, device="cuda")
        y = B.sliding_sum(op, w, x, ctx=ctx)  # auto -> the tuned variant
        torch.cuda.synchronize()
        assert_sampled(op, w, x, y, sample_indices(n - w + 1, np.random.default_rng(w)))
    finally:
        ctx.close()


@pytest.mark.parametrize("op", ["add_i32", "affine_u32", "add_f32"])
@pytest.mark.parametrize("variant", ["warp", "stream", "auto"])
def test_streamed_kernels_with_unaligned_output(op, variant):
    """An aligned input (the tensor copies need it) and an output that starts 4 bytes into its
    buffer: the streamed kernels fall back to element stores."""
    n = (1 << 21) + 5
    x = make_input(op, n, seed=8, device="cuda")
    for w in (16, 64, 1024):
        m = n - w + 1
        buf = torch.empty((m + 1,) + tuple(x.shape[1:]), dtype=x.dtype, device="cuda")
        y = B.sliding_sum(op, w, x, out=buf[1:], variant=variant)
        yr = B.sliding_sum(op, w, x, variant="block_combine")
        torch.cuda.synchronize()
        if op != "add_f32":
            assert torch.equal(y, yr), (op, variant, w)
        assert_sampled(op, w, x, y, sample_indices(m, np.random.default_rng(w)))
