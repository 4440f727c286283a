"""Shared helpers of the GPU parity tests: inputs, oracle calls with caching, comparisons."""

from __future__ import annotations

import functools

import numpy as np
import pytest
import torch

import oracle
from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import build, synth

# fp32 sliding add: |y32 - y64| <= FP32_TOL * max(|y64|, sum of |x| over the window).
FP32_TOL = 1e-5


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    B.load()


def make_input(op: str, n: int, seed: int = 42, full_range: bool = False, device="cpu") -> torch.Tensor:
    if op == "affine_u32":
        return synth.affine_pairs(n, seed=seed, device=device)
    if op == "add_f32":
        return synth.f32_normal(n, seed=seed, device=device)
    if full_range:
        return synth.draws(seed, synth.STREAM_INT32, n, device=device).to(torch.int32)
    return synth.int32_uniform(n, seed=seed, device=device)


def window_abs_sum(x: np.ndarray, w: int) -> np.ndarray:
    a = np.abs(x.astype(np.float64))
    c = np.concatenate([[0.0], np.cumsum(a)])
    return c[w:] - c[:-w]


def assert_sliding_equal(op: str, w: int, x_cpu: torch.Tensor, y_gpu: torch.Tensor, ref: np.ndarray, idx=None):
    y = y_gpu.cpu().numpy()
    if idx is not None:
        y = y[idx]
    if op == "add_f32":
        xs = x_cpu.numpy()
        bound = window_abs_sum(xs, w)
        if idx is not None:
            bound = bound[idx]
        err = np.abs(y.astype(np.float64) - ref)
        lim = FP32_TOL * np.maximum(np.abs(ref), bound)
        bad = np.nonzero(err > lim)[0]
        assert bad.size == 0, f"fp32 tolerance exceeded at {bad[:5]}: err {err[bad[:5]]} lim {lim[bad[:5]]}"
    elif op == "affine_u32":
        yv = y.view(np.uint32).reshape(-1, 2)
        bad = np.nonzero((yv != ref).any(axis=1))[0]
        assert bad.size == 0, f"affine mismatch at {bad[:5]}: {yv[bad[:3]]} vs {ref[bad[:3]]}"
    else:
        bad = np.nonzero(y != ref)[0]
        assert bad.size == 0, f"mismatch at {bad[:5]} (of {y.size}): {y[bad[:5]]} vs {ref[bad[:5]]}"


@functools.lru_cache(maxsize=64)
def oracle_sliding(op: str, w: int, n: int, seed: int, full_range: bool):
    x = make_input(op, n, seed, full_range)
    return x, oracle.sliding_sum(op, w, x)


def to_u64(h: torch.Tensor) -> np.ndarray:
    a = h.cpu().numpy()
    if a.dtype == np.int32:
        return a.view(np.uint32).astype(np.uint64)
    return a.view(np.uint64)


def random_nblocks(n: int, rng: np.random.Generator, count: int, maxlen: int) -> np.ndarray:
    if n == 0 or count == 0:
        return np.zeros((0, 2), dtype=np.int64)
    starts = np.sort(rng.choice(n, size=min(count, n), replace=False))
    iv = []
    last_end = -1
    for s in starts:
        s = int(s)
        if s < last_end:
            continue
        e = min(n, s + int(rng.integers(1, maxlen + 1)))
        iv.append((s, e))
        last_end = e + 1
    return np.array(iv, dtype=np.int64).reshape(-1, 2)


def sample_indices(m: int, rng: np.random.Generator, count: int = 2048) -> np.ndarray:
    """Output indices to check on a large sliding sum: both ends, tile seams, random."""
    parts = [np.arange(min(64, m)), np.arange(max(m - 64, 0), m)]
    for tile in (4096, 8192):
        seams = rng.integers(1, max(m // tile, 2), size=32) * tile
        parts.append((seams[:, None] + np.arange(-3, 3)[None, :]).ravel())
    parts.append(rng.integers(0, m, size=count))
    idx = np.unique(np.concatenate(parts))
    return idx[(idx >= 0) & (idx < m)]


def assert_sampled(op: str, w: int, x: torch.Tensor, y: torch.Tensor, idx: np.ndarray):
    """y (device) against the oracle evaluated window by window at the sampled outputs idx."""
    dev = x.device
    it = torch.from_numpy(idx).to(dev)
    yv = y[it].cpu().numpy()
    win = x[it[:, None] + torch.arange(w, device=dev)[None, :]].cpu()
    flat = win.reshape((-1,) + tuple(x.shape[1:]))
    ref = oracle.sliding_sum_at(op, w, flat, np.arange(idx.size, dtype=np.uint64) * w)
    if op == "add_f32":
        bound = np.abs(win.numpy().astype(np.float64)).sum(axis=1)
        err = np.abs(yv.astype(np.float64) - ref)
        bad = np.nonzero(err > FP32_TOL * np.maximum(np.abs(ref), bound))[0]
    elif op == "affine_u32":
        bad = np.nonzero((yv.view(np.uint32).reshape(-1, 2) != ref).any(axis=1))[0]
    else:
        bad = np.nonzero(yv != ref)[0]
    assert bad.size == 0, (op, w, idx[bad[:5]])
