"""The single-pass sliding minimum over precomputed keys (the paper's timed task, Sec. 4) against
the oracle, element by element: every window length 1..17, inputs from the smallest the kernel
takes (32 keys) to thousands of tiles (so that tiles are placed by counts published by many
CTAs), ragged tails and final partial rows, ties (few distinct values, constant, monotone
inputs), full-range 32-bit keys, capacity overflow, and consecutive calls.  At 2^28 keys (the
benchmark's size) the picks are checked on sampled segments and by invariants."""

import numpy as np
import pytest
import torch

import oracle
from paper_1811_10074_gb300 import binding as B
from paper_1811_10074_gb300 import synth
from gpu_common import require_gpu, to_u64

pytestmark = pytest.mark.gpu

TILE = 4096


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def check_keys(keys: np.ndarray, w: int, what=""):
    kd = torch.from_numpy(keys.astype(np.uint32).view(np.int32)).cuda()
    assert kd.data_ptr() % 16 == 0
    h, p = B.minimizers_from_keys(kd, w)
    rh, rp = oracle.minimizers_from_keys(keys.astype(np.uint64), w)
    assert h.shape[0] == rh.size, (w, what, h.shape[0], rh.size)
    gh, gp = to_u64(h), p.cpu().numpy().view(np.uint32)
    bad = np.nonzero((gh != rh) | (gp != rp))[0]
    assert bad.size == 0, (w, what, bad[:5], gp[bad[:3]], rp[bad[:3]])


@pytest.mark.parametrize("w", list(range(1, 18)))
def test_every_window_length(w):
    rng = np.random.default_rng(300 + w)
    sizes = [32, 33, 63, w + 31, TILE, TILE + w - 1, TILE + w, 3 * TILE + 17, 1000 * TILE + 12_345]
    for m in sizes:
        if m < w:
            continue
        check_keys(rng.integers(0, 1 << 30, size=m, dtype=np.int64), w, f"random m={m}")
    # ties and monotone inputs over a few hundred tiles
    m = 300 * TILE + 7
    check_keys(rng.integers(0, 3, size=m, dtype=np.int64), w, "few values")
    check_keys(np.full(m, 7, dtype=np.int64), w, "constant")
    check_keys(np.arange(m, dtype=np.int64), w, "increasing")
    check_keys(np.arange(m, 0, -1, dtype=np.int64), w, "decreasing")
    check_keys(np.arange(m, dtype=np.int64) % (2 * w + 3), w, "sawtooth")
    check_keys(rng.integers(0, 1 << 32, size=50 * TILE + 29, dtype=np.int64), w, "full range")


def test_hashed_kmers_of_a_genome():
    """The benchmark's keys: hashed canonical 15-mers (sws_kmers) of a uniform sequence."""
    n = 5_000_000 + 14
    seq = synth.acgt_uniform_packed(n, seed=44)
    keys = oracle.kmers(seq, n, 15, "hash")
    for w in (4, 10, 16, 17):
        check_keys(keys.astype(np.int64), w, "hashed 15-mers")
    # and the GPU's own k-mer hashes as the input
    kd = B.kmers(seq.cuda(), n, 15, "hash")
    assert np.array_equal(kd.cpu().numpy().view(np.uint32).astype(np.uint64), keys)


def test_capacity_overflow_keeps_exact_count():
    rng = np.random.default_rng(5)
    m, w = 20 * TILE + 3, 6
    keys = rng.integers(0, 1 << 30, size=m, dtype=np.int64).astype(np.uint32)
    rh, rp = oracle.minimizers_from_keys(keys.astype(np.uint64), w)
    kd = torch.from_numpy(keys.view(np.int32)).cuda()
    cap = rh.size // 2
    h, p, cnt = B.minimizers_from_keys(kd, w, capacity=cap, sync=False)
    torch.cuda.synchronize()
    assert int(cnt.item()) == rh.size
    assert np.array_equal(to_u64(h[:cap]), rh[:cap]) and np.array_equal(p[:cap].cpu().numpy().view(np.uint32), rp[:cap])


def test_consecutive_calls_and_sizes():
    """The workspace (status words, ticket) is reset by every call: calls of shrinking and growing
    size in a row give the oracle's picks."""
    rng = np.random.default_rng(8)
    for m in (800 * TILE + 1, 40, 5 * TILE, 800 * TILE + 1, 2 * TILE + 31):
        keys = rng.integers(0, 1 << 30, size=m, dtype=np.int64)
        check_keys(keys, 10, f"m={m}")


@pytest.mark.parametrize("w", [4, 10, 17])
def test_full_size_sampled(w):
    """2^28 hashed 15-mers (the benchmark's input): counts match the density, positions strictly
    increase, and the picks whose windows lie inside a sampled segment equal the oracle's picks of
    that segment."""
    m = 1 << 28
    seq = synth.acgt_uniform_packed(m + 14, seed=44, device="cuda")
    keys = B.kmers(seq, m + 14, 15, "hash")
    del seq
    h, p, cnt = B.minimizers_from_keys(keys, w, capacity=m // 2, sync=False)
    count = int(cnt.item())
    assert abs(count / m - 2 / (w + 1)) < 0.01
    pos = p[:count].to(torch.int64) & 0xFFFFFFFF
    assert bool((pos[1:] > pos[:-1]).all())
    rng = np.random.default_rng(w)
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
    del keys, h, p
    torch.cuda.empty_cache()
