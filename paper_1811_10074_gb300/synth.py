"""Seeded synthetic inputs for the sliding-window-sum and minimizer workloads.

Every generator draws from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based generator: draw ``i``
of a stream is ``mix(state0 + (i + 1) * GAMMA)``.  The arithmetic is torch int64 (two's
complement, wrapping mod 2^64), so one call gives the same bits on the CPU and on a CUDA
device; large benchmark inputs are therefore generated directly in device memory.

This module holds none of the method's arithmetic (no k-mers, hashes, window sums or
minima).  It only produces inputs in the library's formats:

* DNA is 2-bit packed, ``A=0, C=1, G=2, T=3``, base ``i`` in byte ``i >> 2`` at bits
  ``2 * (i & 3)`` (least significant first); the pad bits of the final byte are zero.
* N-blocks are half-open base intervals ``[start, end)`` (int64 ``[m, 2]``, sorted, disjoint).
* Affine maps are interleaved uint32 pairs ``(a, b)`` stored as int32 bit patterns.
"""

from __future__ import annotations

import math

import numpy as np
import torch

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_STREAM_MUL = 0xD1B54A32D192ED03  # odd constant separating streams of one seed

# Stream ids: one per workload field, so that fields never share draws.
STREAM_SEQ = 1
STREAM_INT32 = 2
STREAM_AFFINE = 3
STREAM_F32 = 4
STREAM_GC = 5
STREAM_NBLOCK = 6
STREAM_READ_LEN = 7
STREAM_READ_SEQ = 8
STREAM_ARRIVAL = 9
STREAM_REQ_LEN = 10
STREAM_REQ_SEQ = 11
STREAM_HASHES = 12
STREAM_SKEW = 13


def _s64(c: int) -> int:
    """Python int in [0, 2^64) -> the int64 with the same bits."""
    c &= MASK64
    return c - (1 << 64) if c >= (1 << 63) else c


def _mix_py(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def stream_state(seed: int, stream: int) -> int:
    """Starting state of stream ``stream`` of ``seed`` (a Python int in [0, 2^64))."""
    return _mix_py(seed * GAMMA + stream * _STREAM_MUL)


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor holding uint64 bits."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def draws(seed: int, stream: int, count: int, device="cpu", start: int = 0) -> torch.Tensor:
    """``count`` raw 64-bit draws (int64 bit patterns) of one stream, beginning at draw ``start``."""
    s0 = _s64(stream_state(seed, stream))
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = i * _s64(GAMMA) + s0
    z = (z ^ _srl(z, 30)) * _s64(_M1)
    z = (z ^ _srl(z, 27)) * _s64(_M2)
    return z ^ _srl(z, 31)


def draws_numpy(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """The same draws as :func:`draws`, computed with numpy uint64 (used to cross-check torch)."""
    s0 = np.uint64(stream_state(seed, stream))
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = i * np.uint64(GAMMA) + s0
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def _u53(d: torch.Tensor) -> torch.Tensor:
    """Draws -> float64 uniforms in [0, 1) with 53 random bits."""
    return _srl(d, 11).to(torch.float64) * (2.0 ** -53)


# ----------------------------------------------------------------------------------------
# DNA
# ----------------------------------------------------------------------------------------

def packed_nbytes(n: int) -> int:
    return (n + 3) // 4


def acgt_uniform_packed(n: int, seed: int = 42, stream: int = STREAM_SEQ, device="cpu") -> torch.Tensor:
    """``n`` i.i.d. uniform bases, 2-bit packed (uint8, ``ceil(n/4)`` bytes).

    Each 64-bit draw supplies 32 bases (its bytes in little-endian order)."""
    nb = packed_nbytes(n)
    d = draws(seed, stream, (nb + 7) // 8, device=device)
    out = d.view(torch.uint8)[:nb].clone()
    if n % 4:
        out[nb - 1] &= (1 << (2 * (n % 4))) - 1
    return out


def pack_codes(codes: torch.Tensor) -> torch.Tensor:
    """Base codes (uint8 values 0..3, length n) -> 2-bit packed bytes."""
    n = codes.numel()
    nb = packed_nbytes(n)
    c = torch.zeros(nb * 4, dtype=torch.uint8, device=codes.device)
    c[:n] = codes.to(torch.uint8)
    c = c.view(nb, 4)
    return c[:, 0] | (c[:, 1] << 2) | (c[:, 2] << 4) | (c[:, 3] << 6)


def unpack_codes(packed: torch.Tensor, n: int) -> torch.Tensor:
    """2-bit packed bytes -> base codes (uint8, length n)."""
    p = packed.to(torch.uint8)
    c = torch.stack([p & 3, (p >> 2) & 3, (p >> 4) & 3, (p >> 6) & 3], dim=1).reshape(-1)
    return c[:n].contiguous()


def codes_from_string(s: str) -> torch.Tensor:
    table = {"A": 0, "C": 1, "G": 2, "T": 3}
    return torch.tensor([table[ch] for ch in s.upper()], dtype=torch.uint8)


def acgt_gc_codes(n: int, gc: float = 0.41, seed: int = 42, device="cpu", chunk: int = 1 << 28) -> torch.Tensor:
    """``n`` i.i.d. base codes with P(C)=P(G)=gc/2 and P(A)=P(T)=(1-gc)/2 (see
    :func:`acgt_gc_codes_range`), generated in chunks so that long sequences fit in memory."""
    out = torch.empty(n, dtype=torch.uint8, device=device)
    per = chunk - chunk % 4
    for b0 in range(0, n, per):
        m = min(per, n - b0)
        out[b0:b0 + m] = acgt_gc_codes_range(b0, m, gc, seed, device)
    return out


def nblock_intervals(n: int, frac: float = 0.05, lmin: int = 10_000, lmax: int = 1_000_000,
                     seed: int = 42, stream: int = STREAM_NBLOCK) -> np.ndarray:
    """N-blocks covering at least ``frac`` of ``n`` bases, lengths log-uniform in [lmin, lmax],
    at uniform disjoint positions.  Returns sorted int64 ``[m, 2]`` half-open intervals."""
    if n <= 0 or frac <= 0:
        return np.zeros((0, 2), dtype=np.int64)
    lens = []
    total = 0
    idx = 0
    target = frac * n
    while total < target:
        u = float(_u53(draws(seed, stream, 1, start=idx))[0]); idx += 1
        L = int(round(math.exp(math.log(lmin) + u * (math.log(lmax) - math.log(lmin)))))
        L = max(1, min(L, n - total - 1))
        if L <= 0:
            break
        lens.append(L)
        total += L
    m = len(lens)
    free = n - total
    g = _u53(draws(seed, stream, m + 1, start=idx)).numpy() + 1e-9
    gaps = np.floor(g / g.sum() * free).astype(np.int64)
    iv = np.zeros((m, 2), dtype=np.int64)
    pos = 0
    for j in range(m):
        pos += int(gaps[j])
        iv[j] = (pos, pos + lens[j])
        pos += lens[j]
    assert pos <= n
    return iv


def genome_packed(n: int, gc: float = 0.41, nfrac: float = 0.05, lmin: int = 10_000, lmax: int = 1_000_000,
                  seed: int = 42, device="cpu", chunk: int = 1 << 28):
    """Synthetic genome: GC-biased i.i.d. bases with N-blocks.  Returns (packed uint8, intervals).

    Bases inside N-blocks are stored as code 0; the intervals say where they are."""
    iv = nblock_intervals(n, nfrac, lmin, lmax, seed=seed)
    nb = packed_nbytes(n)
    packed = torch.empty(nb, dtype=torch.uint8, device=device)
    per = chunk - chunk % 4
    for b0 in range(0, n, per):
        m = min(per, n - b0)
        codes = acgt_gc_codes_range(b0, m, gc, seed, device)
        for s, e in iv:
            lo, hi = max(int(s), b0), min(int(e), b0 + m)
            if lo < hi:
                codes[lo - b0:hi - b0] = 0
        packed[b0 // 4:(b0 + m + 3) // 4] = pack_codes(codes)
        del codes
    return packed, iv


def acgt_gc_codes_range(b0: int, m: int, gc: float, seed: int, device) -> torch.Tensor:
    """Bases ``[b0, b0 + m)`` of the GC-biased sequence (``b0`` a multiple of 4).

    Each draw supplies four 16-bit uniforms; base ``i`` uses 16-bit field ``i & 3`` of draw
    ``i >> 2``, compared against the cumulative thresholds C < G < A < T."""
    assert b0 % 4 == 0
    t_c = int(round(gc / 2 * 65536))
    t_g = int(round(gc * 65536))
    t_a = int(round((gc + (1 - gc) / 2) * 65536))
    d = draws(seed, STREAM_GC, (m + 3) // 4, device=device, start=b0 // 4)
    u = torch.stack([d & 0xFFFF, _srl(d, 16) & 0xFFFF, _srl(d, 32) & 0xFFFF, _srl(d, 48)], 1).reshape(-1)[:m]
    code = torch.full_like(u, 3)
    code = torch.where(u < t_a, torch.zeros_like(u), code)
    code = torch.where(u < t_g, torch.full_like(u, 2), code)
    code = torch.where(u < t_c, torch.ones_like(u), code)
    return code.to(torch.uint8)


# ----------------------------------------------------------------------------------------
# Generic sliding-sum inputs
# ----------------------------------------------------------------------------------------

def int32_uniform(n: int, lo: int = -(1 << 20), hi: int = 1 << 20, seed: int = 42,
                  stream: int = STREAM_INT32, device="cpu") -> torch.Tensor:
    """int32 uniform in [lo, hi) (multiply-shift of the top 32 bits of each draw)."""
    d = draws(seed, stream, n, device=device)
    u32 = _srl(d, 32)
    v = ((u32 * (hi - lo)) >> 32) + lo
    return v.to(torch.int32)


def affine_pairs(n: int, seed: int = 42, stream: int = STREAM_AFFINE, device="cpu") -> torch.Tensor:
    """``n`` affine maps x -> a*x + b mod 2^32, a and b uniform uint32: int32 ``[n, 2]`` = (a, b) bits."""
    d = draws(seed, stream, n, device=device)
    return d.view(torch.int32).reshape(n, 2)


def f32_normal(n: int, seed: int = 42, stream: int = STREAM_F32, device="cpu") -> torch.Tensor:
    """fp32 N(0, 1) by the Box-Muller transform evaluated in fp64, then rounded."""
    m = (n + 1) // 2
    d = draws(seed, stream, 2 * m, device=device)
    u1 = 1.0 - _u53(d[0::2])          # (0, 1]
    u2 = _u53(d[1::2])
    r = torch.sqrt(-2.0 * torch.log(u1))
    z = torch.stack([r * torch.cos(2 * math.pi * u2), r * torch.sin(2 * math.pi * u2)], 1).reshape(-1)[:n]
    return z.to(torch.float32)


def uint32_hashes(n: int, bits: int = 30, seed: int = 42, stream: int = STREAM_HASHES, device="cpu") -> torch.Tensor:
    """``n`` uniform ``bits``-bit values as int32 bit patterns (stand-in for a precomputed hash array)."""
    d = draws(seed, stream, n, device=device)
    return (_srl(d, 64 - bits)).to(torch.int64).to(torch.int32) if bits < 32 else _srl(d, 32).to(torch.int32)


def minimizer_skew_hashes(m: int, hash_bits: int = 38, w: int = 10, drop_bits: int = 2, seed: int = 42,
                          stream: int = STREAM_SKEW, device="cpu", chunk: int = 1 << 24) -> torch.Tensor:
    """``m`` int64 hashes spread like the minimizer picks of i.i.d. keys.

    A key at hash fraction x is some window's leftmost least key exactly when the keys to its
    left that exceed it and the keys to its right that do not undercut it span at least w - 1
    places, which for i.i.d. keys has probability (1 - x)^(w-1) (1 + (w-1) x): small hashes are
    picked far more often than large ones.  Draw 2i gives x, draw 2i + 1 the acceptance test of
    that density (rejection sampling); the hash is x scaled to [0, 2^(hash_bits - drop_bits)),
    i.e. drop_bits > 0 crowds the hits into fewer buckets, as a genome 2^drop_bits times larger
    would."""
    out, have, start = [], 0, 0
    scale = float(1 << (hash_bits - drop_bits))
    while have < m:
        d = draws(seed, stream, 2 * chunk, device=device, start=start)
        start += 2 * chunk
        x = _u53(d[0::2])
        u = _u53(d[1::2])
        keep = x[u < (1.0 - x) ** (w - 1) * (1.0 + (w - 1) * x)]
        out.append((keep * scale).to(torch.int64))
        have += keep.numel()
    return torch.cat(out)[:m]


# ----------------------------------------------------------------------------------------
# Read batches and serving arrivals
# ----------------------------------------------------------------------------------------

def _normals(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    d = draws(seed, stream, 2 * count, start=2 * start)
    u1 = 1.0 - _u53(d[0::2])
    u2 = _u53(d[1::2])
    return (torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2 * math.pi * u2)).numpy()


def read_lengths(n_short: int, n_long: int, short_lo: int = 100, short_hi: int = 250,
                 long_median: float = 10_000.0, long_sigma: float = 1.0, long_max: int = 200_000,
                 long_min: int = 24, seed: int = 42) -> np.ndarray:
    """Lengths of a read batch: ``n_short`` uniform in [short_lo, short_hi] then ``n_long``
    log-normal (ln L ~ N(ln median, sigma)), resampled until ``long_min <= L <= long_max``."""
    d = draws(seed, STREAM_READ_LEN, n_short).numpy().view(np.uint64)
    short = short_lo + ((d >> np.uint64(32)) * np.uint64(short_hi - short_lo + 1) >> np.uint64(32)).astype(np.int64)
    out = []
    idx = 0
    while len(out) < n_long:
        z = _normals(seed, STREAM_READ_LEN + 100, 4 * (n_long - len(out)) + 16, start=idx)
        idx += len(z)
        L = np.round(np.exp(math.log(long_median) + long_sigma * z)).astype(np.int64)
        L = L[(L >= long_min) & (L <= long_max)]
        out.extend(L[: n_long - len(out)].tolist())
    return np.concatenate([short, np.asarray(out, dtype=np.int64)])


def read_batch(lengths: np.ndarray, seed: int = 42, device="cpu"):
    """Concatenate reads of the given lengths into one packed stream of uniform bases.

    Returns (packed uint8, base_offsets int64 [nreads + 1])."""
    offs = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offs[1:])
    total = int(offs[-1])
    packed = acgt_uniform_packed(total, seed=seed, stream=STREAM_READ_SEQ, device=device)
    return packed, offs


def poisson_arrivals(count: int, rate: float, seed: int = 42) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (exponential gaps)."""
    u = 1.0 - _u53(draws(seed, STREAM_ARRIVAL, count)).numpy()
    return np.cumsum(-np.log(u) / rate)


def loguniform_lengths(count: int, lo: int = 150, hi: int = 1_000_000, seed: int = 42) -> np.ndarray:
    u = _u53(draws(seed, STREAM_REQ_LEN, count)).numpy()
    return np.round(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
