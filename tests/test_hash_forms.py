"""The arithmetic forms of the 2k-bit hash that the single-pass kernels use, against the oracle's
hash (Wang's mix truncated to 2k bits after every step).  CPU only.

The kernels never compute the hash in its masked textbook form:
  * 32-bit keys (k <= 16): the mix runs on x << (32 - 2k), where arithmetic modulo 2^(2k) is the
    32-bit word's own overflow and each right shift clears the low 32 - 2k bits it brings in;
    the result is shifted back when a pick is written out;
  * 64-bit keys (16 < k <= 29): an xor-shift by s of a state whose high word holds at most HB
    bits (2k = 32 + HB) leaves nothing in the high word when HB <= s, so it touches the low word
    only (HB = 14 serves k <= 23, HB = 26 serves k <= 29).
These restatements mirror those forms step by step; the oracle decides."""

import numpy as np
import pytest

M32 = 0xFFFFFFFF
M64 = (1 << 64) - 1


def mix_left32(X: int, hm: int) -> int:
    X = (X * 0x1FFFFF + hm) & M32
    X ^= (X >> 24) & hm
    X = (X * 265) & M32
    X ^= (X >> 14) & hm
    X = (X * 21) & M32
    X ^= (X >> 28) & hm
    return (X * 0x80000001) & M32


def mix_hb64(x: int, mhi: int, hb: int) -> int:
    def mask(v):
        return ((((v >> 32) & mhi) << 32) | (v & M32)) & M64

    def xs(v, s):
        lo, hi = v & M32, v >> 32
        if hb <= s:  # the high word of v >> s is empty: only the low word changes
            return (hi << 32) | (lo ^ (((hi << 32 | lo) >> s) & M32))
        return v ^ (v >> s)

    x = mask(x * 0x1FFFFF + M64)
    x = xs(x, 24)
    x = mask(x * 265)
    x = xs(x, 14)
    x = mask(x * 21)
    x = xs(x, 28)
    return mask(x * 0x80000001)


def samples(bits: int, n: int = 1500, seed: int = 0):
    rng = np.random.default_rng(seed + bits)
    m = (1 << bits) - 1
    edge = [0, 1, 2, m, m - 1, m >> 1, (m >> 1) + 1]
    rnd = [int(v) & m for v in rng.integers(0, 1 << 62, size=n, dtype=np.int64)]
    return [v for v in edge if 0 <= v <= m] + rnd


@pytest.mark.parametrize("k", range(1, 17))
def test_left_aligned_32_bit_hash(orc, k):
    bits = 2 * k
    s = 32 - bits
    hm = (M32 << s) & M32
    for x in samples(bits):
        assert mix_left32(x << s, hm) >> s == orc.hash64(x, bits), (k, x)


@pytest.mark.parametrize("k", range(17, 30))
def test_one_word_xor_shift_64_bit_hash(orc, k):
    bits = 2 * k
    mhi = ((1 << bits) - 1) >> 32
    hb = 14 if k <= 23 else 26  # the classes the kernel instantiates
    assert bits - 32 <= hb
    for x in samples(bits):
        assert mix_hb64(x, mhi, hb) == orc.hash64(x, bits), (k, x)


def test_left_aligned_order_is_the_hash_order():
    """The combine compares shifted keys: shifting left by 32 - 2k keeps their order."""
    for k in (5, 11, 15):
        s = 32 - 2 * k
        vals = sorted(samples(2 * k, n=300))
        shifted = [(v << s) & M32 for v in vals]
        assert shifted == sorted(shifted)
