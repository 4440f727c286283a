"""The chunked multi-threaded drivers of the oracle (used to time it on all host cores) give
exactly the plain oracle's picks: the windows split into ranges, each range run by the plain
oracle in its own thread, the ranges joined with the seam pick stored once.  CPU only."""

import numpy as np
import pytest

from paper_1811_10074_gb300 import synth


@pytest.mark.parametrize("threads", [1, 2, 3, 8, 16])
def test_keys_chunked_equals_plain(orc, threads):
    rng = np.random.default_rng(threads)
    for m, hi in ((50_000, 1 << 30), (20_000, 3), (40, 5), (9, 1 << 30)):
        keys = rng.integers(0, hi, size=m, dtype=np.uint64)
        keys[m // 2:m // 2 + m // 10] = 7  # a run of equal keys across range seams
        for w in (1, 4, 10, 17):
            if w > m:
                continue
            want = orc.minimizers_from_keys(keys, w)
            for deque in (False, True):
                got = orc.minimizers_from_keys_chunked(keys, w, threads, deque=deque)
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (m, hi, w, deque)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_dna_chunked_equals_plain(orc, threads):
    for n, k, w in ((200_003, 15, 10), (60_000, 19, 50), (5_000, 4, 3), (30, 5, 4)):
        seq = synth.acgt_uniform_packed(n, seed=n + threads)
        want = orc.minimizers(seq, n, k, w)
        got = orc.minimizers_chunked(seq, n, k, w, threads)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (n, k, w)
    # a low-complexity sequence: equal k-mers repeat inside windows and across range seams
    n = 40_000
    seq = synth.pack_codes(__import__("torch").tensor(([0, 1] * (n // 2)), dtype=__import__("torch").uint8))
    want = orc.minimizers(seq, n, 5, 6)
    got = orc.minimizers_chunked(seq, n, 5, 6, threads)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
