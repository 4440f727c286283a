"""The skewed hit generator used to measure the seed-table sort: its density is the one of
minimizer picks of i.i.d. keys, checked against the oracle's picks on random keys."""

import numpy as np
import torch

import oracle
from paper_1811_10074_gb300 import synth


def test_skew_density_matches_oracle_picks():
    w, n = 10, 400_000
    keys = synth.uint32_hashes(n, bits=30, seed=3).numpy().view(np.uint32)
    vals, _ = oracle.minimizers_from_keys(keys, w)
    frac = vals.astype(np.float64) / float(1 << 30)
    # picks per key, by tenth of the hash range, against the density (1-x)^(w-1) (1 + (w-1) x)
    edges = np.linspace(0.0, 1.0, 11)
    got = np.histogram(frac, bins=edges)[0] / (n / 10)
    xs = np.linspace(0.0, 1.0, 100_001)
    dens = (1 - xs) ** (w - 1) * (1 + (w - 1) * xs)
    want = np.array([dens[(xs >= a) & (xs < b)].mean() for a, b in zip(edges[:-1], edges[1:])])
    assert np.allclose(got, want, atol=0.01), (got, want)
    assert abs(vals.size / n - 2 / (w + 1)) < 0.005


def test_skew_generator_follows_the_density():
    m, w = 300_000, 10
    h = synth.minimizer_skew_hashes(m, hash_bits=30, w=w, drop_bits=0, seed=5)
    assert h.shape == (m,) and h.dtype == torch.int64
    assert int(h.min()) >= 0 and int(h.max()) < (1 << 30)
    frac = h.numpy().astype(np.float64) / float(1 << 30)
    edges = np.linspace(0.0, 1.0, 11)
    got = np.histogram(frac, bins=edges)[0] / m
    xs = np.linspace(0.0, 1.0, 100_001)
    dens = (1 - xs) ** (w - 1) * (1 + (w - 1) * xs)
    want = np.array([dens[(xs >= a) & (xs < b)].mean() for a, b in zip(edges[:-1], edges[1:])])
    want = want / want.sum()
    assert np.allclose(got, want, atol=0.004), (got, want)
    # deterministic, and drop_bits packs into the lower part of the range
    assert torch.equal(h[:1000], synth.minimizer_skew_hashes(1000, hash_bits=30, w=w, drop_bits=0, seed=5))
    h2 = synth.minimizer_skew_hashes(1000, hash_bits=30, w=w, drop_bits=2, seed=5)
    assert int(h2.max()) < (1 << 28)
