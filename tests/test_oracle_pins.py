"""The oracle against facts the paper and mathematics fix (see tests/pins.py).  CPU only."""

import pytest

import pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(orc, check):
    check(orc.load())


@pytest.mark.slow
def test_hash_bijection_30_bits(orc):
    """The k=15 hash (2k = 30 bits) is a bijection, checked over all 2^30 inputs."""
    assert orc.hash_is_bijection(30)
