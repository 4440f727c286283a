"""The seeded input generators (CPU only)."""

import numpy as np
import torch

from paper_1811_10074_gb300 import synth


def test_draws_match_numpy_uint64():
    for stream in (0, 1, 7):
        a = synth.draws(42, stream, 5000, start=123).numpy().view(np.uint64)
        b = synth.draws_numpy(42, stream, 5000, start=123)
        assert (a == b).all()


def test_splitmix64_reference_values():
    """Plain SplitMix64 from state 0 (Steele, Lea & Flood 2014): its first outputs are the
    widely reproduced 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F."""
    def plain(state, count):
        out = []
        for _ in range(count):
            state = (state + synth.GAMMA) & synth.MASK64
            out.append(synth._mix_py(state))
        return out
    assert plain(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    s0 = synth.stream_state(42, 1)
    got = synth.draws_numpy(42, 1, 4)
    assert [int(v) for v in got] == plain(s0, 4)


def test_packing_roundtrip_and_pad_bits():
    for n in (1, 2, 3, 4, 5, 1001):
        p = synth.acgt_uniform_packed(n)
        assert p.numel() == (n + 3) // 4
        if n % 4:
            assert int(p[-1]) >> (2 * (n % 4)) == 0
        c = synth.unpack_codes(p, n)
        assert torch.equal(synth.pack_codes(c), p)
    c = synth.codes_from_string("ACGTTGCA")
    assert synth.pack_codes(c).tolist() == [0b11100100, 0b00011011]


def test_base_composition():
    c = synth.acgt_gc_codes(400_000, gc=0.41)
    f = torch.bincount(c.long(), minlength=4).double() / c.numel()
    assert abs(float(f[1] + f[2]) - 0.41) < 0.005
    u = synth.unpack_codes(synth.acgt_uniform_packed(400_000), 400_000)
    f = torch.bincount(u.long(), minlength=4).double() / u.numel()
    assert (f - 0.25).abs().max() < 0.005


def test_nblocks():
    n = 5_000_000
    iv = synth.nblock_intervals(n, 0.05, 1000, 100_000)
    assert (iv[:, 1] > iv[:, 0]).all() and (iv[1:, 0] >= iv[:-1, 1]).all()
    assert iv[0, 0] >= 0 and iv[-1, 1] <= n
    cov = int((iv[:, 1] - iv[:, 0]).sum())
    assert 0.05 * n <= cov < 0.08 * n
    packed, iv2 = synth.genome_packed(200_000, nfrac=0.05, lmin=100, lmax=5000)
    assert packed.numel() == 50_000 and iv2.shape[1] == 2


def test_reads_and_values():
    L = synth.read_lengths(1000, 200, long_max=200_000)
    assert ((L[:1000] >= 100) & (L[:1000] <= 250)).all()
    assert ((L[1000:] >= 24) & (L[1000:] <= 200_000)).all()
    assert 4000 < np.median(L[1000:]) < 25000
    x = synth.int32_uniform(100_000)
    assert int(x.min()) >= -(1 << 20) and int(x.max()) < (1 << 20)
    z = synth.f32_normal(100_001)
    assert z.dtype == torch.float32 and abs(float(z.mean())) < 0.02 and abs(float(z.std()) - 1) < 0.02
    a = synth.affine_pairs(10)
    assert a.shape == (10, 2) and a.dtype == torch.int32
