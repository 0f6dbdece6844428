"""The seeded input generators (synth/): the counter-based SplitMix64 stream
against its published outputs, counter addressing, the distributions drawn
from it, and the phantom, PSF and noise helpers.  The same inputs are drawn on
the x86 host and on the Arm GPU host, so every value must follow from the
definitions alone."""
import math

import numpy as np

import synth

# SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) from state 0: the first
# outputs of the reference generator (state += 0x9E3779B97F4A7C15, then the
# mix), as quoted with its published reference implementation.
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_splitmix64_follows_the_published_sequence():
    got = [int(v) for v in synth.splitmix64(0, 0, 4)]
    assert got == SPLITMIX64_SEED0


def test_splitmix64_counter_addressing_and_separation():
    full = synth.splitmix64(7, 3, 40)
    assert np.array_equal(synth.splitmix64(7, 3, 15, offset=25), full[25:])
    assert np.array_equal(synth.splitmix64(7, 3, 40), full)  # deterministic
    others = [synth.splitmix64(8, 3, 40), synth.splitmix64(7, 4, 40)]
    for o in others:  # another seed or stream shares no draw in this window
        assert not np.intersect1d(o, full).size


def test_uniform_range_and_moments():
    n = 1_000_000
    u = synth.uniform(11, 0, n)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / n)
    # 53-bit resolution: every value is a multiple of 2^-53
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))


def test_normal_moments_and_odd_lengths():
    n = 1_000_001
    z = synth.normal(12, 1, n)
    assert z.shape == (n,)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * math.sqrt(96 / n)  # Gaussian kurtosis
    assert np.array_equal(synth.normal(12, 1, 5), z[:5])


def test_gaussian_psf_is_normalised_centred_and_separable():
    h = synth.gaussian_psf((1.0, 1.5, 0.7))
    assert h.shape == (7, 11, 7)  # (p_s, p_n, p_m) = 2 ceil(3 sigma) + 1
    assert abs(h.sum() - 1.0) < 1e-14
    c = tuple(p // 2 for p in h.shape)
    assert np.unravel_index(np.argmax(h), h.shape) == c
    assert np.allclose(h, h[::-1, ::-1, ::-1], rtol=0, atol=1e-17)
    fs, fn, fm = h.sum(axis=(1, 2)), h.sum(axis=(0, 2)), h.sum(axis=(0, 1))
    assert np.allclose(h, fs[:, None, None] * fn[None, :, None] * fm[None, None, :], rtol=1e-13, atol=0)
    # ratio of neighbouring taps along m is exp(-(2i+1) / (2 sigma^2))
    r = h[c[0], c[1], c[2] + 1] / h[c[0], c[1], c[2]]
    assert abs(r - math.exp(-1 / (2 * 1.0 ** 2))) < 1e-14


def test_noise_sigma_gives_the_requested_snr():
    clean = synth.uniform(3, 0, 4096).reshape(16, 16, 16)
    for snr in (20.0, 40.0):
        s = synth.noise_sigma(clean, snr)
        assert abs(10 * math.log10(clean.var() / s ** 2) - snr) < 1e-12
    assert np.array_equal(synth.noise_field((4, 4, 4), 9), synth.normal(9, 3, 64).reshape(4, 4, 4))


def test_ellipsoid_phantom_is_seeded_and_bounded():
    a = synth.ellipsoid_phantom((32, 24, 16), 12, 5)
    b = synth.ellipsoid_phantom((32, 24, 16), 12, 5)
    c = synth.ellipsoid_phantom((32, 24, 16), 12, 6)
    assert a.shape == (16, 24, 32) and a.dtype == np.float64
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0 and (a > 0).any() and (a == 0).any()
    # piecewise constant: at most one value per ellipsoid plus the background
    assert len(np.unique(a)) <= 13
    f = synth.ellipsoid_phantom((32, 24, 16), 12, 5, field_amplitude=0.1)
    assert abs(np.abs(f - a).max() - 0.1) < 1e-12
