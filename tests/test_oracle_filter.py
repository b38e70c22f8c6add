"""Pins of the oracle's ISO 16610-61 Gaussian filters (the S- and L-filters
the paper applies to its measured surfaces, Section 4.1.1): transmission
closed forms, invariants and a 2D brute force of the areal definition."""
import math

import numpy as np
import pytest

ALPHA = math.sqrt(math.log(2.0) / math.pi)


def transmission(lam_cut, lam):
    """Amplitude transmission of the Gaussian low-pass: 50 % at the cutoff."""
    return math.exp(-math.pi * (ALPHA * lam_cut / lam) ** 2)


def test_constant_is_kept_everywhere(oracle_mod):
    H = np.full((37, 53), -0.1234)
    out = oracle_mod.gauss_filter(H, 0.005, 0.08)
    assert np.abs(out - H).max() <= 1e-15


def test_plane_is_kept_in_the_interior(oracle_mod):
    """The weighting function is even, so linear terms pass unchanged where
    the whole kernel lies inside the map; the SL-surface of a plane is 0."""
    pitch, lc = 0.005, 0.1
    T = int(lc / pitch)
    y, x = np.mgrid[0:80, 0:90] * pitch
    H = 0.03 * x - 0.02 * y + 0.5
    out = oracle_mod.gauss_filter(H, pitch, lc)
    inner = (slice(T, 80 - T), slice(T, 90 - T))
    assert np.abs(out[inner] - H[inner]).max() <= 1e-12
    sl = oracle_mod.sl_surface(H, pitch, 0.0, lc)
    assert np.abs(sl[inner]).max() <= 1e-12


@pytest.mark.parametrize("ratio", [1.0, 2.0, 0.5, 4.0])
def test_transmission_of_a_sinusoid(oracle_mod, ratio):
    """A sinusoid of wavelength ratio * cutoff comes out scaled by
    exp(-pi (alpha lc / lambda)^2): 50 % at the cutoff (ISO 16610-61)."""
    pitch, lc = 0.002, 0.08
    lam = ratio * lc
    T = int(lc / pitch)
    x = (np.arange(600) + 0.25) * pitch
    H = np.tile(np.sin(2 * math.pi * x / lam), (2 * T + 3, 1)) * 1e-3
    out = oracle_mod.gauss_filter(H, pitch, lc)
    k = T + 1
    exp = transmission(lc, lam) * H[k, T:-T]
    assert np.abs(out[k, T:-T] - exp).max() <= 2e-6 * 1e-3


def test_s_filter_removes_short_wavelengths_and_sl_keeps_the_band(oracle_mod):
    """S-filter at lambda_s = 10 um passes a 5 um sinusoid at 2^-4; the
    L-filter at 0.8 mm takes 2^(-1/16) of a 3.2 mm sinusoid as mean surface,
    leaving 1 - 2^(-1/16) in the SL-surface."""
    pitch = 0.001
    ls, lc = 0.010, 0.8
    x = (np.arange(4000) + 0.5) * pitch
    short = 1e-4 * np.sin(2 * math.pi * x / 0.005)
    long_ = 1e-2 * np.sin(2 * math.pi * x / 3.2)
    H = np.tile(short + long_, (3, 1))
    S = oracle_mod.gauss_filter(H, pitch, ls)
    mid = slice(900, 3100)
    want = transmission(ls, 0.005) * short + transmission(ls, 3.2) * long_
    assert transmission(ls, 0.005) == pytest.approx(2 ** -4)
    assert np.abs(S[1, mid] - want[mid]).max() <= 1e-9
    sl = oracle_mod.sl_surface(H, pitch, ls, lc)
    band = (1 - transmission(lc, 3.2)) * transmission(ls, 3.2) * long_ + \
        (1 - transmission(lc, 0.005)) * transmission(ls, 0.005) * short
    assert 1 - transmission(lc, 3.2) == pytest.approx(1 - 2 ** (-1 / 16))
    assert np.abs(sl[1, mid] - band[mid]).max() <= 2e-8


def test_separable_passes_equal_the_areal_definition(oracle_mod):
    """Brute force of the 2D weighting function with the end correction over
    the rectangle, on a small random map whose edges cut the kernel."""
    rng = np.random.default_rng(7)
    ny, nx, pitch, lam = 23, 31, 0.01, 0.09
    H = rng.normal(size=(ny, nx))
    T = int(lam / pitch + 1e-9)
    a = ALPHA * lam
    t = np.arange(-T, T + 1) * pitch
    w = np.exp(-math.pi * (t / a) ** 2)
    W2 = np.outer(w, w)
    ref = np.empty_like(H)
    for k in range(ny):
        for i in range(nx):
            num = den = 0.0
            for u in range(-T, T + 1):
                for v in range(-T, T + 1):
                    kk, ii = k + u, i + v
                    if 0 <= kk < ny and 0 <= ii < nx:
                        num += W2[u + T, v + T] * H[kk, ii]
                        den += W2[u + T, v + T]
            ref[k, i] = num / den
    out = oracle_mod.gauss_filter(H, pitch, lam)
    assert np.abs(out - ref).max() <= 1e-13


def test_rejects_bad_requests(oracle_mod):
    H = np.zeros((4, 4))
    with pytest.raises(ValueError):
        oracle_mod.gauss_filter(H, 0.0, 0.1)
    with pytest.raises(ValueError):
        oracle_mod.sl_surface(H, 0.01, -1.0, 0.1)
