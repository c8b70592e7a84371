"""Pins of the oracle's filtering stage (Algorithm 1: cosine weight + Ram-Lak row convolution)."""
import os

import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.phantom import (pixel_positions, principal_point, scaled_geometry,
                                            source_positions)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_ramlak_taps_golden():
    """Kak & Slaney, 'Principles of Computerized Tomographic Imaging', ch. 3, the
    spatial band-limited ramp: h(0)=1/4, h(even)=0, h(odd n)=-1/(pi^2 n^2) (unit pitch)."""
    tab = np.loadtxt(os.path.join(GOLDEN, "ramlak_kak_slaney.txt"))
    h = oracle.ramlak(16)
    for n, val in tab:
        assert h[int(n) + 15] == pytest.approx(val, rel=1e-15, abs=1e-18)
        assert h[-int(n) + 15] == pytest.approx(val, rel=1e-15, abs=1e-18)


@pytest.mark.parametrize("n", [64, 511, 2048])
def test_ramlak_frequency_response(n):
    """DTFT of the taps approaches the ramp |w|/(2 pi) on [-pi, pi]; the truncation
    error is at most sum_{|m| >= n} 1/(pi^2 m^2) <= 2/(pi^2 (n-1))."""
    h = oracle.ramlak(n)
    m = np.arange(-(n - 1), n)
    w = np.linspace(-np.pi, np.pi, 401)
    H = (h[None, :] * np.cos(w[:, None] * m[None, :])).sum(axis=1)
    bound = 2.0 / (np.pi ** 2 * (n - 1))
    assert np.max(np.abs(H - np.abs(w) / (2 * np.pi))) <= bound
    assert abs(h.sum()) <= bound                               # zero DC gain
    assert abs(H[-1] - 0.5) <= bound                           # gain 1/2 at Nyquist


def test_cosine_weight_is_ray_angle():
    """F_cos = cos of the angle between the pixel ray and the central ray, measured
    from the scanner's world-space source and pixel positions."""
    g = scaled_geometry(8, 24, 3, n_det_v=18).with_(off_u=0.7, off_v=-1.1)
    fc = oracle.cosine_weight(g)
    uc, vc = principal_point(g)
    beta = g.angles[1]
    S = source_positions(g, [1])[0]
    C = pixel_positions(g, beta, uc, vc)
    iv, iu = np.meshgrid(np.arange(g.nv), np.arange(g.nu), indexing="ij")
    P = pixel_positions(g, beta, iu, iv)
    ray = P - S
    cosang = (ray @ (C - S)) / (np.linalg.norm(ray, axis=-1) * np.linalg.norm(C - S))
    np.testing.assert_allclose(fc, cosang, rtol=1e-13)


@pytest.mark.parametrize("nu", [7, 64, 100, 300])
def test_direct_equals_fft(nu):
    """Direct linear convolution == zero-padded FFT convolution (independent algorithm)."""
    g = scaled_geometry(8, nu, 2, n_det_v=5)
    rng = np.random.default_rng(nu)
    E = rng.normal(size=(10, nu))
    rows = rng.integers(0, g.nv, size=10)
    qd = oracle.filter_rows(g, E, rows, method="direct")
    qf = oracle.filter_rows(g, E, rows, method="fft")
    assert np.max(np.abs(qd - qf)) <= 1e-12 * np.max(np.abs(qd))


def test_impulse_and_constant_rows():
    g = scaled_geometry(8, 41, 1, n_det_v=3)
    fc = oracle.cosine_weight(g)
    h = oracle.ramlak(g.nu)
    # impulse at m0: Q[n] = h(n - m0) F_cos[m0]
    m0, row = 13, 1
    E = np.zeros((1, g.nu))
    E[0, m0] = 1.0
    Q = oracle.filter_rows(g, E, [row], method="direct")[0]
    n = np.arange(g.nu)
    np.testing.assert_allclose(Q, h[n - m0 + g.nu - 1] * fc[row, m0], rtol=1e-14, atol=1e-16)
    # a row that is constant after weighting is mapped near 0 away from the edges
    E = (3.0 / fc[row])[None, :]
    Q = oracle.filter_rows(g, E, [row], method="fft")[0]
    mid = g.nu // 2
    tail = 3.0 * 2.0 / (np.pi ** 2 * (g.nu // 2 - 1))
    assert abs(Q[mid]) <= tail
    # at the edge only one side of the kernel overlaps the row:
    # 3 (h(0) + sum_{odd m>0} h(m)) = 3 (1/4 - 1/8 + truncation tail)
    for edge in (Q[0], Q[-1]):
        assert 3.0 / 8.0 <= edge <= 3.0 / 8.0 + 3.0 / (np.pi ** 2 * (g.nu - 2))
