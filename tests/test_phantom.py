"""Pins of the seeded input generator (analytic ellipsoid line integrals).

Each check compares against something other than the generator's own
quadratic: a closed form, bisection on the implicit surface, additivity, or
the scanner geometry read off the Eq. 2 matrices."""
import numpy as np
import pytest

from paper_1909_02724_gb300.phantom import (Ellipsoids, chord_lengths, line_integrals,
                                            pixel_positions, principal_point, random_ellipsoids,
                                            safe_radius, scaled_geometry, source_positions, sphere,
                                            workload)


def test_sphere_chord_closed_form():
    """Chord of a ball of radius R at distance b from the centre: 2 sqrt(R^2 - b^2)."""
    rng = np.random.default_rng(0)
    R, c = 17.0, np.array([3.0, -2.0, 5.0])
    ball = sphere(R, rho=1.0, centre=c)
    src = np.array([-1000.0, 40.0, 10.0])
    dst = rng.normal(size=(200, 3)) * 15.0 + np.array([500.0, 0.0, 0.0])
    d = (dst - src) / np.linalg.norm(dst - src, axis=1, keepdims=True)
    b = np.linalg.norm(np.cross(c - src, d), axis=1)
    expect = np.where(b < R, 2.0 * np.sqrt(np.maximum(R * R - b * b, 0.0)), 0.0)
    got = chord_lengths(ball, src, dst)
    assert np.max(np.abs(got - expect)) < 1e-9 * R
    assert (b < R).sum() > 50


def _bisect_chord(c, axes, rot, src, d):
    """Entry/exit of the implicit surface |diag(1/a) R^T (x - c)| = 1 along x = src + t d,
    located by scanning for sign changes and bisection (no quadratic formula)."""
    m = rot.T / axes[:, None]

    def q(t):
        return np.sum((m @ (src + t * d - c)) ** 2) - 1.0

    t_mid = float(np.dot(c - src, d))
    span = 2.0 * float(np.max(axes))
    ts = np.linspace(t_mid - span, t_mid + span, 4001)
    vals = np.array([q(t) for t in ts])
    roots = []
    for n in range(len(ts) - 1):
        if vals[n] * vals[n + 1] < 0:
            lo, hi = ts[n], ts[n + 1]
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if q(lo) * q(mid) <= 0:
                    hi = mid
                else:
                    lo = mid
            roots.append(0.5 * (lo + hi))
    if len(roots) < 2:
        return 0.0
    return roots[-1] - roots[0]


def test_ellipsoid_chord_vs_bisection():
    ell = random_ellipsoids(6, 25.0, seed=5)
    rng = np.random.default_rng(1)
    src = np.array([0.0, -1000.0, 0.0])
    for e in range(len(ell)):
        one = Ellipsoids(ell.centre[e:e + 1], ell.axes[e:e + 1], ell.rot[e:e + 1], np.ones(1))
        for _ in range(6):
            target = ell.centre[e] + rng.normal(size=3) * 0.4 * ell.axes[e].min()
            dst = src + 1.5 * (target - src)
            d = (dst - src) / np.linalg.norm(dst - src)
            expect = _bisect_chord(ell.centre[e], ell.axes[e], ell.rot[e], src, d)
            got = float(chord_lengths(one, src, dst[None])[0])
            assert expect > 0
            assert abs(got - expect) < 1e-9 * max(1.0, expect)


def test_additivity_and_density():
    g = scaled_geometry(16, 20, 6)
    a = random_ellipsoids(3, 20.0, seed=2)
    b = random_ellipsoids(4, 20.0, seed=3)
    ab = Ellipsoids(np.concatenate([a.centre, b.centre]), np.concatenate([a.axes, b.axes]),
                    np.concatenate([a.rot, b.rot]), np.concatenate([a.rho, b.rho]))
    Ea, Eb, Eab = line_integrals(a, g), line_integrals(b, g), line_integrals(ab, g)
    np.testing.assert_allclose(Eab, Ea + Eb, rtol=1e-12, atol=1e-12)
    a2 = Ellipsoids(a.centre, a.axes, a.rot, 2.5 * a.rho)
    np.testing.assert_allclose(line_integrals(a2, g), 2.5 * Ea, rtol=1e-12, atol=1e-12)


def test_scanner_positions():
    """Central pixel ray has length D; the detector plane is perpendicular to it;
    pixel pitch along U and V is (Du, Dv)."""
    g = scaled_geometry(16, 33, 7).with_(off_u=0.3, off_v=-0.45)
    uc, vc = principal_point(g)
    for s, beta in enumerate(g.angles):
        S = source_positions(g, [s])[0]
        C = pixel_positions(g, beta, uc, vc)
        assert abs(np.linalg.norm(C - S) - g.sdd) < 1e-9
        n = (C - S) / g.sdd
        assert abs(np.dot(S, n) + g.sid) < 1e-9          # source at distance d before the axis
        P1 = pixel_positions(g, beta, uc + 1.0, vc)
        P2 = pixel_positions(g, beta, uc, vc + 1.0)
        assert abs(np.dot(P1 - C, n)) < 1e-9 and abs(np.dot(P2 - C, n)) < 1e-9
        assert abs(np.linalg.norm(P1 - C) - g.du) < 1e-12
        assert abs(np.linalg.norm(P2 - C) - g.dv) < 1e-12


def test_workloads_fit_the_field_of_view():
    for name in ("fdk64", "fdk512", "grad32"):
        w = workload(name)
        ell = w.phantom()
        r = np.linalg.norm(ell.centre, axis=1) + ell.axes.max(axis=1)
        assert r.max() <= 0.95 * 0.9 * safe_radius(w.geom) + 1e-9
        assert len(ell) == w.n_ellipsoids


def test_untruncated_projections():
    """Inside the safe radius no ray leaves the detector: the detector border is empty."""
    w = workload("fdk64")
    E = line_integrals(w.phantom(), w.geom)
    border = np.concatenate([E[:, 0, :].ravel(), E[:, -1, :].ravel(), E[:, :, 0].ravel(),
                             E[:, :, -1].ravel()])
    assert border.max() == 0.0
    assert E.max() > 1.0


@pytest.mark.parametrize("seed", [1909, 1910])
def test_seeded_phantom_is_reproducible(seed):
    a = random_ellipsoids(5, 10.0, seed)
    b = random_ellipsoids(5, 10.0, seed)
    np.testing.assert_array_equal(a.packed(), b.packed())
