"""Pins of the oracle's short-scan weights (Parker, Med. Phys. 9, 1982).

The redundant partner of a ray is found from the scanner's world geometry
(the second crossing of the ray's line with the source circle), not from the
weight formula, so a wrong sign of gamma or a wrong offset fails the
redundancy pin.  A uniform ball reconstructed from a short scan must have
its density at the centre (the factor 2 that replaces the full-scan 1/2),
and the mid-plane must match the full-scan reconstruction."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.geometry import circular, fan_half_angle, short_scan
from paper_1909_02724_gb300.phantom import (line_integrals, pixel_positions, principal_point, random_ellipsoids,
                                            scaled_geometry, sphere)


def partner(g, beta, iu):
    """(beta2, gamma2) of the ray that measures the line of (beta, column iu) at
    mid-height in the opposite direction."""
    uc, vc = principal_point(g)
    S = np.array([-g.sid * np.sin(beta), -g.sid * np.cos(beta), 0.0])
    d = pixel_positions(g, beta, iu, vc) - S
    d /= np.linalg.norm(d)
    S2 = S - 2.0 * np.dot(S, d) * d                  # second crossing of the source circle
    beta2 = np.arctan2(-S2[0], -S2[1])
    P0, P1 = pixel_positions(g, beta2, 0.0, vc), pixel_positions(g, beta2, 1.0, vc)
    eu = P1 - P0
    nrm = np.cross(eu, [0.0, 0.0, 1.0])
    H = S2 - np.dot(P0 - S2, nrm) / np.dot(-d, nrm) * d   # hits the detector of view beta2
    u2 = np.dot(H - P0, eu) / np.dot(eu, eu)
    return beta2, np.arctan((u2 - uc) * g.du / g.sdd)


def test_redundant_rays_weigh_one_in_total():
    g = short_scan(90, 64, 8, 1.5, 1.5, 8, 8, 8, 1.0, start=0.3)
    delta = 0.5 * (g.angles[-1] - g.angles[0] - np.pi)
    uc, _ = principal_point(g)
    rng = np.random.default_rng(4)
    n_pairs = n_single = 0
    for n in range(400):
        # half of the rays near the scan's ends, where rays are measured twice
        b = rng.uniform(0.0, np.pi + 2 * delta) if n % 2 else rng.choice([1, -1]) * rng.uniform(0, 4 * delta) % (np.pi + 2 * delta)
        iu = rng.uniform(0.0, g.nu - 1)
        gamma = np.arctan((iu - uc) * g.du / g.sdd)
        beta2, gamma2 = partner(g, g.angles[0] + b, iu)
        b2 = (beta2 - g.angles[0]) % (2 * np.pi)
        w = oracle.parker_weight(b, gamma, delta)
        if b2 <= np.pi + 2 * delta:
            n_pairs += 1
            assert w + oracle.parker_weight(b2, gamma2, delta) == pytest.approx(1.0, abs=1e-9)
        else:
            n_single += 1
            assert w == pytest.approx(1.0, abs=1e-12)     # measured once
    assert n_pairs > 100 and n_single > 100


def test_weight_boundaries_and_continuity():
    delta = 0.1
    for gamma in (-0.09, -0.03, 0.0, 0.05, 0.09):
        assert oracle.parker_weight(0.0, gamma, delta) == 0.0
        assert oracle.parker_weight(np.pi + 2 * delta, gamma, delta) == pytest.approx(0.0, abs=1e-15)
        for edge in (2 * delta - 2 * gamma, np.pi - 2 * gamma):
            lo, hi = oracle.parker_weight([edge - 1e-9, edge + 1e-9], gamma, delta)
            assert lo == pytest.approx(hi, abs=1e-6)
        b = np.linspace(-0.1, np.pi + 2 * delta + 0.1, 2001)
        w = oracle.parker_weight(b, gamma, delta)
        assert w.min() >= 0.0 and w.max() <= 1.0
        assert np.all(w[(b < 0) | (b > np.pi + 2 * delta)] == 0.0)


def test_short_scan_table_matches_geometry():
    g = short_scan(40, 32, 8, 1.5, 1.5, 8, 8, 8, 1.0)
    W = oracle.short_scan_weights(g)
    assert W.shape == (g.np, g.nu)
    assert np.all(W[0] == 0.0) and np.allclose(W[-1], 0.0, atol=1e-15)
    assert W.max() == 2.0
    delta = 0.5 * (g.angles[-1] - g.angles[0] - np.pi)
    assert delta > fan_half_angle(g.nu, g.du, g.sdd)


def test_short_scan_sphere_centre_and_full_scan_mid_plane():
    base = scaled_geometry(64, 64, 64).with_(nz=2)
    # the same angular sampling (about 1 view per degree) in both scans
    full = circular(360, base.nu, base.nv, base.du, base.dv, base.nx, base.ny, base.nz, base.dx)
    g = short_scan(190, base.nu, base.nv, base.du, base.dv, base.nx, base.ny, base.nz, base.dx)
    # uniform ball: density at the centre
    vol = oracle.fdk(g, line_integrals(sphere(20.0), g))
    c = g.nx // 2
    assert abs(vol[c - 1:c + 1, c - 1:c + 1, :].mean() - 1.0) <= 5e-3
    # mid-plane of a random phantom: the short scan reconstructs what the full scan does
    ell = random_ellipsoids(6, 15.0, seed=11)
    v_short = oracle.fdk(g, line_integrals(ell, g))
    v_full = oracle.fdk(full, line_integrals(ell, full))
    inner = np.hypot(*np.meshgrid(np.arange(g.nx) - 31.5, np.arange(g.ny) - 31.5, indexing="ij")) < 22
    a, b = v_short[:, :, 0][inner], v_full[:, :, 0][inner]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-2   # 4.4e-3 here, 2.4e-3 at twice the views
