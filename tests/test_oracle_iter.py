"""Pins of the oracle's iterative solvers (SART and MLEM over ordered view subsets,
the iterative methods the paper names for its back-projector, Sec. 1, Sec. 6).

* one update on a 8^3 volume equals the update written with a dense system
  matrix built column by column from the world-space brute force (ray / plane
  intersection, no projection matrices), for SART (one and two subsets) and
  MLEM;
* consistent data p = A x_true make x_true a fixed point of both;
* SIRT (one subset) never increases the R^-1-weighted residual for
  0 < lam < 2 (Landweber on R^-1/2 A C^-1/2, whose norm is at most 1);
* MLEM keeps x >= 0, preserves the counts (sum_j C_j x_j = sum_i p_i after a
  full-subset update) and never decreases the Poisson log-likelihood.
"""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.geometry import circular
from paper_1909_02724_gb300.phantom import scaled_geometry
from tests.test_oracle_bp import brute_force_bp_of_impulse


def dense_A(g):
    """A[pixel, voxel] = the back-projection of a unit impulse at the pixel, at the voxel."""
    cols = []
    for s in range(g.np):
        for r in range(g.nv):
            for c in range(g.nu):
                cols.append(brute_force_bp_of_impulse(g, s, r, c).ravel())
    return np.array(cols)


def tiny():
    return circular(5, 10, 9, 1.4, 1.3, 8, 8, 8, 1.1, 1.0, 0.9, sid=60.0, sdd=95.0, start=0.3)


def cylinder_volume(g, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 1.0, size=(g.nx, g.ny, g.nz))
    i, j = np.meshgrid(np.arange(g.nx) - (g.nx - 1) / 2, np.arange(g.ny) - (g.ny - 1) / 2, indexing="ij")
    x[(i ** 2 + j ** 2) > (0.45 * g.nx) ** 2] = 0.0
    return x


def test_one_update_equals_the_dense_matrix_update():
    g = tiny()
    A = dense_A(g)
    x_true = cylinder_volume(g, 1)
    p = A @ x_true.ravel()
    x0 = np.full(g.nx * g.ny * g.nz, 0.3)
    ranges_of = {1: [[(0, 5)]], 2: [[(0, 2)], [(2, 3)]]}
    for nsub, subsets in ranges_of.items():
        x = x0.copy()
        R = A @ np.ones(A.shape[1])
        for S in subsets:
            rows = np.zeros(A.shape[0], dtype=bool)
            for b, c in S:
                rows[b * g.nv * g.nu:(b + c) * g.nv * g.nu] = True
            As = A[rows]
            C = As.T @ np.ones(As.shape[0])
            r = np.where(R[rows] > 0, (p[rows] - As @ x) / np.where(R[rows] > 0, R[rows], 1), 0)
            x = x + 0.7 * np.where(C > 0, (As.T @ r) / np.where(C > 0, C, 1), 0)
        got = oracle.sart(g, p.reshape(g.np, g.nv, g.nu), x0.reshape(g.nx, g.ny, g.nz), 1, subsets, lam=0.7)[0]
        np.testing.assert_allclose(got.ravel(), x, rtol=1e-10, atol=1e-12)
    # MLEM, one subset
    C = A.T @ np.ones(A.shape[0])
    Ax = A @ x0
    x1 = np.where(C > 0, x0 * (A.T @ np.where(Ax > 0, p / np.where(Ax > 0, Ax, 1), 0)) / np.where(C > 0, C, 1), x0)
    got = oracle.mlem(g, p.reshape(g.np, g.nv, g.nu), x0.reshape(g.nx, g.ny, g.nz), 1, [[(0, 5)]])[0]
    np.testing.assert_allclose(got.ravel(), x1, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("subsets", [[[(0, 12)]], [[(0, 3), (6, 3)], [(3, 3), (9, 3)]]])
def test_consistent_data_make_the_truth_a_fixed_point(subsets):
    g = scaled_geometry(12, 18, 12, nz=10)
    x_true = cylinder_volume(g, 2)
    p = oracle.project(g, x_true)
    xs = oracle.sart(g, p, x_true, 2, subsets, lam=1.0)
    for x in xs:
        assert np.abs(x - x_true).max() <= 1e-11 * x_true.max()
    xm = oracle.mlem(g, p, x_true, 2, subsets)
    for x in xm:
        assert np.abs(x - x_true).max() <= 1e-11 * x_true.max()


@pytest.mark.parametrize("lam", [1.0, 1.9])
def test_sirt_never_increases_the_weighted_residual(lam):
    g = scaled_geometry(12, 18, 12, nz=10)
    x_true = cylinder_volume(g, 3)
    p = oracle.project(g, x_true)
    R = oracle.row_sums(g)
    w = np.where(R > 0, 1.0 / np.where(R > 0, R, 1.0), 0.0)

    def res(x):
        d = p - oracle.project(g, x)
        return float(np.sum(w * d * d))

    xs = oracle.sart(g, p, np.zeros_like(x_true), 6, [[(0, g.np)]], lam=lam)
    vals = [res(np.zeros_like(x_true))] + [res(x) for x in xs]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(vals, vals[1:])), vals
    assert vals[-1] < 0.3 * vals[0]


def test_sart_with_a_flipped_step_fails_the_residual_pin():
    """The residual pin catches a sign error in the update (planted here, on the CPU)."""
    g = scaled_geometry(12, 18, 12, nz=10)
    x_true = cylinder_volume(g, 3)
    p = oracle.project(g, x_true)
    x_bad = oracle.sart(g, p, np.zeros_like(x_true), 1, [[(0, g.np)]], lam=-1.0)[0]
    R = oracle.row_sums(g)
    w = np.where(R > 0, 1.0 / np.where(R > 0, R, 1.0), 0.0)
    assert np.sum(w * (p - oracle.project(g, x_bad)) ** 2) > np.sum(w * p ** 2)


def test_mlem_counts_positivity_and_likelihood():
    g = scaled_geometry(12, 18, 12, nz=10)
    x_true = cylinder_volume(g, 4)
    rng = np.random.default_rng(5)
    p = oracle.project(g, x_true)
    p = np.maximum(p * (1 + 0.05 * rng.normal(size=p.shape)), 0.0)   # inconsistent, non-negative
    x0 = np.ones_like(x_true)
    xs = oracle.mlem(g, p, x0, 5, [[(0, g.np)]])
    C = oracle.column_sums(g, [(0, g.np)])
    seen = C > 0
    for prev, x in zip([x0] + xs[:-1], xs):
        assert x.min() >= 0.0
        # a full-subset update sends the counts of the rays the previous iterate reaches
        # into the voxels it updates: sum_j C_j x_j = sum of p_i over (A x_prev)_i > 0
        assert abs(float(np.sum(C[seen] * x[seen])) - float(p[oracle.project(g, prev) > 0].sum())) <= \
            1e-10 * float(p.sum())

    def loglik(x):
        ax = oracle.project(g, x)
        m = ax > 0
        return float(np.sum(p[m] * np.log(ax[m]) - ax[m]))

    L = [loglik(x0)] + [loglik(x) for x in xs]
    assert all(b >= a - 1e-10 * abs(a) for a, b in zip(L, L[1:])), L
