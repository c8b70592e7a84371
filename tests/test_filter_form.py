"""The summed-by-parts form of the ramp filter that both CUDA filters use.

Algorithm 1's row convolution Q(u) = sum_k h(u - k) w(k) is evaluated on the
GPU as sum_{k=0}^{nu} g(u - k) d(k), with d(k) = w(k) - w(k-1) (w = 0
outside the row) and g(m) = sum_{j=-(nu-1)}^{m} h(j).  These CPU tests check
that the two forms agree exactly (in FP64, with non-zero row edges), and that
the second is the well-conditioned one: with both operands split into BF16
terms as the tensor-core kernel splits them, the difference form keeps
FP32-level accuracy where the direct form loses it."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.geometry import circular


def running_tap_sum(nu):
    h = oracle.ramlak(nu)                                # h(m) at index m + nu - 1
    return np.concatenate([[0.0], np.cumsum(h)])         # g(m) at index m + nu, m in [-nu, nu - 1]


def difference_form(w):
    nu = w.shape[1]
    g = running_tap_sum(nu)
    wp = np.pad(w, ((0, 0), (1, 1)))
    d = wp[:, 1:] - wp[:, :-1]                           # d(k), k = 0..nu
    G = g[np.arange(nu)[None, :] - np.arange(nu + 1)[:, None] + nu]
    return d, G


@pytest.mark.parametrize("nu", [1, 2, 7, 64, 200])
def test_summation_by_parts_equals_direct_convolution(nu):
    g = circular(2, nu, 3, 0.5, 0.5, 4, 4, 4, 1.0)
    w = np.random.default_rng(nu).normal(size=(6, nu)) + 3.0   # large DC, non-zero edges
    ref = oracle.filter_rows(g, w / oracle.cosine_weight(g)[np.arange(6) % g.nv], np.arange(6) % g.nv, method="direct")
    d, G = difference_form(w)
    assert np.max(np.abs(d @ G - ref)) <= 1e-12 * np.max(np.abs(w))


def test_running_tap_sum_shape():
    """What makes the by-parts form well conditioned: g is bounded by ~1/8
    (g(0) = 1/8 + O(1/nu), g(-1) = -1/8 + O(1/nu)), positive right of the
    centre, negative left of it, decays monotonically away from it, and its
    l1 norm grows only like log(nu) / pi^2."""
    for nu in (64, 512, 2048):
        g = running_tap_sum(nu)[1:]                      # m = -(nu-1) .. nu-1, index m + nu - 1
        c = nu - 1
        assert abs(g[c] - 0.125) < 1.0 / nu and abs(g[c - 1] + 0.125) < 1.0 / nu
        assert np.max(np.abs(g)) <= 0.125 + 1.0 / nu
        assert np.all(g[c:] > 0) and np.all(g[:c] < 0)
        right, left = np.abs(g[c:]), np.abs(g[:c][::-1])
        assert np.all(np.diff(right) <= 1e-15) and np.all(np.diff(left) <= 1e-15)
        assert np.sum(np.abs(g)) <= np.log(nu) / np.pi**2 + 0.5


def bf16(x):
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def split(x, n):
    out, r = [], x.copy()
    for _ in range(n):
        t = bf16(r)
        out.append(t)
        r = r - t
    return out


def chord_rows(nu, rows, seed):
    """Rows shaped like ellipsoid projections: sums of sqrt chord profiles."""
    rng = np.random.default_rng(seed)
    x = np.arange(nu)
    w = np.zeros((rows, nu))
    for r in range(rows):
        for _ in range(20):
            c, rad, a = rng.uniform(0.3, 0.7) * nu, rng.uniform(0.02, 0.2) * nu, rng.uniform(0.1, 1.0)
            w[r] += a * np.sqrt(np.clip(rad**2 - (x - c) ** 2, 0.0, None))
    return w


def test_difference_form_is_well_conditioned():
    nu = 1024
    w = chord_rows(nu, 8, 3)
    h = oracle.ramlak(nu)
    T = h[np.arange(nu)[None, :] - np.arange(nu)[:, None] + nu - 1]
    q = w @ T
    rel = lambda a: float(np.linalg.norm(a - q) / np.linalg.norm(q))
    pairs = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]
    # direct form, data rounded to FP32 then split as the kernel would
    w32 = w.astype(np.float32).astype(np.float64)
    direct = sum(a @ b for a, b in ((split(w32, 3)[i], split(T, 3)[j]) for i, j in pairs))
    d, G = difference_form(w)
    d32 = d.astype(np.float32).astype(np.float64)
    by_parts = sum(a @ b for a, b in ((split(d32, 3)[i], split(G, 3)[j]) for i, j in pairs))
    assert np.linalg.norm(w) / np.linalg.norm(q) > 100          # the cancellation is real
    assert rel(by_parts) < 1e-6
    assert rel(direct) > 10 * rel(by_parts)
