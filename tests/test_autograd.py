"""Autograd through the CUDA operators against FP64 finite differences of the oracle.

The operators are linear, so central differences of the FP64 oracle are exact
up to rounding; the FP32 GPU gradients must agree to 1e-4 relative.  The
unrolled reconstruction is checked the same way through all 20 steps."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.phantom import line_integrals, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    from paper_1909_02724_gb300.binding import Plan
    from paper_1909_02724_gb300.build import build
    build()
    w = workload("grad32")
    g = w.geom
    E = line_integrals(w.phantom(), g).astype(np.float32)
    return g, Plan(g), E


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_backproject_grad_vs_fd(setup):
    from paper_1909_02724_gb300 import autograd as A
    g, plan, E = setup
    rng = np.random.default_rng(0)
    Q = rng.normal(size=(g.np, g.nv, g.nu))
    wv = rng.normal(size=(g.nx, g.ny, g.nz))
    Qt = torch.tensor(Q, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = (A.backproject(Qt, plan) * torch.tensor(wv, dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    grad = Qt.grad.double().cpu().numpy()
    idx = [tuple(int(x) for x in (rng.integers(g.np), rng.integers(g.nv), rng.integers(g.nu))) for _ in range(40)]
    eps = 0.5
    fd = []
    for s, v, u in idx:
        Qp, Qm = Q.copy(), Q.copy()
        Qp[s, v, u] += eps
        Qm[s, v, u] -= eps
        fd.append((np.sum(oracle.backproject(g, Qp) * wv) - np.sum(oracle.backproject(g, Qm) * wv)) / (2 * eps))
    got = np.array([grad[i] for i in idx])
    assert rel(got, np.array(fd)) <= 1e-4


def test_project_grad_vs_fd(setup):
    from paper_1909_02724_gb300 import autograd as A
    g, plan, E = setup
    rng = np.random.default_rng(1)
    x = rng.normal(size=(g.nx, g.ny, g.nz))
    yw = rng.normal(size=(g.np, g.nv, g.nu))
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    (A.project(xt, plan) * torch.tensor(yw, dtype=torch.float32, device="cuda")).sum().backward()
    grad = xt.grad.double().cpu().numpy()
    idx = [tuple(int(t) for t in (rng.integers(g.nx), rng.integers(g.ny), rng.integers(g.nz))) for _ in range(40)]
    fd = []
    for i, j, k in idx:
        xp, xm = x.copy(), x.copy()
        xp[i, j, k] += 0.5
        xm[i, j, k] -= 0.5
        fd.append(np.sum((oracle.project(g, xp) - oracle.project(g, xm)) * yw))
    assert rel(np.array([grad[t] for t in idx]), np.array(fd)) <= 1e-4


def test_fdk_grad_through_filter_vs_fd(setup):
    from paper_1909_02724_gb300 import autograd as A
    g, plan, E = setup
    rng = np.random.default_rng(2)
    wv = rng.normal(size=(g.nx, g.ny, g.nz))
    Et = torch.tensor(E, device="cuda", requires_grad=True)
    (A.fdk(Et, plan) * torch.tensor(wv, dtype=torch.float32, device="cuda")).sum().backward()
    grad = Et.grad.double().cpu().numpy()
    E64 = E.astype(np.float64)
    idx = [tuple(int(t) for t in (rng.integers(g.np), rng.integers(g.nv), rng.integers(g.nu))) for _ in range(12)]
    fd = []
    for s, v, u in idx:
        Ep, Em = E64.copy(), E64.copy()
        Ep[s, v, u] += 0.5
        Em[s, v, u] -= 0.5
        fd.append(np.sum((oracle.fdk(g, Ep) - oracle.fdk(g, Em)) * wv))
    assert rel(np.array([grad[t] for t in idx]), np.array(fd)) <= 1e-4


def _oracle_unrolled_loss(g, y, x0, alphas):
    x = x0.copy()
    for a in alphas:
        x = x - a * oracle.backproject(g, oracle.project(g, x) - y)
    r = oracle.project(g, x) - y
    return float(np.sum(r * r))


def test_unrolled_gd_grad_vs_fd(setup):
    """d loss / d alpha_t through 20 unrolled steps (recomputed in backward)."""
    from paper_1909_02724_gb300 import autograd as A
    g, plan, E = setup
    rng = np.random.default_rng(3)
    x_true = rng.uniform(0.0, 1.0, size=(g.nx, g.ny, g.nz))
    y = oracle.project(g, x_true)
    # step size from the largest eigenvalue of A^T A (power iteration, FP64)
    v = rng.normal(size=x_true.shape)
    for _ in range(12):
        v = oracle.backproject(g, oracle.project(g, v))
        lam = np.linalg.norm(v)
        v /= lam
    alphas = (0.8 / lam) * (1.0 + 0.1 * rng.uniform(size=20))
    x0 = np.zeros_like(x_true)
    at = torch.tensor(alphas, dtype=torch.float32, device="cuda", requires_grad=True)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    xT = A.unrolled_gd(plan, yt, torch.zeros(x0.shape, dtype=torch.float32, device="cuda"), at)
    r = A.project(xT, plan) - yt
    loss = (r * r).sum()
    loss.backward()
    grad = at.grad.double().cpu().numpy()
    l0 = _oracle_unrolled_loss(g, y, x0, alphas)
    assert abs(float(loss.detach()) - l0) <= 1e-4 * l0
    fd = []
    check = [0, 5, 12, 19]
    for t in check:
        h = 1e-4 * alphas[t]
        ap, am = alphas.copy(), alphas.copy()
        ap[t] += h
        am[t] -= h
        fd.append((_oracle_unrolled_loss(g, y, x0, ap) - _oracle_unrolled_loss(g, y, x0, am)) / (2 * h))
    assert rel(grad[check], np.array(fd)) <= 1e-4


def test_unrolled_gd_recompute_memory_and_gradients():
    """grad256 workload (256^3, 360 views of 384^2), 20 unrolled steps.  The linear
    operators save no tensors, so with per-step recomputation each step keeps only
    its input volume: the peak stays within 20 volumes plus a constant working set
    (a few projection stacks and the packed views of one back-projection; no
    projection-sized tensor is kept per step); gradients equal the stored-graph run
    and the data misfit decreases."""
    from paper_1909_02724_gb300 import autograd as A
    from paper_1909_02724_gb300.binding import Plan
    from paper_1909_02724_gb300.phantom import workload_projections_gpu
    w = workload("grad256")
    g = w.geom
    plan = Plan(g)
    y = workload_projections_gpu(w)
    y = y / y.abs().max()
    v = torch.randn((g.nx, g.ny, g.nz), device="cuda")
    for _ in range(8):                                   # power iteration on A^T A
        v = plan.backproject(plan.project(v))
        lam = float(v.norm())
        v /= lam
    vol_b, proj_b = 4 * g.nx * g.ny * g.nz, 4 * g.np * g.nv * g.nu
    peaks, losses, grads = {}, {}, {}
    for recompute in (True, False):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        alphas = torch.full((20,), 0.5 / lam, device="cuda", requires_grad=True)
        x = A.unrolled_gd(plan, y, torch.zeros((g.nx, g.ny, g.nz), device="cuda"), alphas, recompute=recompute)
        r = A.project(x, plan) - y
        loss = (r * r).sum()
        loss.backward()
        t1.record()
        torch.cuda.synchronize()
        # operator applications: 20 steps x (project + back-projection) forward, the same
        # again when recomputed, their two transposes in the backward pass, and the loss
        ops = 20 * (6 if recompute else 4) + 2
        ms = t0.elapsed_time(t1)
        print(f"grad256 unrolled GD, 20 steps, recompute={recompute}: {ms:.1f} ms, "
              f"{ops} operator applications, {ops * g.updates / (ms * 1e-3) / 2 ** 30:.0f} GUPS")
        peaks[recompute] = torch.cuda.max_memory_allocated() - base
        losses[recompute] = float(loss.detach())
        grads[recompute] = alphas.grad.detach().double().cpu().numpy()
        assert np.isfinite(grads[recompute]).all()
    # the working set holds the packed views of one back-projection (ifdk_pack_views)
    pk_b = int(np.prod(plan.packed_shape(torch.float32))) * 4 if plan.has_packed(torch.float32) else 0
    assert peaks[True] <= 20 * vol_b + 4 * (vol_b + proj_b) + pk_b, (peaks, vol_b, proj_b, pk_b)
    assert abs(losses[True] - losses[False]) <= 1e-5 * losses[False]
    assert rel(grads[True], grads[False]) <= 1e-5
    assert losses[True] < 0.5 * float((y * y).sum())
