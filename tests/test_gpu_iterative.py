"""GPU parity of the iterative solvers on the back-projection / adjoint pair
(SART and MLEM over ordered view subsets; the paper names them as users of
its back-projector, Sec. 1 and Sec. 6): api.IterativeSolver (ifdk_project,
the packed batch back-projection or ifdk_backproject_views,
ifdk_iter_ratio, ifdk_iter_update) against the FP64 oracle iterate by
iterate on grad32 and fdk64, at the FP32 tolerance (rel-L2 <= 1e-5,
max-abs <= 1e-4 of max |x|); the element-wise kernels against their
definitions, element by element, on aligned and unaligned ranges."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300 import binding as B
from paper_1909_02724_gb300.api import IterativeSolver, half_turn_subsets
from paper_1909_02724_gb300.phantom import scaled_geometry, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def cylinder_volume(g, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 1.0, size=(g.nx, g.ny, g.nz))
    i, j = np.meshgrid(np.arange(g.nx) - (g.nx - 1) / 2, np.arange(g.ny) - (g.ny - 1) / 2, indexing="ij")
    x[(i ** 2 + j ** 2) > (0.45 * g.nx) ** 2] = 0.0
    return x


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


CASES = [("grad32", "sart", 1, False), ("grad32", "sart", 4, True), ("grad32", "mlem", 3, False),
         ("fdk64", "sart", 4, False), ("fdk64", "mlem", 1, False), ("fdk64", "mlem", 4, False),
         ("odd_views", "sart", 3, False), ("odd_views", "mlem", 2, False)]


@pytest.mark.parametrize("name,method,subsets,nonneg", CASES)
def test_iterates_match_the_oracle(name, method, subsets, nonneg):
    g = scaled_geometry(24, 36, 15, nz=20) if name == "odd_views" else workload(name).geom
    x_true = cylinder_volume(g, 11)
    p = oracle.project(g, x_true)
    if nonneg:   # inconsistent data: the clip at 0 takes part
        p = p * (1 + 0.1 * np.random.default_rng(3).normal(size=p.shape))
    x0 = np.zeros_like(x_true) if method == "sart" else np.ones_like(x_true)
    sets = half_turn_subsets(g.np, subsets)
    iters = 3
    if method == "sart":
        ref = oracle.sart(g, p, x0, iters, sets, lam=0.9, nonneg=nonneg)
    else:
        ref = oracle.mlem(g, p, x0, iters, sets)
    plan = B.Plan(g)
    solver = IterativeSolver(plan, method, subsets, lam=0.9, nonneg=nonneg)
    x = torch.from_numpy(x0.astype(np.float32)).cuda()
    got = solver.run(torch.from_numpy(p.astype(np.float32)).cuda(), x, iters, keep=True)
    torch.cuda.synchronize()
    assert plan.device_status() == B.IFDK_OK
    for it, (a, b) in enumerate(zip(got, ref)):
        a = a.double().cpu().numpy()
        err, mx = rel_l2(a, b), float(np.abs(a - b).max() / np.abs(b).max())
        assert err <= 1e-5 and mx <= 1e-4, (it, err, mx)
    # the buffers the kernels keep zeroed between uses
    assert float(solver.Ax.abs().max()) == 0.0 and float(solver.U.abs().max()) == 0.0


@pytest.mark.parametrize("method", [B.IFDK_SART, B.IFDK_MLEM])
@pytest.mark.parametrize("offset", [0, 1])
def test_elementwise_steps_are_their_definitions(method, offset):
    g = scaled_geometry(20, 12, 6, nz=9)                     # 6 x 12 x 12 views, 20 x 20 x 9 voxels
    plan = B.Plan(g)
    rng = np.random.default_rng(4)
    n = g.np * g.nv * g.nu
    Pm = rng.uniform(0, 2, n + 1).astype(np.float32)
    Ax = rng.uniform(0, 2, n + 1).astype(np.float32)
    R = rng.uniform(0, 2, n + 1).astype(np.float32)
    Ax[::7] = 0.0
    R[::5] = 0.0
    d = {k: torch.from_numpy(v).cuda() for k, v in (("Pm", Pm), ("Ax", Ax), ("R", R))}
    out = torch.full((n + 1,), float("nan"), device="cuda")
    sl = slice(offset, offset + n)   # offset 1: 4-byte aligned only (scalar path)
    views = g.np
    B.ifdk_iter_ratio(plan.handle, method, d["Pm"][sl], d["Ax"][sl], d["R"][sl], out[sl], views)
    torch.cuda.synchronize()
    p, a, r = Pm[sl], Ax[sl], R[sl]
    with np.errstate(divide="ignore", invalid="ignore"):
        want = np.where(r > 0, (p - a) / r, 0) if method == B.IFDK_SART else np.where(a > 0, p / a, 0)
    np.testing.assert_array_equal(out[sl].cpu().numpy(), want.astype(np.float32))
    assert float(d["Ax"][sl].abs().max()) == 0.0
    # the volume update
    nv = g.nx * g.ny * g.nz
    x = rng.uniform(0, 1, nv).astype(np.float32)
    U = rng.normal(size=nv).astype(np.float32)
    C = rng.uniform(0, 2, nv).astype(np.float32)
    C[::3] = 0.0
    xt, Ut, Ct = (torch.from_numpy(v).cuda() for v in (x, U, C))
    B.ifdk_iter_update(plan.handle, method, xt, Ut, Ct, 0.75, True)
    torch.cuda.synchronize()
    with np.errstate(divide="ignore", invalid="ignore"):
        if method == B.IFDK_SART:
            want = np.where(C > 0, np.maximum(x + np.float32(0.75) * (U / C), 0), x)
        else:
            want = np.where(C > 0, x * U / C, x)
    # SART's device update is one FMA (numpy rounds the product and the sum apart)
    np.testing.assert_allclose(xt.cpu().numpy(), want, rtol=2e-7, atol=1e-6 if method == B.IFDK_SART else 0)
    assert float(Ut.abs().max()) == 0.0


def test_bad_requests_are_refused_before_any_launch():
    g = scaled_geometry(16, 16, 4)
    plan = B.Plan(g)
    z = torch.zeros(g.np * g.nv * g.nu, device="cuda")
    for args in ((7, z, z, z, z, 4), (B.IFDK_SART, z, z, None, z, 4), (B.IFDK_MLEM, z, z, None, z, 5)):
        with pytest.raises(B.IfdkError) as e:
            B.ifdk_iter_ratio(plan.handle, *args)
        assert e.value.code == B.IFDK_ERR_INVALID
    v = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
    with pytest.raises(B.IfdkError) as e:
        B.ifdk_iter_update(plan.handle, B.IFDK_SART, v, v, None, 1.0, False)
    assert e.value.code == B.IFDK_ERR_INVALID
