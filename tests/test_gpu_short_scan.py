"""Short scans through the CUDA filter (Parker weights with F_cos), against the oracle.

Filter output in every split mode, the FDK of a short scan through both
back-projectors, the adjoint filter's inner-product identity with the weights,
and the plan's refusal of scans the weights do not cover."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.geometry import circular, short_scan
from paper_1909_02724_gb300.phantom import line_integrals, random_ellipsoids, safe_radius

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


GEOMS = {
    "short64": short_scan(100, 64, 48, 1.5, 1.5, 32, 32, 24, 1.0),
    "short_offsets": short_scan(70, 80, 40, 1.2, 1.2, 30, 26, 20, 1.0, off_u=0.9, off_v=-0.6, start=0.7),
}


def phantom_E(g, seed=3):
    return line_integrals(random_ellipsoids(8, 0.9 * safe_radius(g), seed), g).astype(np.float32)


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("split,dtype,tol", [(0, torch.float32, 1e-5), (3, torch.float32, 1e-5),
                                             (2, torch.float16, 2e-3), (2, torch.bfloat16, 4e-3)])
def test_short_scan_filter_matches_oracle(name, split, dtype, tol):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS[name]
    E = phantom_E(g)
    ref = oracle.filter_views(g, E.astype(np.float64))
    plan = Plan(g)
    Q = plan.filter(torch.from_numpy(E).cuda(), dtype=dtype, split_terms=split).float().cpu().double().numpy()
    assert rel_l2(Q, ref) <= tol
    assert np.all(Q[0] == 0.0)                 # the first view has weight 0


@pytest.mark.parametrize("name", list(GEOMS))
def test_short_scan_fdk_matches_oracle(name):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS[name]
    E = phantom_E(g)
    ref = oracle.fdk(g, E.astype(np.float64))
    plan = Plan(g)
    Q = plan.filter(torch.from_numpy(E).cuda())
    vol = plan.backproject(Q).cpu().double().numpy()
    assert rel_l2(vol, ref) <= 1e-5
    assert np.abs(vol - ref).max() <= 1e-4 * np.abs(ref).max()
    if plan.has_packed(torch.float32):
        vp = plan.backproject_packed(plan.pack(Q)).cpu().double().numpy()
        assert rel_l2(vp, ref) <= 1e-5


def test_short_scan_filter_adjoint_identity():
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS["short_offsets"]
    plan = Plan(g)
    rng = np.random.default_rng(2)
    x = torch.from_numpy(rng.standard_normal((g.np, g.nv, g.nu)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.standard_normal((g.np, g.nv, g.nu)).astype(np.float32)).cuda()
    Fx = plan.filter(x, split_terms=0)
    Fty = plan.filter_adjoint(y)
    lhs, rhs = float((Fx.double() * y.double()).sum()), float((x.double() * Fty.double()).sum())
    scale = float(Fx.double().norm() * y.double().norm())
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_short_scan_switch_and_refusals():
    from paper_1909_02724_gb300.binding import IFDK_ERR_GEOMETRY, IfdkError, Plan, ifdk_set_short_scan
    g = GEOMS["short64"]
    plan = Plan(g)
    E = torch.from_numpy(phantom_E(g)).cuda()
    ifdk_set_short_scan(plan.handle, False)               # back to the full-scan weighting
    Q_full = plan.filter(E).cpu().double().numpy()
    ref_full = oracle.filter_views(g.with_(short_scan=False), E.cpu().double().numpy())
    assert rel_l2(Q_full, ref_full) <= 1e-5
    bad = {
        "half turn only": circular(60, 64, 48, 1.5, 1.5, 16, 16, 8, 1.0, arc=np.pi),
        "decreasing": short_scan(40, 64, 48, 1.5, 1.5, 16, 16, 8, 1.0).with_(angles=-np.linspace(0, 3.3, 40)),
        "two views": circular(2, 64, 48, 1.5, 1.5, 16, 16, 8, 1.0, arc=np.pi),
    }
    for name, gb in bad.items():
        p = Plan(gb.with_(short_scan=False))
        with pytest.raises(IfdkError) as e:
            ifdk_set_short_scan(p.handle, True)
        assert e.value.code == IFDK_ERR_GEOMETRY, name


@pytest.mark.parametrize("dtype,split", [(torch.float32, 3), (torch.float16, 2)])
def test_short_scan_noalloc_filter_equals_workspace_filter(dtype, split):
    from paper_1909_02724_gb300.binding import Plan, dtype_code, ifdk_filter_noalloc
    g = GEOMS["short64"]
    plan = Plan(g)
    E = torch.from_numpy(phantom_E(g)).cuda()
    want = plan.filter(E, dtype=dtype, split_terms=split)
    got = torch.empty_like(want)
    ifdk_filter_noalloc(plan.handle, E, got, dtype_code(dtype), split)
    torch.cuda.synchronize()
    # the same kernels on the same 128-row tiles, in launches of at most 16 MiB of operands
    assert float((got.float() - want.float()).abs().max()) <= 1e-6 * float(want.float().abs().max())
    assert torch.equal(got[0], torch.zeros_like(got[0]))       # the first view has weight 0
