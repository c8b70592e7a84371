"""GPU parity over seeded random scanner geometries (tests/random_geometries.py).

Random detector and volume sizes (odd and even), pitches, source distances,
offsets, start angles and view counts: the tensor-core filter, both
back-projectors (packed with and without view pairing where the plan has
them), FP16 storage (pairs and, where the scan allows, quads), BF16 storage (against
the oracle on the stored BF16 values) and the adjoint, each against the FP64
oracle.  The same
geometries pass the host emulation of the packed windows on the CPU."""
import numpy as np
import pytest

import oracle
from tests.random_geometries import random_geometries

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GEOMS = dict(random_geometries())


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("name", list(GEOMS))
def test_random_geometry_parity(name):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS[name]
    rng = np.random.default_rng(sum(map(ord, name)))   # stable across processes
    E = rng.uniform(0.0, 2.0, (g.np, g.nv, g.nu)).astype(np.float32)
    Q_ref = oracle.filter_views(g, E.astype(np.float64))
    ref = oracle.backproject(g, Q_ref)
    plan = Plan(g)
    Ed = torch.from_numpy(E).cuda()
    assert rel_l2(plan.filter(Ed).cpu().double().numpy(), Q_ref) <= 1e-5
    Qd = torch.from_numpy(Q_ref.astype(np.float32)).cuda()
    vol = plan.backproject(Qd).cpu().double().numpy()
    assert rel_l2(vol, ref) <= 1e-5 and np.abs(vol - ref).max() <= 1e-4 * np.abs(ref).max()
    if plan.has_packed(torch.float32):
        Qp = plan.pack(Qd)
        for pairing in (True, False):
            plan.set_view_pairing(pairing)
            vp = plan.backproject_packed(Qp).cpu().double().numpy()
            assert rel_l2(vp, ref) <= 1e-5, pairing
            assert np.abs(vp - ref).max() <= 1e-4 * np.abs(ref).max()
        Q16 = plan.filter(Ed, dtype=torch.float16)
        Qp16 = plan.pack(Q16)
        for mode in (1, 2):          # half-turn pairs; quarter-turn quads where the geometry has them
            plan.set_view_pairing(mode)
            v16 = plan.backproject_packed(Qp16).cpu().double().numpy()
            assert rel_l2(v16, ref) <= 2e-3, mode
        # BF16 packed views (raw taps, BF16 u weights) against the oracle on the stored values
        Qb = plan.filter(Ed, dtype=torch.bfloat16)
        ref_b = oracle.backproject(g, Qb.float().double().cpu().numpy())
        Qpb = plan.pack(Qb)
        for pairing in (True, False):
            plan.set_view_pairing(pairing)
            vb = plan.backproject_packed(Qpb).cpu().double().numpy()
            assert rel_l2(vb, ref_b) <= 2e-3, pairing
    x = rng.standard_normal((g.nx, g.ny, g.nz)).astype(np.float32)
    P = plan.project(torch.from_numpy(x).cuda()).cpu().double().numpy()
    assert rel_l2(P, oracle.project(g, x.astype(np.float64))) <= 1e-5
    assert plan.device_status() == 0
