"""Degenerate volumes and scans through the whole CUDA path, against the oracle.

One or two slices, an odd slice count, a single view, a single half-turn pair,
a single voxel column: filter (tensor cores), back-projection (standard and
packed kernels, with and without view pairing), adjoint and output slices,
each compared with the FP64 oracle at the FP32 tolerances."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.geometry import circular

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


GEOMS = {
    "one_slice": circular(8, 64, 48, 1.5, 1.5, 24, 24, 1, 1.0),
    "two_slices": circular(8, 64, 48, 1.5, 1.5, 24, 24, 2, 1.0),
    "three_slices": circular(8, 64, 48, 1.5, 1.5, 24, 24, 3, 1.0),
    "one_view": circular(1, 64, 48, 1.5, 1.5, 24, 24, 16, 1.0, start=0.4),
    "one_pair": circular(2, 64, 48, 1.5, 1.5, 24, 24, 16, 1.0, start=0.4),
    "one_column": circular(6, 64, 48, 1.5, 1.5, 1, 1, 16, 1.0),
    "one_row_of_columns": circular(6, 64, 48, 1.5, 1.5, 24, 1, 16, 1.0),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_degenerate_fdk_and_adjoint(name):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS[name]
    rng = np.random.default_rng(17)
    E = rng.uniform(0.0, 2.0, (g.np, g.nv, g.nu)).astype(np.float32)
    Q_ref = oracle.filter_views(g, E.astype(np.float64))
    ref = oracle.backproject(g, Q_ref)
    plan = Plan(g)
    Ed = torch.from_numpy(E).cuda()
    Q = plan.filter(Ed)
    assert rel_l2(Q.cpu().double().numpy(), Q_ref) <= 1e-5
    Qd = torch.from_numpy(Q_ref.astype(np.float32)).cuda()
    vol = plan.backproject(Qd).cpu().double().numpy()
    assert rel_l2(vol, ref) <= 1e-5
    assert np.abs(vol - ref).max() <= 1e-4 * np.abs(ref).max()
    if plan.has_packed(torch.float32):
        Qp = plan.pack(Qd)
        for pairing in (True, False):
            plan.set_view_pairing(pairing)
            vp = plan.backproject_packed(Qp).cpu().double().numpy()
            assert rel_l2(vp, ref) <= 1e-5, pairing
            assert np.abs(vp - ref).max() <= 1e-4 * np.abs(ref).max()
    # adjoint of the same operator
    x = rng.standard_normal((g.nx, g.ny, g.nz))
    P = plan.project(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().double().numpy()
    P_ref = oracle.project(g, x.astype(np.float32).astype(np.float64))
    assert rel_l2(P, P_ref) <= 1e-5
    # output slices of the back-projected volume, exact
    vd = plan.backproject(Qd)
    s = plan.slices(vd).cpu().numpy()
    assert np.array_equal(s, oracle.volume_slices(vd.cpu().numpy()))
    assert plan.device_status() == 0
