"""GPU parity of quarter-turn view quads (the packed kernel's NV = 4 form, FP16
storage; the rotational symmetry after Zhao et al. that Sec. 3.2 cites):

* the whole-scan packed back-projection with quads matches the FP64 oracle
  (FP16 storage: rel-L2 <= 2e-3) and the half-turn pair result up to the
  FP32 summation order;
* ifdk_backproject_packed_quads over batches (ragged last batch) sums to the
  whole back-projection, in every pairing mode and storage type (quads for
  FP16, pairs or single views otherwise);
* a pair range over the whole scan takes quads too;
* geometries without a quarter turn (non-square grid) fall back to pairs;
* FDK in batches of quads (api.BatchFdk, group 4) against the oracle FDK;
* the timeout hook (no device fault) reports and recovers with quads.
"""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300 import binding as B
from paper_1909_02724_gb300.phantom import line_integrals, scaled_geometry, workload
from tests.random_geometries import random_square_geometries

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


def rel_np(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


GEOMS = {"fdk64": workload("fdk64").geom, "ragged": scaled_geometry(48, 64, 40, nz=42),
         "odd_nz": scaled_geometry(32, 48, 16, nz=33)}
TDT = {"float32": torch.float32, "float16": torch.float16, "bfloat16": torch.bfloat16}


def random_views(g, tdt, seed=5):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(g.np, g.nv, g.nu)).astype(np.float32)
    return torch.from_numpy(Q).cuda().to(tdt)


@pytest.mark.parametrize("name", list(GEOMS))
def test_quads_match_the_oracle_and_the_pairs(name):
    g = GEOMS[name]
    plan = B.Plan(g)
    Q = random_views(g, torch.float16)
    Qp = plan.pack(Q)
    plan.set_view_pairing(2)
    assert plan.packed_info(torch.float16)["path"] == 4
    quads = plan.backproject_packed(Qp)
    plan.set_view_pairing(1)
    assert plan.packed_info(torch.float16)["path"] == 2
    pairs = plan.backproject_packed(Qp)
    torch.cuda.synchronize()
    assert plan.device_status() == B.IFDK_OK
    # the same sum in another order (and the quad's coordinates come from the own view's terms)
    assert rel(quads, pairs) <= 5e-5
    ref = oracle.backproject(g, Q.float().double().cpu().numpy())
    assert rel_np(quads.cpu().numpy(), ref) <= 2e-3


@pytest.mark.parametrize("name", [n for n, _ in random_square_geometries()])
def test_quads_on_random_square_geometries(name):
    g = dict(random_square_geometries())[name]
    plan = B.Plan(g)
    Q = random_views(g, torch.float16, seed=len(name))
    Qp = plan.pack(Q)
    plan.set_view_pairing(2)
    assert plan.packed_info(torch.float16)["path"] == 4
    quads = plan.backproject_packed(Qp)
    plan.set_view_pairing(1)
    pairs = plan.backproject_packed(Qp)
    torch.cuda.synchronize()
    assert plan.device_status() == B.IFDK_OK
    assert rel(quads, pairs) <= 5e-5
    ref = oracle.backproject(g, Q.float().double().cpu().numpy())
    assert rel_np(quads.cpu().numpy(), ref) <= 2e-3


@pytest.mark.parametrize("dtype", ["float16", "float32", "bfloat16"])
@pytest.mark.parametrize("mode", [2, 1, 0])
def test_quad_batches_sum_to_the_whole(dtype, mode):
    g = GEOMS["ragged"]                        # 40 views: 10 quads, batches of 4, 4, 2
    plan = B.Plan(g)
    tdt = TDT[dtype]
    Q = random_views(g, tdt)
    Qp = plan.pack(Q)
    plan.set_view_pairing(1)
    whole = plan.backproject_packed(Qp)
    plan.set_view_pairing(mode)
    q4 = g.np // 4
    vol = torch.zeros_like(whole)
    for b in range(0, q4, 4):
        n = min(4, q4 - b)
        Qpq = torch.cat([Qp[b + k * q4:b + k * q4 + n] for k in range(4)]).contiguous()
        plan.backproject_packed_quads(Qpq, b, n, vol)
    torch.cuda.synchronize()
    assert plan.device_status() == B.IFDK_OK
    assert rel(vol, whole) <= (1e-5 if dtype == "float32" else 5e-5)
    ref = oracle.backproject(g, Q.float().double().cpu().numpy())
    tol = 1e-5 if dtype == "float32" else 2e-3
    assert rel_np(vol.cpu().numpy(), ref) <= tol


def test_pair_range_over_the_whole_scan_takes_quads():
    g = GEOMS["odd_nz"]
    plan = B.Plan(g)
    Q = random_views(g, torch.float16)
    Qp = plan.pack(Q)
    plan.set_view_pairing(2)
    whole = plan.backproject_packed(Qp)
    part = plan.backproject_packed_pairs(Qp, 3, 6)
    torch.cuda.synchronize()
    nz_out = part.shape[2]
    # the pair-range launch sums each block's views in another order (FP16 products, FP32 sums)
    assert rel(part[:, :, :6], whole[:, :, 3:9]) <= 5e-5
    assert rel(part[:, :, nz_out - 6:], whole[:, :, g.nz - 9:g.nz - 3]) <= 5e-5


def test_non_square_grid_falls_back_to_pairs():
    g = scaled_geometry(48, 64, 40, nz=42).with_(ny=40)
    plan = B.Plan(g)
    plan.set_view_pairing(2)
    assert plan.packed_info(torch.float16)["path"] == 2
    Q = random_views(g, torch.float16)
    vol = plan.backproject_packed(plan.pack(Q))
    ref = oracle.backproject(g, Q.float().double().cpu().numpy())
    assert rel_np(vol.cpu().numpy(), ref) <= 2e-3
    with pytest.raises(B.IfdkError) as e:      # 40 views: np/4 = 10, the batch runs past it
        B.ifdk_backproject_packed_quads(plan.handle, torch.zeros(1, device="cuda"), B.IFDK_F16, 8, 3, vol)
    assert e.value.code == B.IFDK_ERR_INVALID


def test_batch_fdk_in_quads_matches_the_oracle():
    from paper_1909_02724_gb300.api import BatchFdk
    w = workload("fdk64")
    g = w.geom
    E = line_integrals(w.phantom(), g).astype(np.float32)
    ref = oracle.fdk(g, E.astype(np.float64))
    plan = B.Plan(g)
    plan.set_view_pairing(2)
    Ed = torch.from_numpy(E).cuda()
    for batches in (4, 3):                     # 16 quads: 4 each, or 6, 6, 4
        bf = BatchFdk(plan, batches, dtype=torch.float16, group=4)
        vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
        bf.reconstruct(Ed, vol)
        torch.cuda.synchronize()
        assert plan.device_status() == B.IFDK_OK
        assert rel_np(vol.cpu().numpy(), ref) <= 2e-3


@pytest.mark.parametrize("group", [1, 6])
def test_quad_timeout_path_reports_and_recovers(group):
    g = GEOMS["fdk64"]
    plan = B.Plan(g)
    plan.set_view_pairing(2)
    plan.set_view_split(1)
    Q = random_views(g, torch.float16)
    Qp = plan.pack(Q)
    B.ifdk_set_test_abort(plan.handle, group)
    plan.backproject_packed(Qp)
    torch.cuda.synchronize()
    assert plan.device_status() == B.IFDK_ERR_TIMEOUT
    B.ifdk_set_test_abort(plan.handle, -1)
    vol = plan.backproject_packed(Qp)
    assert plan.device_status() == B.IFDK_OK
    ref = oracle.backproject(g, Q.float().double().cpu().numpy())
    assert rel_np(vol.cpu().numpy(), ref) <= 2e-3
