"""GPU parity of the batch path the benchmark times (the paper's pipeline, Sec. 4,
filters and back-projects views in batches):

* ifdk_filter_views on a view range gives the rows ifdk_filter gives those
  views (tensor-core and SIMT kernels, short scans whose per-view weights
  must follow the range), and matches the FP64 oracle;
* ifdk_backproject_packed_batch over batches of half-turn view pairs sums
  to the whole packed back-projection and matches the oracle, with pairing
  on and off, in every storage type, with ragged last batches;
* FDK in batches (api.BatchFdk, and streamed from pinned host memory by
  api.batch_host_pipeline) against the oracle FDK;
* requests outside the batch rules are refused before any launch;
* the arithmetic rate probe (ifdk_arith_rate) reports plausible rates.
"""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300 import binding as B
from paper_1909_02724_gb300.geometry import circular, short_scan
from paper_1909_02724_gb300.phantom import line_integrals, random_ellipsoids, safe_radius, scaled_geometry, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def phantom_E(g, n_ell=8, seed=3):
    ell = random_ellipsoids(n_ell, 0.9 * safe_radius(g), seed)
    return line_integrals(ell, g).astype(np.float32)


TDT = {"float32": torch.float32, "float16": torch.float16, "bfloat16": torch.bfloat16}


@pytest.mark.parametrize("terms", [0, 1, 2, 3])
def test_filter_views_equals_the_whole_filter(terms):
    g = scaled_geometry(40, 72, 30, n_det_v=50)
    plan = B.Plan(g)
    E = torch.from_numpy(phantom_E(g)).cuda()
    whole = plan.filter(E, split_terms=terms)
    for b, n in ((0, 30), (7, 11), (29, 1), (3, 0)):
        Qv = torch.full((n, g.nv, g.nu), float("nan"), device="cuda")
        plan.filter_views(E[b:b + n].contiguous(), Qv, view_begin=b, split_terms=terms)
        torch.cuda.synchronize()
        if n:
            # the same arithmetic per row: equal up to the last bits
            assert float((Qv - whole[b:b + n]).abs().max()) <= 1e-6 * float(whole.abs().max()), (b, n)
    ref = oracle.filter_views(g, E.double().cpu().numpy())
    Qv = plan.filter_views(E[5:25].contiguous(), view_begin=5, split_terms=terms)
    err = rel_l2(Qv.cpu().numpy(), ref[5:25])
    # one BF16 term is the split the precision findings expect to miss 2e-3 (kept for the record)
    assert err <= {0: 1e-5, 1: 1e-2, 2: 2e-3, 3: 1e-5}[terms], err


def test_filter_views_short_scan_weights_follow_the_range():
    g = short_scan(40, 64, 24, 1.5, 1.5, 16, 16, 16, 1.0)
    plan = B.Plan(g)
    E = torch.from_numpy(phantom_E(g)).cuda()
    for terms in (0, 3):
        whole = plan.filter(E, split_terms=terms)
        Qv = plan.filter_views(E[12:31].contiguous(), view_begin=12, split_terms=terms)
        torch.cuda.synchronize()
        assert float((Qv - whole[12:31]).abs().max()) <= 1e-6 * float(whole.abs().max())


def _packed_batches(plan, Qp_all, n):
    """Packed views of the batches of n pairs: views [b, b + n) then [b + h, b + h + n)."""
    h = plan.geom.np // 2
    for b in range(0, h, n):
        m = min(n, h - b)
        yield b, m, torch.cat([Qp_all[b:b + m], Qp_all[h + b:h + b + m]]).contiguous()


@pytest.mark.parametrize("dtype", ["float32", "float16", "bfloat16"])
@pytest.mark.parametrize("pairing", [True, False])
def test_packed_batches_sum_to_the_whole_and_match_the_oracle(dtype, pairing):
    g = scaled_geometry(48, 64, 40, nz=42)
    plan = B.Plan(g)
    plan.set_view_pairing(pairing)
    tdt = TDT[dtype]
    rng = np.random.default_rng(5)
    Q = torch.from_numpy(rng.normal(size=(g.np, g.nv, g.nu)).astype(np.float32)).cuda().to(tdt)
    Qp = plan.pack(Q)
    whole = plan.backproject_packed(Qp)
    vol = torch.zeros_like(whole)
    for b, m, Qpb in _packed_batches(plan, Qp, 7):          # 20 pairs: batches of 7, 7, 6
        plan.backproject_packed_batch(Qpb, b, m, vol)
    torch.cuda.synchronize()
    assert plan.device_status() == B.IFDK_OK
    assert float((vol - whole).norm() / whole.norm()) <= 1e-6
    ref = oracle.backproject(g, Q.float().double().cpu().numpy())
    v = vol.cpu().numpy()
    if dtype == "float32":
        assert rel_l2(v, ref) <= 1e-5 and max_rel(v, ref) <= 1e-4
    else:   # 16-bit packed elements round the tap and its column difference once each
        assert rel_l2(v, ref) <= 2e-3


def test_batch_requests_outside_the_rules_are_refused():
    g = scaled_geometry(32, 32, 12)
    plan = B.Plan(g)
    Qp = torch.zeros((2 * 4,) + plan.packed_shape(torch.float32)[1:], device="cuda")
    vol = torch.full((g.nx, g.ny, g.nz), 3.0, device="cuda")
    for b, n in ((3, 4), (-1, 2), (0, 7)):                 # past np/2, negative, past np/2
        with pytest.raises(B.IfdkError) as e:
            B.ifdk_backproject_packed_batch(plan.handle, Qp, B.IFDK_F32, b, n, vol)
        assert e.value.code == B.IFDK_ERR_INVALID
    odd = B.Plan(scaled_geometry(32, 32, 13))
    with pytest.raises(B.IfdkError) as e:
        B.ifdk_backproject_packed_batch(odd.handle, Qp, B.IFDK_F32, 0, 2, vol)
    assert e.value.code == B.IFDK_ERR_INVALID
    E = torch.zeros((4, g.nv, g.nu), device="cuda")
    with pytest.raises(B.IfdkError) as e:
        B.ifdk_filter_views(plan.handle, E, E, B.IFDK_F32, 0, 10, 4)
    assert e.value.code == B.IFDK_ERR_INVALID
    torch.cuda.synchronize()
    assert float(vol.min()) == 3.0


@pytest.mark.parametrize("dtype,tol", [("float32", 1e-5), ("float16", 2e-3), ("bfloat16", 2e-3)])
def test_batch_fdk_matches_the_oracle(dtype, tol):
    from paper_1909_02724_gb300.api import BatchFdk
    w = workload("fdk64")
    g = w.geom
    E = line_integrals(w.phantom(), g).astype(np.float32)
    ref = oracle.fdk(g, E.astype(np.float64))
    plan = B.Plan(g)
    Ed = torch.from_numpy(E).cuda()
    for batches in (4, 3):                                  # 32 pairs: 8 each, or 11, 11, 10
        bf = BatchFdk(plan, batches, dtype=TDT[dtype])
        vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
        bf.reconstruct(Ed, vol)
        torch.cuda.synchronize()
        assert plan.device_status() == B.IFDK_OK
        v = vol.cpu().numpy()
        assert rel_l2(v, ref) <= tol, (batches, rel_l2(v, ref))
        if dtype == "float32":
            assert max_rel(v, ref) <= 1e-4


def test_batch_host_pipeline_matches_the_device_batches():
    from paper_1909_02724_gb300.api import BatchFdk, batch_host_pipeline
    w = workload("fdk64")
    g = w.geom
    E = torch.from_numpy(line_integrals(w.phantom(), g).astype(np.float32))
    plan = B.Plan(g)
    bf = BatchFdk(plan, 3)
    dev_vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
    bf.reconstruct(E.cuda(), dev_vol)
    E_host = E.pin_memory()
    vol_host = torch.empty((g.nx, g.ny, g.nz), pin_memory=True)
    E_b = [torch.empty((2 * bf.n, g.nv, g.nu), device="cuda") for _ in range(2)]
    vols = [torch.empty_like(dev_vol), torch.empty_like(dev_vol)]
    batch_host_pipeline(bf, E_host, vol_host, E_b, vols, 7)   # two whole reconstructions and a part
    assert torch.equal(vol_host, dev_vol.cpu())


def test_arith_rates_are_plausible():
    r = B.arith_rates(iters=512)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert r["n_sm"] == n_sm
    for k in B.RATE_KINDS:
        assert r[k]["sms_seen"] == n_sm, k
        assert 0 < r[k]["lane_ops_per_clk_sm"] <= 2 * 256, (k, r[k])
    # one FP32 FMA per lane and clock on 128 lanes, at most
    assert 96 <= r["ffma"]["lane_ops_per_clk_sm"] <= 130, r["ffma"]
    print({k: round(v["lane_ops_per_clk_sm"], 1) for k, v in r.items() if k != "n_sm"})
