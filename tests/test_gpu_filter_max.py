"""The 16-bit range check of the filter (ifdk_filter_max) against the oracle.

view_max[s] is the largest |Q| of view s in FP32 before the cast.  It is
checked against the FP64 oracle's filtered views for every split mode and
storage type, on detector heights that make views change in the middle of a
warp's rows (the segmented warp reduction).  It must flag exactly the views
whose values leave the FP16 range, and it must carry a NaN."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.geometry import circular

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TDT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
# relative accuracy of the FP32 values per split mode (0: SIMT FP32)
TOL = {0: 1e-5, 3: 1e-5, 2: 5e-4, 1: 2e-2}
GEOMS = {
    "nv37": circular(5, 200, 37, 0.48, 0.48, 8, 8, 8, 1.0),
    "nv40": circular(6, 64, 40, 1.5, 1.5, 8, 8, 8, 1.0),
    "nv8": circular(9, 96, 8, 1.0, 1.0, 8, 8, 4, 1.0),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def seeded_E(g, seed=5):
    return np.random.default_rng(seed).uniform(0.0, 3.0, (g.np, g.nv, g.nu)).astype(np.float32)


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("dtype", list(TDT))
@pytest.mark.parametrize("split", [0, 1, 2, 3])
def test_view_max_matches_oracle(name, dtype, split):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS[name]
    E = seeded_E(g)
    ref = np.abs(oracle.filter_views(g, E.astype(np.float64))).reshape(g.np, -1).max(axis=1)
    plan = Plan(g)
    vm = torch.full((g.np,), -1.0, device="cuda")
    Q = plan.filter(torch.from_numpy(E).cuda(), dtype=TDT[dtype], split_terms=split, view_max=vm)
    got = vm.cpu().double().numpy()
    np.testing.assert_allclose(got, ref, rtol=TOL[split], atol=0)
    # view_max does not change Q
    Q2 = plan.filter(torch.from_numpy(E).cuda(), dtype=TDT[dtype], split_terms=split)
    assert torch.equal(Q, Q2)


@pytest.mark.parametrize("split", [0, 2])
def test_view_max_flags_fp16_overflow(split):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS["nv40"]
    E = seeded_E(g, 6)
    base = np.abs(oracle.filter_views(g, E.astype(np.float64))).reshape(g.np, -1).max(axis=1)
    scale = np.full(g.np, 0.1 * 65504.0) / base     # every view near 6550
    scale[[0, 3]] *= 100.0                           # views 0 and 3 near 655040
    Es = (E * scale[:, None, None]).astype(np.float32)
    plan = Plan(g)
    vm = torch.zeros(g.np, device="cuda")
    Q = plan.filter(torch.from_numpy(Es).cuda(), dtype=torch.float16, split_terms=split, view_max=vm)
    over = (vm.cpu().numpy() > 65504.0).nonzero()[0].tolist()
    assert over == [0, 3]
    inf_views = torch.isinf(Q.float()).flatten(1).any(dim=1).cpu().numpy().nonzero()[0].tolist()
    assert inf_views == [0, 3]


@pytest.mark.parametrize("split", [0, 3])
def test_view_max_carries_nan(split):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS["nv37"]
    E = seeded_E(g, 7)
    E[2, 5, 7] = np.nan
    plan = Plan(g)
    vm = torch.zeros(g.np, device="cuda")
    plan.filter(torch.from_numpy(E).cuda(), split_terms=split, view_max=vm)
    v = vm.cpu().numpy()
    assert np.isnan(v[2]) and np.isfinite(np.delete(v, 2)).all()


def test_view_max_argument_errors():
    from paper_1909_02724_gb300.binding import (IFDK_ERR_ALIGNMENT, IFDK_ERR_INVALID, IfdkError, Plan,
                                                ifdk_filter_max)
    g = GEOMS["nv8"]
    plan = Plan(g)
    E = torch.zeros((g.np, g.nv, g.nu), device="cuda")
    Q = torch.empty_like(E)
    vm = torch.zeros(g.np + 4, device="cuda")
    with pytest.raises(IfdkError) as e:
        ifdk_filter_max(plan.handle, E, Q, 0, 0, None, 0, None)
    assert e.value.code == IFDK_ERR_INVALID
    with pytest.raises(IfdkError) as e:
        ifdk_filter_max(plan.handle, E, Q, 0, 0, None, 0, int(vm.data_ptr()) + 2)
    assert e.value.code == IFDK_ERR_ALIGNMENT
    with pytest.raises(ValueError):
        plan.filter(E, Q, view_max=torch.zeros(g.np + 1, device="cuda"))
