"""The tensor-core filter (tcgen05 split-BF16 Toeplitz product) against the FP64 oracle.

The kernel sums the convolution by parts (first differences of the weighted
row against the running sum of the taps), so operand rounding is amplified
only ~5x instead of the direct sum's ~1000x; expected rel-L2 of Q: 3 terms
~1e-7 (FP32 level), 2 terms ~1e-6, 1 term ~1e-2.  Sizes cover
ragged row counts, nu below / above / not a multiple of the 128-wide tile,
and workspaces small enough to force many chunks."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.geometry import circular
from paper_1909_02724_gb300.phantom import line_integrals, random_ellipsoids, safe_radius

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GEOMS = {
    "nu64": circular(6, 64, 40, 1.5, 1.5, 8, 8, 8, 1.0),
    "nu200": circular(5, 200, 37, 0.48, 0.48, 8, 8, 8, 1.0),
    "nu384": circular(3, 384, 70, 0.25, 0.25, 8, 8, 8, 1.0),
}
TOL = {3: 1e-6, 2: 2e-4, 1: 5e-2}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def phantom_E(g):
    ell = random_ellipsoids(6, 0.9 * safe_radius(g), 5)
    return line_integrals(ell, g).astype(np.float32)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("terms", [3, 2, 1])
def test_tc_filter_matches_oracle(name, terms):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS[name]
    E = phantom_E(g)
    ref = oracle.filter_views(g, E.astype(np.float64))
    p = plan = Plan(g)
    Q = plan.filter(torch.from_numpy(E).cuda(), split_terms=terms).cpu().numpy()
    assert p.device_status() == 0
    err = rel_l2(Q, ref)
    assert err <= TOL[terms], (name, terms, err)
    if terms == 3:
        assert float(np.max(np.abs(Q - ref)) / np.max(np.abs(ref))) <= 1e-5


@pytest.mark.parametrize("dtype", ["float16", "bfloat16"])
def test_tc_filter_16bit_output(dtype):
    from paper_1909_02724_gb300.binding import Plan
    g = GEOMS["nu200"]
    E = phantom_E(g)
    ref = oracle.filter_views(g, E.astype(np.float64))
    Q = Plan(g).filter(torch.from_numpy(E).cuda(), dtype=getattr(torch, dtype)).float().cpu().numpy()
    assert rel_l2(Q, ref) <= (1e-3 if dtype == "float16" else 5e-3)


def test_tc_filter_small_workspace_many_chunks():
    from paper_1909_02724_gb300 import binding as B
    g = GEOMS["nu64"]
    E = torch.from_numpy(phantom_E(g)).cuda()
    p = B.Plan(g)
    mn, pref = B.ifdk_filter_workspace_size(p.handle, 3)
    assert 0 < mn <= pref
    ws = torch.empty(mn // 2 + 64, dtype=torch.bfloat16, device="cuda")
    base = ws.data_ptr() + (-ws.data_ptr()) % 128
    Q1 = torch.empty_like(E)
    B.ifdk_filter(p.handle, E, Q1, B.IFDK_F32, 3, base, mn)            # 128 rows per launch
    Q2 = p.filter(E, split_terms=3)                                     # preferred workspace
    assert torch.equal(Q1, Q2)
    with pytest.raises(B.IfdkError):
        B.ifdk_filter(p.handle, E, Q1, B.IFDK_F32, 3, base, mn - 2)     # too small: rejected before launch
    with pytest.raises(B.IfdkError):
        B.ifdk_filter(p.handle, E, Q1, B.IFDK_F32, 3, None, 0)
