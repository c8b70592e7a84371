"""ifdk_filter_noalloc: the tensor-core filter with the library's fixed
workspace, for callers that cannot allocate device memory (a C caller that
only owns the E and Q buffers it was handed, or a pipeline that reserves all
device memory at start-up).  It must give the same filtered views as
ifdk_filter with a caller workspace, call after call, although every call
reuses (and leaves behind) the same 16 MiB array.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_1909_02724_gb300.geometry import circular
from paper_1909_02724_gb300.phantom import line_integrals, random_ellipsoids, safe_radius

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _views(g, seed):
    ell = random_ellipsoids(6, 0.9 * safe_radius(g), seed)
    return torch.from_numpy(line_integrals(ell, g).astype(np.float32)).cuda()


def _rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


@pytest.mark.parametrize("dtype,terms,tol", [("float32", 3, 1e-6), ("float16", 2, 1e-6), ("bfloat16", 2, 1e-6)])
def test_noalloc_filter_matches_workspace_filter(dtype, terms, tol):
    from paper_1909_02724_gb300 import binding as B
    from paper_1909_02724_gb300.build import build
    build()
    # 120 views x 100 rows x 320 columns: 12000 rows, two launches of the 16 MiB array for 3 terms
    g = circular(120, 320, 100, 0.3, 0.3, 8, 8, 8, 1.0)
    plan = B.Plan(g)
    tdt = getattr(torch, dtype)
    for seed in (1, 2):                       # two calls in a row, different inputs
        E = _views(g, seed)
        ref = plan.filter(E, dtype=tdt, split_terms=terms)
        Q = torch.full_like(ref, float("nan"))
        B.ifdk_filter_noalloc(plan.handle, E, Q, B.dtype_code(tdt), terms)
        torch.cuda.synchronize()
        assert torch.isfinite(Q.float()).all()
        assert _rel(Q.float(), ref.float()) <= tol
    assert plan.device_status() == B.IFDK_OK


def test_noalloc_filter_rejects_bad_requests_before_work():
    from paper_1909_02724_gb300 import binding as B
    g = circular(4, 64, 16, 1.5, 1.5, 8, 8, 8, 1.0)
    plan = B.Plan(g)
    E = torch.zeros((g.np, g.nv, g.nu), device="cuda")
    Q = torch.full_like(E, 7.0)
    for terms in (0, 4):
        with pytest.raises(B.IfdkError) as e:
            B.ifdk_filter_noalloc(plan.handle, E, Q, B.IFDK_F32, terms)
        assert e.value.code == B.IFDK_ERR_INVALID
    torch.cuda.synchronize()
    assert float(Q.min()) == 7.0
