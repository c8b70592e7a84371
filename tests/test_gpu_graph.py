"""FdkGraph: the FDK launch sequence captured as a CUDA graph replays the eager
result bit for bit, for new projections copied into its input buffer."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.phantom import line_integrals, random_ellipsoids, safe_radius, workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_graph_replay_equals_eager(dtype):
    from paper_1909_02724_gb300.api import FdkGraph, fdk
    from paper_1909_02724_gb300.binding import Plan
    g = workload("fdk64").geom
    plan = Plan(g)
    fg = FdkGraph(plan, dtype=dtype)
    for seed in (1, 2):
        E = line_integrals(random_ellipsoids(8, 0.9 * safe_radius(g), seed), g).astype(np.float32)
        Et = torch.from_numpy(E).cuda()
        fg.E.copy_(Et)
        got = fg.replay().clone()
        want = fdk(plan, Et, dtype=dtype)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        if dtype == torch.float32:
            ref = oracle.fdk(g, E.astype(np.float64))
            v = got.cpu().double().numpy()
            assert np.linalg.norm(v - ref) / np.linalg.norm(ref) <= 1e-5
    assert plan.device_status() == 0
