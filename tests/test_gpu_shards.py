"""The rank decomposition (Sec. 4 of the paper) through the CUDA library.

Each rank's share is run here one after another on one GPU (no kernel waits
on another): the column split back-projects a view range of the whole volume
per rank (ifdk_backproject / the packed path with view_begin, view_count) and
the shares sum to the single-call volume; the row split builds a plan per
z-slab (off-centre slabs) and the slabs, stacked, are the single-call volume.
Both are checked against the FP64 oracle at the FP32 tolerances."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.parallel import slab_shard, view_shard
from paper_1909_02724_gb300.phantom import scaled_geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def case():
    g = scaled_geometry(48, 64, 30, nz=41, n_det_v=56)
    Q = np.random.default_rng(7).standard_normal((g.np, g.nv, g.nu))
    return g, Q, oracle.backproject(g, Q)


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("packed", [False, True])
def test_view_split_sums_to_whole(world, packed):
    from paper_1909_02724_gb300.binding import Plan
    g, Q, ref = case()
    plan = Plan(g)
    Qd = torch.from_numpy(Q).float().cuda()
    vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device="cuda")
    Qp = plan.pack(Qd) if packed else None
    for r in range(world):
        b, c = view_shard(g, world, r)
        part = torch.zeros_like(vol)
        if packed:
            plan.backproject_packed(Qp, part, view_begin=b, view_count=c)
        else:
            plan.backproject(Qd, part, view_begin=b, view_count=c)
        vol += part
    got = vol.cpu().double().numpy()
    assert rel_l2(got, ref) <= 1e-5
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_slab_split_stacks_to_whole(world):
    from paper_1909_02724_gb300.binding import Plan
    g, Q, ref = case()
    Qd = torch.from_numpy(Q).float().cuda()
    got = np.zeros_like(ref)
    for r in range(world):
        s = slab_shard(g, world, r)
        plan = Plan(s.geom)
        v = plan.backproject(Qd)
        got[:, :, s.k_begin:s.k_begin + s.k_count] = v.cpu().double().numpy()
        sl = ref[:, :, s.k_begin:s.k_begin + s.k_count]
        assert rel_l2(got[:, :, s.k_begin:s.k_begin + s.k_count], sl) <= 1e-5
    assert rel_l2(got, ref) <= 1e-5
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
