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
    assert plan.device_status() == 0
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


PAIR_GEOMS = {
    "even_nz": scaled_geometry(48, 64, 30, nz=40, n_det_v=56),
    "odd_nz": scaled_geometry(40, 56, 24, nz=33, n_det_v=48),
    "fdk64": scaled_geometry(64, 64, 64),
}


@pytest.mark.parametrize("name", list(PAIR_GEOMS))
@pytest.mark.parametrize("world", [1, 2, 3, 4])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_pair_shards_place_to_whole(name, world, dtype):
    """The paper's sub-volumes (a slab and its mirror slab) through
    ifdk_backproject_packed_pairs, one rank after another on one GPU."""
    from paper_1909_02724_gb300.binding import Plan
    from paper_1909_02724_gb300.parallel import pair_shard, place_pair_slab
    g = PAIR_GEOMS[name]
    Q = np.random.default_rng(9).standard_normal((g.np, g.nv, g.nu))
    tdt = torch.float32 if dtype == "f32" else torch.float16
    plan = Plan(g)
    Qp = plan.pack(torch.from_numpy(Q).to(tdt).cuda())
    whole = plan.backproject_packed(Qp).cpu().double().numpy()
    got = torch.full((g.nx, g.ny, g.nz), float("nan"), dtype=torch.float64)
    for r in range(world):
        b, c = pair_shard(g, world, r)
        part = plan.backproject_packed_pairs(Qp, b, c)
        place_pair_slab(got, part.cpu().double(), g.nz, b, c)
    got = got.numpy()
    assert np.isfinite(got).all()
    # a range that starts off the whole launch's block grid forms v from another block
    # start (another rounding of v); the oracle bound is the one the parts must meet
    assert rel_l2(got, whole) <= (1e-5 if dtype == "f32" else 1e-3)
    if dtype == "f32":
        ref = oracle.backproject(g, Q)
        assert rel_l2(got, ref) <= 1e-5
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    assert plan.device_status() == 0


def test_pair_range_arguments():
    from paper_1909_02724_gb300.binding import IFDK_ERR_INVALID, IfdkError, Plan, ifdk_backproject_packed_pairs
    g = PAIR_GEOMS["odd_nz"]
    plan = Plan(g)
    Qp = plan.pack(torch.zeros((g.np, g.nv, g.nu), device="cuda"))
    vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
    for b, c in ((-1, 2), (0, 18), (16, 2), (3, -1)):
        with pytest.raises(IfdkError) as e:
            ifdk_backproject_packed_pairs(plan.handle, Qp, 0, 0, g.np, b, c, vol)
        assert e.value.code == IFDK_ERR_INVALID
    ifdk_backproject_packed_pairs(plan.handle, Qp, 0, 0, g.np, 5, 0, vol)   # empty range
    assert plan.device_status() == 0
