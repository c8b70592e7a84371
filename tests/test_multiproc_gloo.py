"""World-size-2 runs of the rank decomposition (Sec. 4 of the paper) on CPU.

Two gloo ranks, spawned as processes, each back-project their share with the
FP64 oracle and combine through paper_1909_02724_gb300.parallel: the column
split (views, summed by a reduce) and the row split (z-slabs, gathered) must
give the single-process volume, and max_over_ranks the slowest rank's time.
The shares are ragged (odd view and slice counts)."""
import os
import socket
import traceback

import numpy as np
import pytest

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from paper_1909_02724_gb300.phantom import scaled_geometry
    g = scaled_geometry(14, 20, 15, nz=11, n_det_v=18).with_(off_u=0.3, off_v=-0.4, vol_off_z=0.7)
    Q = np.random.default_rng(1909).standard_normal((g.np, g.nv, g.nu))
    return g, Q


def _worker(rank, port, q):
    try:
        import torch
        import torch.distributed as dist

        import oracle
        from paper_1909_02724_gb300 import parallel as P

        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=WORLD)
        out = {"rank": rank}
        out["max"] = P.max_over_ranks(rank + 0.25)

        g, Q = _case()
        b, c = P.view_shard(g, WORLD, rank)
        out["views"] = (b, c)
        reduced = torch.from_numpy(oracle.backproject(g, Q, b, c, threads=1))
        P.reduce_volume(reduced, dst=0)

        slab = P.slab_shard(g, WORLD, rank)
        out["slab"] = (slab.k_begin, slab.k_count)
        vs = torch.from_numpy(oracle.backproject(slab.geom, Q, threads=1))
        full = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float64) if rank == 0 else None
        P.gather_slabs(vs, full, dst=0, nz=g.nz)
        made = P.gather_slabs(vs, None, dst=1, nz=g.nz)      # allocated on the destination rank
        # the paper's sub-volumes: mirror pairs, direct slab then mirror slab
        pb, pc = P.pair_shard(g.with_(vol_off_z=0.0), WORLD, rank)
        gc = g.with_(vol_off_z=0.0)
        ks = np.arange(pb, pb + pc)
        depth = 2 * pc - (1 if g.nz % 2 and pb + pc == (g.nz + 1) // 2 else 0)
        ii, jj = np.meshgrid(np.arange(g.nx), np.arange(g.ny), indexing="ij")
        part = np.zeros((g.nx, g.ny, depth))
        for t, k in enumerate(ks):
            for kk, dst_k in ((k, t), (g.nz - 1 - k, depth - 1 - t)):
                vox = np.stack([ii.ravel(), jj.ravel(), np.full(ii.size, kk)], 1)
                part[:, :, dst_k] = oracle.backproject_voxels(gc, Q, vox, threads=1).reshape(g.nx, g.ny)
        pairs_full = P.gather_pair_slabs(torch.from_numpy(part), None, g.nz, dst=0)
        if rank == 0:
            out["reduced"] = reduced.numpy()
            out["gathered"] = full.numpy()
            out["pairs"] = pairs_full.numpy()
            assert made is None
        else:
            out["gathered_on_1"] = made.numpy()
        dist.barrier()
        dist.destroy_process_group()
        q.put(out)
    except Exception:  # reported to the parent, which fails the test
        q.put({"rank": rank, "error": traceback.format_exc()})


@pytest.fixture(scope="module")
def results():
    import multiprocessing as mp

    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(WORLD):
            r = q.get(timeout=180)
            out[r["rank"]] = r
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    for r in out.values():
        assert "error" not in r, r["error"]
    return out


def test_split_range_covers_in_order():
    from paper_1909_02724_gb300.parallel import split_range
    for n in (0, 1, 5, 16, 17):
        for parts in (1, 2, 3, 8):
            spans = [split_range(n, parts, i) for i in range(parts)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        split_range(4, 0, 0)
    with pytest.raises(ValueError):
        split_range(4, 2, 2)


def test_slab_geometry_keeps_voxel_positions():
    """Voxel k of every slab has the world Z of voxel k_begin + k of the volume."""
    from paper_1909_02724_gb300.parallel import slab_shard
    g, _ = _case()

    def z(geom, k):
        return -geom.dz * (k - (geom.nz - 1) / 2.0) + geom.vol_off_z

    for world in (1, 2, 3, 4):
        seen = []
        for r in range(world):
            s = slab_shard(g, world, r)
            ks = np.arange(s.k_count)
            np.testing.assert_allclose(z(s.geom, ks), z(g, s.k_begin + ks), atol=1e-12)
            seen.extend(range(s.k_begin, s.k_begin + s.k_count))
        assert seen == list(range(g.nz))


def test_max_over_ranks(results):
    assert all(r["max"] == WORLD - 1 + 0.25 for r in results.values())


def test_shares_are_ragged_and_disjoint(results):
    g, _ = _case()
    v = sorted(r["views"] for r in results.values())
    s = sorted(r["slab"] for r in results.values())
    assert v == [(0, 8), (8, 7)] and sum(c for _, c in v) == g.np
    assert s == [(0, 6), (6, 5)] and sum(c for _, c in s) == g.nz


def test_view_split_reduce_equals_single_process(results):
    import oracle
    g, Q = _case()
    ref = oracle.backproject(g, Q, threads=1)
    got = results[0]["reduced"]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_slab_split_gather_equals_single_process(results):
    import oracle
    g, Q = _case()
    ref = oracle.backproject(g, Q, threads=1)
    got = results[0]["gathered"]
    # the slab's matrices differ from the volume's only in rounding (the Z shift)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    np.testing.assert_array_equal(results[1]["gathered_on_1"], got)


def test_pair_split_gather_equals_single_process(results):
    """Mirror-pair sub-volumes (pair_shard) of the centred volume, gathered."""
    import oracle
    g, Q = _case()
    gc = g.with_(vol_off_z=0.0)
    ref = oracle.backproject(gc, Q, threads=1)
    np.testing.assert_allclose(results[0]["pairs"], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
