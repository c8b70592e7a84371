"""Streaming back-projection from host memory, and views-only Q buffers.

* ifdk_backproject_views on a buffer holding only the called views gives
  bit-identical volumes to ifdk_backproject on the whole array (same kernels,
  only the TMA / load coordinates move), on the mirror and general paths.
* ifdk_backproject_host streams pinned host views in chunks (ragged last
  chunk, either the plan's own rows or a row window strided out of
  full-height views) and gives bit-identical volumes to the device call.
* A plan cut to the rows ifdk_query_rows reports matches the full plan.
* The large slab (4096 x 4096 x 256 from 2048 views of 4096 x 4096, FP16
  views streamed from pinned host memory in 64-view chunks) against the FP64
  oracle on sampled voxels."""
import time

import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300 import binding as B
from paper_1909_02724_gb300.phantom import line_integrals_gpu, scaled_geometry, workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def chunked(plan, Q, chunk, vol=None):
    """Device back-projection in the launches the streaming call makes (one
    per chunk, each adding its views' sum into the volume)."""
    g = plan.geom
    if vol is None:
        vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
    for v0 in range(0, g.np, chunk):
        plan.backproject(Q, vol, view_begin=v0, view_count=min(chunk, g.np - v0))
    return vol


def rand_views(g, dtype, seed):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    return torch.randn((g.np, g.nv, g.nu), device="cuda", generator=gen).to(dtype)


GEOMS = {
    "mirror": scaled_geometry(64, 96, 40, nz=24),
    "general": scaled_geometry(48, 80, 36, nz=20).with_(vol_off_z=5.0),
}


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_views_only_buffer_is_bit_identical(name, dtype):
    g = GEOMS[name]
    plan = B.Plan(g)
    assert plan.info(dtype)["path"] == (1 if name == "mirror" else 0)
    Q = rand_views(g, dtype, 3)
    ref = plan.backproject(Q, view_begin=5, view_count=17)
    got = plan.backproject_views(Q[5:22].contiguous(), view_begin=5)
    assert torch.equal(got, ref)
    assert plan.device_status() == 0


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
def test_host_streaming_is_bit_identical(dtype):
    g = GEOMS["mirror"]
    plan = B.Plan(g)
    Q = rand_views(g, dtype, 4)
    ref = chunked(plan, Q, 7)
    whole = plan.backproject(Q)
    assert float((ref - whole).abs().max()) <= 1e-6 * float(whole.abs().max())
    Qh = Q.cpu().pin_memory()
    vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
    plan.backproject_host(Qh, vol, chunk_views=7, packed=False)  # 6 chunks, the last one of 5 views
    torch.cuda.synchronize()
    assert torch.equal(vol, ref)
    # view subsets accumulate; one chunk larger than the range
    vol2 = torch.zeros_like(vol)
    plan.backproject_host(Qh, vol2, chunk_views=64, view_begin=0, view_count=11, packed=False)
    plan.backproject_host(Qh, vol2, chunk_views=4, view_begin=11, view_count=29, packed=False)
    torch.cuda.synchronize()
    assert float((vol2 - whole).abs().max()) <= 1e-6 * float(whole.abs().max())
    assert plan.device_status() == 0


def test_row_window_streamed_out_of_full_height_views():
    g = GEOMS["mirror"]
    r0, n = B.ifdk_query_rows(g)
    assert 0 < n < g.nv
    full_plan, cut_plan = B.Plan(g), B.Plan(g.crop_rows(r0, n))
    assert cut_plan.info(torch.float16)["path"] == 1
    Q = rand_views(g, torch.float16, 5)
    ref_full = chunked(full_plan, Q, 8)
    ref_cut = chunked(cut_plan, Q[:, r0:r0 + n].contiguous(), 8)
    # the cut plan reads the same pixels; only FP32 rounding of v differs
    assert float((ref_cut - ref_full).norm() / ref_full.norm()) <= 2e-6
    Qh = Q.cpu().pin_memory()                                     # full-height host views
    vol = torch.zeros_like(ref_cut)
    cut_plan.backproject_host(Qh, vol, chunk_views=8, host_row0=r0, packed=False)
    torch.cuda.synchronize()
    assert torch.equal(vol, ref_cut)
    # the packed streaming path on the same rows: the same sum up to rounding order
    vol_p = torch.zeros_like(ref_cut)
    cut_plan.backproject_host(Qh, vol_p, chunk_views=8, host_row0=r0)
    torch.cuda.synchronize()
    # (the packed FP16 kernel also takes the v-lerp in half2)
    assert float((vol_p - ref_cut).norm() / ref_cut.norm()) <= 5e-4


def test_host_streaming_rejects_bad_arguments():
    g = GEOMS["mirror"]
    plan = B.Plan(g)
    Qh = torch.zeros((g.np, g.nv, g.nu), dtype=torch.float16).pin_memory()
    vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
    st = torch.empty(2 * 8 * g.nv * g.nu + 256, dtype=torch.float16, device="cuda")
    nbytes = 2 * 8 * g.nv * g.nu * 2
    h = plan.handle
    ok = (h, Qh, B.IFDK_F16, g.nv, 0, 0, g.np, 8, st, nbytes, vol)
    B.ifdk_backproject_host(*ok)
    torch.cuda.synchronize()
    bad = [
        (h, Qh, B.IFDK_F16, g.nv, 0, 0, g.np, 8, st, nbytes - 2, vol),          # staging too small
        (h, Qh, B.IFDK_F16, g.nv, 0, 0, g.np, 8, st.data_ptr() + 2, nbytes, vol),   # misaligned staging
        (h, Qh, B.IFDK_F16, g.nv, 1, 0, g.np, 8, st, nbytes, vol),              # rows past the host view
        (h, Qh, B.IFDK_F16, g.nv - 1, 0, 0, g.np, 8, st, nbytes, vol),          # host view too short
        (h, Qh, B.IFDK_F16, g.nv, 0, 0, g.np, 0, st, nbytes, vol),              # empty chunks
        (h, Qh, B.IFDK_F16, g.nv, 0, 30, 20, 8, st, nbytes, vol),               # past the last view
        (h, None, B.IFDK_F16, g.nv, 0, 0, g.np, 8, st, nbytes, vol),
    ]
    for args in bad:
        with pytest.raises(B.IfdkError):
            B.ifdk_backproject_host(*args)
    assert float(vol.abs().max()) == 0.0                          # nothing ran
    B.ifdk_backproject_host(h, Qh, B.IFDK_F16, g.nv, 0, 3, 0, 8, st, nbytes, vol)   # zero views: no-op


def slab_inputs():
    """The slab workload's FP16 filtered views for the rows the slab reads,
    in pinned host memory, with the cut plan and the raw rows."""
    w = workload("slab4096")
    g = w.geom
    r0, n = B.ifdk_query_rows(g)
    gc = g.crop_rows(r0, n)
    E = line_integrals_gpu(w.phantom(), gc)                       # [2048][n][4096] FP32, the full scene's phantom
    plan = B.Plan(gc)
    Q = plan.filter(E, dtype=torch.float16)
    Qh = torch.empty(Q.shape, dtype=torch.float16, pin_memory=True)
    Qh.copy_(Q)
    del Q
    return gc, plan, E, Qh


def test_slab4096_streamed_fp16_against_oracle():
    gc, plan, E, Qh = slab_inputs()
    vol = torch.zeros((gc.nx, gc.ny, gc.nz), device="cuda")      # 16 GiB
    torch.cuda.synchronize()
    t = time.perf_counter()
    plan.backproject_host(Qh, vol, chunk_views=64)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    print(f"slab4096 streamed FP16: {gc.updates / dt / 2**30:.0f} GUPS ({dt:.2f} s)")
    assert plan.device_status() == 0
    rng = np.random.default_rng(55)
    ii, jj, kk = np.meshgrid(np.arange(0, gc.nx, 64), np.arange(0, gc.ny, 64), [0, 128, 255], indexing="ij")
    # three slices (bottom, middle, top): the oracle filters only the ~35 rows
    # per view that they touch
    vox = np.concatenate([np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1),
                          np.stack([rng.integers(0, gc.nx, 768), rng.integers(0, gc.ny, 768),
                                    rng.choice([0, 128, 255], 768)], 1)])
    idx = [torch.from_numpy(vox[:, c]).cuda() for c in range(3)]
    v = vol[idx[0], idx[1], idx[2]].double().cpu().numpy()
    need = oracle.rows_needed(gc, vox)
    s_idx, r_idx = np.nonzero(need)
    rowmap = -np.ones((gc.np, gc.nv), dtype=np.int64)
    rowmap[s_idx, r_idx] = np.arange(len(s_idx))
    E_rows = E[torch.from_numpy(s_idx).cuda(), torch.from_numpy(r_idx).cuda()].double().cpu().numpy()
    ref = oracle.backproject_voxels(gc, oracle.filter_rows(gc, E_rows, r_idx), vox, rowmap=rowmap)
    err = float(np.linalg.norm(v - ref) / np.linalg.norm(ref))
    # the same Q the GPU read (FP16-rounded): back-projection arithmetic alone
    Q16 = Qh[torch.from_numpy(s_idx), torch.from_numpy(r_idx)].double().numpy()
    ref16 = oracle.backproject_voxels(gc, Q16, vox, rowmap=rowmap)
    err16 = float(np.linalg.norm(v - ref16) / np.linalg.norm(ref16))
    print(f"slab4096: rel-L2 vs FP64 oracle {err:.3e}; vs oracle on the FP16 views {err16:.3e}")
    assert err <= 2e-3
    # the FP16 kernel interpolates along u in FP16 (packed half2): one rounding
    # of <= 2^-11 relative per tap pair, averaged over 2048 views
    assert err16 <= 2e-4
