"""GPU parity of the packed-view path (ifdk_pack_views + ifdk_backproject_packed).

* the pack kernel equals a NumPy restatement of the packed layout, bit for bit;
* the packed back-projection matches the FP64 oracle (FP32: rel-L2 <= 1e-5,
  max-abs <= 1e-4 max|vol|) with half-turn view pairing on and off, for
  whole scans and for view ranges that split into pairs and single views;
* FDK end to end (filter, pack, packed back-projection) against the oracle
  FDK in every storage type (reduced precision: rel-L2 <= 2e-3);
* streaming from pinned host views through the packed path;
* geometries without packed views are refused before any launch.
"""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300 import binding as B
from paper_1909_02724_gb300.geometry import circular
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


GEOMS = {
    "fdk64": workload("fdk64").geom,
    "ragged": scaled_geometry(40, 56, 24, nz=50, n_det_v=48),
    "odd_nz_odd_ny": scaled_geometry(33, 48, 16, nz=33),
    "half_pixel_v_offset": circular(10, 64, 48, 1.5, 1.5, 36, 28, 22, 1.0, off_u=-0.4, off_v=0.75),
    "neg_v_offset": circular(12, 64, 48, 1.5, 1.5, 36, 28, 22, 1.0, off_u=0.2, off_v=-4.5),
    "magnified_odd_np": circular(9, 96, 80, 0.5, 0.5, 24, 24, 20, 0.5),
}

TDT = {"float32": torch.float32, "float16": torch.float16, "bfloat16": torch.bfloat16}


def pack_numpy(g, Q, raw=False):
    """The packed layout written out: element (i, e) of detector row r = r0 + i
    and column c = e - 1 holds Q[r][c], Q[2vc-r][c], Q[r][c+1] - Q[r][c],
    Q[2vc-r][c+1] - Q[2vc-r][c] (FP32 differences), Q zero off the detector;
    raw (the BF16 layout): Q[r][c], Q[2vc-r][c], Q[r][c+1], Q[2vc-r][c+1]."""
    vc = (g.nv - 1) / 2 + g.off_v / g.dv
    two_vc = int(round(2 * vc))
    r0 = min(0, two_vc - (g.nv - 1))
    rows = int(np.floor(vc)) + 3 - r0
    nu_p = (g.nu + 2) // 2 * 2
    Z = np.zeros((Q.shape[0], g.nv + 2 * rows + 4, nu_p + 1), dtype=Q.dtype)
    off = rows + 2                                   # Z row of detector row 0
    Z[:, off:off + g.nv, 1:g.nu + 1] = Q             # Z column of detector column c is c + 1

    def rowsof(rr):
        return Z[:, off + rr, :]
    r = r0 + np.arange(rows)
    d, m = rowsof(r), rowsof(two_vc - r)
    a, b = d[..., :nu_p], m[..., :nu_p]
    if raw:
        return np.stack([a, b, d[..., 1:nu_p + 1], m[..., 1:nu_p + 1]], -1)
    return np.stack([a, b, d[..., 1:nu_p + 1] - a, m[..., 1:nu_p + 1] - b], -1)


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("dtype", ["float32", "float16", "bfloat16"])
def test_pack_is_the_packed_layout(name, dtype):
    g = GEOMS[name]
    p = B.Plan(g)
    gen = torch.Generator(device="cuda").manual_seed(7)
    Q = torch.randn((g.np, g.nv, g.nu), device="cuda", generator=gen).to(TDT[dtype])
    Qp = p.pack(Q)
    ref = pack_numpy(g, Q.cpu().float().numpy(), raw=dtype == "bfloat16")   # FP32 arithmetic on the stored values
    ref = torch.from_numpy(ref).to(TDT[dtype]).float().numpy()   # rounded once to the storage type
    assert Qp.shape == ref.shape
    assert np.array_equal(Qp.cpu().float().numpy(), ref)


@pytest.mark.parametrize("pairing", [True, False])
@pytest.mark.parametrize("name", list(GEOMS))
def test_backproject_packed_fp32_matches_oracle(name, pairing):
    g = GEOMS[name]
    Q = oracle.filter_views(g, phantom_E(g).astype(np.float64)).astype(np.float32)
    ref = oracle.backproject(g, Q.astype(np.float64))
    p = B.Plan(g)
    p.set_view_pairing(pairing)
    Qt = torch.from_numpy(Q).cuda()
    vol = p.backproject_packed(p.pack(Qt)).cpu().numpy()
    info = p.packed_info(torch.float32)
    assert info["path"] == (2 if pairing and g.ny % 2 == 0 and g.np % 2 == 0 else 1), info
    assert rel_l2(vol, ref) <= 1e-5, (name, info)
    assert max_rel(vol, ref) <= 1e-4
    # the same sum as the standard-layout kernels, and bitwise reproducible
    std = p.backproject(Qt).cpu().numpy()
    assert max_rel(vol, std) <= 2e-6
    again = p.backproject_packed(p.pack(Qt)).cpu().numpy()
    assert np.array_equal(vol, again)
    assert p.device_status() == 0


@pytest.mark.parametrize("name", ["fdk64", "ragged", "odd_nz_odd_ny", "neg_v_offset"])
@pytest.mark.parametrize("dtype", ["float32", "float16", "bfloat16"])
def test_fdk_packed_end_to_end(name, dtype):
    g = GEOMS[name]
    E = phantom_E(g)
    ref = oracle.fdk(g, E.astype(np.float64))
    p = B.Plan(g)
    Q = p.filter(torch.from_numpy(E).cuda(), dtype=TDT[dtype])
    Qp = p.pack(Q)
    for pairing in (True, False):
        p.set_view_pairing(pairing)
        vol = p.backproject_packed(Qp).cpu().numpy()
        if dtype == "float32":
            assert rel_l2(vol, ref) <= 1e-5, pairing
            assert max_rel(vol, ref) <= 1e-4, pairing
        else:
            assert rel_l2(vol, ref) <= 2e-3, (pairing, rel_l2(vol, ref))


@pytest.mark.parametrize("name", ["fdk64", "ragged", "half_pixel_v_offset"])
@pytest.mark.parametrize("dtype", ["float32", "float16"])
def test_packed_view_ranges_split_into_pairs_and_singles(name, dtype):
    """A call over views [b, e) back-projects the half-turn pairs inside the
    range together and the rest singly: every range matches the oracle's sum
    over exactly those views, and ranges that partition the scan add up."""
    g = GEOMS[name]
    Q = oracle.filter_views(g, phantom_E(g).astype(np.float64)).astype(np.float32)
    Qt = torch.from_numpy(Q).cuda().to(TDT[dtype])
    Qd = Qt.double().cpu().numpy()
    p = B.Plan(g)
    Qp = p.pack(Qt)
    h = g.np // 2
    for b, e in [(0, g.np), (1, g.np - 1), (2, h + 3), (h - 1, h + 2), (0, h), (3, 5)]:
        vol = p.backproject_packed(Qp, view_begin=b, view_count=e - b).cpu().numpy()
        ref = oracle.backproject(g, Qd, view_begin=b, view_count=e - b)
        tol = 1e-5 if dtype == "float32" else 1e-3   # FP16: interpolation in half2
        assert rel_l2(vol, ref) <= tol, (b, e, rel_l2(vol, ref))
    whole = p.backproject_packed(Qp)
    acc = torch.zeros_like(whole)
    for b, e in [(0, 3), (3, h + 4), (h + 4, g.np)]:
        p.backproject_packed(Qp, acc, view_begin=b, view_count=e - b)
    # FP16 taps are interpolated in half2 with du, dv rounded to FP16: paired and
    # single launches form du, dv from different (equal in exact arithmetic) terms
    tol = 2e-6 if dtype == "float32" else 5e-4
    assert float((acc - whole).abs().max()) <= tol * float(whole.abs().max())
    assert p.device_status() == 0


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("chunk", [2, 7, 64])
def test_host_streaming_packed(dtype, chunk):
    """The streaming call packs each chunk on the device (pair chunks first with
    view pairing): the same sum as the device packed call for whole and
    partial ranges, pairing on and off."""
    g = scaled_geometry(64, 96, 40, nz=24)
    p = B.Plan(g)
    gen = torch.Generator(device="cuda").manual_seed(6)
    Q = torch.randn((g.np, g.nv, g.nu), device="cuda", generator=gen).to(dtype)
    Qp = p.pack(Q)
    Qh = Q.cpu().pin_memory()
    for pairing in (True, False):
        p.set_view_pairing(pairing)
        for b, n in [(0, g.np), (3, 30), (15, 25), (0, 21)]:
            ref = p.backproject_packed(Qp, view_begin=b, view_count=n)
            vol = torch.zeros_like(ref)
            p.backproject_host(Qh, vol, chunk_views=chunk, view_begin=b, view_count=n)
            torch.cuda.synchronize()
            tol = 2e-6 if dtype == torch.float32 else 5e-4
            assert float((vol - ref).abs().max()) <= tol * float(ref.abs().max()), (pairing, b, n, chunk)
    assert p.device_status() == 0


def test_packed_path_refuses_what_it_does_not_cover():
    g = circular(12, 64, 48, 1.5, 1.5, 37, 29, 21, 1.0, off_u=0.6, off_v=0.35, vol_off_z=1.3)
    p = B.Plan(g)
    assert p.packed_info(torch.float32)["path"] == 0
    with pytest.raises(B.IfdkError) as e:
        B.ifdk_packed_size(p.handle, B.IFDK_F32)
    assert e.value.code == B.IFDK_ERR_UNSUPPORTED
    Q = torch.zeros((g.np, g.nv, g.nu), device="cuda")
    vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
    with pytest.raises(B.IfdkError) as e:
        B.ifdk_backproject_packed(p.handle, Q, B.IFDK_F32, 0, g.np, vol)
    assert e.value.code == B.IFDK_ERR_UNSUPPORTED
    with pytest.raises(B.IfdkError) as e:
        B.ifdk_pack_views(p.handle, Q, B.IFDK_F32, g.np, vol)
    assert e.value.code == B.IFDK_ERR_UNSUPPORTED
    # the standard kernels serve it; bad arguments of the packed calls are caught first
    g2 = GEOMS["fdk64"]
    p2 = B.Plan(g2)
    Qp = torch.zeros(p2.packed_shape(torch.float32), device="cuda")
    v2 = torch.zeros((g2.nx, g2.ny, g2.nz), device="cuda")
    with pytest.raises(B.IfdkError) as e:
        B.ifdk_backproject_packed(p2.handle, Qp, B.IFDK_F32, 5, g2.np, v2)
    assert e.value.code == B.IFDK_ERR_INVALID
    raw = torch.zeros(Qp.numel() + 4, device="cuda")
    with pytest.raises(B.IfdkError) as e:
        B.ifdk_backproject_packed(p2.handle, raw.data_ptr() + 4, B.IFDK_F32, 0, g2.np, v2)
    assert e.value.code == B.IFDK_ERR_ALIGNMENT
    assert float(v2.abs().max()) == 0.0


def test_fdk_host_pipeline_matches_device_fdk():
    """The pipelined host-to-host FDK (copies of one step overlapping its
    neighbours' computation) returns the device FDK's volume."""
    from paper_1909_02724_gb300.api import fdk, fdk_host_pipeline
    g = GEOMS["ragged"]
    E = torch.from_numpy(phantom_E(g)).cuda()
    p = B.Plan(g)
    ref = fdk(p, E)
    E_host = E.cpu().pin_memory()
    vol_host = torch.empty((g.nx, g.ny, g.nz), pin_memory=True)
    E2 = [torch.empty_like(E), torch.empty_like(E)]
    vol2 = [torch.empty_like(ref), torch.empty_like(ref)]
    Q = torch.empty_like(E)
    Qp = torch.empty(p.packed_shape(torch.float32), device="cuda")
    for n in (1, 3):
        vol_host.zero_()
        fdk_host_pipeline(p, E_host, vol_host, E2, Q, vol2, Qp_dev=Qp, n_steps=n)
        assert torch.equal(vol_host, ref.cpu())
    assert p.device_status() == 0


@pytest.mark.parametrize("name", ["fdk64", "ragged", "odd_nz_odd_ny", "magnified_odd_np"])
@pytest.mark.parametrize("dtype", ["float32", "float16"])
def test_view_split_small_volumes(name, dtype):
    """Small volumes split the view range over grid layers (partial volumes summed
    in part order): reproducible, accumulating, equal to the unsplit launch up to
    the grouping of the FP32 sums, and within the oracle tolerances."""
    g = GEOMS[name]
    p = B.Plan(g)
    E = phantom_E(g)
    Q = p.filter(torch.from_numpy(E).cuda(), dtype=TDT[dtype])
    Qp = p.pack(Q)
    S = p.view_split(TDT[dtype])
    assert S >= 2, S                      # these grids cover less than half a wave
    vol = p.backproject_packed(Qp)
    assert torch.equal(vol, p.backproject_packed(Qp))
    ones = torch.ones_like(vol)
    p.backproject_packed(Qp, ones)
    assert max_rel((ones - 1).cpu().numpy(), vol.cpu().numpy()) <= 1e-6
    # a view range that is neither the whole scan nor whole pairs
    part = p.backproject_packed(Qp, view_begin=1, view_count=g.np - 3)
    p.set_view_split(3)
    assert 2 <= p.view_split(TDT[dtype]) <= 3
    p.set_view_split(1)
    assert p.view_split(TDT[dtype]) == 1
    whole = p.backproject_packed(Qp).cpu().numpy()
    whole_part = p.backproject_packed(Qp, view_begin=1, view_count=g.np - 3).cpu().numpy()
    v = vol.cpu().numpy()
    assert max_rel(v, whole) <= 2e-6
    assert max_rel(part.cpu().numpy(), whole_part) <= 2e-6
    if dtype == "float32":
        Qh = Q.cpu().double().numpy()
        assert rel_l2(v, oracle.backproject(g, Qh)) <= 1e-5
        assert rel_l2(part.cpu().numpy(), oracle.backproject(g, Qh, 1, g.np - 3)) <= 1e-5
    assert p.device_status() == 0


def test_view_split_off_for_volumes_that_fill_the_gpu():
    g = scaled_geometry(256, 64, 16)
    p = B.Plan(g)
    for dt in TDT.values():
        assert p.view_split(dt) == 1
    with pytest.raises(B.IfdkError):
        p.set_view_split(-1)
