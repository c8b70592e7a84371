"""GPU parity of the output stage (ifdk_volume_slices) against the oracle.

Bit-exact: the FP32 copy is exact and the 16-bit outputs are one rounding to
nearest even on both sides.  Ragged sizes span several 64 x 64 tiles with
partial tiles in i and k; the full-size case is the fdk512 volume in the
launch the benchmark times."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.phantom import scaled_geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_02724_gb300.build import build
    build()


def host_bits(t):
    """The output's bit patterns (bf16 as uint16), f32 / f16 as numpy arrays."""
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def seeded_volume(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((nx, ny, nz)).astype(np.float32) * np.float32(3.0)
    v.reshape(-1)[::97] = 0.0           # exact zeros and a few large values
    v.reshape(-1)[::131] *= np.float32(1e4)
    return v


@pytest.mark.parametrize("dtype", list(DT))
@pytest.mark.parametrize("kb,kc", [(0, None), (5, 60), (130, 1), (64, 67), (7, 0)])
def test_slices_bit_exact_ragged(dtype, kb, kc):
    from paper_1909_02724_gb300.binding import Plan
    g = scaled_geometry(70, 32, 4, nz=131).with_(ny=3)
    vol_h = seeded_volume(g.nx, g.ny, g.nz, 11)
    plan = Plan(g)
    vol = torch.from_numpy(vol_h).cuda()
    n = g.nz - kb if kc is None else kc
    out = torch.full((n, g.ny, g.nx), 7.0, dtype=DT[dtype], device="cuda")
    plan.slices(vol, out, k_begin=kb, k_count=n)
    torch.cuda.synchronize()
    ref = oracle.volume_slices(vol_h, kb, n, dtype)
    got = host_bits(out)
    assert got.shape == ref.shape
    assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_slices_fullsize_fdk512(dtype):
    from paper_1909_02724_gb300.binding import Plan
    g = scaled_geometry(512, 512, 512)
    vol_h = seeded_volume(g.nx, g.ny, g.nz, 12)
    plan = Plan(g)
    vol = torch.from_numpy(vol_h).cuda()
    out = plan.slices(vol, dtype=DT[dtype])
    torch.cuda.synchronize()
    got = host_bits(out)
    ref = oracle.volume_slices(vol_h, 0, g.nz, dtype)
    assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))
    # a chunk of slices in the middle, as a streamed writer takes them
    part = plan.slices(vol, dtype=DT[dtype], k_begin=200, k_count=37)
    assert np.array_equal(host_bits(part).view(np.uint8), ref[200:237].view(np.uint8))


def test_slices_rejects_bad_arguments():
    from paper_1909_02724_gb300.binding import IFDK_ERR_ALIGNMENT, IFDK_ERR_INVALID, IfdkError, Plan, ifdk_volume_slices
    g = scaled_geometry(16, 16, 4, nz=8)
    plan = Plan(g)
    vol = torch.zeros((g.nx, g.ny, g.nz), device="cuda")
    out = torch.zeros((g.nz + 4) * g.ny * g.nx, device="cuda")
    for kb, kc in ((-1, 1), (0, 9), (5, 4), (2, -1)):
        with pytest.raises(IfdkError) as e:
            ifdk_volume_slices(plan.handle, vol, out, 0, kb, kc)
        assert e.value.code == IFDK_ERR_INVALID
    with pytest.raises(IfdkError) as e:
        ifdk_volume_slices(plan.handle, vol, out, 3, 0, 1)
    assert e.value.code == IFDK_ERR_INVALID
    with pytest.raises(IfdkError) as e:
        ifdk_volume_slices(plan.handle, vol, int(out.data_ptr()) + 4, 0, 0, 1)
    assert e.value.code == IFDK_ERR_ALIGNMENT
    ifdk_volume_slices(plan.handle, vol, out, 0, 3, 0)      # empty range: nothing to do
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0


@pytest.mark.parametrize("dtype,chunk", [("f32", 7), ("f16", 64), ("bf16", 1), ("f32", 500)])
def test_slices_to_host_in_chunks(dtype, chunk):
    from paper_1909_02724_gb300.api import volume_slices_host
    from paper_1909_02724_gb300.binding import Plan
    g = scaled_geometry(70, 32, 4, nz=131).with_(ny=3)
    vol_h = seeded_volume(g.nx, g.ny, g.nz, 13)
    plan = Plan(g)
    vol = torch.from_numpy(vol_h).cuda()
    out = torch.empty((g.nz, g.ny, g.nx), dtype=DT[dtype], pin_memory=True)
    volume_slices_host(plan, vol, out, chunk_slices=chunk)
    got = out.view(torch.int16).numpy().view(np.uint16) if dtype == "bf16" else out.numpy()
    ref = oracle.volume_slices(vol_h, 0, g.nz, dtype)
    assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))
