"""GPU parity of the out-of-core path (ecc_compute_stream, Sec. 3.4): host
images cut along dims[0] into chunks with a one-slab collar, streamed
through a ring of three device buffers under a byte budget.  Every result
is compared bit-exactly with the CPU oracle (or, at full size, with the
device-resident path that the other tests pin to the oracle)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MODES = {"vertex": 0, "topcell": 1}


def ecc_mod():
    import paper_2203_09087_gb300 as ecc
    return ecc


def budget_for(shape, itemsize, planes):
    """Device budget that gives chunks of `planes` outer slabs (rows padded to 16 bytes)."""
    row = -(-shape[-1] * itemsize // 16) * 16
    slab = row * (shape[1] if len(shape) == 3 else 1)
    per_buf = -(-(planes + 2) * slab // 256) * 256
    assert per_buf < (planes + 3) * slab
    return 3 * per_buf


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("planes", [1, 2, 5, 1000])
def test_stream_3d_u8(mode, planes):
    import synth
    ecc = ecc_mod()
    img = synth.smoothed_field((37, 61, 130), 2.0, np.uint8, seed=11, device="cpu").numpy()
    plan = ecc.ecc_plan("u8", 0, 255, complex_mode=MODES[mode], max_voxels=img.size)
    got = ecc.ecc_compute_stream(plan, img, budget_for(img.shape, 1, planes))
    assert np.array_equal(got, oracle.ecc(img, 0, 255, mode))


@pytest.mark.parametrize("planes", [1, 3, 64])
def test_stream_2d_rows(planes):
    rng = np.random.default_rng(12)
    ecc = ecc_mod()
    img = rng.integers(0, 7, size=(333, 517)).astype(np.uint8)   # plateaus: many ties across chunk cuts
    for mode in MODES:
        plan = ecc.ecc_plan("u8", 0, 255, complex_mode=MODES[mode], max_voxels=img.size)
        got = ecc.ecc_compute_stream(plan, img, budget_for(img.shape, 1, planes))
        assert np.array_equal(got, oracle.ecc(img, 0, 255, mode))


def test_stream_u16_pitched_and_subrange():
    rng = np.random.default_rng(13)
    ecc = ecc_mod()
    base = rng.integers(100, 1100, size=(23, 40, 77)).astype(np.uint16)
    sub = base[2:21, 3:37, 5:70]                 # pitched host view: rows and slices not contiguous
    plan = ecc.ecc_plan("u16", 100, 1099, max_voxels=sub.size)
    got = ecc.ecc_compute_stream(plan, sub, budget_for(sub.shape, 2, 2))
    assert np.array_equal(got, oracle.ecc(np.ascontiguousarray(sub), 100, 1099, "vertex"))


def test_stream_larger_than_plan_and_repeated():
    """The image may exceed the plan's max_voxels; calls leave the plan clean."""
    rng = np.random.default_rng(14)
    ecc = ecc_mod()
    img = rng.integers(0, 256, size=(50, 48, 64)).astype(np.uint8)
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=1000)
    want = oracle.ecc(img, 0, 255, "vertex")
    for planes in (1, 4):
        assert np.array_equal(ecc.ecc_compute_stream(plan, img, budget_for(img.shape, 1, planes)), want)
    with pytest.raises(ecc.EccError):
        ecc.ecc_compute(plan, torch.from_numpy(img).cuda())   # the device path keeps its limit


def test_stream_budget_too_small_and_range_error():
    ecc = ecc_mod()
    img = np.zeros((10, 20, 30), np.uint8)
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=img.size)
    with pytest.raises(ecc.EccError) as e:
        ecc.ecc_compute_stream(plan, img, 3 * 2 * 20 * 32)   # two slabs per buffer
    assert e.value.status == ecc.ECC_E_INVALID
    plan2 = ecc.ecc_plan("u8", 0, 9, max_voxels=img.size)
    bad = img.copy()
    bad[5, 5, 5] = 200
    with pytest.raises(ecc.EccError) as e:
        ecc.ecc_compute_stream(plan2, bad, budget_for(bad.shape, 1, 2))
    assert e.value.status == ecc.ECC_E_RANGE
    # the plan is usable after the error
    assert np.array_equal(ecc.ecc_compute_stream(plan2, img, budget_for(img.shape, 1, 2)),
                          oracle.ecc(img, 0, 9, "vertex"))


def test_stream_full_size_512cube_against_device_path():
    """The 512^3 uint8 benchmark volume streamed through 64 MiB of chunk
    buffers equals the device-resident ECC."""
    import synth
    ecc = ecc_mod()
    vol = synth.smooth_3d_512(device="cuda")
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=vol.numel())
    want = ecc.ecc_compute(plan, vol).cpu().numpy()
    host = vol.cpu().numpy()
    got = ecc.ecc_compute_stream(plan, host, 64 << 20)
    assert np.array_equal(got, want)
    assert got[-1] == 1


def test_host_path_many_chunks_against_device_path():
    """ecc_compute_host with more chunks than the plan's chunk events (157 MB
    in 8 MiB chunks) equals the device-resident ECC."""
    import synth
    ecc = ecc_mod()
    vol = synth.smooth_3d_512(device="cuda", shape=(600, 512, 512))
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=vol.numel())
    want = ecc.ecc_compute(plan, vol).cpu().numpy()
    host = vol.cpu().pin_memory().numpy()
    assert np.array_equal(ecc.ecc_compute_host(plan, host), want)
