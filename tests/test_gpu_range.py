"""The gray-range contract on every kernel path (-m gpu).

A plan over [lo, hi] reports ECC_E_RANGE when the image holds a value
outside the range, whether or not that voxel changes any ECC value: the
checked voxels below all have a signed cell count of zero (a bright voxel on
the image boundary, whose star is a cone, and the regular points of a ramp,
Sec. 2.3), so only a comparison of every voxel with the bounds can see them.
ECC_FLAG_NO_RANGE_CHECK skips that comparison; the offending voxels still
never reach the histogram, so above-range values leave the ECC at levels
lo..hi equal to the full-range oracle's.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def ecc_mod():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2203_09087_gb300 as ecc
    return ecc


def ramp(shape, dtype, scale):
    """Values scale * x along the fastest axis, constant elsewhere."""
    x = np.arange(shape[-1], dtype=np.int64) * scale
    return np.broadcast_to(x, shape).astype(dtype).copy()


def bright_boundary(shape, dtype, value):
    """A constant image with one voxel on a boundary face set to `value`."""
    img = np.full(shape, 10, dtype=dtype)
    idx = (0,) + tuple(n // 2 for n in shape[1:])
    img[idx] = value
    return img


def _expect_range(ecc, plan, fn):
    fn()
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_status_get(plan)
    assert ei.value.status == ecc.ECC_E_RANGE


CASES = [
    # (name, image, lo, hi)
    ("2d ramp", ramp((40, 200), np.uint8, 1), 0, 150),
    ("2d boundary", bright_boundary((30, 77), np.uint8, 200), 0, 100),
    ("3d aligned ramp", ramp((12, 40, 64), np.uint8, 3), 0, 120),
    ("3d aligned boundary", bright_boundary((9, 33, 48), np.uint8, 250), 0, 200),
    ("3d unaligned ramp", ramp((10, 23, 70), np.uint8, 3), 0, 120),
    ("3d u16 sub-range", ramp((6, 31, 40), np.uint16, 700), 500, 20000),
]


@pytest.mark.parametrize("name,img,lo,hi", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kernel", ["default", "direct"])
def test_every_voxel_is_range_checked(name, img, lo, hi, kernel):
    ecc = ecc_mod()
    flags = ecc.ECC_FLAG_KERNEL_DIRECT if kernel == "direct" else 0
    dt = "u8" if img.dtype == np.uint8 else "u16"
    plan = ecc.ecc_plan(dt, lo, hi, flags=flags, max_voxels=img.size)
    t = torch.from_numpy(img).cuda()
    _expect_range(ecc, plan, lambda: ecc.ecc_compute(plan, t))
    # the same plan computes an in-range image correctly right after
    ok = np.clip(img, lo, hi).astype(img.dtype)
    got = ecc.ecc_compute(plan, torch.from_numpy(ok).cuda())
    assert ecc.ecc_status_get(plan) == ecc.ECC_OK
    assert np.array_equal(got.cpu().numpy(), oracle.ecc(ok, lo, hi, oracle.VERTEX))


def test_top_cell_complex_is_range_checked():
    ecc = ecc_mod()
    img = ramp((10, 35, 48), np.uint8, 4)
    plan = ecc.ecc_plan("u8", 0, 100, complex_mode=ecc.ECC_TOPCELL_MIN, max_voxels=img.size)
    _expect_range(ecc, plan, lambda: ecc.ecc_compute(plan, torch.from_numpy(img).cuda()))


def test_below_lo_is_reported():
    ecc = ecc_mod()
    img = ramp((8, 33, 64), np.uint8, 2) + 40
    img[3, 5, 0] = 12          # below lo, its neighbours too
    img[3, 5, 1] = 11
    plan = ecc.ecc_plan("u8", 20, 255, max_voxels=img.size)
    _expect_range(ecc, plan, lambda: ecc.ecc_compute(plan, torch.from_numpy(img).cuda()))


def test_full_range_plan_checks_nothing_and_is_exact():
    ecc = ecc_mod()
    img = ramp((12, 40, 64), np.uint8, 4)
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=img.size)
    got = ecc.ecc_compute(plan, torch.from_numpy(img).cuda())
    assert ecc.ecc_status_get(plan) == ecc.ECC_OK
    assert np.array_equal(got.cpu().numpy(), oracle.ecc(img, 0, 255, oracle.VERTEX))


@pytest.mark.parametrize("shape", [(12, 40, 64), (10, 23, 70), (40, 200)])
def test_no_range_check_keeps_offenders_out_of_the_histogram(shape):
    """Above-range voxels with the per-voxel check off: not reported (their
    counts are zero), and the ECC over lo..hi equals the oracle's over the
    full range, truncated (cells entering above hi are in no sublevel set of
    a level <= hi)."""
    ecc = ecc_mod()
    img = ramp(shape, np.uint8, 1 if len(shape) == 2 else 3)
    lo, hi = 0, 120
    plan = ecc.ecc_plan("u8", lo, hi, flags=ecc.ECC_FLAG_NO_RANGE_CHECK, max_voxels=img.size)
    got = ecc.ecc_compute(plan, torch.from_numpy(img).cuda())
    assert ecc.ecc_status_get(plan) == ecc.ECC_OK
    full = oracle.ecc(img, 0, 255, oracle.VERTEX)
    assert np.array_equal(got.cpu().numpy(), full[lo:hi + 1])


def test_batch_is_range_checked():
    ecc = ecc_mod()
    good = [torch.from_numpy(np.full((20, 30), 7, np.uint8)).cuda(),
            torch.from_numpy(np.full((9, 12, 40), 9, np.uint8)).cuda()]
    bad2 = torch.from_numpy(ramp((25, 90), np.uint8, 2)).cuda()
    bad3 = torch.from_numpy(ramp((7, 20, 50), np.uint8, 3)).cuda()
    for bad in (bad2, bad3):
        plan = ecc.ecc_plan("u8", 0, 100, max_images=3, max_voxels=1 << 20)
        _expect_range(ecc, plan, lambda: ecc.ecc_compute_batch(plan, good + [bad]))
        out = ecc.ecc_compute_batch(plan, good)
        assert ecc.ecc_status_get(plan) == ecc.ECC_OK
        for i, t in enumerate(good):
            assert np.array_equal(out[i].cpu().numpy(), oracle.ecc(t.cpu().numpy(), 0, 100, oracle.VERTEX))


def test_nd_is_range_checked():
    ecc = ecc_mod()
    img = ramp((4, 5, 33, 40), np.uint8, 3)
    plan = ecc.ecc_plan("u8", 0, 90, max_voxels=img.size)
    _expect_range(ecc, plan, lambda: ecc.ecc_compute_nd(plan, torch.from_numpy(img).cuda()))


def test_host_streaming_is_range_checked():
    ecc = ecc_mod()
    img = ramp((14, 40, 64), np.uint8, 3)
    plan = ecc.ecc_plan("u8", 0, 120, max_voxels=img.size)
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_compute_stream(plan, img, device_budget_bytes=1 << 16)
    assert ei.value.status == ecc.ECC_E_RANGE
