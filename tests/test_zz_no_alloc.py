"""ecc_compute_noalloc -- the entry point for callers that cannot allocate.

Some callers must not allocate device memory once they run: a real-time
pipeline whose device budget is fixed at start-up, or code running inside
another framework's memory pool.  ecc_compute_noalloc serves them from one
fixed scratch array of the library instead of a plan's cudaMalloc'd
workspace.  These tests call it through the C ABI and check it against the
plan-based ecc_compute and against the CPU oracle on the same images, exactly
(integer results), on two calls in a row, so a second call cannot inherit the
first call's scratch contents unnoticed.

The file name sorts last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _ecc():
    import paper_2203_09087_gb300 as ecc
    return ecc


def _noalloc_cabi(img_t, lo, hi, mode, out, flags=0):
    """Call the C entry point directly (no binding-side allocation)."""
    ecc = _ecc()
    lib = ecc.library()
    d = ecc._binding.image_desc(img_t)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ecc_compute_noalloc(ctypes.byref(d), lo, hi, mode, flags, ctypes.c_void_p(out.data_ptr()), None,
                                   stream)


def _with_plan(img_t, lo, hi, mode):
    ecc = _ecc()
    dt = "u8" if img_t.dtype == torch.uint8 else "u16"
    plan = ecc.ecc_plan(dt, lo, hi, complex_mode=mode, max_voxels=img_t.numel())
    out = ecc.ecc_compute(plan, img_t)
    ecc.ecc_status_get(plan)
    return out.cpu().numpy()


def _images(kind):
    rng = np.random.default_rng(17)
    if kind == "3d_u8_aligned":       # TMA-staged bit-sliced kernel
        a = rng.integers(0, 256, size=(40, 70, 96), dtype=np.uint8)
        b = rng.integers(0, 4, size=(33, 50, 64), dtype=np.uint8)
        return a, b, 0, 255
    if kind == "3d_u8_unaligned":     # the batch kernel, its work list in the scratch
        a = rng.integers(0, 256, size=(21, 33, 45), dtype=np.uint8)
        b = rng.integers(0, 9, size=(5, 60, 77), dtype=np.uint8)
        return a, b, 0, 255
    if kind == "3d_u16_unaligned":    # the same with 16-bit rows of 2 x 37 bytes, a narrow range
        a = rng.integers(300, 700, size=(14, 29, 37)).astype(np.uint16)
        b = rng.integers(300, 304, size=(40, 7, 37)).astype(np.uint16)
        return a, b, 300, 699
    if kind == "2d_u8":
        a = rng.integers(0, 256, size=(300, 517), dtype=np.uint8)
        b = rng.integers(0, 3, size=(64, 2000), dtype=np.uint8)
        return a, b, 0, 255
    if kind == "3d_u16_full_range":   # the largest scratch use: 65536 levels
        a = rng.integers(0, 65536, size=(16, 40, 64)).astype(np.uint16)
        b = rng.integers(60000, 60010, size=(24, 30, 32)).astype(np.uint16)
        return a, b, 0, 65535
    raise ValueError(kind)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kind", ["3d_u8_aligned", "3d_u8_unaligned", "2d_u8", "3d_u16_full_range",
                                  "3d_u16_unaligned"])
def test_two_calls_in_a_row_match_ecc_compute(kind, mode):
    a, b, lo, hi = _images(kind)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    n = hi - lo + 1
    out_a = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    out_b = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    assert _noalloc_cabi(ta, lo, hi, mode, out_a) == 0, _ecc().ecc_last_error()
    assert _noalloc_cabi(tb, lo, hi, mode, out_b) == 0, _ecc().ecc_last_error()
    assert np.array_equal(out_a.cpu().numpy(), _with_plan(ta, lo, hi, mode))
    assert np.array_equal(out_b.cpu().numpy(), _with_plan(tb, lo, hi, mode))
    om = oracle.VERTEX if mode == 0 else oracle.TOPCELL
    assert np.array_equal(out_a.cpu().numpy(), oracle.ecc(a, lo, hi, om))
    assert np.array_equal(out_b.cpu().numpy(), oracle.ecc(b, lo, hi, om))


def test_wrapper_with_vcec_on_a_side_stream():
    """The Python wrapper, a VCEC output and a non-default stream: ECC and
    VCEC equal the plan path's and the oracle's."""
    ecc = _ecc()
    rng = np.random.default_rng(23)
    img = rng.integers(0, 256, size=(18, 45, 80), dtype=np.uint8)
    t = torch.from_numpy(img).cuda()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        out = torch.full((256,), -1, dtype=torch.int64, device="cuda")
        vcec = torch.full((256,), -1, dtype=torch.int64, device="cuda")
        ecc.ecc_compute_noalloc(t, 0, 255, 0, out=out, vcec_out=vcec, stream=side)
    side.synchronize()
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=img.size)
    p_vcec = torch.empty(256, dtype=torch.int64, device="cuda")
    p_out = ecc.ecc_compute(plan, t, vcec_out=p_vcec)
    ecc.ecc_status_get(plan)
    assert np.array_equal(out.cpu().numpy(), p_out.cpu().numpy())
    assert np.array_equal(vcec.cpu().numpy(), p_vcec.cpu().numpy())
    want_v = oracle.vcec(img, 0, 255)
    assert np.array_equal(vcec.cpu().numpy(), want_v)
    assert np.array_equal(out.cpu().numpy(), np.cumsum(want_v))


def test_rejects_bad_requests_with_a_clear_error():
    ecc = _ecc()
    t = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    out = torch.empty(256, dtype=torch.int64, device="cuda")
    assert _noalloc_cabi(t, 10, 5, 0, out) == ecc.ECC_E_INVALID
    assert "gray range" in ecc.ecc_last_error()
    bad = torch.full((8, 8), 200, dtype=torch.uint8, device="cuda")
    bad[3, 3] = 7
    assert _noalloc_cabi(bad, 0, 100, 0, out) == ecc.ECC_E_RANGE
    # the scratch is cleared per call: a good call right after the failed one is exact
    good = torch.from_numpy(np.random.default_rng(3).integers(0, 101, size=(30, 40), dtype=np.uint8)).cuda()
    out2 = torch.empty(101, dtype=torch.int64, device="cuda")
    assert _noalloc_cabi(good, 0, 100, 0, out2) == 0
    assert np.array_equal(out2.cpu().numpy(), _with_plan(good, 0, 100, 0))
