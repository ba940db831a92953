"""GPU parity of the iterated ECC + smoothing pipeline (the paper's GPU-only
pipeline, Sec. 4, Table 2) against the oracle: the ECC after every round
and the final smoothed image are compared bit for bit."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MODES = {"vertex": 0, "topcell": 1}


def ecc_mod():
    import paper_2203_09087_gb300 as ecc
    return ecc


def _levels(img, m):
    return np.linspace(float(img.min()), float(img.max()), m).astype(np.float32)


def _run(img_t, taps, iters, levels, mode):
    ecc = ecc_mod()
    m = len(levels)
    plan = ecc.ecc_plan("u16", 0, m, complex_mode=MODES[mode], max_voxels=img_t.numel())
    out = ecc.ecc_pipeline_gaussian(plan, img_t, taps, iters, torch.from_numpy(levels).cuda())
    ecc.ecc_status_get(plan)
    return out.cpu().numpy()


@pytest.mark.parametrize("mode", list(MODES))
def test_2d_rounds_and_final_image_bit_exact(mode):
    ecc = ecc_mod()
    rng = np.random.default_rng(61)
    img = rng.normal(size=(96, 130)).astype(np.float32)
    taps = ecc.gaussian_taps(2.0)
    levels = _levels(img, 64)
    t = torch.from_numpy(img).cuda()
    got = _run(t, taps, 6, levels, mode)
    want, final = oracle.gaussian_pipeline(img, taps, levels.astype(np.float64), 6, mode)
    assert np.array_equal(got, want)
    assert np.array_equal(t.cpu().numpy(), final)


def test_3d_pitched_view_and_untouched_gaps():
    ecc = ecc_mod()
    rng = np.random.default_rng(62)
    base = rng.normal(size=(14, 30, 41)).astype(np.float32)
    parent = torch.from_numpy(base.copy()).cuda()
    view = parent[2:12, 3:27, 4:37]                 # rows and slices pitched
    sub = np.ascontiguousarray(base[2:12, 3:27, 4:37])
    taps = ecc.gaussian_taps(1.3, radius=4)
    levels = _levels(sub, 40)
    got = _run(view, taps, 3, levels, "vertex")
    want, final = oracle.gaussian_pipeline(sub, taps, levels.astype(np.float64), 3, "vertex")
    assert np.array_equal(got, want)
    after = parent.cpu().numpy()
    assert np.array_equal(after[2:12, 3:27, 4:37], final)
    mask = np.ones(base.shape, bool)
    mask[2:12, 3:27, 4:37] = False
    assert np.array_equal(after[mask], base[mask])  # the rest of the parent is untouched


def test_zero_rounds_and_bad_taps():
    ecc = ecc_mod()
    img = torch.ones((8, 9), dtype=torch.float32, device="cuda")
    plan = ecc.ecc_plan("u16", 0, 4, max_voxels=img.numel())
    lv = torch.tensor([0.0, 1.0, 2.0, 3.0], device="cuda")
    out = ecc.ecc_pipeline_gaussian(plan, img, ecc.gaussian_taps(1.0), 0, lv)
    assert out.numel() == 0 and torch.equal(img, torch.ones_like(img))
    with pytest.raises(ecc.EccError):
        ecc.ecc_pipeline_gaussian(plan, img, np.ones(4, np.float32) / 4, 1, lv)   # even tap count


def test_paper_size_1024_square_grf():
    """The paper's setting: a 1024^2 Gaussian random field, 13 taps, here 12
    rounds at 256 levels fixed from the initial range."""
    import synth
    ecc = ecc_mod()
    g = torch.Generator().manual_seed(63)
    img = synth.smooth(torch.randn((1024, 1024), generator=g), 3.0).numpy().astype(np.float32)
    taps = ecc.gaussian_taps(2.0)
    levels = _levels(img, 256)
    t = torch.from_numpy(img).cuda()
    got = _run(t, taps, 12, levels, "vertex")
    want, final = oracle.gaussian_pipeline(img, taps, levels.astype(np.float64), 12, "vertex", threads=16)
    assert np.array_equal(got, want)
    assert np.array_equal(t.cpu().numpy(), final)


# ----------------------------------------------------------------------------
# 2D images with at most 255 levels take one fused kernel per round (tile read
# once: level search, bit-sliced cell count, both filter passes); the cases
# below cover its tile edges, halo widths, round parity and inputs.

@pytest.mark.parametrize("shape,iters,ntaps,m,mode", [
    ((96, 130), 5, 13, 64, "vertex"),      # odd rounds: result copied back from the scratch image
    ((121, 241), 4, 13, 255, "topcell"),   # one past a tile in both axes, the largest fused level count
    ((7, 5), 3, 13, 20, "vertex"),         # smaller than the filter: reflection wraps several times
    ((64, 120), 2, 1, 30, "vertex"),       # one tap: the filter is the identity, halo of one pixel
    ((200, 333), 3, 33, 100, "topcell"),   # the widest filter, ragged tiles
    ((1, 300), 2, 5, 17, "vertex"),        # one row
    ((300, 1), 2, 5, 17, "topcell"),       # one column
    # enough tiles of 64 rows to fill the GPU twice: the 64-row tile (the
    # smaller images above take 32-row tiles), ragged in both axes
    ((1350, 2530), 2, 13, 255, "vertex"),
    ((1350, 2530), 3, 7, 90, "topcell"),
])
def test_fused_rounds_bit_exact(shape, iters, ntaps, m, mode):
    ecc = ecc_mod()
    rng = np.random.default_rng(70 + ntaps + m)
    img = rng.normal(size=shape).astype(np.float32)
    r = ntaps // 2
    if ntaps == 1:
        taps = np.ones(1, np.float32)
    else:
        taps = ecc.gaussian_taps(max(1.0, r / 3.0), radius=r)
    levels = _levels(img, m)
    t = torch.from_numpy(img).cuda()
    got = _run(t, taps, iters, levels, mode)
    want, final = oracle.gaussian_pipeline(img, taps, levels.astype(np.float64), iters, mode)
    assert np.array_equal(got, want)
    assert np.array_equal(t.cpu().numpy(), final)


def test_fused_pitched_rows_and_special_values():
    """A view with pitched rows (the gaps untouched), NaN and infinities in
    the image, levels with ties."""
    ecc = ecc_mod()
    rng = np.random.default_rng(81)
    base = rng.normal(size=(150, 260)).astype(np.float32)
    base[10, 20] = np.nan
    base[40, 7] = np.inf
    base[99, 200] = -np.inf
    parent = torch.from_numpy(base.copy()).cuda()
    view = parent[5:140, 9:250]
    sub = np.ascontiguousarray(base[5:140, 9:250])
    taps = ecc.gaussian_taps(1.5, radius=4)
    levels = np.sort(np.concatenate([np.linspace(-2, 2, 40), [0.0, 0.0, 0.5]])).astype(np.float32)
    got = _run(view, taps, 3, levels, "vertex")
    want, final = oracle.gaussian_pipeline(sub, taps, levels.astype(np.float64), 3, "vertex")
    assert np.array_equal(got, want)
    after = parent.cpu().numpy()
    assert np.array_equal(after[5:140, 9:250], final, equal_nan=True)
    mask = np.ones(base.shape, bool)
    mask[5:140, 9:250] = False
    assert np.array_equal(after[mask], base[mask], equal_nan=True)


def test_fused_paper_size_1024_square_255_levels():
    """The paper's 1024^2 GRF with 13 taps through the fused kernel: 255
    levels (the fused path's limit), 11 rounds (captured as a graph)."""
    import synth
    ecc = ecc_mod()
    g = torch.Generator().manual_seed(64)
    img = synth.smooth(torch.randn((1024, 1024), generator=g), 3.0).numpy().astype(np.float32)
    taps = ecc.gaussian_taps(2.0)
    levels = _levels(img, 255)
    t = torch.from_numpy(img).cuda()
    got = _run(t, taps, 11, levels, "vertex")
    want, final = oracle.gaussian_pipeline(img, taps, levels.astype(np.float64), 11, "vertex", threads=16)
    assert np.array_equal(got, want)
    assert np.array_equal(t.cpu().numpy(), final)


def test_one_plan_pipeline_then_out_of_core_then_pipeline():
    """A plan that grows its out-of-core chunk buffers between two pipeline
    calls keeps its pipeline scratch image: both pipeline calls and the
    streamed ECC are exact."""
    ecc = ecc_mod()
    rng = np.random.default_rng(64)
    img = rng.normal(size=(200, 180)).astype(np.float32)
    taps = ecc.gaussian_taps(1.5)
    levels = _levels(img, 300)
    plan = ecc.ecc_plan("u16", 0, 300, max_voxels=1 << 22)
    lv = torch.from_numpy(levels).cuda()
    want, _ = oracle.gaussian_pipeline(img, taps, levels.astype(np.float64), 2, "vertex")
    t = torch.from_numpy(img.copy()).cuda()
    got = ecc.ecc_pipeline_gaussian(plan, t, taps, 2, lv)
    ecc.ecc_status_get(plan)
    assert np.array_equal(got.cpu().numpy(), want)
    vol = rng.integers(0, 301, size=(40, 64, 96)).astype(np.uint16)
    streamed = ecc.ecc_compute_stream(plan, vol, device_budget_bytes=1 << 20)
    assert np.array_equal(streamed, oracle.ecc(vol, 0, 300))
    t = torch.from_numpy(img.copy()).cuda()
    got = ecc.ecc_pipeline_gaussian(plan, t, taps, 2, lv)
    ecc.ecc_status_get(plan)
    assert np.array_equal(got.cpu().numpy(), want)
