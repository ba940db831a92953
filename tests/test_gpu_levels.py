"""GPU parity of float32 images at given thresholds (ecc_compute_levels,
Eq. 1 with the t_i given) against the oracle's float path, which counts
every cell at the first level at or above its float value.  Bit-exact."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MODES = {"vertex": 0, "topcell": 1}


def ecc_mod():
    import paper_2203_09087_gb300 as ecc
    return ecc


def _run(img, levels, mode, dtype="u16", hi=None):
    ecc = ecc_mod()
    m = len(levels)
    nvox = img.size if isinstance(img, np.ndarray) else img.numel()
    plan = ecc.ecc_plan(dtype, 0, hi if hi is not None else m, complex_mode=MODES[mode], max_voxels=nvox)
    lv = torch.tensor(np.asarray(levels, np.float32), device="cuda")
    t = torch.from_numpy(np.ascontiguousarray(img)).cuda() if isinstance(img, np.ndarray) else img
    out = ecc.ecc_compute_levels(plan, t, lv)
    ecc.ecc_status_get(plan)
    return out.cpu().numpy()


def _rand_img(rng, shape):
    vals = np.array([-np.inf, -1.5, -0.25, 0.0, 0.5, 0.5000001, 2.0, 3.75, np.inf, np.nan], np.float32)
    return vals[rng.integers(0, vals.size, size=shape)]


@pytest.mark.parametrize("mode", list(MODES))
def test_small_images_with_ties_nan_inf(mode):
    rng = np.random.default_rng(41)
    cand = np.array([-2.0, -1.5, -0.3, 0.0, 0.4, 0.5, 0.5000001, 1.0, 2.0, 3.75, 5.0], np.float32)
    for shape in [(1, 1), (7, 5), (33, 70), (3, 4, 5), (9, 40, 70), (1, 31, 33)]:
        img = _rand_img(rng, shape)
        levels = np.sort(rng.choice(cand, size=int(rng.integers(1, 12))))
        want = oracle.ecc_levels(img, levels.astype(np.float64), mode)
        for dt in ("u8", "u16"):
            assert np.array_equal(_run(img, levels, mode, dt), want), (shape, dt)


@pytest.mark.parametrize("mode", list(MODES))
def test_smooth_float_volume_many_levels(mode):
    import synth
    g = torch.Generator().manual_seed(42)
    f = synth.smooth(torch.randn((48, 90, 130), generator=g), 2.0).numpy().astype(np.float32)
    levels = np.quantile(f, np.linspace(0.0, 1.0, 300)).astype(np.float32)   # 300 levels: u16 plan
    want = oracle.ecc_levels(f, levels.astype(np.float64), mode, threads=8)
    assert np.array_equal(_run(f, levels, mode, "u16"), want)
    lv8 = levels[::2][:200]
    want8 = oracle.ecc_levels(f, lv8.astype(np.float64), mode, threads=8)
    assert np.array_equal(_run(f, lv8, mode, "u8"), want8)


def test_integer_valued_floats_equal_the_integer_path():
    ecc = ecc_mod()
    rng = np.random.default_rng(43)
    img = rng.integers(0, 256, size=(40, 64, 96)).astype(np.uint8)
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=img.size)
    want = ecc.ecc_compute(plan, torch.from_numpy(img).cuda()).cpu().numpy()
    got = _run(img.astype(np.float32), np.arange(255, dtype=np.float32), "vertex", "u8", hi=255)
    assert np.array_equal(got, want[:255])


def test_many_levels_in_global_memory_and_pitched_view():
    rng = np.random.default_rng(44)
    base = rng.normal(size=(20, 60, 90)).astype(np.float32)
    sub = torch.from_numpy(base).cuda()[3:18, 5:55, 7:88]       # pitched device view
    levels = np.sort(rng.normal(size=20000)).astype(np.float32)  # beyond the shared-memory limit
    want = oracle.ecc_levels(np.ascontiguousarray(base[3:18, 5:55, 7:88]), levels.astype(np.float64), "vertex",
                             threads=8)
    assert np.array_equal(_run(sub, levels, "vertex", "u16"), want)


def test_errors():
    ecc = ecc_mod()
    img = torch.zeros((10, 12), dtype=torch.float32, device="cuda")
    lv = torch.tensor([0.0, 1.0, 2.0], device="cuda")
    with pytest.raises(ecc.EccError):
        ecc.ecc_compute_levels(ecc.ecc_plan("u16", 1, 100), img, lv)     # lo must be 0
    with pytest.raises(ecc.EccError):
        ecc.ecc_compute_levels(ecc.ecc_plan("u16", 0, 2), img, lv)       # hi must be >= m
    plan = ecc.ecc_plan("u16", 0, 3, max_voxels=img.numel())
    bad = torch.tensor([0.0, 2.0, 1.0], device="cuda")
    ecc.ecc_compute_levels(plan, img, bad)
    with pytest.raises(ecc.EccError) as e:
        ecc.ecc_status_get(plan)
    assert e.value.status == ecc.ECC_E_INVALID
    out = ecc.ecc_compute_levels(plan, img, lv)                          # usable afterwards
    ecc.ecc_status_get(plan)
    assert out.cpu().tolist() == [1, 1, 1]
