"""Pins of the oracle's float32 threshold path (oracle.ecc_levels: ECC_i =
chi(K_{<= t_i}) at given ascending levels, Eq. 1), against things other
than itself: the naive thresholding method on tiny images (with ties, NaN
and infinities), beta0 - beta1 by flood fill in 2D, the pinned integer
oracle on integer-valued data, invariance under strictly increasing maps
of values and levels together, and planted mistakes that must be caught."""
from pathlib import Path

import numpy as np
import pytest

import oracle
from tests import pins

MODES = ["vertex", "topcell"]


def _rand_img(rng, shape):
    """Floats with ties (few distinct values), NaN and infinities mixed in."""
    vals = np.array([-np.inf, -1.5, -0.25, 0.0, 0.5, 0.5000001, 2.0, 3.75, np.inf, np.nan], np.float32)
    return vals[rng.integers(0, vals.size, size=shape)]


def _rand_levels(rng, m):
    """Ascending levels, with repeats and values outside the image range."""
    cand = np.array([-2.0, -1.5, -0.3, 0.0, 0.4, 0.5, 0.5000001, 1.0, 2.0, 3.75, 5.0, np.inf], np.float64)
    return np.sort(rng.choice(cand, size=m, replace=True))


@pytest.mark.parametrize("mode", MODES)
def test_random_small_float_images_vs_bruteforce(mode):
    rng = np.random.default_rng(31)
    for _ in range(150):
        nd = int(rng.integers(2, 4))
        shape = tuple(int(x) for x in rng.integers(1, 6 if nd == 2 else 4, size=nd))
        img = _rand_img(rng, shape)
        levels = _rand_levels(rng, int(rng.integers(1, 8)))
        got = oracle.ecc_levels(img, levels, mode)
        assert np.array_equal(got, pins.bruteforce_ecc_levels(img, levels, mode)), (img, levels)


@pytest.mark.parametrize("mode", MODES)
def test_2d_float_vs_flood_fill(mode):
    rng = np.random.default_rng(32)
    for _ in range(30):
        img = rng.normal(size=(int(rng.integers(2, 12)), int(rng.integers(2, 12)))).astype(np.float32)
        levels = np.sort(rng.normal(size=6))
        got = oracle.ecc_levels(img, levels, mode)
        for i, t in enumerate(levels):
            # integer image that is 0 where img <= t: flood fill at level 0
            bin_img = (~(img <= t)).astype(np.uint8)
            assert got[i] == pins.betti_ecc_2d(bin_img, 0, 0, mode)[0]


@pytest.mark.parametrize("mode", MODES)
def test_integer_valued_floats_equal_the_integer_oracle(mode):
    rng = np.random.default_rng(33)
    for shape in [(17, 23), (6, 7, 9), (1, 5, 8)]:
        img = rng.integers(0, 40, size=shape).astype(np.uint8)
        want = oracle.ecc(img, 0, 39, mode)
        assert np.array_equal(oracle.ecc_levels(img.astype(np.float32), np.arange(40.0), mode), want)
        # a level between two integers sees the same sublevel set as the lower one
        got = oracle.ecc_levels(img.astype(np.float32), np.arange(40.0) + 0.5, mode)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", MODES)
def test_strictly_increasing_map_of_values_and_levels(mode):
    rng = np.random.default_rng(34)
    img = rng.normal(size=(7, 8, 9)).astype(np.float32)
    levels = np.sort(rng.normal(size=9))
    f = lambda x: np.float32(3.0) * np.asarray(x, np.float32) ** 3 + np.float32(1.0)
    a = oracle.ecc_levels(img, levels, mode)
    b = oracle.ecc_levels(f(img), f(levels).astype(np.float64), mode)
    assert np.array_equal(a, b)


def test_closed_forms_and_errors():
    box = np.zeros((4, 5, 6), np.float32)
    assert list(oracle.ecc_levels(box, [-1.0, 0.0, 1.0], "vertex")) == [0, 1, 1]
    one = box.copy()
    one[2, 2, 2] = 1.0                       # bright interior voxel: a cavity at t = 0
    assert list(oracle.ecc_levels(one, [0.0, 1.0], "vertex")) == [2, 1]
    nan = box.copy()
    nan[2, 2, 2] = np.nan                    # NaN is above every level
    assert list(oracle.ecc_levels(nan, [0.0, 1e30], "vertex")) == [2, 2]
    with pytest.raises(oracle.OracleError):
        oracle.ecc_levels(box, [1.0, 0.0], "vertex")   # levels must ascend


LEVEL_MUTANTS = [
    ("level search strict", "if (levels[mid] < v) lo = mid + 1; else hi = mid;",
     "if (levels[mid] <= v) lo = mid + 1; else hi = mid;", 0),
    ("cells above the last level kept", "if (i < m) bins[i] += (dim % 2 == 0) ? 1 : -1;",
     "bins[i < m ? i : m - 1] += (dim % 2 == 0) ? 1 : -1;", 0),
    ("float max replaced by last vertex", "if (v > value) value = v;", "value = v;", 1),
    ("float min replaced by first coface", "if (v < value) value = v;", "if (value == (double)INFINITY) value = v;", 1),
    ("sign dropped in float top cells", "if (i < m) bins[i] += (dim % 2 == 0) ? 1 : -1;",
     "if (i < m) bins[i] += 1;", 1),
    ("NaN vertex ignored", "if (v != v) nan_vertex = 1;", "if (v != v) nan_vertex = 0;", 0),
    ("NaN cofaces counted at +infinity", "if (!any_coface) continue;", "", 0),
]


def _level_pins_pass(lib) -> bool:
    rng = np.random.default_rng(35)
    # fixed cases first: NaN inside (a hole at every level, +infinity
    # included), at a corner and in a row, with +infinity a level
    fixed = [(np.array([[1.0, 0.0, 2.0], [0.5, np.nan, 1.0], [3.0, 0.0, -1.0]], np.float32),
              np.array([0.0, 2.0, np.inf])),
             (np.array([[np.nan, 1.0, 2.0], [0.5, np.inf, np.nan]], np.float32), np.array([0.0, 2.0, np.inf])),
             (np.array([[[np.nan, np.nan], [3.0, -1.0]]], np.float32), np.array([-1.0, np.inf]))]
    for mode in MODES:
        fn = lib.oracle_levels_vertex_rows if mode == "vertex" else lib.oracle_levels_topcell_rows
        for k in range(60 + len(fixed)):
            if k < len(fixed):
                img, levels = fixed[k]
                shape = img.shape
            else:
                nd = int(rng.integers(2, 4))
                shape = tuple(int(x) for x in rng.integers(1, 5, size=nd))
                img = np.ascontiguousarray(_rand_img(rng, shape))
                levels = _rand_levels(rng, int(rng.integers(1, 6)))
            dims = np.asarray(shape, np.int64)
            bins = np.zeros(levels.size, np.int64)
            import ctypes
            rc = fn(img.ctypes.data, img.ndim, dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 0,
                    oracle.row_extent(shape, mode), levels.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    levels.size, bins.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
            if rc != 0 or not np.array_equal(np.cumsum(bins), pins.bruteforce_ecc_levels(img, levels, mode)):
                return False
    return True


def test_level_pins_pass_on_the_real_oracle():
    assert _level_pins_pass(oracle.load())


@pytest.mark.parametrize("name,old,new,which", LEVEL_MUTANTS, ids=[m[0] for m in LEVEL_MUTANTS])
def test_level_mutants_are_caught(tmp_path, name, old, new, which):
    src = (Path(oracle.__file__).parent / "ecc_oracle.c").read_text()
    starts = [i for i in range(len(src)) if src.startswith(old, i)]
    assert len(starts) > which, f"mutation anchor not found: {old!r}"
    at = starts[which]
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src[:at] + new + src[at + len(old):])
    lib_path = oracle.build(src=mutated, out=tmp_path / "libmutant.so")
    assert not _level_pins_pass(oracle.load(lib_path)), f"mutant survived: {name}"
