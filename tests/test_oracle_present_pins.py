"""Pins of the oracle's present-value thresholds (oracle.present_levels and
oracle.ecc_present: the paper's ECC sequence of a float image, Eq. 1, with
t_1 < ... < t_n the distinct values present, Sec. 2.2).  They are checked
against things other than themselves:
- a plain set-of-values construction by float equality;
- the naive thresholding method on tiny images;
- the integer oracle on integer-valued data;
- the full-box invariant;
- planted mistakes that must be caught."""
import numpy as np
import pytest

import oracle
from tests import pins

MODES = ["vertex", "topcell"]


def _distinct_by_equality(img):
    """Distinct non-NaN values by float equality, in a Python set (-0.0 and
    0.0 compare and hash equal, so they are one value), ascending."""
    seen = set()
    for v in np.asarray(img, np.float32).ravel().tolist():
        if v == v:
            seen.add(float(v))
    return sorted(seen)


def _rand_img(rng, shape):
    vals = np.array([-np.inf, -1.5, -0.0, 0.0, 0.5, 0.5000001, 2.0, np.inf, np.nan], np.float32)
    return vals[rng.integers(0, vals.size, size=shape)]


def test_levels_are_the_distinct_values_by_equality():
    rng = np.random.default_rng(41)
    for _ in range(200):
        shape = tuple(int(x) for x in rng.integers(1, 7, size=int(rng.integers(1, 4))))
        img = _rand_img(rng, shape)
        got = oracle.present_levels(img)
        want = _distinct_by_equality(img)
        assert got.dtype == np.float32
        assert got.tolist() == want, (img, got)
        assert np.all(np.diff(got) > 0)
        # a zero threshold is +0.0
        assert not np.any(np.signbit(got[got == 0]))


def test_nan_only_and_single_value_images():
    assert oracle.present_levels(np.full((3, 4), np.nan, np.float32)).size == 0
    lv, e = oracle.ecc_present(np.full((3, 4, 2), 2.5, np.float32))
    assert lv.tolist() == [2.5]
    assert e.tolist() == [1]  # the full box at its one level


@pytest.mark.parametrize("mode", MODES)
def test_tiny_images_against_bruteforce(mode):
    rng = np.random.default_rng(42)
    for _ in range(120):
        nd = int(rng.integers(2, 4))
        shape = tuple(int(x) for x in rng.integers(1, 6 if nd == 2 else 4, size=nd))
        img = _rand_img(rng, shape)
        lv, e = oracle.ecc_present(img, mode)
        assert np.array_equal(e, pins.bruteforce_ecc_levels(img, lv.astype(np.float64), mode)), img


@pytest.mark.parametrize("mode", MODES)
def test_integer_valued_floats_are_the_integer_ecc_at_present_values(mode):
    rng = np.random.default_rng(43)
    for shape in [(19, 13), (5, 6, 7), (2, 1, 9), (40, 3)]:
        img = rng.choice(np.array([3, 7, 8, 20, 21, 33], np.uint8), size=shape)
        full = oracle.ecc(img, 0, 40, mode)  # every gray level 0..40
        lv, e = oracle.ecc_present(img.astype(np.float32), mode)
        present = np.unique(img)
        assert lv.tolist() == present.astype(np.float32).tolist()
        assert np.array_equal(e, full[present.astype(np.int64)])


@pytest.mark.parametrize("mode", MODES)
def test_last_level_is_the_full_box_without_nan(mode):
    rng = np.random.default_rng(44)
    for shape in [(8, 9), (4, 5, 6)]:
        img = rng.normal(size=shape).astype(np.float32)
        img[0] = -0.0
        lv, e = oracle.ecc_present(img, mode)
        assert lv.size == np.unique(img).size
        assert e[-1] == 1


# ---------------------------------------------------------------- mutants
# Each one is a plausible mistake in present_levels or ecc_present; the pins
# above, run on the mutant instead of the oracle, must fail.

def _finite(img):
    v = np.asarray(img, np.float32).ravel()
    return v[~np.isnan(v)]


def _levels_keep_nan(img):
    return np.unique(np.asarray(img, np.float32).ravel() + np.float32(0.0))


def _levels_negzero_apart(img):
    return np.unique(_finite(img).view(np.uint32)).view(np.float32)


def _levels_negzero_kept(img):
    return np.unique(_finite(img))  # a zero threshold may come out as -0.0


def _levels_first_seen_order(img):
    return np.array(list(dict.fromkeys(_finite(img).tolist())), np.float32)


def _levels_descending(img):
    return oracle.present_levels(img)[::-1].copy()


def _present_with(levels_fn):
    def fn(img, mode=oracle.VERTEX, threads=1):
        lv = levels_fn(img)
        if lv.size == 0:
            return lv, np.zeros(0, np.int64)
        return lv, oracle.ecc_levels(img, lv, mode, threads)
    return fn


def _present_nan_at_infinity(img, mode=oracle.VERTEX, threads=1):
    lv = oracle.present_levels(img)
    if lv.size == 0:
        return lv, np.zeros(0, np.int64)
    filled = np.where(np.isnan(img), np.float32(np.inf), img).astype(np.float32)
    return lv, oracle.ecc_levels(filled, lv, mode, threads)


def _present_strict_sublevel(img, mode=oracle.VERTEX, threads=1):
    lv = oracle.present_levels(img)
    if lv.size == 0:
        return lv, np.zeros(0, np.int64)
    below = np.nextafter(lv, np.float32(-np.inf)).astype(np.float32)  # v < t instead of v <= t
    return lv, oracle.ecc_levels(img, below, mode, threads)


def _present_shifted_one_level(img, mode=oracle.VERTEX, threads=1):
    lv, e = oracle.ecc_present(img, mode, threads)
    return lv, np.concatenate([np.zeros(min(1, e.size), np.int64), e[:-1]])


def _pins_hold(levels_fn, present_fn) -> bool:
    rng = np.random.default_rng(45)
    for _ in range(60):
        shape = tuple(int(x) for x in rng.integers(1, 6, size=int(rng.integers(2, 4))))
        img = _rand_img(rng, shape)
        got = np.asarray(levels_fn(img))
        want = _distinct_by_equality(img)
        if got.dtype != np.float32 or got.tolist() != want:
            return False
        if np.any(np.signbit(got[got == 0])):
            return False
        for mode in MODES:
            lv, e = present_fn(img, mode)
            if not np.array_equal(np.asarray(lv).view(np.uint32), got.view(np.uint32)):
                return False
            if not np.array_equal(e, pins.bruteforce_ecc_levels(img, got.astype(np.float64), mode)):
                return False
    return True


def test_pins_hold_for_the_oracle():
    assert _pins_hold(oracle.present_levels, oracle.ecc_present)


LEVEL_MUTANTS = [_levels_keep_nan, _levels_negzero_apart, _levels_negzero_kept, _levels_first_seen_order,
                 _levels_descending]
PRESENT_MUTANTS = [_present_nan_at_infinity, _present_strict_sublevel, _present_shifted_one_level]


@pytest.mark.parametrize("mutant", LEVEL_MUTANTS, ids=[m.__name__ for m in LEVEL_MUTANTS])
def test_planted_level_mistakes_are_caught(mutant):
    assert not _pins_hold(mutant, _present_with(mutant))


@pytest.mark.parametrize("mutant", PRESENT_MUTANTS, ids=[m.__name__ for m in PRESENT_MUTANTS])
def test_planted_ecc_mistakes_are_caught(mutant):
    assert not _pins_hold(oracle.present_levels, mutant)
