"""Pins of the oracle's iterated pipeline (``oracle.gaussian_pipeline``).

Sec. 4 "Case study: GPU-only pipeline", paragraph "Pipeline" (and Table 2):
each round first computes the ECC of the image held in memory and then
applies the smoothing filter to that image; rounds repeat on the smoothed
result.  The pins below fix that order and the round count with filters
whose effect is known in closed form, independently of ``oracle.blur``:

* one round is exactly (ECC of the input, one smoothing of the input);
* the identity filter leaves every round's ECC equal to the first and the
  image unchanged;
* the one-sided filter w = (0, 0, 1) maps index x to min(x + 1, n - 1) on
  every axis under half-sample reflection, so after k rounds the image is
  img[min(x + k, n - 1), ...] and round k's ECC is that image's ECC;
* planted mistakes (smoothing before the first ECC, one round too many, the
  ECC taken after the smoothing, rounds that restart from the input) each
  fail one of these pins.
"""
import numpy as np
import pytest

import oracle

SHIFT = np.array([0.0, 0.0, 1.0], np.float32)     # out[x] = in[reflect(x + 1)]
IDENT = np.array([0.0, 1.0, 0.0], np.float32)


def shifted_k(img: np.ndarray, k: int) -> np.ndarray:
    """The image after k one-sided shifts on every axis, by the closed form
    index map x -> min(x + k, n - 1) (no use of the oracle's filter)."""
    out = np.asarray(img, np.float32)
    for axis, n in enumerate(img.shape):
        idx = np.minimum(np.arange(n) + k, n - 1)
        out = np.take(out, idx, axis=axis)
    return out


def blob_image(shape, seed):
    """Float32 image with several small bright features near the low corner,
    which the one-sided shift pushes out one index per round, so the ECC at
    the levels changes from round to round."""
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 0.2, size=shape).astype(np.float32)
    for c in range(6):
        pos = tuple(int(rng.integers(0, min(4, n))) if i == 0 else int(rng.integers(0, n)) for i, n in enumerate(shape))
        img[pos] = np.float32(0.5 + 0.08 * c)
    # a ring far from the low edges keeps a 1-cycle for several rounds
    if len(shape) == 2:
        img[6:10, 6:10] = 0.9
        img[7:9, 7:9] = 0.1
    return img


LEVELS = np.array([0.05, 0.1, 0.15, 0.3, 0.55, 0.62, 0.7, 0.85, 0.95], np.float32)


def reference_rounds(img, weights_image_fn, iterations):
    """Expected (eccs, final) from a closed-form image sequence."""
    eccs = [oracle.ecc_levels(weights_image_fn(img, k), LEVELS) for k in range(iterations)]
    return np.stack(eccs), weights_image_fn(img, iterations)


@pytest.mark.parametrize("shape", [(14, 15), (6, 7, 8)])
def test_one_round_is_ecc_then_one_smoothing(shape):
    rng = np.random.default_rng(61)
    img = rng.normal(size=shape).astype(np.float32)
    taps = np.array([0.1, 0.2, 0.4, 0.2, 0.1], np.float32)
    levels = np.sort(rng.normal(size=7)).astype(np.float32)
    eccs, final = oracle.gaussian_pipeline(img, taps, levels, 1)
    assert eccs.shape == (1, levels.size)
    assert np.array_equal(eccs[0], oracle.ecc_levels(img, levels))
    assert np.array_equal(final, oracle.blur(img, taps))


@pytest.mark.parametrize("shape", [(12, 13), (5, 6, 7)])
def test_identity_filter_keeps_every_round(shape):
    img = blob_image(shape, 62)
    eccs, final = oracle.gaussian_pipeline(img, IDENT, LEVELS, 4)
    assert eccs.shape == (4, LEVELS.size)
    for k in range(4):
        assert np.array_equal(eccs[k], oracle.ecc_levels(img, LEVELS))
    assert np.array_equal(final, img)


@pytest.mark.parametrize("shape", [(12, 13), (6, 7, 8)])
def test_shift_filter_round_k_sees_the_image_shifted_k_times(shape):
    img = blob_image(shape, 63)
    iters = 5
    eccs, final = oracle.gaussian_pipeline(img, SHIFT, LEVELS, iters)
    want_eccs, want_final = reference_rounds(img, shifted_k, iters)
    assert np.array_equal(final, want_final)
    assert np.array_equal(eccs, want_eccs)
    # the pins below are only as strong as the rounds are distinct
    assert len({tuple(e) for e in want_eccs}) >= 3


def test_shift_closed_form_matches_reflection_rule():
    # half-sample reflection: index n reflects to n - 1, so one shift is x -> min(x + 1, n - 1)
    x = np.arange(10, dtype=np.float32).reshape(1, 10)
    assert list(shifted_k(x, 1)[0]) == [1, 2, 3, 4, 5, 6, 7, 8, 9, 9]
    assert list(shifted_k(x, 3)[0]) == [3, 4, 5, 6, 7, 8, 9, 9, 9, 9]


# ---------------------------------------------------------------- mutants

def _smooth_first(img, weights, levels, iterations, mode=oracle.VERTEX, threads=1):
    cur = np.asarray(img, np.float32)
    eccs = []
    for _ in range(iterations):
        cur = oracle.blur(cur, weights)
        eccs.append(oracle.ecc_levels(cur, levels, mode, threads))
    return np.stack(eccs), cur


def _one_round_too_many(img, weights, levels, iterations, mode=oracle.VERTEX, threads=1):
    return oracle.gaussian_pipeline(img, weights, levels, iterations + 1, mode, threads)


def _extra_smoothing(img, weights, levels, iterations, mode=oracle.VERTEX, threads=1):
    eccs, cur = oracle.gaussian_pipeline(img, weights, levels, iterations, mode, threads)
    return eccs, oracle.blur(cur, weights)


def _restart_each_round(img, weights, levels, iterations, mode=oracle.VERTEX, threads=1):
    cur = np.asarray(img, np.float32)
    eccs = []
    for _ in range(iterations):
        eccs.append(oracle.ecc_levels(cur, levels, mode, threads))
        out = oracle.blur(cur, weights)
    return np.stack(eccs), out


def _pins_hold(fn) -> bool:
    for shape in [(12, 13), (6, 7, 8)]:
        img = blob_image(shape, 63)
        eccs, final = fn(img, SHIFT, LEVELS, 5)
        want_eccs, want_final = reference_rounds(img, shifted_k, 5)
        if eccs.shape != want_eccs.shape or not np.array_equal(eccs, want_eccs):
            return False
        if not np.array_equal(final, want_final):
            return False
        e1, f1 = fn(img, IDENT, LEVELS, 3)
        if e1.shape != (3, LEVELS.size) or not np.array_equal(f1, img):
            return False
    return True


def test_pins_hold_for_the_oracle():
    assert _pins_hold(oracle.gaussian_pipeline)


@pytest.mark.parametrize("mutant", [_smooth_first, _one_round_too_many, _extra_smoothing, _restart_each_round])
def test_planted_pipeline_mistakes_are_caught(mutant):
    assert not _pins_hold(mutant)
