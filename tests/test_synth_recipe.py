"""The seeded input generators (`synth`) follow their stated recipe: the
same seed gives the same bytes, values span the stated ranges, smoothed
fields are smooth, the uneven batch and the Poisson request stream have the
stated counts and size distributions, and serving crops stay inside their
base fields with 16-element-aligned rows.  CPU only, small sizes."""
import math

import numpy as np
import torch

import synth


def test_uniform_noise_is_seeded_and_spans_the_range():
    a, b = synth.uniform_2d_256(), synth.uniform_2d_256()
    assert a.shape == (256, 256) and a.dtype == np.uint8
    assert np.array_equal(a, b)
    assert a.min() == 0 and a.max() == 255
    assert abs(float(a.mean()) - 127.5) < 1.5
    c = synth.uniform((64, 64), np.uint16, seed=1, lo=10, hi=20)
    assert c.dtype == np.uint16 and c.min() == 10 and c.max() == 20


def test_gaussian_taps_are_normalised_and_truncated_at_four_sigma():
    for sigma in (0.5, 2.0, 4.0, 8.0):
        t = synth._gauss_taps(sigma)
        r = max(1, math.ceil(4 * sigma))
        assert t.numel() == 2 * r + 1
        assert abs(float(t.sum()) - 1.0) < 1e-6
        assert torch.equal(t, t.flip(0))
        assert int(t.argmax()) == r


def test_smoothing_keeps_constants_and_reflects_at_the_edge():
    f = torch.full((7, 9), 3.25)
    assert torch.allclose(synth.smooth(f, 1.5), f)
    # reflect without repeating the edge: an impulse at x = 0 spreads as if
    # mirrored about the first sample
    g = torch.zeros(1, 21)
    g[0, 0] = 1.0
    taps = synth._gauss_taps(1.0)
    out = synth._smooth_axis(g, taps, 1)[0]
    r = (taps.numel() - 1) // 2
    for x in range(1, r + 1):
        assert abs(float(out[x]) - float(taps[r - x])) < 1e-7


def test_smoothed_fields_are_seeded_full_range_and_smooth():
    a = synth.smoothed_field((20, 24, 28), 2.0, np.uint8, seed=1)
    b = synth.smoothed_field((20, 24, 28), 2.0, np.uint8, seed=1)
    c = synth.smoothed_field((20, 24, 28), 2.0, np.uint8, seed=2)
    assert a.dtype == torch.uint8 and torch.equal(a, b) and not torch.equal(a, c)
    assert int(a.min()) == 0 and int(a.max()) == 255  # min-max rescaled
    step = (a[:, :, 1:].to(torch.int32) - a[:, :, :-1].to(torch.int32)).abs().float().mean()
    noise = torch.from_numpy(synth.uniform((20, 24, 28), np.uint8, seed=3).astype(np.int32))
    noise_step = (noise[:, :, 1:] - noise[:, :, :-1]).abs().float().mean()
    assert float(step) < 0.25 * float(noise_step)
    w = synth.smoothed_field((16, 40), 1.0, np.uint16, seed=5)
    assert w.dtype == torch.uint16 and int(w.to(torch.int32).max()) == 65535


def test_blobs_paint_integer_balls_in_their_value_range():
    vol = torch.zeros((40, 40, 40), dtype=torch.uint16)
    out = synth.add_blobs(vol, 5, seed=2, r_range=(3, 5), v_range=(60000, 65535))
    v = out.to(torch.int32)
    painted = v > 0
    assert int(painted.sum()) > 0
    assert int(v[painted].min()) >= 60000 and int(v.max()) <= 65535
    assert torch.equal(out, synth.add_blobs(vol, 5, seed=2, r_range=(3, 5), v_range=(60000, 65535)))
    # one ball alone is exactly the lattice points within its radius
    rng = np.random.default_rng(7)
    r, val = int(rng.integers(3, 6)), int(rng.integers(60000, 65536))
    one = synth.add_blobs(vol, 1, seed=7, r_range=(3, 5), v_range=(60000, 65535)).to(torch.int32)
    assert int((one == val).sum()) == int((one > 0).sum())
    assert int((one > 0).sum()) <= sum(1 for x in range(-r, r + 1) for y in range(-r, r + 1)
                                       for z in range(-r, r + 1) if x * x + y * y + z * z <= r * r)


def test_uneven_batch_counts_and_size_ranges():
    specs = synth.batch_specs()
    assert specs == synth.batch_specs()
    two = [s for s, _ in specs if len(s) == 2]
    three = [s for s, _ in specs if len(s) == 3]
    assert len(two) == 4096 and len(three) == 256
    assert all(64 <= x <= 1024 for s in two for x in s)
    assert all(32 <= x <= 256 for s in three for x in s)
    assert all(1.0 <= sig <= 6.0 for _, sig in specs)
    sides = np.array(two).ravel()
    assert abs(sides.mean() - 544) < 10  # U{64..1024} has mean 544
    assert sides.min() == 64 and sides.max() == 1024


def test_poisson_request_stream():
    reqs = synth.poisson_requests(2000.0, 2.0)
    assert reqs == synth.poisson_requests(2000.0, 2.0)
    n = len(reqs)
    assert abs(n - 4000) < 4 * math.sqrt(4000)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 2.0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 2000) < 4 / 2000 / math.sqrt(n)  # exponential gaps
    two = [r for r in reqs if len(r["shape"]) == 2]
    three = [r for r in reqs if len(r["shape"]) == 3]
    frac = len(two) / n
    assert abs(frac - 0.7) < 4 * math.sqrt(0.21 / n)
    assert all(r["dtype"] == "u8" for r in two)
    u16 = sum(r["dtype"] == "u16" for r in three) / len(three)
    assert abs(u16 - 0.5) < 4 * math.sqrt(0.25 / len(three))
    s2 = np.array([r["shape"][0] for r in two])
    s3 = np.array([r["shape"][0] for r in three])
    assert s2.min() >= 128 and s2.max() <= 4096 and s3.min() >= 64 and s3.max() <= 768
    # log-uniform: log sides have the mean of their interval
    assert abs(np.log(s2).mean() - 0.5 * (math.log(128) + math.log(4096))) < 0.1
    assert abs(np.log(s3).mean() - 0.5 * (math.log(64) + math.log(768))) < 0.15
    assert all(len(set(r["shape"])) == 1 for r in reqs)  # square and cubic requests


class _Base:
    """Stands in for a resident field: slicing returns the index tuple."""

    def __init__(self, shape):
        self.shape = shape

    def __getitem__(self, idx):
        return idx


def test_serving_crops_stay_inside_with_aligned_rows():
    reqs = synth.poisson_requests(2000.0, 0.5)
    bases = {"2d": _Base((4096, 4096)), "u8": _Base((768,) * 3), "u16": _Base((768,) * 3)}
    views = synth.serving_crops(reqs, bases)
    assert len(views) == len(reqs)
    for r, (idx, hi) in zip(reqs, views):
        assert hi == (65535 if r["dtype"] == "u16" else 255)
        dim = 4096 if len(r["shape"]) == 2 else 768
        assert len(idx) == len(r["shape"])
        for sl, s in zip(idx, r["shape"]):
            assert 0 <= sl.start and sl.stop - sl.start == s and sl.stop <= dim
        assert idx[-1].start % 16 == 0
