"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only -- no part of the ECC computation.
Both the CUDA path and the CPU oracle consume the bytes it produces; neither
imports the other.  The paper's datasets (CMB projections, VICTRE phantoms,
Gaussian random fields, uniform noise; Sec. 4 "Datasets") are not available,
so these generators stand in for the last two with the shapes of the
benchmark configurations:

* ``uniform``: iid uniform integer noise (the paper's "uniform noise").
* ``smoothed_field``: an iid N(0,1) field convolved with an isotropic
  Gaussian, min-max rescaled to the full integer range and rounded (the
  paper's "Gaussian random fields" of varying smoothness, Fig. 2).
* ``add_blobs``: bright constant spheres painted over a field (large
  plateaus of ties for the 16-bit configuration).
* ``batch_specs`` / ``batch_images``: thousands of images and volumes of
  uneven sizes (Table 3's many-small-files case, made uneven).
* ``poisson_requests``: a seeded Poisson request stream for serving.

Recorded choices (the configurations leave them open): the Gaussian kernel is
truncated at 4 sigma and applied separably with reflect boundaries in float32;
rescaling is (f - min) / (max - min) * maxval, rounded half-to-even, then
clamped; integer sizes are drawn inclusive of both ends; blobs use integer
radius, value and centre, are clipped at the volume edge, and later blobs
overwrite earlier ones.
"""
from __future__ import annotations

import math

import numpy as np
import torch

_MAXVAL = {torch.uint8: 255, torch.uint16: 65535, np.uint8: 255, np.uint16: 65535}


def _torch_dtype(dtype):
    if dtype in (np.uint8, torch.uint8, "u8", "uint8"):
        return torch.uint8
    if dtype in (np.uint16, torch.uint16, "u16", "uint16"):
        return torch.uint16
    raise TypeError(f"unsupported dtype {dtype}")


def uniform(shape, dtype=np.uint8, seed: int = 0, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """iid uniform integers in [lo, hi] from numpy's default_rng(seed)."""
    dt = np.dtype(dtype)
    if hi is None:
        hi = 255 if dt == np.uint8 else 65535
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=tuple(shape), dtype=dt)


def _gauss_taps(sigma: float) -> torch.Tensor:
    r = max(1, int(math.ceil(4.0 * sigma)))
    x = torch.arange(-r, r + 1, dtype=torch.float64)
    k = torch.exp(-0.5 * (x / sigma) ** 2)
    return (k / k.sum()).to(torch.float32)


def _smooth_axis(f: torch.Tensor, taps: torch.Tensor, axis: int) -> torch.Tensor:
    r = (taps.numel() - 1) // 2
    n = f.shape[axis]
    g = f.movedim(axis, -1)
    shp = g.shape
    g = g.reshape(-1, 1, n)
    if r >= n:  # reflect padding needs r < n; replicate the edge values for tiny axes
        left = g[..., :1].expand(-1, -1, r)
        right = g[..., -1:].expand(-1, -1, r)
    else:       # reflect (edge not repeated), built with flips: no batch-size limit
        left = g[..., 1:r + 1].flip(-1)
        right = g[..., n - 1 - r:n - 1].flip(-1)
    g = torch.cat([left, g, right], dim=-1)
    out = torch.empty(g.shape[0], 1, n, dtype=g.dtype, device=g.device)
    step = 1 << 20  # bound the rows per convolution call
    for i in range(0, g.shape[0], step):
        out[i:i + step] = torch.nn.functional.conv1d(g[i:i + step], taps.to(g.device).view(1, 1, -1))
    return out.reshape(shp).movedim(-1, axis)


def smooth(f: torch.Tensor, sigma: float) -> torch.Tensor:
    """Separable isotropic Gaussian blur (float32, 4-sigma truncation, reflect)."""
    taps = _gauss_taps(sigma)
    for axis in range(f.dim()):
        f = _smooth_axis(f, taps, axis)
    return f


def quantize(f: torch.Tensor, dtype) -> torch.Tensor:
    """Min-max rescale to [0, maxval], round half-to-even, clamp, cast."""
    tdt = _torch_dtype(dtype)
    maxval = float(_MAXVAL[tdt])
    lo, hi = f.min(), f.max()
    scale = maxval / (hi - lo).clamp_min(1e-30)
    q = torch.round((f - lo) * scale).clamp_(0, maxval)
    if tdt == torch.uint16:
        return q.to(torch.int32).to(torch.uint16)
    return q.to(tdt)


def smoothed_field(shape, sigma: float, dtype=np.uint8, seed: int = 1, device="cpu") -> torch.Tensor:
    """N(0,1) field from torch.Generator(device).manual_seed(seed), smoothed and quantized."""
    gen = torch.Generator(device=device).manual_seed(seed)
    f = torch.randn(tuple(shape), generator=gen, device=device, dtype=torch.float32)
    f = smooth(f, sigma)
    return quantize(f, dtype)


def add_blobs(vol: torch.Tensor, count: int, seed: int, r_range=(3, 12), v_range=(60000, 65535)) -> torch.Tensor:
    """Paint ``count`` constant-valued balls (integer radius, value, centre) in order."""
    rng = np.random.default_rng(seed)
    dims = vol.shape
    radii = rng.integers(r_range[0], r_range[1] + 1, size=count)
    values = rng.integers(v_range[0], v_range[1] + 1, size=count)
    centres = np.stack([rng.integers(0, d, size=count) for d in dims], axis=1)
    dev = vol.device
    out = vol.to(torch.int32)  # index_put is not implemented for uint16
    for r, v, c in zip(radii.tolist(), values.tolist(), centres.tolist()):
        sl = tuple(slice(max(0, ci - r), min(d, ci + r + 1)) for ci, d in zip(c, dims))
        grids = torch.meshgrid(*[torch.arange(s.start, s.stop, device=dev) - ci for s, ci in zip(sl, c)],
                               indexing="ij")
        inside = sum(g * g for g in grids) <= r * r
        view = out[sl]
        view[inside] = v
    return out.to(vol.dtype)


# --- the five benchmark configurations ---------------------------------------

def uniform_2d_256() -> np.ndarray:
    """One 256x256 uint8 image, iid uniform in [0,255], seed 0."""
    return uniform((256, 256), np.uint8, seed=0)


def smooth_3d_512(device="cuda", shape=(512, 512, 512)) -> torch.Tensor:
    """512^3 uint8: N(0,1) seed 1 smoothed with sigma=4, rescaled to [0,255]."""
    return smoothed_field(shape, 4.0, np.uint8, seed=1, device=device)


def smooth_blobs_u16_1024(device="cuda", shape=(1024, 1024, 1024), blobs: int = 2000) -> torch.Tensor:
    """1024^3 uint16: N(0,1) seed 2 smoothed with sigma=8, rescaled to [0,65535], plus blobs."""
    v = smoothed_field(shape, 8.0, np.uint16, seed=2, device=device)
    return add_blobs(v, blobs, seed=2)


def batch_specs(n2d: int = 4096, n3d: int = 256, seed: int = 3,
                side2d=(64, 1024), side3d=(32, 256), sigma=(1.0, 6.0)):
    """Shapes and smoothing widths of the uneven batch (seeded, inclusive ranges)."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n2d):
        h, w = rng.integers(side2d[0], side2d[1] + 1, size=2).tolist()
        specs.append(((h, w), float(rng.uniform(*sigma))))
    for _ in range(n3d):
        d, h, w = rng.integers(side3d[0], side3d[1] + 1, size=3).tolist()
        specs.append(((d, h, w), float(rng.uniform(*sigma))))
    return specs


def batch_images(specs, seed: int = 3, device="cuda", dtype=np.uint8):
    """One smoothed, quantized field per spec; image i uses seed ``seed*100003 + i``."""
    return [smoothed_field(shape, sig, dtype, seed=seed * 100003 + i, device=device)
            for i, (shape, sig) in enumerate(specs)]


def poisson_requests(rate_hz: float, duration_s: float, seed: int = 4, frac_2d: float = 0.7,
                     side2d=(128, 4096), side3d=(64, 768)):
    """Seeded Poisson arrivals with log-uniform sizes.

    Returns a list of dicts: t (arrival, s), shape, dtype ('u8'/'u16'), sigma.
    """
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        if rng.uniform() < frac_2d:
            s = int(round(math.exp(rng.uniform(math.log(side2d[0]), math.log(side2d[1])))))
            shape, dt = (s, s), "u8"
        else:
            s = int(round(math.exp(rng.uniform(math.log(side3d[0]), math.log(side3d[1])))))
            shape, dt = (s, s, s), ("u8" if rng.uniform() < 0.5 else "u16")
        out.append({"t": t, "shape": shape, "dtype": dt, "sigma": float(rng.uniform(1.0, 6.0))})
    return out


def serving_bases(device="cuda"):
    """Resident seeded fields the serving requests are cut from: one 4096^2
    uint8 image and one 768^3 volume each of uint8 and uint16 (sigma 3)."""
    return {"2d": smoothed_field((4096, 4096), 3.0, np.uint8, seed=41, device=device),
            "u8": smoothed_field((768, 768, 768), 3.0, np.uint8, seed=42, device=device),
            "u16": smoothed_field((768, 768, 768), 3.0, np.uint16, seed=43, device=device)}


def serving_crops(reqs, bases, seed: int = 4):
    """One (view, hi) per request: a crop of the request's shape from its base
    field at a seeded origin, the innermost origin rounded down to a multiple
    of 16 elements.  Views share the bases' storage."""
    rng = np.random.default_rng(seed)
    views = []
    for r in reqs:
        s = r["shape"][0]
        if len(r["shape"]) == 2:
            o = [int(rng.integers(0, 4096 - s + 1)) for _ in range(2)]
            o[1] -= o[1] % 16
            views.append((bases["2d"][o[0]:o[0] + s, o[1]:o[1] + s], 255))
        else:
            base, hi = (bases["u8"], 255) if r["dtype"] == "u8" else (bases["u16"], 65535)
            o = [int(rng.integers(0, 768 - s + 1)) for _ in range(3)]
            o[2] -= o[2] % 16
            views.append((base[o[0]:o[0] + s, o[1]:o[1] + s, o[2]:o[2] + s], hi))
    return views
