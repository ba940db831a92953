"""CPU oracle for the Euler characteristic curve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  The
product library never imports it, and it imports nothing from the product.

The arithmetic lives in ``ecc_oracle.c`` (plain single-threaded C, one cell at
a time, following Sec. 2.1-2.3 of Wang, Wagner, Chen, SoCG 2022).  This module
only compiles it with gcc, marshals numpy arrays, and -- for full-size checks
-- runs the oracle's own slab entry points (the chunking of Sec. 3.4) on
several host threads and sums their histograms.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (brute force on tiny inputs, Betti numbers by
flood fill, closed forms, symmetries, and a mutation check), the float
thresholds by ``tests/test_oracle_levels_pins.py``, the smoothing filter by
``tests/test_oracle_blur_pins.py`` and the iterated pipeline by
``tests/test_oracle_pipeline_pins.py`` (closed-form filters fix the order
ECC-then-smooth and the round count).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "ecc_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libecc_oracle.so"

VERTEX = "vertex"    # cells enter at the max of their vertices (pixels as vertices)
TOPCELL = "topcell"  # voxels are top cells; lower cells take the min of their cofaces (Sec. 2.1)

_lib = None
_lock = threading.Lock()


def build(src: Path = _SRC, out: Path = _LIB_PATH, extra_flags=()) -> Path:
    """Compile the oracle with gcc into a shared library; returns its path."""
    out.parent.mkdir(parents=True, exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra_flags, str(src), "-o", str(out)]
    subprocess.run(cmd, check=True)
    return out


def load(path: Path | None = None):
    """Load (building if needed) the oracle library and declare its signatures."""
    global _lib
    if path is None:
        with _lock:
            if _lib is not None:
                return _lib
            if not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
                build()
            _lib = _declare(ctypes.CDLL(str(_LIB_PATH)))
            return _lib
    return _declare(ctypes.CDLL(str(path)))


def _declare(lib):
    i64p = ctypes.POINTER(ctypes.c_int64)
    for name in ("oracle_vcec_vertex_rows", "oracle_vcec_topcell_rows"):
        f = getattr(lib, name)
        f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, i64p,
                      ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, i64p]
        f.restype = ctypes.c_int
    for name in ("oracle_vcec_vertex", "oracle_vcec_topcell"):
        f = getattr(lib, name)
        f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, i64p,
                      ctypes.c_int32, ctypes.c_int32, i64p]
        f.restype = ctypes.c_int
    lib.oracle_ecc_from_vcec.argtypes = [i64p, ctypes.c_int64, i64p]
    lib.oracle_ecc_from_vcec.restype = None
    for name in ("oracle_levels_vertex_rows", "oracle_levels_topcell_rows"):
        f = getattr(lib, name)
        f.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_int64,
                      ctypes.POINTER(ctypes.c_double), ctypes.c_int64, i64p]
        f.restype = ctypes.c_int
    return lib


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.uint8:
        return 1
    if a.dtype == np.uint16:
        return 2
    raise TypeError(f"oracle supports uint8/uint16 images, got {a.dtype}")


def _i64p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class OracleError(RuntimeError):
    pass


def _check(rc: int):
    if rc == 1:
        raise OracleError("invalid arguments")
    if rc == 2:
        raise OracleError("image value outside [lo, hi]")


def _default_range(img: np.ndarray, lo, hi):
    if lo is None:
        lo = 0
    if hi is None:
        hi = 255 if img.dtype == np.uint8 else 65535
    return int(lo), int(hi)


def vcec(img: np.ndarray, lo=None, hi=None, mode: str = VERTEX, lib=None) -> np.ndarray:
    """VCEC (int64[hi-lo+1]) of a dense uint8/uint16 image, single-threaded."""
    lib = lib or load()
    img = np.ascontiguousarray(img)
    lo, hi = _default_range(img, lo, hi)
    dims = np.asarray(img.shape, dtype=np.int64)
    out = np.zeros(hi - lo + 1, dtype=np.int64)
    fn = lib.oracle_vcec_vertex if mode == VERTEX else lib.oracle_vcec_topcell
    _check(fn(img.ctypes.data, _dtype_code(img), img.ndim, _i64p(dims), lo, hi, _i64p(out)))
    return out


def ecc_from_vcec(v: np.ndarray, lib=None) -> np.ndarray:
    lib = lib or load()
    v = np.ascontiguousarray(v, dtype=np.int64)
    out = np.empty_like(v)
    lib.oracle_ecc_from_vcec(_i64p(v), v.size, _i64p(out))
    return out


def ecc(img: np.ndarray, lo=None, hi=None, mode: str = VERTEX, lib=None) -> np.ndarray:
    """ECC (int64[hi-lo+1]): ECC[g] = chi(K_{<= lo+g})."""
    lib = lib or load()
    return ecc_from_vcec(vcec(img, lo, hi, mode, lib), lib)


def vcec_rows(img: np.ndarray, begin: int, end: int, lo=None, hi=None, mode: str = VERTEX,
              lib=None) -> np.ndarray:
    """VCEC of the cells whose dims[0] index lies in [begin, end).

    V-mode indexes base points 0..dims[0]-1; T-mode indexes elementary
    intervals 0..2*dims[0] (even = degenerate).  Disjoint ranges add up.
    """
    lib = lib or load()
    img = np.ascontiguousarray(img)
    lo, hi = _default_range(img, lo, hi)
    dims = np.asarray(img.shape, dtype=np.int64)
    out = np.zeros(hi - lo + 1, dtype=np.int64)
    fn = lib.oracle_vcec_vertex_rows if mode == VERTEX else lib.oracle_vcec_topcell_rows
    _check(fn(img.ctypes.data, _dtype_code(img), img.ndim, _i64p(dims), int(begin), int(end),
              lo, hi, _i64p(out)))
    return out


def level_bins_rows(img: np.ndarray, levels, begin: int, end: int, mode: str = VERTEX, lib=None) -> np.ndarray:
    """Signed cell counts of a float32 image per threshold index (int64[m]):
    bin i holds the cells whose value's first level at or above it is
    levels[i] (Eq. 1 with the t_i given), for the dims[0] indices in
    [begin, end).  Disjoint ranges add up."""
    lib = lib or load()
    img = np.ascontiguousarray(img, dtype=np.float32)
    lv = np.ascontiguousarray(levels, dtype=np.float64)
    dims = np.asarray(img.shape, dtype=np.int64)
    out = np.zeros(lv.size, dtype=np.int64)
    fn = lib.oracle_levels_vertex_rows if mode == VERTEX else lib.oracle_levels_topcell_rows
    _check(fn(img.ctypes.data, img.ndim, _i64p(dims), int(begin), int(end),
              lv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), lv.size, _i64p(out)))
    return out


def ecc_levels(img: np.ndarray, levels, mode: str = VERTEX, threads: int = 1) -> np.ndarray:
    """ECC of a float32 image at ascending thresholds: int64[m], entry i =
    chi(K_{<= levels[i]}).  A NaN voxel is in no sublevel set: it lies above
    every level, +infinity included."""
    lib = load()
    img = np.ascontiguousarray(img, dtype=np.float32)
    end = row_extent(img.shape, mode)
    threads = max(1, min(threads, end))
    cuts = np.linspace(0, end, threads + 1).round().astype(np.int64)
    parts = [None] * threads
    errors = []

    def work(i):
        try:
            parts[i] = level_bins_rows(img, levels, cuts[i], cuts[i + 1], mode, lib)
        except Exception as e:  # surfaced below
            errors.append(e)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errors:
        raise errors[0]
    return ecc_from_vcec(np.sum(parts, axis=0).astype(np.int64), lib)


def present_levels(img: np.ndarray) -> np.ndarray:
    """Eq. 1's thresholds of a float32 image: the values present in it,
    distinct and ascending (t_1 < t_2 < ... < t_n, Sec. 2.2).  NaN voxels
    define no threshold and lie in no sublevel set (v <= t is false for
    every t, +infinity included), and -0.0 is the value 0.0 (it compares
    equal to it, so it is the same threshold), returned as +0.0.  A library
    sort-unique is the step."""
    v = np.asarray(img, dtype=np.float32).ravel()
    v = v[~np.isnan(v)]
    return np.unique(v + np.float32(0.0)).astype(np.float32)


def ecc_present(img: np.ndarray, mode: str = VERTEX, threads: int = 1):
    """The paper's ECC sequence of a float32 image (Eq. 1): (levels, ecc)
    with levels = present_levels(img) and ecc[i] = chi(K_{<= levels[i]})."""
    lv = present_levels(img)
    if lv.size == 0:  # every voxel NaN: no threshold
        return lv, np.zeros(0, np.int64)
    return lv, ecc_levels(img, lv, mode, threads)


def row_extent(img_shape, mode: str = VERTEX) -> int:
    """Number of dims[0] indices the *_rows entry points range over."""
    return img_shape[0] if mode == VERTEX else 2 * img_shape[0] + 1


def vcec_parallel(img: np.ndarray, lo=None, hi=None, mode: str = VERTEX, threads: int | None = None,
                  rows: tuple[int, int] | None = None) -> np.ndarray:
    """Run the single-threaded oracle on disjoint dims[0] slabs in host threads
    (ctypes releases the GIL) and sum the slab histograms.  ``rows`` restricts
    the work to a sub-range of the dims[0] indices."""
    lib = load()
    img = np.ascontiguousarray(img)
    lo, hi = _default_range(img, lo, hi)
    begin, end = rows if rows is not None else (0, row_extent(img.shape, mode))
    threads = max(1, min(threads or os.cpu_count() or 1, end - begin))
    cuts = np.linspace(begin, end, threads + 1).round().astype(np.int64)
    parts = [None] * threads
    errors = []

    def work(i):
        try:
            parts[i] = vcec_rows(img, cuts[i], cuts[i + 1], lo, hi, mode, lib)
        except Exception as e:  # surfaced below
            errors.append(e)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errors:
        raise errors[0]
    return np.sum(parts, axis=0).astype(np.int64)


def reflect_index(j: np.ndarray, n: int) -> np.ndarray:
    """Half-sample symmetric reflection of indices into [0, n): ... 1 0 | 0 1 ... n-1 | n-1 n-2 ..."""
    p = np.mod(j, 2 * n)
    return np.where(p >= n, 2 * n - 1 - p, p)


def blur_axis(img: np.ndarray, weights: np.ndarray, axis: int) -> np.ndarray:
    """One pass of a discrete convolution along `axis` in float32 (the
    smoothing step of the paper's iterated ECC + Gaussian pipeline, Sec. 4
    "GPU-only pipeline"): out[x] = sum over taps k = -r..r, in that order, of
    w[k + r] * in[reflect(x + k)], every product and partial sum rounded to
    float32 (no fused multiply-add)."""
    img = np.asarray(img, np.float32)
    w = np.asarray(weights, np.float32)
    r = (w.size - 1) // 2
    n = img.shape[axis]
    acc = np.zeros_like(img, dtype=np.float32)
    for k in range(-r, r + 1):
        idx = reflect_index(np.arange(n) + k, n)
        term = np.take(img, idx, axis=axis) * w[k + r]          # float32 product
        acc = (acc + term).astype(np.float32)                    # float32 sum
    return acc


def blur(img: np.ndarray, weights) -> np.ndarray:
    """Separable smoothing: one pass per axis, last axis first."""
    out = np.asarray(img, np.float32)
    for axis in range(out.ndim - 1, -1, -1):
        out = blur_axis(out, weights, axis)
    return out


def gaussian_pipeline(img: np.ndarray, weights, levels, iterations: int, mode: str = VERTEX, threads: int = 1):
    """The iterated pipeline: ECC at the levels, then smooth, `iterations`
    times.  Returns (int64[iterations, m] ECCs, final image)."""
    cur = np.asarray(img, np.float32)
    eccs = []
    for _ in range(iterations):
        eccs.append(ecc_levels(cur, levels, mode, threads))
        cur = blur(cur, weights)
    return np.stack(eccs), cur
