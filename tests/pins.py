"""Independent checks that pin the CPU oracle to mathematics, not to itself.

Nothing here reuses the oracle's cell enumeration.  Each check computes the
Euler characteristic curve some other way:

* ``bruteforce_ecc``: the naive O(mn) method of Sec. 2.3 -- threshold the
  image at every level, build the indicator of every cell type by shifting
  and AND-ing (V-mode: all vertices present) or OR-dilating (T-mode: some
  coface present) the thresholded array, and form sum (-1)^dim * count.
* ``betti_ecc_2d``: beta_0 - beta_1 from connected components (the
  Euler-Poincare equality in Eq. 1), with the digital-topology pairing each
  complex induces: (4, 8) connectivity for V-mode, (8, 4) for T-mode.
* closed forms for shapes whose homotopy type is known.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy import ndimage


def _levels(lo, hi):
    return range(lo, hi + 1)


def _vertex_cell_counts(B: np.ndarray):
    """sum over axis subsets A of (-1)^|A| * #{p : all of p + {0,1}^A in B}."""
    d = B.ndim
    chi = 0
    for A in itertools.product((0, 1), repeat=d):
        arr = B
        for a in range(d):
            if A[a]:
                n = arr.shape[a]
                lo = [slice(None)] * d
                hi = [slice(None)] * d
                lo[a] = slice(0, n - 1)
                hi[a] = slice(1, n)
                arr = arr[tuple(lo)] & arr[tuple(hi)]
        chi += (-1) ** sum(A) * int(arr.sum())
    return chi


def _topcell_cell_counts(B: np.ndarray):
    """sum over interval types of (-1)^dim * #{cells with some coface voxel in B}.

    Along an axis, degenerate intervals [k,k] (k = 0..n) touch voxels k-1 and
    k; non-degenerate [k,k+1] touch voxel k only.
    """
    d = B.ndim
    chi = 0
    for deg in itertools.product((0, 1), repeat=d):
        arr = B
        for a in range(d):
            if deg[a]:
                pad = [(0, 0)] * d
                pad[a] = (1, 1)
                p = np.pad(arr, pad, constant_values=False)
                n = p.shape[a]
                lo = [slice(None)] * d
                hi = [slice(None)] * d
                lo[a] = slice(0, n - 1)
                hi[a] = slice(1, n)
                arr = p[tuple(lo)] | p[tuple(hi)]
        dim = d - sum(deg)
        chi += (-1) ** dim * int(arr.sum())
    return chi


def bruteforce_ecc(img: np.ndarray, lo: int, hi: int, mode: str) -> np.ndarray:
    count = _vertex_cell_counts if mode == "vertex" else _topcell_cell_counts
    return np.array([count(img <= t) for t in _levels(lo, hi)], dtype=np.int64)


def _components(mask: np.ndarray, full: bool) -> int:
    structure = ndimage.generate_binary_structure(mask.ndim, mask.ndim if full else 1)
    return int(ndimage.label(mask, structure=structure)[1])


def betti_ecc_2d(img: np.ndarray, lo: int, hi: int, mode: str) -> np.ndarray:
    """beta_0 - beta_1 of K_{<=t} for a 2D image, at every level t."""
    out = []
    for t in _levels(lo, hi):
        F = img <= t
        # background plus a one-pixel frame that stands for the outside
        bg = np.pad(~F, 1, constant_values=True)
        if mode == "vertex":
            b0 = _components(F, full=False)          # 4-connected foreground
            b1 = _components(bg, full=True) - 1      # 8-connected background
        else:
            b0 = _components(F, full=True)           # 8-connected foreground
            b1 = _components(bg, full=False) - 1     # 4-connected background
        out.append(b0 - b1)
    return np.array(out, dtype=np.int64)


def vcec_of(ecc: np.ndarray) -> np.ndarray:
    v = ecc.copy()
    v[1:] -= ecc[:-1]
    return v


def symmetries(img: np.ndarray):
    """All axis permutations combined with all axis flips."""
    d = img.ndim
    for perm in itertools.permutations(range(d)):
        t = np.transpose(img, perm)
        for flips in itertools.product((False, True), repeat=d):
            u = t
            for a, f in enumerate(flips):
                if f:
                    u = np.flip(u, axis=a)
            yield np.ascontiguousarray(u)


def bruteforce_ecc_levels(img: np.ndarray, levels, mode: str) -> np.ndarray:
    """The naive method at given thresholds of a float image (Eq. 1 with the
    t_i given): threshold at each level and count cells.  A NaN voxel is at
    no level, i.e. above all of them."""
    count = _vertex_cell_counts if mode == "vertex" else _topcell_cell_counts
    return np.array([count(img <= t) for t in levels], dtype=np.int64)
