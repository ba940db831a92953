"""CPU checks of the bit-sliced building blocks used by the CUDA stencil
(transpose to bit planes, bit-serial comparison, carry-save counting and the
per-voxel cell count), each against naive per-voxel Python."""
import ctypes
import itertools
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent
CSRC = ROOT / "paper_2203_09087_gb300" / "csrc"


@pytest.fixture(scope="module")
def h(tmp_path_factory):
    out = tmp_path_factory.mktemp("bs") / "libbs.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", str(CSRC),
                    str(ROOT / "tests" / "bitslice_harness.cpp"), "-o", str(out)], check=True)
    lib = ctypes.CDLL(str(out))
    u32p = ctypes.POINTER(ctypes.c_uint32)
    for n in ("h_transpose_u8", "h_transpose_u16", "h_count12", "h_split_pm1_2d", "h_split_pm1_3d"):
        getattr(lib, n).argtypes = [u32p, u32p]
    for n in ("h_ge8", "h_ge16"):
        getattr(lib, n).argtypes = [u32p, u32p]
        getattr(lib, n).restype = ctypes.c_uint32
    lib.h_kappa3d.argtypes = [u32p, u32p]
    lib.h_kappa3d.restype = ctypes.c_uint32
    lib.h_kappa2d.argtypes = [u32p, u32p]
    lib.h_kappa3d_many.argtypes = [u32p, ctypes.c_int64, u32p, u32p]
    lib.h_kappa2d.restype = ctypes.c_uint32
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def planes_naive(vox: np.ndarray, k: int) -> np.ndarray:
    out = np.zeros(k, np.uint32)
    for b in range(k):
        for x in range(32):
            out[b] |= np.uint32(((int(vox[x]) >> b) & 1) << x)
    return out


def test_transpose_u8(h):
    rng = np.random.default_rng(0)
    for _ in range(200):
        vox = rng.integers(0, 256, size=32, dtype=np.uint8)
        r = np.frombuffer(vox.tobytes(), dtype=np.uint32).copy()
        p = np.zeros(8, np.uint32)
        h.h_transpose_u8(_p(r), _p(p))
        assert np.array_equal(p, planes_naive(vox, 8))


def test_transpose_u16(h):
    rng = np.random.default_rng(1)
    for _ in range(200):
        vox = rng.integers(0, 65536, size=32, dtype=np.uint16)
        r = np.frombuffer(vox.tobytes(), dtype=np.uint32).copy()
        p = np.zeros(16, np.uint32)
        h.h_transpose_u16(_p(r), _p(p))
        assert np.array_equal(p, planes_naive(vox, 16))


@pytest.mark.parametrize("k", [8, 16])
def test_bit_serial_compare(h, k):
    rng = np.random.default_rng(2)
    f = h.h_ge8 if k == 8 else h.h_ge16
    for levels in (2, 5, 1 << k):
        for _ in range(100):
            a = rng.integers(0, levels, size=32)
            b = rng.integers(0, levels, size=32)
            got = f(_p(planes_naive(a, k)), _p(planes_naive(b, k)))
            want = sum(1 << x for x in range(32) if a[x] >= b[x])
            assert got == want


def _vals(planes, nbits):
    return [sum(((int(planes[k]) >> x) & 1) << k for k in range(nbits)) for x in range(32)]


@pytest.mark.parametrize("n,fn,planes", [(12, "h_count12", 4)])
def test_counters(h, n, fn, planes):
    rng = np.random.default_rng(3)
    for density in (0.1, 0.5, 0.9, 1.0):
        for _ in range(100):
            x = np.array([sum(int(rng.uniform() < density) << b for b in range(32)) for _ in range(n)], np.uint32)
            o = np.zeros(planes, np.uint32)
            getattr(h, fn)(_p(x), _p(o))
            want = [sum((int(x[i]) >> b) & 1 for i in range(n)) for b in range(32)]
            assert _vals(o, planes) == want


def kappa3d_scalar(w):
    """1 - faces + squares - cubes from the 26 wins w[dz][dy][dx] (0/1)."""
    k = 1
    faces = [(0, 1, 1), (2, 1, 1), (1, 0, 1), (1, 2, 1), (1, 1, 0), (1, 1, 2)]
    k -= sum(w[f] for f in faces)
    for a in (0, 2):
        for b in (0, 2):
            k += w[1, a, 1] & w[1, 1, b] & w[1, a, b]
            k += w[a, 1, 1] & w[1, 1, b] & w[a, 1, b]
            k += w[a, 1, 1] & w[1, b, 1] & w[a, b, 1]
    for c in (0, 2):
        for b in (0, 2):
            for a in (0, 2):
                k -= (w[c, 1, 1] & w[1, b, 1] & w[1, 1, a] & w[c, b, 1] & w[c, 1, a] & w[1, b, a] & w[c, b, a])
    return k


def test_kappa3d(h):
    rng = np.random.default_rng(4)
    for density in (0.1, 0.5, 0.9, 0.97):
        for _ in range(40):
            bits = (rng.uniform(size=(27, 32)) < density).astype(np.uint64)
            w27 = np.array([sum(int(bits[i, x]) << x for x in range(32)) for i in range(27)], np.uint32)
            T = np.zeros(4, np.uint32)
            nz = h.h_kappa3d(_p(w27), _p(T))
            t = _vals(T, 4)
            for x in range(32):
                w = bits[:, x].reshape(3, 3, 3).astype(int)
                kap = kappa3d_scalar(w)
                assert t[x] - 5 == kap
                assert ((nz >> x) & 1) == (kap != 0)


def test_kappa3d_exhaustive(h):
    """The chain grouping of the signed cell count is an identity of the 26
    win bits: check every one of the 2^26 win patterns against
    1 - faces + squares - cubes evaluated term by term."""
    n_cfg = 1 << 26
    words = n_cfg // 32
    j = np.arange(words, dtype=np.uint32)
    # input bit b of configuration 32*j + x is bit b of that index
    win_idx = [i for i in range(27) if i != 13]           # skip the centre
    w27 = np.zeros((27, words), np.uint32)
    low = [np.uint32(sum(1 << x for x in range(32) if (x >> b) & 1)) for b in range(5)]
    for b, i in enumerate(win_idx):
        w27[i] = low[b] if b < 5 else np.where((j >> (b - 5)) & 1, np.uint32(0xFFFFFFFF), np.uint32(0))
    T = np.zeros((4, words), np.uint32)
    nz = np.zeros(words, np.uint32)
    h.h_kappa3d_many(_p(w27), words, _p(T), _p(nz))
    # reference: per configuration, from the index bits (in chunks)
    bit = lambda arr: ((arr[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1).astype(np.int8)
    chunk = 1 << 22
    for c0 in range(0, n_cfg, chunk):
        cfg = np.arange(c0, c0 + chunk, dtype=np.uint32)
        wb = {i: ((cfg >> b) & 1).astype(np.int8) for b, i in enumerate(win_idx)}
        W = lambda dz, dy, dx: wb[9 * dz + 3 * dy + dx]
        kap = np.ones(chunk, np.int8)
        for f in [(0, 1, 1), (2, 1, 1), (1, 0, 1), (1, 2, 1), (1, 1, 0), (1, 1, 2)]:
            kap -= W(*f)
        for a in (0, 2):
            for b in (0, 2):
                kap += W(1, a, 1) & W(1, 1, b) & W(1, a, b)
                kap += W(a, 1, 1) & W(1, 1, b) & W(a, 1, b)
                kap += W(a, 1, 1) & W(1, b, 1) & W(a, b, 1)
        for c in (0, 2):
            for b in (0, 2):
                for a in (0, 2):
                    kap -= (W(c, 1, 1) & W(1, b, 1) & W(1, 1, a) & W(c, b, 1) & W(c, 1, a) & W(1, b, a)
                            & W(c, b, a))
        sl = slice(c0 // 32, (c0 + chunk) // 32)
        t = bit(T[0, sl]) + 2 * bit(T[1, sl]) + 4 * bit(T[2, sl]) + 8 * bit(T[3, sl])
        assert np.array_equal(t - 5, kap)
        assert np.array_equal(bit(nz[sl]), (kap != 0).astype(np.int8))


def test_kappa2d(h):
    rng = np.random.default_rng(5)
    for density in (0.2, 0.5, 0.8):
        for _ in range(60):
            bits = (rng.uniform(size=(9, 32)) < density).astype(np.uint64)
            w9 = np.array([sum(int(bits[i, x]) << x for x in range(32)) for i in range(9)], np.uint32)
            X = np.zeros(3, np.uint32)
            nz = h.h_kappa2d(_p(w9), _p(X))
            for x in range(32):
                xs = [(int(X[j]) >> x) & 1 for j in range(3)]
                w = bits[:, x].reshape(3, 3).astype(int)
                kap = 1 - (w[1, 0] + w[1, 2] + w[0, 1] + w[2, 1])
                for a in (0, 2):
                    for b in (0, 2):
                        kap += w[a, 1] & w[1, b] & w[a, b]
                assert xs[0] + xs[1] + 2 * xs[2] - 3 == kap
                assert ((nz >> x) & 1) == (kap != 0)


def _kappa4_scalar(w):
    """1 - edges + squares - cubes + tesseracts over the 81 cells of 4D
    containing the voxel, from the 80 wins w[dw][dz][dy][dx] (0/1): a cell
    (axis subset A, a side per axis) is won when every nonempty sub-sum of
    its sides is."""
    k = 0
    for A in itertools.product((0, 1), repeat=4):
        axes = [i for i in range(4) if A[i]]
        for sides in itertools.product((-1, 1), repeat=len(axes)):
            won = 1
            for B in itertools.product((0, 1), repeat=len(axes)):
                if not any(B):
                    continue
                d = [0, 0, 0, 0]
                for j, ax in enumerate(axes):
                    if B[j]:
                        d[ax] = sides[j]
                won &= w[d[0] + 1, d[1] + 1, d[2] + 1, d[3] + 1]
            k += (-1) ** len(axes) * won
    return k


def test_kappa4d_against_the_81_cells(h):
    rng = np.random.default_rng(6)
    h.h_kappa4d.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32)]
    h.h_kappa4d.restype = ctypes.c_uint32
    for density in (0.2, 0.5, 0.8, 0.95, 0.99):
        for _ in range(12):
            bits = (rng.uniform(size=(81, 32)) < density).astype(np.uint64)
            w81 = np.array([sum(int(bits[i, x]) << x for x in range(32)) for i in range(81)], np.uint32)
            kap = np.zeros(32, np.int32)
            nz = h.h_kappa4d(_p(w81), kap.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
            for x in range(32):
                want = _kappa4_scalar(bits[:, x].reshape(3, 3, 3, 3).astype(int))
                assert kap[x] == want
                assert ((nz >> x) & 1) == (want != 0)


def test_kappa4_nonzero_exhaustive(h):
    """The 6-plane adder that decides kappa4 != 0 from the three chain counts
    (each 0..12) and the two w-wins, against the integer formula, for every
    combination."""
    I32 = ctypes.POINTER(ctypes.c_int32)
    h.h_kappa4_nonzero.argtypes = [I32] * 5
    h.h_kappa4_nonzero.restype = ctypes.c_uint32
    cases = np.array([(a, b, c, p, m) for a in range(13) for b in range(13) for c in range(13)
                      for p in (0, 1) for m in (0, 1)], np.int32)
    pad = (-len(cases)) % 32
    cases = np.concatenate([cases, np.tile(cases[:1], (pad, 1))])
    want = ((cases[:, 0] - 5) - cases[:, 3] * (cases[:, 1] - 5) - cases[:, 4] * (cases[:, 2] - 5)) != 0
    for g in range(0, len(cases), 32):
        blk = np.ascontiguousarray(cases[g:g + 32].T)
        nz = h.h_kappa4_nonzero(*[blk[j].ctypes.data_as(I32) for j in range(5)])
        got = np.array([(nz >> i) & 1 for i in range(32)], bool)
        assert np.array_equal(got, want[g:g + 32]), g


# ---------------------------------------------------------------------------
# The 3D walker's bit logic (ecc_bitlogic.cuh): explicit three-input logic
# operations and multiply shifts, against naive code and the plain forms.

def _w3(h):
    u32p = ctypes.POINTER(ctypes.c_uint32)
    for n in ("h_w3_transpose_u8", "h_w3_transpose_u16", "h_w3_count12"):
        getattr(h, n).argtypes = [u32p, u32p]
    for n in ("h_w3_ge8", "h_w3_ge16"):
        getattr(h, n).argtypes = [u32p, u32p]
        getattr(h, n).restype = ctypes.c_uint32
    h.h_w3_kappa3.argtypes = [u32p, ctypes.c_uint32, u32p]
    h.h_w3_kappa3.restype = ctypes.c_uint32
    return h


@pytest.mark.parametrize("bits", [8, 16])
def test_walker_transpose_matches_naive(h, bits):
    w3 = _w3(h)
    rng = np.random.default_rng(40 + bits)
    dt = np.uint8 if bits == 8 else np.uint16
    fn = w3.h_w3_transpose_u8 if bits == 8 else w3.h_w3_transpose_u16
    for _ in range(200):
        vox = rng.integers(0, 1 << bits, size=32, dtype=dt)
        r = np.frombuffer(vox.tobytes(), dtype=np.uint32).copy()
        p = np.zeros(bits, np.uint32)
        fn(_p(r), _p(p))
        assert np.array_equal(p, planes_naive(vox, bits))


@pytest.mark.parametrize("bits", [8, 16])
def test_walker_ge_matches_naive(h, bits):
    w3 = _w3(h)
    rng = np.random.default_rng(50 + bits)
    fn = w3.h_w3_ge8 if bits == 8 else w3.h_w3_ge16
    for levels in (2, 5, 1 << bits):
        for _ in range(100):
            a = rng.integers(0, levels, size=32)
            b = rng.integers(0, levels, size=32)
            pa, pb = planes_naive(a, bits), planes_naive(b, bits)
            want = sum(1 << x for x in range(32) if a[x] >= b[x])
            assert fn(_p(pa), _p(pb)) == want


def test_walker_count12_matches_plain(h):
    w3 = _w3(h)
    rng = np.random.default_rng(60)
    for _ in range(300):
        x = rng.integers(0, 1 << 32, size=12, dtype=np.uint64).astype(np.uint32)
        o1 = np.zeros(4, np.uint32)
        o2 = np.zeros(4, np.uint32)
        h.h_count12(_p(x), _p(o1))
        w3.h_w3_count12(_p(x), _p(o2))
        assert np.array_equal(o1, o2)


def test_walker_cell_count_equals_plain_on_random_and_structured_wins(h):
    """kappa3w (the walker's polarities, explicit truth tables) against
    bs::kappa3d, which the chain identity pins on all 2^26 win patterns."""
    w3 = _w3(h)
    rng = np.random.default_rng(61)
    for density in (0.05, 0.3, 0.5, 0.7, 0.95):
        for _ in range(200):
            w = (rng.uniform(size=(27, 32)) < density)
            w27 = np.array([sum(int(w[i, x]) << x for x in range(32)) for i in range(27)], np.uint32)
            w27[13] = 0
            t1 = np.zeros(4, np.uint32)
            t2 = np.zeros(4, np.uint32)
            nz1 = h.h_kappa3d(_p(w27), _p(t1))
            out_x = int(rng.integers(0, 1 << 32))
            nz2 = w3.h_w3_kappa3(_p(w27), out_x, _p(t2))
            assert np.array_equal(t1, t2)
            assert nz2 == (nz1 & out_x)


def test_2d_walker_cell_count_equals_plain(h):
    """kappa2w (the 2D walker's polarities, explicit truth tables) against
    bs::kappa2d on random win masks of every density, and exhaustively on
    all 2^8 patterns of one voxel."""
    u32p = ctypes.POINTER(ctypes.c_uint32)
    h.h_w2_kappa2.argtypes = [u32p, ctypes.c_uint32, u32p]
    h.h_w2_kappa2.restype = ctypes.c_uint32
    rng = np.random.default_rng(62)
    for density in (0.1, 0.5, 0.9):
        for _ in range(300):
            w9 = rng.integers(0, 1 << 32, size=9, dtype=np.uint64).astype(np.uint32)
            if density != 0.5:
                bits = rng.uniform(size=(9, 32)) < density
                w9 = np.array([sum(int(bits[i, x]) << x for x in range(32)) for i in range(9)], np.uint32)
            w9[4] = 0
            x1 = np.zeros(3, np.uint32)
            x2 = np.zeros(3, np.uint32)
            nz1 = h.h_kappa2d(_p(w9), _p(x1))
            out_x = int(rng.integers(0, 1 << 32))
            nz2 = h.h_w2_kappa2(_p(w9), out_x, _p(x2))
            assert np.array_equal(x1, x2)
            assert nz2 == (nz1 & out_x)
    # every pattern of the 8 neighbours at once: bit x of input i is bit i of x's pattern
    pats = np.arange(256, dtype=np.uint32)
    for base in range(0, 256, 32):
        w9 = np.zeros(9, np.uint32)
        nbr = [0, 1, 2, 3, 5, 6, 7, 8]
        for j, i in enumerate(nbr):
            w9[i] = np.uint32(sum(((int(p) >> j) & 1) << x for x, p in enumerate(pats[base:base + 32])))
        x1 = np.zeros(3, np.uint32)
        x2 = np.zeros(3, np.uint32)
        assert h.h_w2_kappa2(_p(w9), 0xffffffff, _p(x2)) == h.h_kappa2d(_p(w9), _p(x1))
        assert np.array_equal(x1, x2)


@pytest.mark.parametrize("dim", [2, 3])
def test_emission_split_of_unit_counts(h, dim):
    """The emission's split of the counts: pm marks exactly the voxels whose
    count is +1 or -1 and plus exactly the +1 among them, for every value
    of the count planes (bit x of the planes holds pattern x)."""
    nplanes = 3 if dim == 2 else 4
    pats = np.arange(1 << nplanes)
    planes = np.array([sum(((int(p) >> k) & 1) << x for x, p in enumerate(pats)) for k in range(nplanes)],
                      np.uint32)
    out = np.zeros(2, np.uint32)
    getattr(h, f"h_split_pm1_{dim}d")(_p(planes), _p(out))
    for x, p in enumerate(pats):
        bits = [(int(p) >> k) & 1 for k in range(nplanes)]
        count = bits[0] + bits[1] + 2 * bits[2] - 3 if dim == 2 else int(p) - 5
        assert ((int(out[0]) >> x) & 1) == (count in (1, -1)), (dim, p)
        if count in (1, -1):
            assert ((int(out[1]) >> x) & 1) == (count == 1), (dim, p)
