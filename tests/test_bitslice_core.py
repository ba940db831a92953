"""CPU checks of the bit-sliced building blocks used by the CUDA stencil
(transpose to bit planes, bit-serial comparison, carry-save counting and the
per-voxel cell count), each against naive per-voxel Python."""
import ctypes
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
    for n in ("h_transpose_u8", "h_transpose_u16", "h_count26"):
        getattr(lib, n).argtypes = [u32p, u32p]
    for n in ("h_ge8", "h_ge16"):
        getattr(lib, n).argtypes = [u32p, u32p]
        getattr(lib, n).restype = ctypes.c_uint32
    lib.h_kappa3d.argtypes = [u32p, u32p]
    lib.h_kappa3d.restype = ctypes.c_uint32
    lib.h_kappa2d.argtypes = [u32p, u32p, u32p]
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


@pytest.mark.parametrize("n,fn", [(26, "h_count26")])
def test_counters(h, n, fn):
    rng = np.random.default_rng(3)
    for _ in range(300):
        x = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        o = np.zeros(5, np.uint32)
        getattr(h, fn)(_p(x), _p(o))
        want = [sum((int(x[i]) >> b) & 1 for i in range(n)) for b in range(32)]
        assert _vals(o, 5) == want


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
            T = np.zeros(5, np.uint32)
            nz = h.h_kappa3d(_p(w27), _p(T))
            t = _vals(T, 5)
            for x in range(32):
                w = bits[:, x].reshape(3, 3, 3).astype(int)
                kap = kappa3d_scalar(w)
                assert t[x] - 13 == kap
                assert ((nz >> x) & 1) == (kap != 0)


def test_kappa2d(h):
    rng = np.random.default_rng(5)
    for density in (0.2, 0.5, 0.8):
        for _ in range(60):
            bits = (rng.uniform(size=(9, 32)) < density).astype(np.uint64)
            w9 = np.array([sum(int(bits[i, x]) << x for x in range(32)) for i in range(9)], np.uint32)
            F = np.zeros(3, np.uint32)
            Q = np.zeros(3, np.uint32)
            nz = h.h_kappa2d(_p(w9), _p(F), _p(Q))
            f, q = _vals(F, 3), _vals(Q, 3)
            for x in range(32):
                w = bits[:, x].reshape(3, 3).astype(int)
                kap = 1 - (w[1, 0] + w[1, 2] + w[0, 1] + w[2, 1])
                for a in (0, 2):
                    for b in (0, 2):
                        kap += w[a, 1] & w[1, b] & w[a, b]
                assert 1 - f[x] + q[x] == kap
                assert ((nz >> x) & 1) == (kap != 0)
