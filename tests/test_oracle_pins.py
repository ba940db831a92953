"""Pins for the CPU oracle (no GPU).

The oracle enumerates cells one by one (Sec. 2.1-2.3).  These tests tie it to
results fixed by mathematics rather than to itself: the naive per-threshold
method (Sec. 2.3), Betti numbers from flood fill (Eq. 1 via Euler-Poincare),
closed forms for shapes of known homotopy type, symmetry invariance, the
exact top-cell/vertex duality, and the additivity of chunks (Sec. 3.4).
``test_mutants_are_caught`` plants plausible mistakes in a copy of the oracle
and checks that these pins catch every one.
"""
import itertools
from pathlib import Path

import numpy as np
import pytest

import oracle
from tests import pins

MODES = (oracle.VERTEX, oracle.TOPCELL)


def _ecc(img, lo, hi, mode, lib=None):
    return oracle.ecc(img, lo, hi, mode, lib=lib)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("mode", MODES)
def test_exhaustive_3x3_three_levels(mode):
    """All 3^9 images of size 3x3 over {0,1,2}: oracle == naive method == beta0-beta1."""
    lib = oracle.load()
    vals = np.array(list(itertools.product(range(3), repeat=9)), dtype=np.uint8).reshape(-1, 3, 3)
    for img in vals:
        got = _ecc(img, 0, 2, mode, lib)
        assert np.array_equal(got, pins.bruteforce_ecc(img, 0, 2, mode)), img
        assert np.array_equal(got, pins.betti_ecc_2d(img, 0, 2, mode)), img


@pytest.mark.parametrize("mode", MODES)
def test_exhaustive_2x2x2_three_levels(mode):
    lib = oracle.load()
    vals = np.array(list(itertools.product(range(3), repeat=8)), dtype=np.uint8).reshape(-1, 2, 2, 2)
    for img in vals:
        assert np.array_equal(_ecc(img, 0, 2, mode, lib), pins.bruteforce_ecc(img, 0, 2, mode)), img


@pytest.mark.parametrize("mode", MODES)
def test_random_small_2d_vs_bruteforce_and_betti(mode):
    rng = np.random.default_rng(11)
    for _ in range(300):
        h, w = rng.integers(1, 8, size=2)
        levels = int(rng.integers(1, 7))
        img = rng.integers(0, levels, size=(h, w)).astype(np.uint8)
        got = _ecc(img, 0, levels - 1, mode)
        assert np.array_equal(got, pins.bruteforce_ecc(img, 0, levels - 1, mode))
        assert np.array_equal(got, pins.betti_ecc_2d(img, 0, levels - 1, mode))


@pytest.mark.parametrize("mode", MODES)
def test_random_small_3d_vs_bruteforce(mode):
    rng = np.random.default_rng(12)
    for _ in range(150):
        d, h, w = rng.integers(1, 6, size=3)
        levels = int(rng.integers(1, 7))
        img = rng.integers(0, levels, size=(d, h, w)).astype(np.uint8)
        assert np.array_equal(_ecc(img, 0, levels - 1, mode), pins.bruteforce_ecc(img, 0, levels - 1, mode))


def test_uint16_and_offset_range_vs_bruteforce():
    rng = np.random.default_rng(13)
    for mode in MODES:
        img = rng.integers(1000, 1006, size=(4, 5, 3)).astype(np.uint16)
        assert np.array_equal(_ecc(img, 998, 1007, mode), pins.bruteforce_ecc(img, 998, 1007, mode))


def test_one_dimensional_components():
    """In 1D the Euler characteristic of a sublevel set is its number of runs."""
    rng = np.random.default_rng(14)
    for _ in range(100):
        n = int(rng.integers(1, 20))
        img = rng.integers(0, 4, size=n).astype(np.uint8)
        got = _ecc(img, 0, 3, oracle.VERTEX)
        runs = []
        for t in range(4):
            b = (img <= t).astype(np.int8)
            runs.append(int(np.sum(np.diff(np.concatenate([[0], b])) == 1)))
        assert np.array_equal(got, runs)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", [(1, 1), (5, 7), (1, 1, 1), (3, 4, 5)])
def test_constant_image_is_a_single_step(mode, shape):
    img = np.full(shape, 7, dtype=np.uint8)
    v = oracle.vcec(img, 0, 9, mode)
    expect = np.zeros(10, dtype=np.int64)
    expect[7] = 1
    assert np.array_equal(v, expect)


@pytest.mark.parametrize("mode", MODES)
def test_full_box_ends_at_one(mode):
    rng = np.random.default_rng(15)
    for shape in [(9, 13), (4, 6, 5), (1, 17), (17, 1, 3)]:
        img = rng.integers(0, 256, size=shape).astype(np.uint8)
        assert oracle.vcec(img, 0, 255, mode).sum() == 1
        assert _ecc(img, 0, 255, mode)[-1] == 1


@pytest.mark.parametrize("mode", MODES)
def test_one_bright_interior_voxel(mode):
    """Box minus the open star of an interior point: circle in 2D, sphere in 3D."""
    a, b = 3, 7
    img2 = np.full((5, 6), a, np.uint8)
    img2[2, 3] = b
    v2 = oracle.vcec(img2, 0, 9, mode)
    assert (v2[a], v2[b]) == (0, 1) and np.count_nonzero(v2) == 1
    img3 = np.full((5, 6, 4), a, np.uint8)
    img3[2, 3, 1] = b
    v3 = oracle.vcec(img3, 0, 9, mode)
    assert (v3[a], v3[b]) == (2, -1) and np.count_nonzero(v3) == 2


@pytest.mark.parametrize("mode", MODES)
def test_one_bright_corner_voxel_changes_nothing_topologically(mode):
    a, b = 2, 5
    for shape, corner in [((4, 5), (0, 4)), ((3, 4, 5), (2, 0, 4))]:
        img = np.full(shape, a, np.uint8)
        img[corner] = b
        v = oracle.vcec(img, 0, 9, mode)
        assert (v[a], v[b]) == (1, 0) and np.count_nonzero(v) == 1


@pytest.mark.parametrize("mode", MODES)
def test_one_dark_voxel_in_bright_box(mode):
    a, b = 1, 8
    img = np.full((4, 5, 6), b, np.uint8)
    img[1, 2, 3] = a
    v = oracle.vcec(img, 0, 9, mode)
    assert (v[a], v[b]) == (1, 0) and np.count_nonzero(v) == 1


def _binary(shape, fg_slices, holes=()):
    img = np.ones(shape, np.uint8)
    for s in fg_slices:
        img[s] = 0
    for h in holes:
        img[h] = 1
    return img


CLOSED_FORMS = [
    # (name, image, chi of the foreground complex; same in both complexes)
    ("solid box", _binary((7, 7, 7), [np.s_[1:5, 2:6, 1:4]]), 1),
    ("three boxes", _binary((9, 9, 9), [np.s_[0:2, 0:2, 0:2], np.s_[4:6, 4:6, 4:6], np.s_[7:9, 0:3, 6:9]]), 3),
    ("hollow shell (sphere)", _binary((7, 7, 7), [np.s_[2:5, 2:5, 2:5]], holes=[(3, 3, 3)]), 2),
    ("two cavities", _binary((7, 7, 9), [np.s_[2:5, 2:5, 2:7]], holes=[(3, 3, 3), (3, 3, 5)]), 3),
    ("planar ring (circle / solid torus)", _binary((5, 7, 7), [np.s_[2, 2:5, 2:5]], holes=[(2, 3, 3)]), 0),
    ("tube through a block", _binary((9, 7, 7), [np.s_[2:7, 2:5, 2:5]], holes=[np.s_[2:7, 3, 3]]), 0),
    ("plate with two holes", _binary((9, 11), [np.s_[1:8, 1:10]], holes=[(3, 3), (5, 7)]), -1),
    ("annulus", _binary((8, 8), [np.s_[1:7, 1:7]], holes=[np.s_[3:5, 3:5]]), 0),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name,img,chi", CLOSED_FORMS, ids=[c[0] for c in CLOSED_FORMS])
def test_shapes_of_known_topology(mode, name, img, chi):
    e = _ecc(img, 0, 1, mode)
    assert e[0] == chi, name
    assert e[1] == 1


# ---------------------------------------------------------------- symmetries

@pytest.mark.parametrize("mode", MODES)
def test_invariance_under_flips_and_transposes(mode):
    rng = np.random.default_rng(16)
    img3 = rng.integers(0, 6, size=(3, 4, 5)).astype(np.uint8)
    ref = oracle.vcec(img3, 0, 5, mode)
    for s in pins.symmetries(img3):
        assert np.array_equal(oracle.vcec(s, 0, 5, mode), ref)
    img2 = rng.integers(0, 6, size=(5, 7)).astype(np.uint8)
    ref2 = oracle.vcec(img2, 0, 5, mode)
    for s in pins.symmetries(img2):
        assert np.array_equal(oracle.vcec(s, 0, 5, mode), ref2)


@pytest.mark.parametrize("mode", MODES)
def test_depth_one_volume_equals_the_image(mode):
    rng = np.random.default_rng(17)
    img = rng.integers(0, 256, size=(9, 14)).astype(np.uint8)
    ref = oracle.vcec(img, 0, 255, mode)
    assert np.array_equal(oracle.vcec(img[None], 0, 255, mode), ref)
    assert np.array_equal(oracle.vcec(img[:, None, :], 0, 255, mode), ref)


def test_value_remap_permutes_bins():
    """A strictly increasing relabelling of gray levels moves bins, nothing else."""
    rng = np.random.default_rng(18)
    img = rng.integers(0, 5, size=(4, 5, 6)).astype(np.uint8)
    remap = np.array([2, 3, 9, 20, 21], np.uint8)
    for mode in MODES:
        v = oracle.vcec(img, 0, 4, mode)
        w = oracle.vcec(remap[img], 0, 21, mode)
        assert np.array_equal(w[remap], v) and w.sum() == v.sum()


@pytest.mark.parametrize("ndim", [2, 3])
def test_topcell_vertex_duality(ndim):
    """Top-cell cells of I <-> vertex cells of (lo+hi-I) with a collar below every level.

    Each top-cell cell is a box of voxels (its cofaces); it is the vertex cell
    of the reflected image with those vertices once the image is padded by a
    collar whose value is below every real level, and its dimension becomes
    d - dim.  So VCEC_T(I)[t] = (-1)^d VCEC_V(pad(lo+hi-I))[lo+hi-t].
    """
    rng = np.random.default_rng(19)
    lo, hi = 1, 6
    for _ in range(30):
        shape = tuple(rng.integers(1, 6, size=ndim))
        img = rng.integers(lo, hi + 1, size=shape).astype(np.uint8)
        t = oracle.vcec(img, lo, hi, oracle.TOPCELL)
        refl = np.pad((lo + hi - img.astype(np.int32)).astype(np.uint8), 1, constant_values=lo - 1)
        v = oracle.vcec(refl, lo - 1, hi, oracle.VERTEX)
        for level in range(lo, hi + 1):
            assert t[level - lo] == (-1) ** ndim * v[(lo + hi - level) - (lo - 1)]


# ---------------------------------------------------------------- chunking

@pytest.mark.parametrize("mode", MODES)
def test_chunks_add_up(mode):
    """Sec. 3.4: disjoint chunks along dims[0] with a one-voxel collar sum to the whole."""
    rng = np.random.default_rng(20)
    img = rng.integers(0, 256, size=(11, 6, 7)).astype(np.uint8)
    full = oracle.vcec(img, 0, 255, mode)
    n = oracle.row_extent(img.shape, mode)
    for cuts in ([0, n], [0, 1, n], [0, 3, 4, 9, n], list(range(n + 1))):
        parts = sum(oracle.vcec_rows(img, a, b, 0, 255, mode) for a, b in zip(cuts[:-1], cuts[1:]))
        assert np.array_equal(parts, full)
    assert np.array_equal(oracle.vcec_parallel(img, 0, 255, mode, threads=4), full)


def test_errors():
    img = np.array([[0, 5], [3, 9]], np.uint8)
    with pytest.raises(oracle.OracleError):
        oracle.vcec(img, 0, 8)          # 9 is outside [0, 8]
    with pytest.raises(oracle.OracleError):
        oracle.vcec(img, 5, 4)          # hi < lo
    with pytest.raises(TypeError):
        oracle.vcec(img.astype(np.float32))


# ---------------------------------------------------------------- golden file

def test_golden_256sq_uniform():
    """The stored ECC of the 256x256 uniform image was written by
    tests/golden/make_golden.py, which calls only the oracle."""
    import synth
    path = Path(__file__).parent / "golden" / "uniform_256x256_seed0_vertex.txt"
    want = np.loadtxt(path, dtype=np.int64)
    img = synth.uniform_2d_256()
    assert np.array_equal(oracle.ecc(img, 0, 255, oracle.VERTEX), want)
    # the same image checked independently at a few thresholds by flood fill
    for t in (0, 37, 128, 200, 255):
        assert pins.betti_ecc_2d(img, t, t, "vertex")[0] == want[t]


# ---------------------------------------------------------------- mutation check

MUTANTS = [
    # (name, anchor, replacement, which occurrence of the anchor)
    ("sign dropped in vertex cells", "vcec[value - lo] += (dim % 2 == 0) ? 1 : -1;",
     "vcec[value - lo] += 1;", 0),
    ("sign dropped in top cells", "vcec[value - lo] += (dim % 2 == 0) ? 1 : -1;",
     "vcec[value - lo] += 1;", 1),
    ("cubes dropped", "if (!exists) continue;", "if (!exists || dim == 3) continue;", 0),
    ("max replaced by last vertex", "if (v > value) value = v;", "value = v;", 0),
    ("min replaced by max", "if (v < value) value = v;", "if (v > value || value == INT64_MAX) value = v;", 0),
    ("lower coface dropped", "last[a] = (k > dims[a] - 1) ? dims[a] - 1 : k;", "last[a] = first[a];", 0),
    ("top-cell dim not counted", "++dim;\n                first[a] = k;", "first[a] = k;", 0),
    ("prefix sum not accumulated", "run += vcec[g];", "run = vcec[g];", 0),
    ("far corner instead of each vertex", "q[a] = p[a] + ((B >> a) & 1u);", "q[a] = p[a] + ((A >> a) & 1u);", 0),
]


def _run_pins(lib) -> bool:
    """True when every quick pin passes for the given oracle build."""
    rng = np.random.default_rng(21)
    for mode in MODES:
        for _ in range(40):
            shape = tuple(rng.integers(1, 5, size=int(rng.integers(2, 4))))
            img = rng.integers(0, 3, size=shape).astype(np.uint8)
            if not np.array_equal(_ecc(img, 0, 2, mode, lib), pins.bruteforce_ecc(img, 0, 2, mode)):
                return False
        for name, img, chi in CLOSED_FORMS:
            if _ecc(img, 0, 1, mode, lib)[0] != chi:
                return False
    return True


def test_pins_pass_on_the_real_oracle():
    assert _run_pins(oracle.load())


@pytest.mark.parametrize("name,old,new,which", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutants_are_caught(tmp_path, name, old, new, which):
    src = (Path(oracle.__file__).parent / "ecc_oracle.c").read_text()
    starts = [i for i in range(len(src)) if src.startswith(old, i)]
    assert len(starts) > which, f"mutation anchor not found: {old!r}"
    at = starts[which]
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src[:at] + new + src[at + len(old):])
    lib_path = oracle.build(src=mutated, out=tmp_path / "libmutant.so")
    assert not _run_pins(oracle.load(lib_path)), f"mutant survived: {name}"


# ---------------------------------------------------------------- four dimensions

@pytest.mark.parametrize("mode", MODES)
def test_random_small_4d_vs_bruteforce(mode):
    rng = np.random.default_rng(71)
    for _ in range(80):
        shape = tuple(int(x) for x in rng.integers(1, 4, size=4))
        img = rng.integers(0, 3, size=shape).astype(np.uint8)
        assert np.array_equal(oracle.ecc(img, 0, 2, mode), pins.bruteforce_ecc(img, 0, 2, mode))


@pytest.mark.parametrize("mode", MODES)
def test_2x2x2x2_two_level_patterns(mode):
    for code in range(1 << 16):
        img = np.array([(code >> i) & 1 for i in range(16)], np.uint8).reshape(2, 2, 2, 2)
        if code % 97 and code not in (0, 1, 0xFFFF, 0x8000):
            continue   # every 97th of the 65536 patterns plus the extremes keeps this quick
        assert np.array_equal(oracle.ecc(img, 0, 1, mode), pins.bruteforce_ecc(img, 0, 1, mode))


def test_4d_closed_forms():
    box = np.zeros((4, 5, 3, 6), np.uint8)
    assert oracle.ecc(box, 0, 3, "vertex")[-1] == 1
    assert list(pins.vcec_of(oracle.ecc(box + 2, 0, 3, "vertex"))) == [0, 0, 1, 0]
    one = box.copy()
    one[2, 2, 1, 3] = 3                         # the dark level is a box minus a vertex star: a 3-sphere
    assert list(pins.vcec_of(oracle.ecc(one, 0, 3, "vertex"))) == [0, 0, 0, 1]
    corner = box.copy()
    corner[0, 0, 0, 0] = 3                      # a corner changes nothing topologically
    assert list(pins.vcec_of(oracle.ecc(corner, 0, 3, "vertex"))) == [1, 0, 0, 0]
    # a depth-1 4D image is the 3D volume
    rng = np.random.default_rng(72)
    vol = rng.integers(0, 5, size=(3, 4, 5)).astype(np.uint8)
    for mode in MODES:
        assert np.array_equal(oracle.ecc(vol[None], 0, 4, mode), oracle.ecc(vol, 0, 4, mode))
