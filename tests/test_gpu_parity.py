"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer work, so every comparison is bit-exact.  Inputs are seeded; shapes
span several tiles with ragged tails, size-1 axes, pitched (non-contiguous)
views, plateaus of ties, sub-ranges of gray levels, both complexes, both
element types, and both stencil kernels (the bit-sliced fast path and the
one-thread-per-voxel kernel).
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MODES = {"vertex": 0, "topcell": 1}
KERNELS = {"default": 0, "direct": 0x10}


def ecc_mod():
    import paper_2203_09087_gb300 as ecc
    return ecc


def _gpu(img: np.ndarray):
    return torch.from_numpy(img).cuda()


def _expect(img: np.ndarray, lo, hi, mode):
    return oracle.ecc(img, lo, hi, mode)


def _run(img_t, lo, hi, mode, kernel="default", with_vcec=False):
    ecc = ecc_mod()
    dt = "u8" if img_t.dtype == torch.uint8 else "u16"
    plan = ecc.ecc_plan(dt, lo, hi, complex_mode=MODES[mode], max_voxels=max(img_t.numel(), 1),
                        flags=KERNELS[kernel])
    out = torch.full((hi - lo + 1,), -777, dtype=torch.int64, device="cuda")
    v = torch.full((hi - lo + 1,), -777, dtype=torch.int64, device="cuda") if with_vcec else None
    ecc.ecc_compute(plan, img_t, out, v)
    ecc.ecc_status_get(plan)
    res = out.cpu().numpy()
    if with_vcec:
        return res, v.cpu().numpy()
    return res


SHAPES_2D = [(1, 1), (1, 37), (37, 1), (2, 2), (31, 33), (100, 77), (256, 256), (129, 1030), (700, 45),
             # either side of the 2D kernel's narrow mapping (one 30-column window per lane below 960)
             (64, 30), (2, 61), (3, 959), (5, 960), (33, 991)]
SHAPES_3D = [(1, 1, 1), (1, 5, 7), (4, 1, 9), (3, 33, 65), (17, 40, 129), (40, 64, 64), (9, 97, 31), (2, 130, 300)]


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D)
def test_uniform_u8(shape, mode, kernel):
    rng = np.random.default_rng(hash(shape) % 1000)
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    assert np.array_equal(_run(_gpu(img), 0, 255, mode, kernel), _expect(img, 0, 255, mode))


# 3D shapes whose rows are 16-byte aligned take the TMA-staged bit-sliced kernel
TMA_SHAPES = [(40, 64, 64), (33, 48, 96), (7, 35, 160), (100, 31, 32), (3, 64, 208), (65, 100, 112),
              (1, 80, 48), (2, 2, 16), (31, 61, 512), (9, 33, 1008)]


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("levels", [3, 256])
def test_tma_path_u8(shape, mode, levels):
    rng = np.random.default_rng(sum(shape) + levels)
    img = rng.integers(0, levels, size=shape, dtype=np.uint8)
    assert np.array_equal(_run(_gpu(img), 0, 255, mode), _expect(img, 0, 255, mode))


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", [(20, 40, 72), (9, 33, 136), (50, 17, 8), (4, 70, 256)])
@pytest.mark.parametrize("levels", [5, 65536])
def test_tma_path_u16(shape, mode, levels):
    rng = np.random.default_rng(sum(shape) + levels)
    img = rng.integers(0, levels, size=shape).astype(np.uint16)
    assert np.array_equal(_run(_gpu(img), 0, 65535, mode), _expect(img, 0, 65535, mode))


@pytest.mark.parametrize("mode", list(MODES))
def test_tma_path_pitched_view(mode):
    rng = np.random.default_rng(6)
    big = rng.integers(0, 7, size=(40, 90, 256), dtype=np.uint8)
    view = _gpu(big)[3:37, 2:85, 32:232]   # 16-byte aligned start, pitches 256 and 90*256
    want = _expect(np.ascontiguousarray(big[3:37, 2:85, 32:232]), 0, 255, mode)
    assert np.array_equal(_run(view, 0, 255, mode), want)


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", [(61, 70), (5, 66, 40), (33, 31, 130)])
@pytest.mark.parametrize("levels", [1, 2, 3, 7])
def test_plateaus_and_ties(shape, mode, kernel, levels):
    rng = np.random.default_rng(levels)
    img = rng.integers(0, levels, size=shape, dtype=np.uint8)
    assert np.array_equal(_run(_gpu(img), 0, 255, mode, kernel), _expect(img, 0, 255, mode))


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", [(50, 300), (7, 45, 90), (20, 64, 140)])
def test_uint16_full_range(shape, mode, kernel):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 65536, size=shape, dtype=np.uint16)
    assert np.array_equal(_run(_gpu(img), 0, 65535, mode, kernel), _expect(img, 0, 65535, mode))


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("mode", list(MODES))
def test_uint16_smooth_with_blobs(mode, kernel):
    import synth
    v = synth.smoothed_field((48, 64, 96), 3.0, np.uint16, seed=5, device="cuda")
    v = synth.add_blobs(v, 20, seed=5, r_range=(2, 6))
    img = v.cpu().numpy()
    assert np.array_equal(_run(v, 0, 65535, mode, kernel), _expect(img, 0, 65535, mode))


@pytest.mark.parametrize("mode", list(MODES))
def test_subrange_and_vcec_output(mode):
    rng = np.random.default_rng(3)
    img = rng.integers(40, 61, size=(9, 30, 70), dtype=np.uint8)
    ecc_v, vcec_v = _run(_gpu(img), 37, 64, mode, with_vcec=True)
    assert np.array_equal(ecc_v, _expect(img, 37, 64, mode))
    assert np.array_equal(vcec_v, oracle.vcec(img, 37, 64, mode))


@pytest.mark.parametrize("mode", list(MODES))
def test_fused_scan_in_the_stencils(mode):
    """The 3D and 2D stencils' last CTA scans histograms of up to 4096 bins
    itself (no scan launch).  ECC and VCEC equal the oracle's on both sides
    of that limit (4096 bins fused, 4097 and 65536 through the scan kernel),
    for 3D volumes whose rows the TMA addresses and 2D images, spanning many
    CTAs, over repeated calls on one plan (the accumulator and the CTA
    counters are left clean for the next call)."""
    ecc = ecc_mod()
    rng = np.random.default_rng(17)
    img8 = rng.integers(0, 256, size=(37, 61, 96), dtype=np.uint8)
    img16 = rng.integers(0, 4096, size=(29, 70, 128), dtype=np.uint16)
    img2 = rng.integers(0, 256, size=(700, 1333), dtype=np.uint8)
    img2w = rng.integers(0, 4096, size=(301, 2900), dtype=np.uint16)
    for img, lo, hi in ((img8, 0, 255), (img8, 0, 199), (img16, 0, 4095), (img16, 0, 4096), (img16, 0, 65535),
                        (img2, 0, 255), (img2w, 0, 4095), (img2w, 0, 4096)):
        if img.max() > hi:
            img = np.minimum(img, hi).astype(img.dtype)
        t = _gpu(img)
        dt = "u8" if img.dtype == np.uint8 else "u16"
        plan = ecc.ecc_plan(dt, lo, hi, complex_mode=MODES[mode], max_voxels=img.size)
        want_e, want_v = _expect(img, lo, hi, mode), oracle.vcec(img, lo, hi, mode)
        for _ in range(3):
            out = torch.full((hi - lo + 1,), -777, dtype=torch.int64, device="cuda")
            v = torch.full((hi - lo + 1,), -777, dtype=torch.int64, device="cuda")
            ecc.ecc_compute(plan, t, out, v)
            ecc.ecc_status_get(plan)
            assert np.array_equal(out.cpu().numpy(), want_e), (img.dtype, hi)
            assert np.array_equal(v.cpu().numpy(), want_v), (img.dtype, hi)
        assert ecc.ecc_plan_last_launches(plan) == (1 if hi - lo + 1 <= 4096 else 2)
        plan.close()


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("kernel", list(KERNELS))
def test_pitched_views(mode, kernel):
    rng = np.random.default_rng(4)
    big = rng.integers(0, 256, size=(12, 70, 200), dtype=np.uint8)
    t = _gpu(big)
    view3 = t[2:11, 3:60, 5:150]          # both pitches non-dense, odd offset
    img3 = np.ascontiguousarray(big[2:11, 3:60, 5:150])
    assert np.array_equal(_run(view3, 0, 255, mode, kernel), _expect(img3, 0, 255, mode))
    view2 = t[4, 1:69, 7:190]
    img2 = np.ascontiguousarray(big[4, 1:69, 7:190])
    assert np.array_equal(_run(view2, 0, 255, mode, kernel), _expect(img2, 0, 255, mode))


def test_out_of_range_is_reported():
    ecc = ecc_mod()
    img = torch.full((4, 40), 10, dtype=torch.uint8, device="cuda")
    img[2, 7] = 200
    plan = ecc.ecc_plan("u8", 0, 100)
    ecc.ecc_compute(plan, img)
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_status_get(plan)
    assert ei.value.status == ecc.ECC_E_RANGE
    # the status word is cleared after it was read
    ecc.ecc_compute(plan, torch.full((4, 40), 10, dtype=torch.uint8, device="cuda"))
    assert ecc.ecc_status_get(plan) == ecc.ECC_OK


def test_invalid_arguments():
    ecc = ecc_mod()
    with pytest.raises(ecc.EccError):
        ecc.ecc_plan("u8", 10, 5)
    with pytest.raises(ecc.EccError):
        ecc.ecc_plan("u8", 0, 300)
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=100)
    with pytest.raises(ecc.EccError):
        ecc.ecc_compute(plan, torch.zeros((20, 20), dtype=torch.uint8, device="cuda"))
    plan16 = ecc.ecc_plan("u16", 0, 65535)
    with pytest.raises(ecc.EccError):
        ecc.ecc_compute(plan16, torch.zeros((20, 20), dtype=torch.uint8, device="cuda"))


def test_repeated_calls_are_independent():
    """The workspace is self-cleaning: the second call must not see the first."""
    ecc = ecc_mod()
    rng = np.random.default_rng(9)
    a = rng.integers(0, 256, size=(30, 40, 50), dtype=np.uint8)
    b = rng.integers(0, 5, size=(30, 40, 50), dtype=np.uint8)
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=a.size)
    for img in (a, b, a):
        out = ecc.ecc_compute(plan, _gpu(img))
        assert np.array_equal(out.cpu().numpy(), _expect(img, 0, 255, "vertex"))


@pytest.mark.parametrize("mode", list(MODES))
def test_host_streaming_path(mode):
    """ecc_compute_host copies in chunks along dims[0] and overlaps the kernels."""
    import synth
    ecc = ecc_mod()
    img = synth.smoothed_field((70, 90, 130), 2.0, np.uint8, seed=8, device="cpu").numpy()
    plan = ecc.ecc_plan("u8", 0, 255, complex_mode=MODES[mode], max_voxels=img.size)
    assert np.array_equal(ecc.ecc_compute_host(plan, img), _expect(img, 0, 255, mode))
    sub = img[:, 5:80, 3:120]  # pitched host view
    assert np.array_equal(ecc.ecc_compute_host(plan, sub), _expect(np.ascontiguousarray(sub), 0, 255, mode))
    # a 2D image of several 8 MiB chunks: the 2D stencil on row ranges
    img2 = synth.smoothed_field((3100, 4100), 3.0, np.uint8, seed=9, device="cpu").numpy()
    plan2 = ecc.ecc_plan("u8", 0, 255, complex_mode=MODES[mode], max_voxels=img2.size)
    assert np.array_equal(ecc.ecc_compute_host(plan2, img2), _expect(img2, 0, 255, mode))


def test_256sq_uniform_matches_golden():
    import synth
    from pathlib import Path
    img = synth.uniform_2d_256()
    for mode in MODES:
        want = np.loadtxt(Path(__file__).parent / "golden" / f"uniform_256x256_seed0_{mode}.txt",
                          dtype=np.int64)
        for kernel in KERNELS:
            assert np.array_equal(_run(_gpu(img), 0, 255, mode, kernel), want)


@pytest.mark.parametrize("tile", ["61", "62", "42", "31"])
def test_every_3d_tile_variant(tile, monkeypatch):
    """Each tile shape / histogram-copy variant the autotuner may pick is exact."""
    monkeypatch.setenv("ECC_TILE3D", tile)
    rng = np.random.default_rng(int(tile))
    for shape, dt, levels in [((37, 70, 208), np.uint8, 256), ((21, 45, 96), np.uint8, 4),
                              ((19, 33, 136), np.uint16, 65536)]:
        img = rng.integers(0, levels, size=shape).astype(dt)
        hi = 255 if dt == np.uint8 else 65535
        for mode in MODES:
            assert np.array_equal(_run(_gpu(img), 0, hi, mode), _expect(img, 0, hi, mode)), (tile, shape, mode)


def _nonzero_kappa_count(img: np.ndarray) -> int:
    """Voxels whose signed count of introduced cells is nonzero (vertex
    complex), by brute force over the cells around each voxel: p introduces
    a cell iff it beats every other vertex, where p beats q iff I[p] > I[q]
    or I[p] == I[q] and p comes first in memory; cells with a vertex outside
    the image do not exist (the neighbour is padded with +infinity)."""
    import itertools
    d = img.ndim
    n = img.size
    lin = np.arange(n, dtype=np.int64).reshape(img.shape)
    key = img.astype(np.int64) * n + (n - 1 - lin)
    big = np.iinfo(np.int64).max
    pad = np.pad(key, 1, constant_values=big)
    center = tuple(slice(1, 1 + s) for s in img.shape)
    c = pad[center]

    def beats(off):
        sl = tuple(slice(1 + o, 1 + o + s) for o, s in zip(off, img.shape))
        return c > pad[sl]

    kappa = np.ones(img.shape, np.int64)
    for sgn in itertools.product((-1, 0, 1), repeat=d):
        if not any(sgn):
            continue
        dim = sum(1 for s in sgn if s)
        verts = [t for t in itertools.product(*[(0, s) if s else (0,) for s in sgn]) if any(t)]
        m = np.ones(img.shape, bool)
        for t in verts:
            m &= beats(t)
        kappa += (-1) ** dim * m
    return int(np.count_nonzero(kappa))


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("shape", [(100, 77), (17, 40, 129), (9, 97, 31)])
def test_emitted_count_is_the_nonzero_kappa_count(shape, kernel):
    ecc = ecc_mod()
    rng = np.random.default_rng(7)
    img = rng.integers(0, 6, size=shape, dtype=np.uint8)   # plateaus and ties
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=img.size, flags=KERNELS[kernel] | ecc.ECC_FLAG_COUNT_EMITTED)
    out = torch.empty(256, dtype=torch.int64, device="cuda")
    ecc.ecc_compute(plan, _gpu(img), out)
    ecc.ecc_status_get(plan)
    assert ecc.ecc_plan_emitted(plan) == _nonzero_kappa_count(img)
    assert ecc.ecc_plan_emitted(plan) == 0   # read resets
    assert np.array_equal(out.cpu().numpy(), _expect(img, 0, 255, "vertex"))
