"""GPU parity of 4D images (ecc_compute_nd: the method for d > 3) against
the CPU oracle, bit-exact: random images with ties, size-1 axes, smoothed
fields, pitched views, both complexes and element types; 2D and 3D images
through the same entry point equal ecc_compute."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MODES = {"vertex": 0, "topcell": 1}


def ecc_mod():
    import paper_2203_09087_gb300 as ecc
    return ecc


def _run(t, lo, hi, mode, with_vcec=False):
    ecc = ecc_mod()
    dt = "u8" if t.dtype == torch.uint8 else "u16"
    plan = ecc.ecc_plan(dt, lo, hi, complex_mode=MODES[mode], max_voxels=t.numel())
    v = torch.empty(hi - lo + 1, dtype=torch.int64, device="cuda") if with_vcec else None
    out = ecc.ecc_compute_nd(plan, t, vcec_out=v)
    ecc.ecc_status_get(plan)
    return (out.cpu().numpy(), v.cpu().numpy()) if with_vcec else out.cpu().numpy()


@pytest.mark.parametrize("mode", list(MODES))
def test_random_4d_with_ties(mode):
    rng = np.random.default_rng(81)
    for shape in [(1, 1, 1, 1), (2, 3, 1, 4), (3, 3, 3, 3), (5, 4, 7, 9), (1, 6, 5, 40)]:
        for levels in (2, 5, 256):
            img = rng.integers(0, levels, size=shape).astype(np.uint8)
            got = _run(torch.from_numpy(img).cuda(), 0, 255, mode)
            assert np.array_equal(got, oracle.ecc(img, 0, 255, mode)), (shape, levels)


@pytest.mark.parametrize("mode", list(MODES))
def test_smoothed_4d_u8_and_u16(mode):
    import synth
    g = torch.Generator().manual_seed(82)
    f = synth.smooth(torch.randn((10, 14, 17, 23), generator=g), 1.5)
    img8 = synth.quantize(f, np.uint8).numpy()
    got, vcec = _run(torch.from_numpy(img8).cuda(), 0, 255, mode, with_vcec=True)
    assert np.array_equal(got, oracle.ecc(img8, 0, 255, mode))
    assert np.array_equal(vcec, oracle.vcec(img8, 0, 255, mode))
    img16 = (synth.quantize(f, np.uint16).numpy() // 64).astype(np.uint16)
    assert np.array_equal(_run(torch.from_numpy(img16).cuda(), 0, 1023, mode), oracle.ecc(img16, 0, 1023, mode))


@pytest.mark.parametrize("mode", list(MODES))
def test_4d_row_tiles_windows_and_w_chunks(mode):
    """Shapes spanning several 30-row tiles and 30-column windows with
    ragged tails, and (the first) enough (z, tile, window) columns that the
    w axis is cut into chunks of several hyperplanes with a short last one."""
    rng = np.random.default_rng(85)
    for shape, levels, dt, hi in [((40, 64, 40, 40), 7, np.uint8, 255), ((9, 5, 65, 70), 3, np.uint8, 255),
                                  ((6, 7, 33, 95), 300, np.uint16, 1023), ((7, 3, 31, 61), 4, np.uint16, 65535)]:
        img = rng.integers(0, levels, size=shape).astype(dt)
        got = _run(torch.from_numpy(img).cuda(), 0, hi, mode)
        assert np.array_equal(got, oracle.ecc(img, 0, hi, mode)), (shape, levels)


def test_pitched_4d_view():
    rng = np.random.default_rng(83)
    base = rng.integers(0, 6, size=(6, 9, 11, 40)).astype(np.uint8)
    t = torch.from_numpy(base).cuda()[1:5, 2:8, 1:10, 3:35]
    want = oracle.ecc(np.ascontiguousarray(base[1:5, 2:8, 1:10, 3:35]), 0, 255, "vertex")
    assert np.array_equal(_run(t, 0, 255, "vertex"), want)


def test_2d_and_3d_through_the_nd_entry():
    ecc = ecc_mod()
    rng = np.random.default_rng(84)
    for shape in [(40, 70), (9, 33, 65)]:
        img = torch.from_numpy(rng.integers(0, 256, size=shape).astype(np.uint8)).cuda()
        plan = ecc.ecc_plan("u8", 0, 255, max_voxels=img.numel())
        assert torch.equal(ecc.ecc_compute_nd(plan, img), ecc.ecc_compute(plan, img))


def test_nd_errors():
    ecc = ecc_mod()
    img = torch.zeros((3, 4, 5, 6), dtype=torch.uint8, device="cuda")
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=100)
    with pytest.raises(ecc.EccError):
        ecc.ecc_compute_nd(plan, img)                      # more voxels than max_voxels
    plan = ecc.ecc_plan("u8", 0, 9, max_voxels=img.numel())
    bad = img.clone()
    bad[1, 2, 3, 4] = 50
    ecc.ecc_compute_nd(plan, bad)
    with pytest.raises(ecc.EccError) as e:
        ecc.ecc_status_get(plan)
    assert e.value.status == ecc.ECC_E_RANGE
