"""The paper's ECC sequence of a float32 image on the GPU (Eq. 1 at the
values present, Sec. 2.2): ecc_levels_present finds the distinct values,
ecc_compute_present then computes the ECC at them.  Both are compared
exactly with the oracle:
- levels bit for bit (so +0.0, never -0.0) against oracle.present_levels;
- the ECC against oracle.ecc_levels at those levels.
The cases cover ties, NaN, infinities, signed zeros, pitched views, the
paper's 11 and 1024 distinct values, nearly all-distinct values, an image
of NaN alone, and an image with more distinct values than allowed."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MODES = [0, 1]


def ecc_mod():
    import paper_2203_09087_gb300 as ecc
    return ecc


def _plan(ecc, nvox, mode):
    return ecc.ecc_plan("u16", 0, 65535, complex_mode=mode, max_voxels=max(nvox, 1))


def _check(img, mode, view=None):
    ecc = ecc_mod()
    t = torch.from_numpy(img).cuda() if view is None else view
    host = t.cpu().numpy()
    plan = _plan(ecc, host.size, mode)
    lv, e = ecc.ecc_compute_present(plan, t)
    ecc.ecc_status_get(plan)
    want_lv = oracle.present_levels(host)
    got_lv = lv.cpu().numpy()
    assert np.array_equal(got_lv.view(np.uint32), want_lv.view(np.uint32)), (got_lv[:8], want_lv[:8])
    om = oracle.VERTEX if mode == 0 else oracle.TOPCELL
    want = oracle.ecc_levels(host, want_lv, om, threads=8) if want_lv.size else np.zeros(0, np.int64)
    assert np.array_equal(e.cpu().numpy(), want)


def _from_values(rng, shape, values):
    return np.asarray(values, np.float32)[rng.integers(0, len(values), size=shape)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (45, 1), (33, 70), (300, 257), (5, 6, 7), (17, 40, 65)])
def test_ties_nan_infinities_signed_zeros(shape, mode):
    rng = np.random.default_rng(sum(shape) + mode)
    vals = [-np.inf, -3.5, -1.0, -0.0, 0.0, 1e-30, 0.5, 0.5000001, 2.0, 7.25, np.inf, np.nan]
    _check(_from_values(rng, shape, vals), mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("ndistinct", [11, 1024])
def test_the_papers_distinct_value_counts(ndistinct, mode):
    """The paper's float datasets hold 11 to 1024 distinct values."""
    rng = np.random.default_rng(ndistinct)
    vals = np.sort(rng.normal(size=ndistinct)).astype(np.float32)
    _check(_from_values(rng, (40, 96, 130), vals), mode)


@pytest.mark.parametrize("mode", MODES)
def test_nearly_all_values_distinct(mode):
    rng = np.random.default_rng(7)
    img = rng.normal(size=(150, 200)).astype(np.float32)  # 30000 voxels, ~30000 values
    _check(img, mode)


@pytest.mark.parametrize("mode", MODES)
def test_pitched_views(mode):
    rng = np.random.default_rng(8)
    base = torch.from_numpy(_from_values(rng, (30, 50, 70), [0.25, -1.0, 3.0, np.nan, 9.5])).cuda()
    _check(None, mode, view=base[3:27, 5:44, 2:61])
    base2 = torch.from_numpy(rng.normal(size=(90, 130)).astype(np.float32)).cuda()
    _check(None, mode, view=base2[7:80, 3:121])


def test_nan_only_and_single_value():
    ecc = ecc_mod()
    t = torch.full((20, 30), float("nan"), device="cuda")
    plan = _plan(ecc, t.numel(), 0)
    lv, e = ecc.ecc_compute_present(plan, t)
    assert lv.numel() == 0 and e.numel() == 0
    t = torch.full((4, 5, 6), -0.0, device="cuda")
    lv, e = ecc.ecc_compute_present(plan, t)
    assert lv.cpu().numpy().view(np.uint32).tolist() == [0]  # +0.0
    assert e.cpu().tolist() == [1]


def test_more_distinct_values_than_allowed():
    ecc = ecc_mod()
    rng = np.random.default_rng(9)
    img = torch.from_numpy(rng.permutation(5000).astype(np.float32).reshape(50, 100)).cuda()
    plan = _plan(ecc, img.numel(), 0)
    lv, cnt = ecc.ecc_levels_present(plan, img, max_levels=1000)
    assert int(cnt.item()) == 1001  # max_levels + 1: more than allowed
    lv, cnt = ecc.ecc_levels_present(plan, img, max_levels=5000)
    assert int(cnt.item()) == 5000
    assert np.array_equal(lv.cpu().numpy(), np.arange(5000, dtype=np.float32))
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_compute_present(plan, img, max_levels=100)
    assert ei.value.status == ecc.ECC_E_BUSY
    # a plan whose levels do not reach n
    small = ecc.ecc_plan("u16", 0, 1000, max_voxels=img.numel())
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_compute_present(small, img)
    assert ei.value.status == ecc.ECC_E_BUSY
    # the plan's table is clean for the next call
    _check(_from_values(rng, (64, 64), [1.0, 2.0, 3.0]), 0)


def test_repeated_calls_and_a_large_volume():
    ecc = ecc_mod()
    rng = np.random.default_rng(10)
    vals = np.sort(rng.uniform(-5, 5, size=1024)).astype(np.float32)
    img = _from_values(rng, (96, 128, 160), vals)
    t = torch.from_numpy(img).cuda()
    plan = _plan(ecc, img.size, 0)
    want_lv = oracle.present_levels(img)
    want = oracle.ecc_levels(img, want_lv, oracle.VERTEX, threads=16)
    for _ in range(3):
        lv, e = ecc.ecc_compute_present(plan, t)
        assert np.array_equal(lv.cpu().numpy(), want_lv)
        assert np.array_equal(e.cpu().numpy(), want)


@pytest.mark.parametrize("mode", MODES)
def test_an_8bit_plan_for_up_to_255_values(mode):
    """ecc_compute_present on an ECC_U8 plan (hi = 255): the level indices
    are bytes."""
    ecc = ecc_mod()
    rng = np.random.default_rng(11 + mode)
    vals = np.sort(rng.normal(size=200)).astype(np.float32)
    img = _from_values(rng, (33, 45, 70), vals)
    plan = ecc.ecc_plan("u8", 0, 255, complex_mode=mode, max_voxels=img.size)
    lv, e = ecc.ecc_compute_present(plan, torch.from_numpy(img).cuda())
    ecc.ecc_status_get(plan)
    want_lv = oracle.present_levels(img)
    assert np.array_equal(lv.cpu().numpy(), want_lv)
    om = oracle.VERTEX if mode == 0 else oracle.TOPCELL
    assert np.array_equal(e.cpu().numpy(), oracle.ecc_levels(img, want_lv, om, threads=8))
