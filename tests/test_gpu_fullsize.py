"""Full-size parity at the benchmark configurations, in the launch
configuration the benchmark times.  The oracle runs on disjoint dims[0] slabs
in host threads (its own chunk entry points, Sec. 3.4) and the slab
histograms are summed; the comparison is exact."""
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _ecc_gpu(vol, lo, hi, mode=0):
    import paper_2203_09087_gb300 as ecc
    dt = "u8" if vol.dtype == torch.uint8 else "u16"
    plan = ecc.ecc_plan(dt, lo, hi, complex_mode=mode, max_voxels=vol.numel())
    out = ecc.ecc_compute(plan, vol)
    ecc.ecc_status_get(plan)
    return out.cpu().numpy()


def test_512cube_u8_smooth():
    import synth
    vol = synth.smooth_3d_512(device="cuda")
    got = _ecc_gpu(vol, 0, 255)
    host = vol.cpu().numpy()
    want = oracle.ecc_from_vcec(oracle.vcec_parallel(host, 0, 255, oracle.VERTEX, threads=os.cpu_count()))
    assert np.array_equal(got, want)
    assert got[-1] == 1


def test_1024cube_u16_blobs():
    import synth
    vol = synth.smooth_blobs_u16_1024(device="cuda")
    got = _ecc_gpu(vol, 0, 65535)
    host = vol.cpu().numpy()
    del vol
    torch.cuda.empty_cache()
    want = oracle.ecc_from_vcec(oracle.vcec_parallel(host, 0, 65535, oracle.VERTEX, threads=os.cpu_count()))
    assert np.array_equal(got, want)
    assert got[-1] == 1


def test_512cube_topcell_matches_oracle_on_a_slab():
    """Top-cell complex at full size, checked on a slab of planes (chunk
    additivity: the GPU result of the slab as an image equals the oracle's)."""
    import synth
    vol = synth.smooth_3d_512(device="cuda")
    slab = vol[100:164].contiguous()
    got = _ecc_gpu(slab, 0, 255, mode=1)
    want = oracle.ecc_from_vcec(oracle.vcec_parallel(slab.cpu().numpy(), 0, 255, oracle.TOPCELL))
    assert np.array_equal(got, want)


def test_largest_2d_image_16384_square():
    """The 2D stencil at 16384^2 uint8 (a smoothed field, sigma 3): long
    row chunks across many warps, against the slab-parallel oracle."""
    import synth
    img = synth.smoothed_field((16384, 16384), 3.0, "u8", seed=9, device="cuda")
    got = _ecc_gpu(img, 0, 255)
    host = img.cpu().numpy()
    del img
    want = oracle.ecc_from_vcec(oracle.vcec_parallel(host, 0, 255, oracle.VERTEX, threads=os.cpu_count()))
    assert np.array_equal(got, want)
    assert got[-1] == 1


def test_1024cube_u8_smooth():
    """The 8-bit 3D stencil at 1024^3 (1 GiB, eight times the benchmark's
    volume): TMA coordinates past 512 and the launcher's z-chunk choice at
    that depth, against the slab-parallel oracle."""
    import synth
    vol = synth.smoothed_field((1024, 1024, 1024), 4.0, "u8", seed=12, device="cuda")
    got = _ecc_gpu(vol, 0, 255)
    host = vol.cpu().numpy()
    del vol
    torch.cuda.empty_cache()
    want = oracle.ecc_from_vcec(oracle.vcec_parallel(host, 0, 255, oracle.VERTEX, threads=os.cpu_count()))
    assert np.array_equal(got, want)
    assert got[-1] == 1
