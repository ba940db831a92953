"""The C ABI library builds, loads, and exports every function include/ecc.h
declares; argument validation that needs no GPU.  No compute calls."""
import ctypes
import subprocess

import pytest

import paper_2203_09087_gb300 as ecc
from paper_2203_09087_gb300 import build as cuda_build


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return ecc.library()


def test_header_declares_the_boundary():
    names = set(ecc.exported_symbols())
    for want in ("ecc_plan", "ecc_compute", "ecc_compute_batch", "ecc_submit", "ecc_plan_destroy",
                 "ecc_status_get", "ecc_last_error", "ecc_server_create", "ecc_wait", "ecc_server_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", str(ecc.library_path())], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in ecc.exported_symbols() if n not in exported]
    assert not missing, f"declared in include/ecc.h but not exported: {missing}"
    for n in ecc.exported_symbols():
        assert getattr(lib, n) is not None


def test_plan_validation_without_gpu(lib):
    d = ecc._binding.EccPlanDesc(dtype=1, lo=10, hi=5, complex_mode=0, max_images=1, reserved=0,
                                 max_voxels=10, flags=0, reserved2=0)
    h = ctypes.c_void_p()
    assert lib.ecc_plan(ctypes.byref(h), ctypes.byref(d)) == ecc.ECC_E_INVALID
    assert b"hi < lo" in lib.ecc_last_error()
    d.hi, d.lo, d.dtype = 300, 0, 1
    assert lib.ecc_plan(ctypes.byref(h), ctypes.byref(d)) == ecc.ECC_E_INVALID
    d.hi, d.complex_mode = 255, 7
    assert lib.ecc_plan(ctypes.byref(h), ctypes.byref(d)) == ecc.ECC_E_INVALID
    assert lib.ecc_plan(None, ctypes.byref(d)) == ecc.ECC_E_INVALID


def test_null_handles_are_rejected(lib):
    assert lib.ecc_plan_nbins(None) == -1
    assert lib.ecc_compute(None, None, None, None, None) == ecc.ECC_E_INVALID
    assert lib.ecc_compute_batch(None, 1, None, None, None) == ecc.ECC_E_INVALID
    assert lib.ecc_plan_destroy(None) == ecc.ECC_E_INVALID
    gave = (ctypes.c_int32 * 2)()
    assert lib.ecc_selftest_wait_timeout(0, gave, None) == ecc.ECC_E_INVALID
    assert lib.ecc_selftest_wait_timeout(1000, None, None) == ecc.ECC_E_INVALID


def test_python_image_descriptor_from_numpy():
    import numpy as np
    a = np.zeros((5, 6, 7), np.uint16)[:, 1:5, 2:]
    d = ecc._binding.host_image_desc(a)
    assert (d.ndim, d.dtype, list(d.dims)) == (3, ecc.ECC_U16, [5, 4, 5])
    assert d.row_pitch == 7 * 2 and d.slice_pitch == 6 * 7 * 2


def test_null_plan_is_rejected_by_every_plan_entry_point(lib):
    """Each entry point that takes a plan reports ECC_E_INVALID for a NULL
    plan, with a message naming it, before it touches the device (so this
    runs without a GPU)."""
    inval = ecc.ECC_E_INVALID
    calls = {
        "ecc_compute_host": lambda: lib.ecc_compute_host(None, None, None, None),
        "ecc_compute_stream": lambda: lib.ecc_compute_stream(None, None, None, 0, None),
        "ecc_compute_levels": lambda: lib.ecc_compute_levels(None, None, None, 1, None, None),
        "ecc_compute_nd": lambda: lib.ecc_compute_nd(None, None, None, None, None),
        "ecc_pipeline_gaussian": lambda: lib.ecc_pipeline_gaussian(None, None, None, 13, 1, None, 1, None, None),
        "ecc_status_get": lambda: lib.ecc_status_get(None, None),
        "ecc_levels_present": lambda: lib.ecc_levels_present(None, None, None, 1, None, None),
        "ecc_compute_present": lambda: lib.ecc_compute_present(None, None, None, 1, None, None, None),
        "ecc_server_prepare": lambda: lib.ecc_server_prepare(None, ecc.ECC_U8, 0, 255, ecc.ECC_VERTEX_MAX),
    }
    for name, call in calls.items():
        assert call() == inval, name
        assert name.encode() in lib.ecc_last_error(), name
    ms, n = ctypes.c_double(), ctypes.c_int64()
    assert lib.ecc_plan_kernel_time(None, ctypes.byref(ms), ctypes.byref(n)) == inval
    assert lib.ecc_plan_last_launches(None) == -1


def test_a_missing_library_is_an_error_not_a_fallback(monkeypatch, tmp_path):
    """Without the built CUDA library every call raises: there is no CPU path."""
    from paper_2203_09087_gb300 import _binding
    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "library_path", lambda: tmp_path / "libecc_gb300.so")
    with pytest.raises(RuntimeError, match="missing"):
        _binding.library()
    with pytest.raises(RuntimeError, match="missing"):
        ecc.ecc_last_error()
