"""GB300 (sm_103a) Euler characteristic curves of 2D/3D integer images.

A thin ctypes binding over the C ABI in ``include/ecc.h``; every step of the
computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams only.  The functions keep the C names:

    plan = ecc_plan(dtype="u8", lo=0, hi=255)           # ecc_plan
    ecc = ecc_compute(plan, volume_cuda_tensor)         # ecc_compute
    eccs = ecc_compute_batch(plan, [img0, img1, ...])   # ecc_compute_batch
    ecc_host = ecc_compute_host(plan, numpy_array)      # ecc_compute_host
    ecc_big = ecc_compute_stream(plan, huge_array, 1 << 30)  # ecc_compute_stream (out of core)
    ecc_t = ecc_compute_levels(plan_u16, f32_tensor, levels)  # ecc_compute_levels (float thresholds)
    eccs = ecc_pipeline_gaussian(plan_u16, f32_tensor, gaussian_taps(2.0), 100, levels)  # Table 2 loop
    ecc4 = ecc_compute_nd(plan, tensor_4d)               # ecc_compute_nd (2D, 3D or 4D)
    srv = ecc_server_create(budget_bytes, n_streams=4)  # ecc_server_create / ecc_submit / ...

There is no CPU fallback: importing works anywhere, but the first call loads
``_build/libecc_gb300.so`` and raises if it is missing or no CUDA device is
present.
"""
from ._binding import (  # noqa: F401
    ECC_E_BUSY,
    ECC_E_CANCELLED,
    ECC_E_CUDA,
    ECC_E_INVALID,
    ECC_E_NOMEM,
    ECC_E_RANGE,
    ECC_E_SHUTDOWN,
    ECC_E_TIMEOUT,
    ECC_FLAG_BATCH_PER_IMAGE,
    ECC_FLAG_KERNEL_BITSLICE,
    ECC_FLAG_KERNEL_DIRECT,
    ECC_FLAG_NO_AUTOTUNE,
    ECC_FLAG_NO_RANGE_CHECK,
    ECC_FLAG_TIME_KERNELS,
    ECC_FLAG_COUNT_EMITTED,
    ECC_OK,
    ECC_TOPCELL_MIN,
    ECC_U8,
    ECC_U16,
    ECC_F32,
    ECC_VERTEX_MAX,
    EccError,
    ImageDescs,
    Plan,
    Server,
    ecc_compute,
    ecc_compute_batch,
    ecc_compute_host,
    ecc_compute_levels,
    ecc_compute_present,
    ecc_levels_present,
    ecc_compute_nd,
    ecc_pipeline_gaussian,
    gaussian_taps,
    ecc_compute_stream,
    ecc_compute_noalloc,
    ecc_last_error,
    ecc_plan,
    ecc_plan_destroy,
    ecc_plan_kernel_time,
    ecc_plan_emitted,
    ecc_plan_last_launches,
    ecc_plan_nbins,
    ecc_selftest_wait_timeout,
    ecc_server_create,
    ecc_server_destroy,
    ecc_server_prepare,
    ecc_server_stats,
    ecc_status_get,
    ecc_submit,
    ecc_wait,
    exported_symbols,
    image_descs,
    library,
    library_path,
)
