"""ctypes marshalling for include/ecc.h.  No computation happens here."""
from __future__ import annotations

import ctypes
import re
import threading
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
_HEADER = _PKG.parent / "include" / "ecc.h"

ECC_OK, ECC_E_INVALID, ECC_E_RANGE, ECC_E_NOMEM, ECC_E_CUDA = 0, 1, 2, 3, 4
ECC_E_TIMEOUT, ECC_E_BUSY, ECC_E_SHUTDOWN, ECC_E_CANCELLED = 5, 6, 7, 8
ECC_U8, ECC_U16, ECC_F32 = 1, 2, 3
ECC_VERTEX_MAX, ECC_TOPCELL_MIN = 0, 1
ECC_FLAG_NO_RANGE_CHECK = 0x1
ECC_FLAG_NO_AUTOTUNE = 0x2
ECC_FLAG_KERNEL_DIRECT = 0x10
ECC_FLAG_KERNEL_BITSLICE = 0x20
ECC_FLAG_BATCH_PER_IMAGE = 0x40
ECC_FLAG_TIME_KERNELS = 0x80
ECC_FLAG_COUNT_EMITTED = 0x100

_STATUS_NAMES = {0: "ECC_OK", 1: "ECC_E_INVALID", 2: "ECC_E_RANGE", 3: "ECC_E_NOMEM", 4: "ECC_E_CUDA",
                 5: "ECC_E_TIMEOUT", 6: "ECC_E_BUSY", 7: "ECC_E_SHUTDOWN", 8: "ECC_E_CANCELLED"}


class EccError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class EccImage(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("ndim", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("dims", ctypes.c_int64 * 3), ("row_pitch", ctypes.c_int64), ("slice_pitch", ctypes.c_int64)]


class EccImageNd(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("ndim", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("dims", ctypes.c_int64 * 4), ("pitches", ctypes.c_int64 * 3)]


class EccPlanDesc(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("lo", ctypes.c_int32), ("hi", ctypes.c_int32),
                ("complex_mode", ctypes.c_int32), ("max_images", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_voxels", ctypes.c_int64), ("flags", ctypes.c_uint32), ("reserved2", ctypes.c_uint32)]


class EccServerDesc(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("n_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("max_job_voxels", ctypes.c_int64), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


DONE_FN = ctypes.CFUNCTYPE(None, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p)

_VP, _I32, _I64, _U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_SIGNATURES = {
    "ecc_plan": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(EccPlanDesc)]),
    "ecc_plan_destroy": (ctypes.c_int, [_VP]),
    "ecc_plan_nbins": (_I32, [_VP]),
    "ecc_plan_last_launches": (_I32, [_VP]),
    "ecc_compute": (ctypes.c_int, [_VP, ctypes.POINTER(EccImage), _VP, _VP, _VP]),
    "ecc_compute_host": (ctypes.c_int, [_VP, ctypes.POINTER(EccImage), _VP, _VP]),
    "ecc_compute_batch": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(EccImage), _VP, _VP]),
    "ecc_compute_stream": (ctypes.c_int, [_VP, ctypes.POINTER(EccImage), _VP, _I64, _VP]),
    "ecc_compute_levels": (ctypes.c_int, [_VP, ctypes.POINTER(EccImage), _VP, _I32, _VP, _VP]),
    "ecc_levels_present": (ctypes.c_int, [_VP, ctypes.POINTER(EccImage), _VP, _I32, _VP, _VP]),
    "ecc_compute_present": (ctypes.c_int, [_VP, ctypes.POINTER(EccImage), _VP, _I32, ctypes.POINTER(_I32), _VP,
                                           _VP]),
    "ecc_compute_nd": (ctypes.c_int, [_VP, ctypes.POINTER(EccImageNd), _VP, _VP, _VP]),
    "ecc_pipeline_gaussian": (ctypes.c_int, [_VP, ctypes.POINTER(EccImage), _VP, _I32, _I32, _VP, _I32, _VP, _VP]),
    "ecc_compute_noalloc": (ctypes.c_int, [ctypes.POINTER(EccImage), _I32, _I32, _I32, ctypes.c_uint32, _VP, _VP,
                                           _VP]),
    "ecc_status_get": (ctypes.c_int, [_VP, _VP]),
    "ecc_plan_kernel_time": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    "ecc_plan_emitted": (ctypes.c_int, [_VP, ctypes.POINTER(_I64), _VP]),
    "ecc_last_error": (ctypes.c_char_p, []),
    "ecc_selftest_wait_timeout": (ctypes.c_int, [_I64, ctypes.POINTER(ctypes.c_int32), _VP]),
    "ecc_server_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(EccServerDesc)]),
    "ecc_submit": (ctypes.c_int, [_VP, ctypes.POINTER(EccImage), _I32, _I32, _I32, _I32, _VP, DONE_FN, _VP,
                                  ctypes.POINTER(_U64)]),
    "ecc_wait": (ctypes.c_int, [_VP, _U64, _I64]),
    "ecc_server_prepare": (ctypes.c_int, [_VP, _I32, _I32, _I32, _I32]),
    "ecc_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), _I32, _I32]),
    "ecc_server_destroy": (ctypes.c_int, [_VP, _I32]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> Path:
    from . import build as _build
    return _build.LIB


def library():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not path.exists():
                raise RuntimeError(f"the CUDA library {path} is missing: run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'` first")
            lib = ctypes.CDLL(str(path))
            for name, (res, args) in _SIGNATURES.items():
                try:
                    f = getattr(lib, name)
                except AttributeError:
                    continue  # reported by the export test
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def exported_symbols():
    """Function names declared in include/ecc.h."""
    text = _HEADER.read_text()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ecc_\w+)\s*\(", text, flags=re.M)))


def ecc_last_error() -> str:
    msg = library().ecc_last_error()
    return msg.decode() if msg else ""


def _check(status: int):
    if status != ECC_OK:
        raise EccError(status, ecc_last_error())


def _dtype_code(dtype) -> int:
    s = str(dtype).lower()
    if s in ("u8", "uint8", "torch.uint8", "<class 'numpy.uint8'>") or dtype is np.uint8:
        return ECC_U8
    if s in ("u16", "uint16", "torch.uint16", "<class 'numpy.uint16'>") or dtype is np.uint16:
        return ECC_U16
    if isinstance(dtype, int) and dtype in (ECC_U8, ECC_U16):
        return dtype
    raise TypeError(f"unsupported dtype {dtype!r} (uint8 or uint16)")


def _stream_handle(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def image_desc(t) -> EccImage:
    """Descriptor of a CUDA tensor (uint8/uint16, 2D/3D, unit innermost stride)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("the image must be a CUDA tensor (use ecc_compute_host for host arrays)")
    return _desc(t.data_ptr(), t.dim(), _dtype_code(t.dtype), tuple(t.shape), tuple(t.stride()), t.element_size())


def host_image_desc(a: np.ndarray) -> EccImage:
    if a.dtype not in (np.uint8, np.uint16):
        raise TypeError(f"unsupported dtype {a.dtype}")
    strides = tuple(s // a.itemsize for s in a.strides)
    return _desc(a.ctypes.data, a.ndim, _dtype_code(a.dtype.type), a.shape, strides, a.itemsize)


def _desc(ptr, ndim, code, shape, strides, esize) -> EccImage:
    if ndim not in (2, 3):
        raise ValueError("the image must be 2D or 3D")
    if strides[-1] != 1:
        raise ValueError("the innermost axis must be contiguous")
    d = EccImage()
    d.data = ptr
    d.ndim = ndim
    d.dtype = code
    for i, n in enumerate(shape):
        d.dims[i] = int(n)
    d.row_pitch = int(strides[-2]) * esize
    d.slice_pitch = int(strides[-3]) * esize if ndim == 3 else 0
    return d


class Plan:
    """Owns an ecc_plan_t; destroyed with the object."""

    def __init__(self, handle: int, desc: EccPlanDesc):
        self.handle = ctypes.c_void_p(handle)
        self.desc = desc
        self.nbins = desc.hi - desc.lo + 1

    def close(self):
        if self.handle and self.handle.value:
            library().ecc_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ecc_plan(dtype="u8", lo: int = 0, hi: int | None = None, complex_mode: int = ECC_VERTEX_MAX,
             max_images: int = 1, max_voxels: int = 1 << 31, flags: int = 0) -> Plan:
    code = _dtype_code(dtype)
    if hi is None:
        hi = 255 if code == ECC_U8 else 65535
    d = EccPlanDesc(dtype=code, lo=int(lo), hi=int(hi), complex_mode=int(complex_mode),
                    max_images=int(max_images), reserved=0, max_voxels=int(max_voxels), flags=int(flags),
                    reserved2=0)
    h = ctypes.c_void_p()
    _check(library().ecc_plan(ctypes.byref(h), ctypes.byref(d)))
    return Plan(h.value, d)


def ecc_plan_destroy(plan: Plan):
    plan.close()


def ecc_plan_nbins(plan: Plan) -> int:
    return int(library().ecc_plan_nbins(plan.handle))


def ecc_plan_last_launches(plan: Plan) -> int:
    return int(library().ecc_plan_last_launches(plan.handle))


def ecc_compute(plan: Plan, image, out=None, vcec_out=None, stream=None):
    """ECC of one CUDA image; returns the int64 CUDA tensor ``out`` (allocated if None)."""
    import torch
    d = image_desc(image)
    if out is None:
        out = torch.empty(plan.nbins, dtype=torch.int64, device=image.device)
    _check_out(out, plan.nbins)
    vptr = None
    if vcec_out is not None:
        _check_out(vcec_out, plan.nbins)
        vptr = vcec_out.data_ptr()
    _check(library().ecc_compute(plan.handle, ctypes.byref(d), out.data_ptr(), vptr, _stream_handle(stream)))
    return out


def _check_out(t, n):
    import torch
    if not (t.is_cuda and t.dtype == torch.int64 and t.is_contiguous() and t.numel() >= n):
        raise ValueError(f"output must be a contiguous CUDA int64 tensor with >= {n} elements")


def ecc_compute_host(plan: Plan, array: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
    """ECC of a host array (streamed to the device in chunks); returns a host int64 array."""
    d = host_image_desc(array)
    if out is None:
        out = np.empty(plan.nbins, dtype=np.int64)
    if out.dtype != np.int64 or not out.flags.c_contiguous or out.size < plan.nbins:
        raise ValueError("out must be a contiguous int64 array")
    _check(library().ecc_compute_host(plan.handle, ctypes.byref(d), out.ctypes.data, _stream_handle(stream)))
    return out


def ecc_compute_levels(plan: Plan, image, levels, out=None, stream=None):
    """ECC of a float32 CUDA image at the ascending thresholds ``levels`` (a float32 CUDA
    tensor of m entries); returns the int64 CUDA tensor ``out`` of m entries."""
    import torch
    if image.dtype != torch.float32 or levels.dtype != torch.float32:
        raise TypeError("image and levels must be float32 tensors")
    if not image.is_cuda or not levels.is_cuda:
        raise ValueError("image and levels must be CUDA tensors")
    if not levels.is_contiguous() or levels.dim() != 1:
        raise ValueError("levels must be a contiguous 1-D tensor")
    m = levels.numel()
    d = _desc(image.data_ptr(), image.dim(), ECC_F32, tuple(image.shape), tuple(image.stride()), 4)
    if out is None:
        out = torch.empty(m, dtype=torch.int64, device=image.device)
    _check_out(out, m)
    _check(library().ecc_compute_levels(plan.handle, ctypes.byref(d), levels.data_ptr(), m, out.data_ptr(),
                                        _stream_handle(stream)))
    return out


def _f32_image_desc(image):
    import torch
    if not isinstance(image, torch.Tensor) or image.dtype != torch.float32 or not image.is_cuda:
        raise TypeError("the image must be a float32 CUDA tensor")
    return _desc(image.data_ptr(), image.dim(), ECC_F32, tuple(image.shape), tuple(image.stride()), 4)


def ecc_levels_present(plan: Plan, image, max_levels: int = 65536, levels_out=None, count_out=None, stream=None):
    """Eq. 1's thresholds of a float32 CUDA image (its distinct values, ascending;
    NaN left out, -0.0 as 0.0), on the device.  Returns (levels, count): a float32
    CUDA tensor of max_levels entries whose first n hold the levels, and an int32
    CUDA tensor of one entry holding n (max_levels + 1 when there are more).
    Asynchronous."""
    import torch
    d = _f32_image_desc(image)
    if levels_out is None:
        levels_out = torch.empty(max_levels, dtype=torch.float32, device=image.device)
    if count_out is None:
        count_out = torch.empty(1, dtype=torch.int32, device=image.device)
    if levels_out.dtype != torch.float32 or not levels_out.is_contiguous() or levels_out.numel() < max_levels:
        raise ValueError("levels_out must be a contiguous float32 CUDA tensor of max_levels entries")
    if count_out.dtype != torch.int32 or count_out.numel() < 1:
        raise ValueError("count_out must be an int32 CUDA tensor")
    _check(library().ecc_levels_present(plan.handle, ctypes.byref(d), levels_out.data_ptr(), int(max_levels),
                                        count_out.data_ptr(), _stream_handle(stream)))
    return levels_out, count_out


def ecc_compute_present(plan: Plan, image, max_levels: int = 65535, stream=None):
    """The paper's ECC sequence of a float32 CUDA image (Eq. 1 at its distinct
    values): returns (levels, ecc), CUDA tensors of n entries, ecc[i] =
    chi(K_{<= levels[i]}).  Synchronizes the stream once, to read n."""
    import torch
    d = _f32_image_desc(image)
    levels = torch.empty(max_levels, dtype=torch.float32, device=image.device)
    out = torch.empty(max_levels, dtype=torch.int64, device=image.device)
    n = ctypes.c_int32(0)
    _check(library().ecc_compute_present(plan.handle, ctypes.byref(d), levels.data_ptr(), int(max_levels),
                                         ctypes.byref(n), out.data_ptr(), _stream_handle(stream)))
    return levels[:n.value], out[:n.value]


def ecc_compute_nd(plan: Plan, image, out=None, vcec_out=None, stream=None):
    """ECC of a 2D, 3D or 4D uint8/uint16 CUDA tensor; returns the int64 CUDA tensor ``out``."""
    import torch
    if not isinstance(image, torch.Tensor) or not image.is_cuda:
        raise ValueError("the image must be a CUDA tensor")
    if image.dim() not in (2, 3, 4) or image.stride(-1) != 1:
        raise ValueError("the image must be 2D, 3D or 4D with a contiguous innermost axis")
    d = EccImageNd()
    d.data = image.data_ptr()
    d.ndim = image.dim()
    d.dtype = _dtype_code(image.dtype)
    es = image.element_size()
    for i, n in enumerate(image.shape):
        d.dims[i] = int(n)
    for i in range(image.dim() - 1):
        d.pitches[i] = int(image.stride(i)) * es
    if out is None:
        out = torch.empty(plan.nbins, dtype=torch.int64, device=image.device)
    _check_out(out, plan.nbins)
    vptr = None
    if vcec_out is not None:
        _check_out(vcec_out, plan.nbins)
        vptr = vcec_out.data_ptr()
    _check(library().ecc_compute_nd(plan.handle, ctypes.byref(d), out.data_ptr(), vptr, _stream_handle(stream)))
    return out


def gaussian_taps(sigma: float, radius: int = 6) -> np.ndarray:
    """Normalized float32 Gaussian taps (2 radius + 1 of them; the paper's filter has 13)."""
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-0.5 * (k / float(sigma)) ** 2)
    return (w / w.sum()).astype(np.float32)


def ecc_pipeline_gaussian(plan: Plan, image, taps, iterations: int, levels, out=None, stream=None):
    """Iterated (ECC at ``levels``, then smoothing with ``taps``) on a float32 CUDA image,
    in place; returns the int64 CUDA tensor [iterations, m] of ECCs."""
    import torch
    if image.dtype != torch.float32 or levels.dtype != torch.float32:
        raise TypeError("image and levels must be float32 tensors")
    if not image.is_cuda or not levels.is_cuda:
        raise ValueError("image and levels must be CUDA tensors")
    taps = np.ascontiguousarray(taps, dtype=np.float32)
    m = levels.numel()
    d = _desc(image.data_ptr(), image.dim(), ECC_F32, tuple(image.shape), tuple(image.stride()), 4)
    if out is None:
        out = torch.empty((int(iterations), m), dtype=torch.int64, device=image.device)
    _check_out(out, int(iterations) * m)
    _check(library().ecc_pipeline_gaussian(plan.handle, ctypes.byref(d), taps.ctypes.data, taps.size,
                                           int(iterations), levels.data_ptr(), m, out.data_ptr(),
                                           _stream_handle(stream)))
    return out


def ecc_compute_stream(plan: Plan, array: np.ndarray, device_budget_bytes: int = 0, out: np.ndarray | None = None,
                       stream=None) -> np.ndarray:
    """Out-of-core ECC of a host array of any size through at most ``device_budget_bytes`` of device
    chunk buffers (0 = 1 GiB); returns a host int64 array."""
    d = host_image_desc(array)
    if out is None:
        out = np.empty(plan.nbins, dtype=np.int64)
    if out.dtype != np.int64 or not out.flags.c_contiguous or out.size < plan.nbins:
        raise ValueError("out must be a contiguous int64 array")
    _check(library().ecc_compute_stream(plan.handle, ctypes.byref(d), out.ctypes.data, int(device_budget_bytes),
                                        _stream_handle(stream)))
    return out


class ImageDescs:
    """A reusable array of ecc_image descriptors for ecc_compute_batch.

    Building one descriptor per tensor costs host time per image; a caller
    that runs the same images repeatedly builds the array once.  The
    descriptors hold the tensors' addresses, shapes and strides at build
    time: the tensors must stay alive and keep their storage."""

    def __init__(self, images):
        self.images = list(images)   # keeps the tensors alive
        self.n = len(self.images)
        self.array = (EccImage * self.n)(*[image_desc(t) for t in self.images])
        self.device = self.images[0].device if self.n else None


def image_descs(images) -> ImageDescs:
    return ImageDescs(images)


def ecc_compute_batch(plan: Plan, images, out=None, stream=None):
    """ECC of every image in ``images`` (CUDA tensors of mixed shapes, or an
    ImageDescs built from them); returns int64 [n, nbins]."""
    import torch
    descs = images if isinstance(images, ImageDescs) else ImageDescs(images)
    n = descs.n
    if out is None:
        out = torch.empty((n, plan.nbins), dtype=torch.int64, device=descs.device)
    _check_out(out, n * plan.nbins)
    _check(library().ecc_compute_batch(plan.handle, n, descs.array, out.data_ptr(), _stream_handle(stream)))
    return out


def ecc_plan_kernel_time(plan: Plan):
    """(total stencil device ms, launches) recorded since the last call (needs ECC_FLAG_TIME_KERNELS)."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(library().ecc_plan_kernel_time(plan.handle, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def ecc_plan_emitted(plan: Plan, stream=None) -> int:
    """Voxels with a nonzero signed count since the last call (needs ECC_FLAG_COUNT_EMITTED)."""
    n = ctypes.c_int64()
    _check(library().ecc_plan_emitted(plan.handle, ctypes.byref(n), _stream_handle(stream)))
    return n.value


def ecc_compute_noalloc(image, lo: int = 0, hi: int | None = None, complex_mode: int = ECC_VERTEX_MAX,
                        out=None, vcec_out=None, flags: int = 0, stream=None):
    """ECC of one CUDA image with no device allocation inside the library
    (fixed scratch array; synchronous).  ``out`` must be given by callers that
    cannot let this binding allocate it."""
    import torch
    d = image_desc(image)
    if hi is None:
        hi = 255 if d.dtype == ECC_U8 else 65535
    n = hi - lo + 1
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=image.device)
    _check_out(out, n)
    vptr = None
    if vcec_out is not None:
        _check_out(vcec_out, n)
        vptr = vcec_out.data_ptr()
    _check(library().ecc_compute_noalloc(ctypes.byref(d), int(lo), int(hi), int(complex_mode), int(flags),
                                         out.data_ptr(), vptr, _stream_handle(stream)))
    return out


def ecc_selftest_wait_timeout(limit_us: int = 50_000, stream=None):
    """Run the bounded-wait self-test; returns (status, [flag wait gave up, mbarrier wait gave up])."""
    gave = (ctypes.c_int32 * 2)()
    st = library().ecc_selftest_wait_timeout(int(limit_us), gave, _stream_handle(stream))
    if st not in (ECC_OK, ECC_E_TIMEOUT):
        _check(st)
    return st, [int(gave[0]), int(gave[1])]


def ecc_status_get(plan: Plan, stream=None) -> int:
    """Synchronizes and returns the device status; raises EccError on a device-reported error."""
    st = library().ecc_status_get(plan.handle, _stream_handle(stream))
    _check(st)
    return st


# ------------------------------------------------------------------ serving

class Server:
    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)
        self._callbacks = {}

    def close(self, cancel: bool = False):
        if self.handle and self.handle.value:
            _check(library().ecc_server_destroy(self.handle, int(cancel)))
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ecc_server_create(hbm_budget_bytes: int, n_streams: int = 4, max_batch: int = 64,
                      max_job_voxels: int = 1 << 31, flags: int = 0) -> Server:
    d = EccServerDesc(hbm_budget_bytes=int(hbm_budget_bytes), n_streams=int(n_streams), max_batch=int(max_batch),
                      max_job_voxels=int(max_job_voxels), flags=int(flags), reserved=0)
    h = ctypes.c_void_p()
    _check(library().ecc_server_create(ctypes.byref(h), ctypes.byref(d)))
    return Server(h.value)


def ecc_submit(server: Server, image, lo: int, hi: int, complex_mode: int = ECC_VERTEX_MAX, out=None,
               host_input: bool | None = None) -> int:
    """Submit one job; ``image`` is a CUDA tensor or a host numpy array; ``out``
    (host int64 array of hi-lo+1 values) receives the ECC at completion."""
    import torch
    if isinstance(image, np.ndarray):
        d = host_image_desc(image)
        host_input = True
    else:
        d = image_desc(image) if image.is_cuda else host_image_desc(image.numpy())
        host_input = not image.is_cuda
    optr = None
    if out is not None:
        if out.dtype != np.int64 or out.size < hi - lo + 1:
            raise ValueError("out must be an int64 host array of hi-lo+1 values")
        optr = out.ctypes.data
    ticket = ctypes.c_uint64()
    _check(library().ecc_submit(server.handle, ctypes.byref(d), int(host_input), int(lo), int(hi),
                                int(complex_mode), optr, DONE_FN(0), None, ctypes.byref(ticket)))
    return int(ticket.value)


def ecc_wait(server: Server, ticket: int, timeout_us: int = -1) -> int:
    st = library().ecc_wait(server.handle, ctypes.c_uint64(ticket), int(timeout_us))
    if st not in (ECC_OK, ECC_E_TIMEOUT):
        _check(st)
    return st


def ecc_server_stats(server: Server, reset: bool = False) -> dict:
    vals = (ctypes.c_double * 8)()
    _check(library().ecc_server_stats(server.handle, vals, 8, int(reset)))
    keys = ["jobs", "voxels", "p50_us", "p99_us", "max_us", "launches", "busy_us", "peak_bytes"]
    return dict(zip(keys, list(vals)))


def ecc_server_prepare(server: Server, dtype, lo: int, hi: int, complex_mode: int = ECC_VERTEX_MAX):
    """Make the plans (and batch graphs) of one job key on every slot ahead of its first jobs."""
    _check(library().ecc_server_prepare(server.handle, _dtype_code(dtype), int(lo), int(hi), int(complex_mode)))


def ecc_server_destroy(server: Server, cancel: bool = False):
    server.close(cancel)
