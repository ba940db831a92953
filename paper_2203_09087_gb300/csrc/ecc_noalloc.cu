// ecc_noalloc.cu -- ecc_compute_noalloc: one image, no device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// real-time pipeline whose device memory budget is fixed at start-up, code
// running inside another framework's memory pool or allocator callback, or a
// process whose device memory is fully reserved by such a pool.  A plan
// (ecc_plan) allocates its workspace with cudaMalloc, so those callers get
// this entry point instead.  Its scratch memory -- the int64 VCEC
// accumulator of up to kNoallocMaxBins gray levels, the device status word
// and the look-back state of the scan -- is one file-scope __device__ array
// of fixed size that every GPU loading this library holds until the process
// exits.  The caller still owns the image and the output buffers.
//
// The same stencil and scan kernels as ecc_compute run on it; only the
// scratch pointer differs.  In host code the array's name is not a device
// address, so the first call on each device looks its address up with
// cudaGetSymbolAddress (with that device current), clears it, and makes the
// CUDA runtime load every kernel this entry point may launch: CUDA loads the
// library's modules lazily, at a kernel's first use, and loading a module can
// take device memory.  The first call on each device therefore does set-up
// work and belongs at start-up, before any memory pool reserves the device's
// memory and before any stream capture (or the process runs with
// CUDA_MODULE_LOADING=EAGER).
//
// A 3D image whose rows the TMA cannot address (row pitch not a multiple of
// 16 bytes) goes through the batch kernel with its one-image work list in
// the scratch array, as ecc_compute runs it from a plan.
//
// Every call on a device shares the array: each call clears the parts that
// must start at zero before using them, and calls whose work overlaps on the
// GPU (different streams, or host threads racing) corrupt each other's
// results.
#include <cuda_runtime.h>

#include <mutex>

#include "ecc.h"
#include "ecc_internal.h"
#include "ecc_plan.h"

namespace ecc {
namespace {

constexpr int kNoallocMaxBins = 65536;
constexpr int kNoallocTiles = (kNoallocMaxBins + kScanTile - 1) / kScanTile;

// Layout (8-byte words): [0, kNoallocMaxBins) accumulator;
// then 32 words for the status word (32-bit word 0), the two scan counters
// (words 2, 3) and the stencil's work counters (words 4, 5);
// then kNoallocTiles words of tile status (ints, 2 per word) rounded up;
// then 2 * kNoallocTiles words of tile values;
// then kBatchWords words for the batch kernel's one-image work list.
constexpr int kAccWords = kNoallocMaxBins;
constexpr int kCtlWords = 32;
constexpr int kStatWords = (kNoallocTiles + 1) / 2;
constexpr int kValWords = 2 * kNoallocTiles;
constexpr int kBatchWords = (int)(kBatchSingleWsBytes / 8);  // one-image work list of the batch kernel
constexpr int kScratchWords = kAccWords + kCtlWords + kStatWords + kValWords + kBatchWords;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long *g_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// The scratch array's device address and the SM count of the current device;
// the first call per device also clears the array and loads the kernels.
ecc_status scratch_for_current_device(unsigned long long **out, int *sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("ecc_compute_noalloc: device ordinal beyond the supported range");
        return ECC_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_noalloc: cudaGetSymbolAddress");
        e = clear_device_now(p, sizeof(g_noalloc_scratch));
        if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_noalloc: scratch clear");
        if ((e = preload_bs3d()) != cudaSuccess || (e = preload_bs2d()) != cudaSuccess ||
            (e = preload_batch()) != cudaSuccess || (e = preload_direct()) != cudaSuccess ||
            (e = preload_scan()) != cudaSuccess)
            return cuda_fail(e, "ecc_compute_noalloc: kernel loading");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_noalloc: device query");
        g_sms[dev] = n;
        g_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_ptr[dev];
    *sms = g_sms[dev];
    return ECC_OK;
}

}  // namespace
}  // namespace ecc

using namespace ecc;

extern "C" ecc_status ecc_compute_noalloc(const ecc_image *img, int32_t lo, int32_t hi, int32_t complex_mode,
                                          uint32_t flags, int64_t *d_ecc, int64_t *d_vcec, void *stream)
{
    if (!img || !d_ecc) {
        set_error("ecc_compute_noalloc: NULL argument");
        return ECC_E_INVALID;
    }
    const int64_t maxval = img->dtype == ECC_U8 ? 255 : 65535;
    if (hi < lo || lo < 0 || hi > maxval) {
        set_error("ecc_compute_noalloc: invalid gray range");
        return ECC_E_INVALID;
    }
    const int64_t nbins = (int64_t)hi - lo + 1;
    if (nbins > kNoallocMaxBins) {
        set_error("ecc_compute_noalloc: more gray levels than the fixed scratch holds (65536)");
        return ECC_E_INVALID;
    }
    if (complex_mode != ECC_VERTEX_MAX && complex_mode != ECC_TOPCELL_MIN) {
        set_error("ecc_compute_noalloc: invalid complex");
        return ECC_E_INVALID;
    }
    Geom g;
    ecc_status st = image_geom(img, 0, 0, &g, nullptr, false);
    if (st != ECC_OK) return st;
    unsigned long long *base = nullptr;
    int sms = 0;
    st = scratch_for_current_device(&base, &sms);
    if (st != ECC_OK) return st;

    unsigned long long *acc = base;
    unsigned int *ctl = reinterpret_cast<unsigned int *>(base + kAccWords);
    unsigned int *status = ctl;  // word 0
    ScanWs ws{ctl + 2, ctl + 3, reinterpret_cast<int *>(base + kAccWords + kCtlWords),
              reinterpret_cast<long long *>(base + kAccWords + kCtlWords + kStatWords), kNoallocTiles};

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // clear what must start at zero: this call's accumulator bins, the status
    // word, the scan counters and tile flags
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)nbins, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(unsigned long long) * (kCtlWords + kStatWords), s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_noalloc: clear");

    const bool range = !(flags & ECC_FLAG_NO_RANGE_CHECK);
    HistDst h{acc, lo, (int32_t)nbins};
    const int64_t outer = g.ndim == 3 ? g.nz : g.ny;
    e = cudaErrorNotSupported;
    if (!(flags & ECC_FLAG_KERNEL_DIRECT) && bitslice_supported(g))
        e = launch_bitslice(g, 0, outer, h, complex_mode, range, status, ctl + 4, sms, 0, s);
    // a 3D image whose rows the TMA cannot address: the batch kernel on a
    // one-image work list in the scratch, as ecc_compute does from its plan
    if (e == cudaErrorNotSupported && !(flags & ECC_FLAG_KERNEL_DIRECT) && g.ndim == 3)
        e = launch_batch_single_ws(g, h, complex_mode, range, base + kAccWords + kCtlWords + kStatWords + kValWords,
                                   status, sms, s);
    if (e == cudaErrorNotSupported) e = launch_direct(g, 0, outer, h, complex_mode, range, status, sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_noalloc: stencil launch");
    e = launch_scan(acc, reinterpret_cast<long long *>(d_ecc), reinterpret_cast<long long *>(d_vcec), 1,
                    (int32_t)nbins, ws, status, s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_noalloc: scan launch");

    // device-detected errors of this call
    unsigned int word = 0;
    e = cudaMemcpyAsync(&word, status, sizeof(word), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_noalloc: status read");
    if (word & DEV_TIMEOUT) {
        set_error("a bounded device-side wait gave up");
        return ECC_E_TIMEOUT;
    }
    if (word & DEV_STATE) {
        set_error("the scan's look-back state was not clean (scratch corrupted)");
        return ECC_E_CUDA;
    }
    if (word & DEV_RANGE) {
        set_error("an image value lies outside [lo, hi]");
        return ECC_E_RANGE;
    }
    return ECC_OK;
}
