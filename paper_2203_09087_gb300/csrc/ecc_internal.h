// ecc_internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/ecc.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ecc.h"

namespace ecc {

// Device status word bits (reported through ecc_status_get).
enum : uint32_t {
    DEV_RANGE = 1u,    // an image value outside [lo, hi]
    DEV_TIMEOUT = 2u,  // a bounded spin-wait gave up
    DEV_LEVELS = 4u,   // threshold levels not in ascending order
    DEV_STATE = 8u,    // a scan tile claimed an index past its grid (look-back state not clean)
};

// Upper bound for every device-side spin-wait (nanoseconds of %globaltimer).
constexpr unsigned long long kSpinLimitNs = 200ull * 1000ull * 1000ull;

// Shared-memory histogram limit of the stencil kernels (int32 bins).
constexpr int kSmemBinsMax = 16384;

// Geometry of one image as the kernels see it: always three axes (z, y, x),
// 2D images have nz == 1.  Pitches in bytes.
struct Geom {
    const unsigned char *data;  // address of voxel (0, 0, 0)
    int64_t nz, ny, nx;
    int64_t pitch_y, pitch_z;
    int32_t ndim;
    int32_t esize;              // bytes per voxel
};

// A histogram destination: int64 accumulator of nbins levels.
struct HistDst {
    unsigned long long *acc;    // int64 bins, accumulated with atomics
    int32_t lo;
    int32_t nbins;
    unsigned long long *emitted = nullptr;  // if set: += voxels with a nonzero count
};

// Decoupled-lookback scan workspace (self-cleaning: the last CTA of every
// scan launch resets it to zero for the next launch).
struct ScanWs {
    unsigned int *tile_counter;
    unsigned int *done_counter;
    int *tile_status;           // 0 = not ready, 1 = aggregate, 2 = inclusive prefix
    long long *tile_value;      // [2 * max_tiles]: aggregates, then inclusive prefixes
    int32_t max_tiles;
};

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Arguments of the scan kernel.  When n_seg_dev is set, the number of
// segments is read from device memory (*n_seg_dev) instead of n, so a
// captured graph can scan a different number of images on every launch;
// CTAs beyond the data then only take part in the workspace reset.
struct ScanArgs {
    unsigned long long *acc;
    long long *ecc;
    long long *vcec;
    int64_t n;
    int32_t nbins;
    int32_t ntiles;
    ScanWs ws;
    unsigned int *status;
    const int *n_seg_dev;
};

// The scan kernel's entry (for graph nodes); grid = scan_tiles(), block = kScanThreads.
const void *scan_kernel_entry();

// --------------------------------------------------------------- launchers

// One-thread-per-voxel stencil + histogram over the voxels whose outer index
// (z for 3D, y for 2D) lies in [outer_begin, outer_end).
cudaError_t launch_direct(const Geom &g, int64_t outer_begin, int64_t outer_end, const HistDst &h,
                          int complex_mode, bool range_check, unsigned int *status,
                          int num_sms, cudaStream_t s);

// A stencil launch over a whole image may also do the scan in its last CTA
// when the histogram is small (no second launch): where the ECC (and VCEC,
// if not null) go; `done` is set when the launch took the scan on.
struct FusedScan {
    long long *ecc = nullptr;
    long long *vcec = nullptr;
    bool done = false;
};
constexpr int kFusedScanMaxBins = 4096;

// Bit-sliced stencil + histogram (3D and 2D, uint8 / uint16, both complexes).
// Returns cudaErrorNotSupported when the geometry does not qualify.
bool bitslice_supported(const Geom &g);
// sched: two device words, zero before the first launch; the kernel leaves
// them zero again (its dynamic item counter and finished-CTA count).
cudaError_t launch_bitslice(const Geom &g, int64_t outer_begin, int64_t outer_end, const HistDst &h,
                            int complex_mode, bool range_check, unsigned int *status, unsigned int *sched,
                            int num_sms, int tune_param, cudaStream_t s, FusedScan *fs = nullptr);

// The 3D bit-sliced kernel (ecc_bs3d.cu); tune = warps per CTA (4 or 8).
cudaError_t launch_bs3d(const Geom &g, int64_t zb, int64_t ze, const HistDst &h, int mode, bool range_check,
                        unsigned int *status, unsigned int *sched, int num_sms, int tune, cudaStream_t s,
                        FusedScan *fs);

// Force the loading of the kernels a plan-free call may launch (CUDA loads
// modules lazily by default: a kernel's module, with its __device__ data, is
// loaded at its first use unless something asks for it earlier).
cudaError_t preload_bs3d();
cudaError_t preload_bs2d();
cudaError_t preload_direct();
cudaError_t preload_scan();

// Segmented inclusive scan of n_seg * nbins int64 values (segment i =
// elements [i*nbins, (i+1)*nbins)).  Reads acc, writes ecc (and vcec if not
// null), and zeroes acc for the next call.
cudaError_t launch_scan(unsigned long long *acc, long long *ecc, long long *vcec, int64_t n_seg,
                        int32_t nbins, const ScanWs &ws, unsigned int *status, cudaStream_t s);

int64_t scan_tiles(int64_t n_seg, int32_t nbins);

// Zeroes device memory and returns once the zeros are in place (a private
// non-blocking stream, synchronized).  A plain cudaMemset runs on the legacy
// default stream, which work launched later on a non-blocking stream does
// not wait for: that launch could run first and have its results cleared.
cudaError_t clear_device_now(void *p, size_t bytes);

// --------------------------------------------------------------- errors

void set_error(const std::string &msg);
ecc_status cuda_fail(cudaError_t e, const char *what);
ecc_status invalid(const std::string &msg);  // sets the message, returns ECC_E_INVALID

}  // namespace ecc
