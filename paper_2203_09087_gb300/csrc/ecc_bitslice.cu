// ecc_bitslice.cu -- bit-sliced stencil + histogram for 2D images (sm_103a),
// and the dispatch of the bit-sliced kernels (3D: ecc_bs3d.cu).
//
// The per-voxel rule is the paper's (Sec. 2.3, Algorithm 1; Sec. 3.2-3.3):
// a pixel introduces the cells it wins against every other member of, and
// adds (-1)^dim of each to the histogram bin of its gray level.
//
//  * Bit-slicing.  A lane holds a window of 32 pixels of one row as
//    K = 8*sizeof(T) bit planes (transpose in registers, ecc_bitslice.cuh).
//    Every comparison of two windows is then K majority operations for 32
//    pixel pairs, and all cell logic is 32 pixels per 32-bit operation.
//  * Overlapped windows.  A window covers pixels [x0-1, x0+31) and produces
//    the 30 pixels x0..x0+29, so the +-1 shifts along x stay inside the
//    register: no halo bits have to be fetched from neighbouring windows.
//  * Lanes along x, warps walk rows; rows come from aligned 32-bit global
//    words (any pitch).  Each of the four neighbour directions is compared
//    once per pixel pair; a pixel's wins over earlier neighbours are the
//    negations of those neighbours' comparisons (ties go to the lower
//    linear index).
//  * Histogram.  Only pixels whose signed cell count is nonzero are emitted,
//    into replicated shared-memory int32 histograms flushed once per CTA
//    into the int64 accumulator, or directly into global int64 bins when
//    nbins is too large for shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "ecc_bitslice.cuh"
#include "ecc_internal.h"
#include "ecc_scan_block.cuh"
#include "ecc_sync.cuh"
#include "ecc_walk.cuh"
#include "ecc_walk2.cuh"

namespace ecc {
namespace {

constexpr int kOut = 30;  // output voxels per 32-voxel window (and per warp in y)

template <typename T>
struct Cfg {
    static constexpr int ES = (int)sizeof(T);
    static constexpr int K = 8 * ES;           // bit planes
    static constexpr int WORDS = 8 * ES;       // 32-bit words of a window
    static constexpr int CHUNKS = 2 * ES + 1;  // 16-byte loads covering a window at any offset
};

// ----------------------------------------------------------------- 2D kernel
//
// A lane holds a window [30 t - 1, 30 t + 31) of a row and walks a chunk
// of rows; the lanes of a warp take consecutive (window, row chunk) pairs,
// windows fastest, so in a wide image they sit side by side in one row (a
// warp covers 960 columns) and in a narrow one they go on into the next
// chunks instead of idling (a 256-wide image keeps all 32 lanes busy, not
// 9).  Rows come straight from global memory as aligned 32-bit words
// (coalesced across the lanes of a row; any pitch and alignment; words that
// hold no byte of the row are not read).  Each voxel pair is compared once:
// the row pair (y, y+1) in three x offsets and the in-row pair, the earlier
// voxel's wins being the negations.  Warps are independent work-list
// walkers; the CTA only shares the privatized histogram.

struct Bs2dArgs {
    const unsigned char *data;
    int64_t nx, ny, pitch;
    int64_t y_begin, y_end;
    int32_t nwin, nyc, ychunk, nitems;  // 30-column windows per row, row chunks, rows per chunk, warp items
    int32_t smem_hist, range_check;
    int32_t check_all;       // compare every output pixel with [lo, hi] (range narrower than the type)
    uint32_t lo_bits, hi_bits;
    walk3::Mul mu;
    HistDst h;
    unsigned int *status;
    long long *ecc_out;      // non-null: the last CTA also scans the bins (whole image, small histogram)
    long long *vcec_out;
    unsigned int *done;      // finished-CTA count for the fused scan (zero between launches)
};

constexpr int kWarps2d = 4;

template <typename T, bool TOP, int HREP>
__global__ void __launch_bounds__(kWarps2d * 32, 4) bs2d_kernel(const Bs2dArgs a)
{
    using C = Cfg<T>;
    constexpr int K = C::K, ES = C::ES;
    extern __shared__ __align__(16) int hist2[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (a.smem_hist)
        for (int i = tid; i < HREP * a.h.nbins; i += kWarps2d * 32) hist2[i] = 0;
    __syncthreads();
    int *my_hist = hist2 + (warp % HREP) * a.h.nbins;
    const int64_t row_bytes = a.nx * ES;

    for (int item = blockIdx.x * kWarps2d + warp; item < a.nitems; item += gridDim.x * kWarps2d) {
        // lane l takes (window, row chunk) pair q = 32 item + l, windows
        // fastest: in a wide image the warp's 32 windows sit side by side
        // in one row chunk; in a narrow one (or where a row's windows run
        // out) the lanes go on into the next chunks, so every lane has work
        const int64_t q = 32 * (int64_t)item + lane;
        const bool active = q < (int64_t)a.nwin * a.nyc;
        const int64_t yc = q / a.nwin, xt = q - yc * a.nwin;
        const int64_t yb = a.y_begin + yc * a.ychunk;
        const int64_t ye = !active ? yb - 1 : (yb + a.ychunk < a.y_end ? yb + a.ychunk : a.y_end);
        const int64_t xw = kOut * xt - 1;  // voxel of window bit 0
        const int64_t first = xw * ES;     // may be negative at x = 0
        const uint32_t xex = active ? walk::x_exist_mask(xw, a.nx) : 0u;
        const uint32_t out_x = xex & 0x7ffffffeu;
        // row yy as K planes and the existence plane (a row outside the
        // image, or a window wholly outside the row, is all missing)
        auto fetch = [&](int64_t yy, uint32_t *P) {
            if (yy < 0 || yy >= a.ny || !xex) {
#pragma unroll
                for (int i = 0; i < K; ++i) P[i] = 0u;
                P[K] = 0xffffffffu;
                return;
            }
            walk2::load_window<K>(a.data + yy * a.pitch, row_bytes, first, P, a.mu);
            P[K] = ~xex;
        };
        // values of emitted voxels come from the row just read (cached)
        const walk::Bins bins{a.smem_hist ? my_hist : nullptr, a.h.acc, a.h.lo, a.h.nbins, a.range_check,
                              a.status};
        int64_t y1 = yb;
        auto emit = [&](uint32_t m, const uint32_t *X) {
            if (a.h.emitted && m) atomicAdd(a.h.emitted, (unsigned long long)__popc(m));  // diagnostic count
            const unsigned char *row = a.data + (y1 - 1) * a.pitch + xw * ES;
            walk2::emit2(
                m, X,
                [&](int i) {
                    return ES == 1 ? (int)__ldg(row + i) : (int)__ldg(reinterpret_cast<const unsigned short *>(row) + i);
                },
                [&](int v, int k) { bins.add(v, k); });
        };
        uint32_t P[K + 1];
        fetch(yb - 1, P);
        walk2::Walk<K, TOP> wk;
        wk.begin(P, a.mu);
        uint32_t bad = 0;  // output pixels outside [lo, hi] (when checked)
        for (; y1 <= ye; ++y1) {
            uint32_t B[K + 1];
            fetch(y1, B);
            if (a.check_all && y1 < ye) bad |= ~walk::in_range<K>(B, a.lo_bits, a.hi_bits) & out_x;
            wk.step(B, y1 - 1 >= yb, out_x, a.mu, emit);
        }
        if (a.check_all && __any_sync(0xffffffffu, bad != 0u) && lane == 0) atomicOr(a.status, DEV_RANGE);
    }
    __syncthreads();
    if (a.smem_hist)
        for (int i = tid; i < a.h.nbins; i += kWarps2d * 32) {
            int v = 0;
#pragma unroll
            for (int r = 0; r < HREP; ++r) v += hist2[r * a.h.nbins + i];
            if (v) atomicAdd(a.h.acc + i, (unsigned long long)(long long)v);
        }
    if (a.ecc_out) {
        // the last CTA to finish scans the bins (as the 3D kernel does)
        __shared__ int s_last2;
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            s_last2 = atomicAdd(a.done, 1u) == gridDim.x - 1;
            if (s_last2) {
                *a.done = 0u;
                __threadfence();
            }
        }
        __syncthreads();
        if (s_last2) scan_bins<kWarps2d * 32>(a.h.acc, a.ecc_out, a.vcec_out, a.h.nbins, tid);
    }
}

template <typename T, bool TOP>
cudaError_t launch_2d_t(const Geom &g, int64_t yb, int64_t ye, const HistDst &h, bool range_check,
                        unsigned int *status, int num_sms, cudaStream_t s, unsigned int *done, FusedScan *fs)
{
    constexpr int HREP = 2;
    Bs2dArgs a{};
    const bool fuse = fs && fs->ecc && done && yb == 0 && ye == g.ny && h.nbins <= kFusedScanMaxBins;
    a.ecc_out = fuse ? fs->ecc : nullptr;
    a.vcec_out = fuse ? fs->vcec : nullptr;
    a.done = done;
    a.data = g.data;
    a.nx = g.nx;
    a.ny = g.ny;
    a.pitch = g.pitch_y;
    a.y_begin = yb;
    a.y_end = ye;
    a.h = h;
    // bins are guarded whenever values can fall outside them; every output
    // pixel is compared with the bounds unless the caller opted out
    a.range_check = walk::range_is_narrow(h.lo, h.nbins, g.esize);
    a.check_all = range_check && a.range_check;
    a.lo_bits = (uint32_t)h.lo;
    a.hi_bits = (uint32_t)(h.lo + h.nbins - 1);
    a.mu = walk3::make_mul();
    a.status = status;
    if ((g.nx + kOut - 1) / kOut > 2147483647) return cudaErrorNotSupported;
    a.nwin = (int32_t)((g.nx + kOut - 1) / kOut);
    a.smem_hist = (size_t)HREP * h.nbins * 4 <= 160 * 1024;
    const size_t smem = a.smem_hist ? (size_t)HREP * h.nbins * 4 : 0;
    auto kern = bs2d_kernel<T, TOP, HREP>;
    static size_t attr_smem = 48 * 1024;
    if (smem > attr_smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cudaErrorNotSupported;
        }
        attr_smem = smem;
    }
    static int per_sm_cached = -1;
    static size_t smem_cached = 0;
    if (per_sm_cached < 0 || smem_cached != smem) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_cached, kern, kWarps2d * 32, smem);
        if (e != cudaSuccess) return e;
        smem_cached = smem;
    }
    if (per_sm_cached < 1) return cudaErrorNotSupported;
    const int64_t warps_max = (int64_t)num_sms * per_sm_cached * kWarps2d;
    const int64_t depth = ye - yb;
    // about three warp items per resident warp, in chunks of at least 16
    // rows (each re-reads one halo row) unless that leaves fewer than four
    // warps per SM: small images walk single rows (a lane's walk is a chain
    // of dependent row steps)
    int64_t nyc = (3 * warps_max * 32 + a.nwin - 1) / a.nwin;
    const int64_t cap16 = (depth + 15) / 16;
    const int64_t cap = cap16 * a.nwin >= 4 * (int64_t)num_sms * 32 ? cap16 : depth;
    if (nyc > cap) nyc = cap;
    if (nyc < 1) nyc = 1;
    a.ychunk = (int32_t)((depth + nyc - 1) / nyc);
    a.nyc = (int32_t)((depth + a.ychunk - 1) / a.ychunk);
    const int64_t items = ((int64_t)a.nwin * a.nyc + 31) / 32;
    if (items > 2147483647) return cudaErrorNotSupported;
    a.nitems = (int32_t)items;
    int64_t ctas = (items + kWarps2d - 1) / kWarps2d;
    const int64_t ctas_max = (int64_t)num_sms * per_sm_cached;
    if (ctas > ctas_max) ctas = ctas_max;
    kern<<<(unsigned)ctas, kWarps2d * 32, smem, s>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && fuse) fs->done = true;
    return e;
}

}  // namespace

// ----------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Loads (under lazy module loading) every 2D kernel a plan-free call can launch.
cudaError_t preload_bs2d()
{
    const void *fns[] = {
        (const void *)bs2d_kernel<unsigned char, false, 2>, (const void *)bs2d_kernel<unsigned char, true, 2>,
        (const void *)bs2d_kernel<unsigned short, false, 2>, (const void *)bs2d_kernel<unsigned short, true, 2>};
    cudaFuncAttributes fa;
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool bitslice_supported(const Geom &g)
{
    if (g.esize != 1 && g.esize != 2) return false;
    if (g.ndim == 2) return g.nx <= (int64_t(1) << 31) && g.ny <= (int64_t(1) << 31);
    if (g.ndim != 3) return false;
    if (reinterpret_cast<uintptr_t>(g.data) % 16) return false;
    if (g.pitch_y % 16 || g.pitch_z % 16) return false;
    if (g.nx > (int64_t(1) << 31) || g.ny > (int64_t(1) << 31) || g.nz > (int64_t(1) << 31)) return false;
    return encode_fn() != nullptr;
}

// tune_param (3D): warps per CTA of the 3D kernel, 4 or 8 (the autotuner's
// candidates); anything else picks 4.
cudaError_t launch_bitslice(const Geom &g, int64_t outer_begin, int64_t outer_end, const HistDst &h, int mode,
                            bool range_check, unsigned int *status, unsigned int *sched, int num_sms, int tune_param,
                            cudaStream_t s, FusedScan *fs)
{
    if (outer_end <= outer_begin) return cudaSuccess;
    if (!bitslice_supported(g)) return cudaErrorNotSupported;
    if (g.ndim == 2) {
        const bool top = mode == ECC_TOPCELL_MIN;
        // the fused scan's finished-CTA count: a word of the scheduling block
        // the 3D kernel does not use
        unsigned int *done = sched ? sched + 2 : nullptr;
        if (g.esize == 1)
            return top ? launch_2d_t<unsigned char, true>(g, outer_begin, outer_end, h, range_check, status, num_sms,
                                                          s, done, fs)
                       : launch_2d_t<unsigned char, false>(g, outer_begin, outer_end, h, range_check, status, num_sms,
                                                           s, done, fs);
        return top ? launch_2d_t<unsigned short, true>(g, outer_begin, outer_end, h, range_check, status, num_sms, s,
                                                       done, fs)
                   : launch_2d_t<unsigned short, false>(g, outer_begin, outer_end, h, range_check, status, num_sms,
                                                        s, done, fs);
    }
    return launch_bs3d(g, outer_begin, outer_end, h, mode, range_check, status, sched, num_sms, tune_param, s, fs);
}

}  // namespace ecc
