// ecc_bitslice.cu -- bit-sliced stencil + histogram for 3D volumes (sm_103a).
//
// The per-voxel rule is the paper's (Sec. 2.3, Algorithm 1; Sec. 3.2-3.3):
// a voxel introduces the cells it wins against every other member of, and
// adds (-1)^dim of each to the histogram bin of its gray level.  What changes
// is how the work maps onto GB300:
//
//  * Bit-slicing.  A lane holds a window of 32 voxels of one row as
//    K = 8*sizeof(T) bit planes (transpose in registers, ecc_bitslice.cuh).
//    Every comparison of two windows is then K majority operations for 32
//    voxel pairs, and all cell logic is 32 voxels per 32-bit operation.
//  * Overlapped windows.  A window covers voxels [x0-1, x0+31) and produces
//    the 30 voxels x0..x0+29, so the +-1 shifts along x stay inside the
//    register: no halo bits have to be fetched from neighbouring windows.
//  * Lanes along y, CTA walks z.  Lane l of a warp holds row y0-1+l (lanes 0
//    and 31 are the y halo); the CTA walks planes z upward.  Each of the 13
//    neighbour directions is compared once per voxel pair (ecc_walk.cuh):
//    plane z against plane z+1 and the in-plane pairs of z+1, the pairs
//    with rows y-1 and y+1 exchanged by warp shuffles.  A voxel's wins over
//    earlier neighbours are the negations of those neighbours' comparisons
//    (ties go to the lower linear index).  The cell count groups the 26
//    signed cell terms into 12 one-bit chains (ecc_bitslice.cuh).
//  * TMA ring.  One elected thread streams one tile plane per step
//    (cp.async.bulk.tensor, mbarrier completion) into a ring of stages; the
//    box starts 16-byte aligned and is an odd number of 16-byte units wide so
//    the per-lane 16-byte shared loads are bank-conflict free.  The
//    boundary is an extra bit plane set from coordinates (a missing voxel
//    compares as 2^K), never the zero fill.
//  * Histogram.  Only voxels whose signed cell count is nonzero (rare in
//    smooth fields) are emitted, into replicated shared-memory int32
//    histograms flushed once per CTA into the int64 accumulator, or
//    directly into global int64 bins when nbins is too large for shared
//    memory.
//  * Persistent CTAs take (x-tile, y-tile, z-chunk) items; every wait on an
//    mbarrier is bounded by %globaltimer and reports DEV_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "ecc_bitslice.cuh"
#include "ecc_internal.h"
#include "ecc_scan_block.cuh"
#include "ecc_sync.cuh"
#include "ecc_walk.cuh"

namespace ecc {
namespace {

constexpr int kOut = 30;  // output voxels per 32-voxel window (and per warp in y)

__host__ __device__ constexpr int box_bytes(int nw, int es)
{
    // from the 16-byte aligned box start to the last window's end plus the
    // 4-byte word overread, as an odd number of 16-byte units
    int need = 16 + (kOut * nw + 1) * es + 4;
    int units = (need + 15) / 16;
    if ((units & 1) == 0) ++units;
    return units * 16;
}

template <typename T>
struct Cfg {
    static constexpr int ES = (int)sizeof(T);
    static constexpr int K = 8 * ES;           // bit planes
    static constexpr int S = ES == 1 ? 8 : 6;  // ring stages
    static constexpr int WORDS = 8 * ES;       // 32-bit words of a window
    static constexpr int CHUNKS = 2 * ES + 1;  // 16-byte loads covering a window at any offset
};

struct Bs3dArgs {
    unsigned int *sched;     // [0] next item, [1] finished CTAs (reset by the last CTA)
    int64_t nx, ny, nz;
    int64_t z_begin, z_end;  // outer range of output planes
    int32_t ntx, nty, nzc;   // tiles along x, y and z-chunks
    int32_t zchunk;
    int32_t nitems;
    int32_t smem_hist;
    int32_t range_check;
    HistDst h;
    unsigned int *status;
    long long *ecc_out;      // non-null: the last CTA also scans the bins (whole image, small histogram)
    long long *vcec_out;
};

// ----------------------------------------------------------------- TMA

using sync::mbar_arrive;
using sync::mbar_expect_tx;
using sync::mbar_init;
using sync::mbar_wait;
using sync::smem_u32;
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Read this lane's 32-voxel window from the staged tile row and transpose it.
template <typename T>
__device__ __forceinline__ void load_window(const unsigned char *row, int off, uint32_t *planes)
{
    using C = Cfg<T>;
    const int base = off & ~15;
    const int sh = off & 15;
    uint32_t v[4 * C::CHUNKS];
#pragma unroll
    for (int c = 0; c < C::CHUNKS; ++c) {
        const uint4 q = *reinterpret_cast<const uint4 *>(row + base + 16 * c);
        v[4 * c + 0] = q.x;
        v[4 * c + 1] = q.y;
        v[4 * c + 2] = q.z;
        v[4 * c + 3] = q.w;
    }
    uint32_t r[C::WORDS];
    const int wsh = (sh & 3) * 8;
    const uint32_t m = bs::kPow2[(32 - wsh) & 31];  // unused when wsh == 0
    // the word offset is uniform across the warp (all lanes read the same
    // columns); the byte shift is done as two multiplies on the FMA pipe
    switch (sh >> 2) {
#define ECC_WIN(W)                                                                     \
    case W:                                                                            \
        if (wsh == 0) {                                                                \
            _Pragma("unroll") for (int i = 0; i < C::WORDS; ++i) r[i] = v[i + W];      \
        } else {                                                                       \
            _Pragma("unroll") for (int i = 0; i < C::WORDS; ++i) r[i] =                \
                v[i + W + 1] * m + __umulhi(v[i + W], m);                              \
        }                                                                              \
        break;
        ECC_WIN(0)
        ECC_WIN(1)
        ECC_WIN(2)
        ECC_WIN(3)
#undef ECC_WIN
    }
    if (C::ES == 1)
        bs::transpose_u8(r, planes);
    else
        bs::transpose_u16(r, planes);
}

// NW compute warps and one producer warp.  Stage s of the ring has a "full"
// barrier (the TMA's transaction count) and an "empty" barrier (one arrival
// per compute warp once it has copied its window out of the stage), so the
// warps never wait for each other, only for data.  The producer claims items
// from a global counter (dynamic load balance) and tags every stage with its
// item; a stage tagged -1 (no copy, plain arrival) ends the CTA.  The last
// CTA to finish resets the counter for the next launch.
// Blocks per SM the register allocation must allow: the walk is latency
// bound, so more resident warps beat more registers per thread.
template <typename T, int NW>
constexpr int bs3d_min_blocks()
{
    return sizeof(T) == 1 ? (NW == 3 ? 5 : (NW == 4 ? 4 : 2)) : (NW == 3 ? 3 : (NW == 4 ? 2 : 1));
}

template <typename T, int NW, bool TOP, int HREP>
__global__ void __launch_bounds__((NW + 1) * 32, bs3d_min_blocks<T, NW>())
    bs3d_kernel(const __grid_constant__ CUtensorMap tmap, const Bs3dArgs a)
{
    using C = Cfg<T>;
    constexpr int K = C::K, S = C::S, ES = C::ES;
    constexpr int BWB = box_bytes(NW, ES);
    constexpr int STAGE = 32 * BWB;
    constexpr int NTH = (NW + 1) * 32;
    constexpr int ALIGN_EL = 16 / ES;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *stages = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * STAGE);
    uint64_t *empty = full + S;
    int *hist = reinterpret_cast<int *>(empty + S);
    __shared__ int s_abort;
    __shared__ int s_item[S];        // item of the plane held by each stage, -1 = end
    __shared__ long long s_consumed[NW];
    __shared__ long long s_issued;
    __shared__ int s_last;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (a.smem_hist)
        for (int i = tid; i < HREP * a.h.nbins; i += NTH) hist[i] = 0;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_issued = 0;
    }
    __syncthreads();

    auto decode = [&](int item, int &xt, int &yt, int64_t &zb, int64_t &ze) {
        xt = item % a.ntx;
        const int r = item / a.ntx;
        yt = r % a.nty;
        const int zc = r / a.nty;
        zb = a.z_begin + (int64_t)zc * a.zchunk;
        ze = zb + a.zchunk < a.z_end ? zb + a.zchunk : a.z_end;
    };
    auto box_x = [&](int xt) -> int64_t {
        const int64_t xm = (int64_t)xt * (kOut * NW) - 1;
        return (xm >= 0 ? xm / ALIGN_EL : -((-xm + ALIGN_EL - 1) / ALIGN_EL)) * ALIGN_EL;
    };

    if (warp == NW) {
        // ------------------------------------------------------ producer warp
        if (lane == 0) {
            int64_t g = 0;
            bool live = true;
            while (live) {
                const unsigned int claimed = atomicAdd(a.sched, 1u);
                const bool more = claimed < (unsigned int)a.nitems;   // unsigned: never a negative item
                const int item = more ? (int)claimed : 0;
                int xt = 0, yt = 0;
                int64_t zb = 0, ze = -1;
                if (more) decode(item, xt, yt, zb, ze);
                const int bx = (int)box_x(xt);
                const int y0 = yt * kOut - 1;
                // planes zb-1 .. ze, or one terminal stage
                for (int64_t z = zb - 1; more ? z <= ze : z == zb - 1; ++z, ++g) {
                    const int s = (int)(g % S);
                    if (g >= S && !mbar_wait(&empty[s], (uint32_t)(((g / S) - 1) & 1))) {
                        atomicOr(a.status, DEV_TIMEOUT);
                        atomicExch(&s_abort, 1);
                        live = false;
                        break;
                    }
                    if (*(volatile int *)&s_abort) {
                        live = false;
                        break;
                    }
                    s_item[s] = more ? item : -1;
                    if (more) {
                        mbar_expect_tx(&full[s], STAGE);
                        tma_load_3d(stages + (size_t)s * STAGE, &tmap, bx, y0, (int)z, &full[s]);
                    } else {
                        mbar_arrive(&full[s]);
                        live = false;
                    }
                    s_issued = g + 1;
                }
            }
        }
    } else {
        // ------------------------------------------------------ compute warps
        int *my_hist = hist + (warp % HREP) * a.h.nbins;
        unsigned n_emitted = 0;  // ECC_FLAG_COUNT_EMITTED
        int g = 0, g_slot = 0;  // planes consumed; ring slot and phase of plane g
        uint32_t g_phase = 0;
        bool ok = true;
        auto wait_full = [&]() -> int {
            // warp-uniform outcome: the phase completed if any lane saw it
            if (!__any_sync(0xffffffffu, mbar_wait(&full[g_slot], g_phase))) {
                if (lane == 0) {
                    atomicOr(a.status, DEV_TIMEOUT);
                    atomicExch(&s_abort, 1);
                }
                ok = false;
                return -1;
            }
            return g_slot;
        };
        auto next_plane = [&]() {
            ++g;
            if (++g_slot == S) {
                g_slot = 0;
                g_phase ^= 1u;
            }
        };
        int off = 0;
        // Copy this lane's window of plane g out of its stage.  The stage is
        // released after the plane's emission, which reads voxel values there.
        // e_row: the existence plane of this lane's window in a plane that
        // exists (set per item); a plane outside the image is all missing.
        uint32_t e_row = 0;
        auto fetch = [&](walk::Rows3<K> &r, bool plane_exists) -> int {
            const int s = ok ? wait_full() : -1;
            if (s >= 0) load_window<T>(stages + (size_t)s * STAGE + lane * BWB, off, r.P);
            r.P[K] = plane_exists ? e_row : 0xffffffffu;
            next_plane();
            walk::complete_rows<K>(r);
            return s;
        };
        auto release = [&](int s) {
            if (s >= 0) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
        };
        while (ok) {
            // the stage of the next item's first plane says which item it is
            const int s0 = wait_full();
            if (s0 < 0) break;
            const int item = s_item[s0];
            if (item < 0) {
                next_plane();
                break;
            }
            int xt, yt;
            int64_t zb, ze;
            decode(item, xt, yt, zb, ze);
            const int64_t X0 = (int64_t)xt * (kOut * NW);
            const int64_t y0 = (int64_t)yt * kOut - 1;
            const int64_t y = y0 + lane;
            const int64_t xw = X0 + kOut * warp - 1;  // voxel of window bit 0
            off = (int)((xw - box_x(xt)) * ES);
            const uint32_t xex = walk::x_exist_mask(xw, a.nx);
            const bool lane_out = lane >= 1 && lane <= kOut && y < a.ny;
            const uint32_t out_x = lane_out ? (xex & 0x7ffffffeu) : 0u;
            e_row = (y >= 0 && y < a.ny) ? ~xex : 0xffffffffu;
            // plane indices fit in int: TMA coordinates are 32-bit
            const int nz = (int)a.nz, z_first = (int)zb, z_last = (int)ze;
            walk::Walk3d<K, TOP> wk;
            wk.begin();
            // The plane being emitted: this lane's window in its stage (bit i
            // of the window is element i), read only for emitted voxels.
            const unsigned char *vals = stages;
            const walk::Bins bins{a.smem_hist ? my_hist : nullptr, a.h.acc, a.h.lo, a.h.nbins, a.range_check,
                                  a.status};
            auto emit = [&](uint32_t m, const uint32_t *Tc, const uint32_t *) {
                if (a.h.emitted) n_emitted += __popc(m);
                walk::emit_sparse3d<TOP>(
                    m, Tc,
                    [&](int i) {
                        return ES == 1 ? (int)vals[i] : (int)reinterpret_cast<const unsigned short *>(vals)[i];
                    },
                    bins);
            };
            // one walk step per plane; r0 holds plane z1-1, r1 plane z1
            walk::Rows3<K> r0, r1;
            int s_cur = fetch(r0, z_first >= 1);  // plane zb-1 (its full barrier already passed)
            for (int z1 = z_first; ok; ++z1) {
                const int s_nxt = fetch(r1, z1 < nz);
                if (!ok) break;
                vals = stages + (size_t)s_cur * STAGE + lane * BWB + off;
                wk.step(r0, r1, z1 > z_first, out_x, emit);
                release(s_cur);
                s_cur = s_nxt;
                r0 = r1;
                if (z1 >= z_last) break;
            }
            release(s_cur);
        }
        if (lane == 0) s_consumed[warp] = (long long)g;
        if (a.h.emitted) {
            const unsigned n = __reduce_add_sync(0xffffffffu, n_emitted);
            if (lane == 0 && n) atomicAdd(a.h.emitted, (unsigned long long)n);
        }
    }

    __syncthreads();
    if (s_abort && tid == 0) {
        // wait (bounded) for copies still in flight before leaving
        long long lo = s_issued;
        for (int w = 0; w < NW; ++w) lo = s_consumed[w] < lo ? s_consumed[w] : lo;
        for (long long q = lo; q < s_issued; ++q) mbar_wait(&full[q % S], (uint32_t)((q / S) & 1));
    }
    __syncthreads();
    if (a.smem_hist)
        for (int i = tid; i < a.h.nbins; i += NTH) {
            int v = 0;
#pragma unroll
            for (int r = 0; r < HREP; ++r) v += hist[r * a.h.nbins + i];
            if (v) atomicAdd(a.h.acc + i, (unsigned long long)(long long)v);
        }
    // The last CTA to finish resets the item counter for the next launch and,
    // when asked, scans the bins: the CTA's adds to acc (ordered before thread
    // 0 by the barrier) are made visible device-wide by its fence before the
    // CTA counts itself finished.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(a.sched + 1, 1u) == gridDim.x - 1;
        if (s_last) {
            a.sched[0] = 0u;
            a.sched[1] = 0u;
            __threadfence();
        }
    }
    if (a.ecc_out) {
        __syncthreads();
        if (s_last) scan_bins<NTH>(a.h.acc, a.ecc_out, a.vcec_out, a.h.nbins, tid);
    }
}

// ----------------------------------------------------------------- 2D kernel
//
// Lanes along x: lane l of a warp holds the window [x0-1, x0+31) with
// x0 = X0 + 30 l, so a warp covers 960 columns; the warp walks rows.  Rows
// come straight from global memory as aligned 32-bit words (coalesced across
// the warp; any pitch and alignment; words that hold no byte of the row are
// not read), with the next row prefetched while the current one is
// processed.  Each voxel pair is compared once: the row pair (y, y+1) in
// three x offsets and the in-row pair, the earlier voxel's wins being the
// negations.  Warps are independent work-list walkers; the CTA only shares
// the privatized histogram.

struct Bs2dArgs {
    const unsigned char *data;
    int64_t nx, ny, pitch;
    int64_t y_begin, y_end;
    int32_t ntx, nyc, ychunk, nitems;
    int32_t smem_hist, range_check;
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
        const int xt = item % a.ntx, yc = item / a.ntx;
        const int64_t yb = a.y_begin + (int64_t)yc * a.ychunk;
        const int64_t ye = yb + a.ychunk < a.y_end ? yb + a.ychunk : a.y_end;
        const int64_t xw = (int64_t)xt * (32 * kOut) + kOut * lane - 1;  // voxel of window bit 0
        const int64_t first = xw * ES;                                    // may be negative at x = 0
        const uint32_t xex = walk::x_exist_mask(xw, a.nx);
        const uint32_t out_x = xex & 0x7ffffffeu;
        // the byte shift of the window inside its aligned words depends on the
        // row's address (pitches need not be multiples of 4)
        auto fetch = [&](int64_t yy, uint32_t *w) -> int {
            if (yy < 0 || yy >= a.ny || !xex) {
#pragma unroll
                for (int i = 0; i <= K; ++i) w[i] = 0;
                return 0;
            }
            return walk::load_row_words<K>(a.data + yy * a.pitch, row_bytes, first, w);
        };
        // values of emitted voxels come from the row just read (cached)
        const walk::Bins bins{a.smem_hist ? my_hist : nullptr, a.h.acc, a.h.lo, a.h.nbins, a.range_check,
                              a.status};
        int64_t y1 = yb;
        auto emit = [&](uint32_t m, const uint32_t *X, const uint32_t *) {
            if (a.h.emitted && m) atomicAdd(a.h.emitted, (unsigned long long)__popc(m));  // diagnostic count
            const unsigned char *row = a.data + (y1 - 1) * a.pitch + xw * ES;
            walk::emit_sparse2d(
                m, X,
                [&](int i) {
                    return ES == 1 ? (int)__ldg(row + i) : (int)__ldg(reinterpret_cast<const unsigned short *>(row) + i);
                },
                bins);
        };
        uint32_t wn[K + 1], P[K];
        int sh = fetch(yb - 1, wn);
        walk::planes_from_words<K>(wn, sh, P);
        walk::Walk2d<K, TOP> wk;
        wk.begin(P, xex);
        sh = fetch(yb, wn);
        for (; y1 <= ye; ++y1) {
            uint32_t B[K];
            walk::planes_from_words<K>(wn, sh, B);
            if (y1 + 1 <= ye) sh = fetch(y1 + 1, wn);  // prefetch the next row
            wk.step(B, y1 < a.ny, y1 - 1 >= 0, y1 - 1 >= yb, out_x, emit);
        }
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
    a.range_check = range_check;
    a.status = status;
    a.ntx = (int32_t)((g.nx + 32 * kOut - 1) / (32 * kOut));
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
    int64_t nyc = (3 * warps_max + a.ntx - 1) / a.ntx;
    // chunks of at least 16 rows (each re-reads one halo row), unless that
    // leaves fewer than four warps per SM: small images walk 4-row chunks
    // (a warp's walk is a chain of dependent row steps)
    const int64_t cap16 = (depth + 15) / 16, cap4 = (depth + 3) / 4;
    const int64_t cap = cap16 * a.ntx >= 4 * (int64_t)num_sms ? cap16 : cap4;
    if (nyc > cap) nyc = cap;
    if (nyc < 1) nyc = 1;
    a.ychunk = (int32_t)((depth + nyc - 1) / nyc);
    a.nyc = (int32_t)((depth + a.ychunk - 1) / a.ychunk);
    const int64_t items = (int64_t)a.ntx * a.nyc;
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

template <typename T, int NW, bool TOP, int HREP>
cudaError_t launch_t(const Geom &g, int64_t zb, int64_t ze, const HistDst &h, bool range_check,
                     unsigned int *status, unsigned int *sched, int num_sms, cudaStream_t s, FusedScan *fs)
{
    using C = Cfg<T>;
    constexpr int BWB = box_bytes(NW, C::ES);
    auto encode = encode_fn();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch_y, (cuuint64_t)g.pitch_z};
    const cuuint32_t box[3] = {(cuuint32_t)(BWB / C::ES), 32u, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = encode(&map, C::ES == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                        const_cast<unsigned char *>(g.data), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorNotSupported;

    Bs3dArgs a{};
    a.sched = sched;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.z_begin = zb;
    a.z_end = ze;
    a.ntx = (int32_t)((g.nx + kOut * NW - 1) / (kOut * NW));
    a.nty = (int32_t)((g.ny + kOut - 1) / kOut);
    a.h = h;
    a.range_check = range_check;
    a.status = status;
    const bool fuse = fs && fs->ecc && zb == 0 && ze == g.nz && h.nbins <= kFusedScanMaxBins;
    a.ecc_out = fuse ? fs->ecc : nullptr;
    a.vcec_out = fuse ? fs->vcec : nullptr;
    const size_t stage_bytes = (size_t)C::S * 32 * BWB + (size_t)C::S * 16;
    a.smem_hist = (size_t)HREP * h.nbins * 4 + stage_bytes <= 160 * 1024;
    const size_t smem = stage_bytes + (a.smem_hist ? (size_t)HREP * h.nbins * 4 : 0);
    auto kern = bs3d_kernel<T, NW, TOP, HREP>;
    static size_t attr_smem = 48 * 1024;  // per instantiation: dynamic smem allowed so far
    static size_t occ_smem = 0;
    static int per_sm = 0;
    if (smem > attr_smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cudaErrorNotSupported;
        }
        attr_smem = smem;
    }
    static bool carveout = false;
    if (!carveout) {  // let the ring stages of several CTAs share an SM
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaGetLastError();
        carveout = true;
    }
    if (occ_smem != smem || per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (NW + 1) * 32, smem);
        if (e != cudaSuccess) return e;
        occ_smem = smem;
    }
    if (per_sm < 1) return cudaErrorNotSupported;
    const int64_t ctas_max = (int64_t)num_sms * per_sm;
    const int64_t cols = (int64_t)a.ntx * a.nty;
    const int64_t depth = ze - zb;
    // z-chunks.  An item costs its planes plus two (the halo plane and the
    // step that emits nothing); CTAs take items dynamically, so the launch
    // costs about (waves of ctas_max items) x (item cost), a partial last
    // wave costing a whole one.  Candidates fill k waves (k = 1, 2, ...);
    // a single wave is charged 10 % more, as nothing then hides a CTA's
    // start-up (ring fill, histogram clear and flush) -- measured.
    int64_t nzc = 1;
    {
        double best = -1.0;
        for (int64_t k = 1; k <= 64; ++k) {
            int64_t n = k * ctas_max / cols;
            if (n < 1) n = 1;
            const int64_t zc = (depth + n - 1) / n;
            n = (depth + zc - 1) / zc;
            if (zc < 8 && k > 1) break;
            const int64_t waves = (cols * n + ctas_max - 1) / ctas_max;
            const double cost = (double)waves * (double)(zc + 2) * (waves == 1 ? 1.1 : 1.0);
            if (best < 0.0 || cost < best) {
                best = cost;
                nzc = n;
            }
        }
    }
    a.zchunk = (int32_t)((depth + nzc - 1) / nzc);
    a.nzc = (int32_t)((depth + a.zchunk - 1) / a.zchunk);
    const int64_t items = cols * a.nzc;
    if (items > 2147483647) return cudaErrorNotSupported;
    a.nitems = (int32_t)items;
    const int64_t ctas = items < ctas_max ? items : ctas_max;
    kern<<<(unsigned)ctas, (NW + 1) * 32, smem, s>>>(map, a);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && fuse) fs->done = true;
    return e;
}

template <int NW, int HREP>
cudaError_t launch_nw(const Geom &g, int64_t zb, int64_t ze, const HistDst &h, int mode, bool rc, unsigned int *st,
                      unsigned int *sched, int sms, cudaStream_t s, FusedScan *fs)
{
    const bool top = mode == ECC_TOPCELL_MIN;
    if (g.esize == 1)
        return top ? launch_t<unsigned char, NW, true, HREP>(g, zb, ze, h, rc, st, sched, sms, s, fs)
                   : launch_t<unsigned char, NW, false, HREP>(g, zb, ze, h, rc, st, sched, sms, s, fs);
    return top ? launch_t<unsigned short, NW, true, HREP>(g, zb, ze, h, rc, st, sched, sms, s, fs)
               : launch_t<unsigned short, NW, false, HREP>(g, zb, ze, h, rc, st, sched, sms, s, fs);
}

}  // namespace

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

// tune_param: 0 = choose by wasted columns; otherwise 10 * (windows per CTA)
// + (shared histogram copies): 61, 62, 42, 31 (the autotuner's candidates).
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
    int tp = tune_param;
    if (tp != 61 && tp != 62 && tp != 42 && tp != 31) {
        // fewest wasted columns; ties to the wider tile
        int64_t best = -1;
        for (int cand : {62, 42, 31}) {
            const int64_t w = kOut * (cand / 10);
            const int64_t waste = (g.nx + w - 1) / w * w - g.nx;
            if (best < 0 || waste < best) {
                best = waste;
                tp = cand;
            }
        }
    }
    switch (tp) {
    case 61: return launch_nw<6, 1>(g, outer_begin, outer_end, h, mode, range_check, status, sched, num_sms, s, fs);
    case 62: return launch_nw<6, 2>(g, outer_begin, outer_end, h, mode, range_check, status, sched, num_sms, s, fs);
    case 42: return launch_nw<4, 2>(g, outer_begin, outer_end, h, mode, range_check, status, sched, num_sms, s, fs);
    default: return launch_nw<3, 1>(g, outer_begin, outer_end, h, mode, range_check, status, sched, num_sms, s, fs);
    }
}

}  // namespace ecc
