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
//    neighbour directions is compared once per voxel pair: a lane compares
//    its rows (z,y), (z,y+1) against (z+1,y), (z+1,y+1) and the in-plane
//    pairs, and receives the pairs it shares with row y-1 by warp shuffles.
//    A voxel's wins over earlier neighbours are the negations of those
//    neighbours' comparisons (ties go to the lower linear index).
//  * TMA ring.  One elected thread streams one tile plane per step
//    (cp.async.bulk.tensor, mbarrier completion) into a ring of stages; the
//    box starts 16-byte aligned and is an odd number of 16-byte units wide so
//    the per-lane 16-byte shared loads are bank-conflict free.  The
//    boundary is handled by existence masks, never by the zero fill.
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
    int64_t nx, ny, nz;
    int64_t z_begin, z_end;  // outer range of output planes
    int32_t ntx, nty, nzc;   // tiles along x, y and z-chunks
    int32_t zchunk;
    int32_t nitems;
    int32_t smem_hist;
    int32_t range_check;
    HistDst h;
    unsigned int *status;
};

// ----------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait: false after kSpinLimitNs without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > kSpinLimitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t shfl_from_next(uint32_t v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ uint32_t shfl_from_prev(uint32_t v) { return __shfl_up_sync(0xffffffffu, v, 1); }

// r[x] = m[x + dx]
template <int DX>
__device__ __forceinline__ uint32_t at_offset(uint32_t m)
{
    return DX > 0 ? (m >> 1) : (DX < 0 ? (m << 1) : m);
}

// win mask from a comparison and the neighbour's existence: in the vertex
// complex a missing neighbour means the cell does not exist (no win); in the
// top-cell complex the voxel alone owns it (win) -- the +infinity collar.
template <bool TOP>
__device__ __forceinline__ uint32_t with_exist(uint32_t cmp, uint32_t exist)
{
    return TOP ? (cmp | ~exist) : (cmp & exist);
}

// a beats b, b later in linear order (ties go to a).
template <int K, bool TOP>
__device__ __forceinline__ uint32_t beats_later(const uint32_t *a, const uint32_t *b)
{
    return TOP ? bs::ge<K>(b, a) : bs::ge<K>(a, b);
}

template <int K>
__device__ __forceinline__ void shifted(const uint32_t *a, uint32_t *p, uint32_t *m)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        p[k] = a[k] >> 1;  // bit x holds voxel x+1
        m[k] = a[k] << 1;  // bit x holds voxel x-1
    }
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
    // the word offset is uniform across the warp (all lanes read the same columns)
    switch (sh >> 2) {
#define ECC_WIN(W)                                                                     \
    case W:                                                                            \
        _Pragma("unroll") for (int i = 0; i < C::WORDS; ++i) r[i] =                    \
            __funnelshift_r(v[i + W], v[i + W + 1], wsh);                              \
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

template <typename T, int NW, bool TOP, int HREP>
__global__ void __launch_bounds__(NW * 32) bs3d_kernel(const __grid_constant__ CUtensorMap tmap, const Bs3dArgs a)
{
    using C = Cfg<T>;
    constexpr int K = C::K, S = C::S, ES = C::ES;
    constexpr int BWB = box_bytes(NW, ES);
    constexpr int STAGE = 32 * BWB;
    constexpr int NTH = NW * 32;
    constexpr int ALIGN_EL = 16 / ES;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *stages = smem;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S * STAGE);
    int *hist = reinterpret_cast<int *>(bar + S);
    __shared__ int s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (a.smem_hist)
        for (int i = tid; i < HREP * a.h.nbins; i += NTH) hist[i] = 0;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();
    int *my_hist = hist + (warp % HREP) * a.h.nbins;

    // -------------------------------------------------------------- producer
    // Steps are the tile planes of this CTA's items in order; item i covers
    // output planes [zb, ze) and loads planes zb-1 .. ze.
    auto decode = [&](int item, int &xt, int &yt, int64_t &zb, int64_t &ze) {
        xt = item % a.ntx;
        const int r = item / a.ntx;
        yt = r % a.nty;
        const int zc = r / a.nty;
        zb = a.z_begin + (int64_t)zc * a.zchunk;
        ze = zb + a.zchunk < a.z_end ? zb + a.zchunk : a.z_end;
    };
    int p_item = blockIdx.x;
    int64_t p_j = 0, p_g = 0;
    auto issue_one = [&]() {
        if (p_item >= a.nitems) return;
        int xt, yt;
        int64_t zb, ze;
        decode(p_item, xt, yt, zb, ze);
        const int64_t X0 = (int64_t)xt * (kOut * NW);
        const int64_t xm = X0 - 1;
        const int64_t bx = (xm >= 0 ? xm / ALIGN_EL : -((-xm + ALIGN_EL - 1) / ALIGN_EL)) * ALIGN_EL;
        const int64_t Y0 = (int64_t)yt * kOut - 1;
        const int64_t z = zb - 1 + p_j;
        const int s = (int)(p_g % S);
        mbar_expect_tx(&bar[s], STAGE);
        tma_load_3d(stages + (size_t)s * STAGE, &tmap, (int)bx, (int)Y0, (int)z, &bar[s]);
        ++p_g;
        if (++p_j == ze - zb + 2) {
            p_j = 0;
            p_item += gridDim.x;
        }
    };
    if (tid == 0)
        for (int i = 0; i < S; ++i) issue_one();

    // -------------------------------------------------------------- consumer
    int64_t g = 0;
    bool aborted = false;
    auto end_step = [&]() {
        __syncthreads();  // every warp is done with step g-1's stage
        if (s_abort) aborted = true;
        if (tid == 0 && g >= 1 && !aborted) issue_one();
        ++g;
    };
    auto wait_stage = [&]() -> const unsigned char * {
        const int s = (int)(g % S);
        if (!mbar_wait(&bar[s], (uint32_t)((g / S) & 1))) {
            if (lane == 0) {
                atomicOr(a.status, DEV_TIMEOUT);
                atomicExch(&s_abort, 1);
            }
            return nullptr;
        }
        return stages + (size_t)s * STAGE;
    };

    for (int item = blockIdx.x; item < a.nitems && !aborted; item += gridDim.x) {
        int xt, yt;
        int64_t zb, ze;
        decode(item, xt, yt, zb, ze);
        const int64_t X0 = (int64_t)xt * (kOut * NW);
        const int64_t xm = X0 - 1;
        const int64_t bx = (xm >= 0 ? xm / ALIGN_EL : -((-xm + ALIGN_EL - 1) / ALIGN_EL)) * ALIGN_EL;
        const int64_t y = (int64_t)yt * kOut - 1 + lane;
        const int64_t xw = X0 + kOut * warp - 1;  // voxel of window bit 0
        const int off = (int)((xw - bx) * ES);

        // x existence of each window bit's voxel, and of its +-1 neighbours
        uint32_t xex = 0;
        {
            const int64_t lo_i = -xw, hi_i = a.nx - xw;  // bits i with 0 <= xw+i < nx
            const int l = lo_i < 0 ? 0 : (lo_i > 32 ? 32 : (int)lo_i);
            const int h = hi_i < 0 ? 0 : (hi_i > 32 ? 32 : (int)hi_i);
            if (h > l) xex = (h - l == 32 ? 0xffffffffu : (((1u << (h - l)) - 1u) << l));
        }
        const uint32_t ex_p = xex >> 1, ex_m = xex << 1;  // neighbour at x+1 / x-1 exists
        const uint32_t ex_x[3] = {ex_m, 0xffffffffu, ex_p};
        const bool lane_out = lane >= 1 && lane <= kOut && y < a.ny;
        const uint32_t out_x = xex & 0x7ffffffeu;
        const uint32_t ey_m = (y - 1 >= 0 && y - 1 < a.ny) ? 0xffffffffu : 0u;
        const uint32_t ey_p = (y + 1 >= 0 && y + 1 < a.ny) ? 0xffffffffu : 0u;
        const uint32_t ey[3] = {ey_m, 0xffffffffu, ey_p};

        uint32_t A[K], Au[K];
        uint32_t wx[3] = {0, 0, 0}, wyp[3] = {0, 0, 0}, wym[3] = {0, 0, 0}, Wm[3][3] = {};
        // prologue: plane zb-1
        {
            const unsigned char *st = wait_stage();
            if (st) {
                load_window<T>(st + lane * BWB, off, A);
#pragma unroll
                for (int k = 0; k < K; ++k) Au[k] = shfl_from_next(A[k]);
            }
            end_step();
        }
        for (int64_t z1 = zb; z1 <= ze && !aborted; ++z1) {
            const unsigned char *st = wait_stage();
            if (st) {
                const unsigned char *st_prev = stages + (size_t)((g - 1) % S) * STAGE;
                uint32_t B[K], Bu[K];
                load_window<T>(st + lane * BWB, off, B);
#pragma unroll
                for (int k = 0; k < K; ++k) Bu[k] = shfl_from_next(B[k]);

                // inter-plane comparisons, (z, .) earlier than (z+1, .)
                uint32_t H0[3], Hp[3], Kp[3];
                {
                    uint32_t Ap[K], Am[K];
                    shifted<K>(A, Ap, Am);
                    H0[0] = beats_later<K, TOP>(Ap, B);  // [x] = A[x+1] vs B[x]
                    H0[1] = beats_later<K, TOP>(A, B);
                    H0[2] = beats_later<K, TOP>(Am, B);  // [x] = A[x-1] vs B[x]
                    Hp[0] = beats_later<K, TOP>(Ap, Bu);
                    Hp[1] = beats_later<K, TOP>(A, Bu);
                    Hp[2] = beats_later<K, TOP>(Am, Bu);
                    uint32_t Aup[K], Aum[K];
                    shifted<K>(Au, Aup, Aum);
                    Kp[0] = beats_later<K, TOP>(Aup, B);
                    Kp[1] = beats_later<K, TOP>(Au, B);
                    Kp[2] = beats_later<K, TOP>(Aum, B);
                }
                uint32_t Hp_dn[3], Kp_dn[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    Hp_dn[d] = shfl_from_prev(Hp[d]);
                    Kp_dn[d] = shfl_from_prev(Kp[d]);
                }
                // in-plane comparisons of plane z+1
                uint32_t E, F[3], F_dn[3];
                {
                    uint32_t Bp[K], Bm[K];
                    shifted<K>(B, Bp, Bm);
                    E = beats_later<K, TOP>(Bm, B);       // [x] = B[x-1] vs B[x]
                    F[0] = beats_later<K, TOP>(Bp, Bu);   // [x] = B[x+1] vs Bu[x]
                    F[1] = beats_later<K, TOP>(B, Bu);
                    F[2] = beats_later<K, TOP>(Bm, Bu);   // [x] = B[x-1] vs Bu[x]
                }
#pragma unroll
                for (int d = 0; d < 3; ++d) F_dn[d] = shfl_from_prev(F[d]);

                const int64_t z = z1 - 1;
                const uint32_t ez_p = z1 < a.nz ? 0xffffffffu : 0u;   // plane z+1 exists
                const uint32_t ez_m1 = z >= 0 ? 0xffffffffu : 0u;     // plane z exists (for z+1's wins)

                // wins of (z, y, x) over plane z+1: [dy][dx]
                uint32_t Wp[3][3];
                Wp[1][0] = at_offset<-1>(H0[0]);
                Wp[1][1] = H0[1];
                Wp[1][2] = at_offset<+1>(H0[2]);
                Wp[2][0] = at_offset<-1>(Hp[0]);
                Wp[2][1] = Hp[1];
                Wp[2][2] = at_offset<+1>(Hp[2]);
                Wp[0][0] = at_offset<-1>(Kp_dn[0]);
                Wp[0][1] = Kp_dn[1];
                Wp[0][2] = at_offset<+1>(Kp_dn[2]);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) Wp[dy][dx] = with_exist<TOP>(Wp[dy][dx], ez_p & ey[dy] & ex_x[dx]);

                if (z >= zb && lane_out) {
                    uint32_t w[3][3][3];
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            w[0][dy][dx] = Wm[dy][dx];
                            w[2][dy][dx] = Wp[dy][dx];
                        }
                    w[1][1][0] = wx[0];
                    w[1][1][2] = wx[2];
                    w[1][1][1] = 0;
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        w[1][0][dx] = wym[dx];
                        w[1][2][dx] = wyp[dx];
                    }
                    uint32_t Sq[4], Nc[4];
                    uint32_t m = bs::kappa3d(w, Sq, Nc) & out_x;
                    const unsigned char *vrow = st_prev + lane * BWB + off;
                    while (m) {
                        const int i = __ffs(m) - 1;
                        m &= m - 1;
                        int kap = 1 + bs::bits_at<4>(Sq, i) - bs::bits_at<4>(Nc, i);
                        if (TOP) kap = -kap;  // (-1)^d, d = 3
                        const int v = ES == 1 ? (int)vrow[i] : (int)*reinterpret_cast<const unsigned short *>(vrow + 2 * i);
                        const int bin = v - a.h.lo;
                        if (a.range_check && (unsigned)bin >= (unsigned)a.h.nbins) {
                            atomicOr(a.status, DEV_RANGE);
                            continue;
                        }
                        if (a.smem_hist)
                            atomicAdd(&my_hist[bin], kap);
                        else
                            atomicAdd(a.h.acc + bin, (unsigned long long)(long long)kap);
                    }
                }

                // wins of (z+1, y, x) over plane z, kept for the next step
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    // neighbour (z, y+dy, x+dx) is earlier: win = not (it beats us)
                    Wm[1][dx] = with_exist<TOP>(~H0[2 - dx], ez_m1 & ey[1] & ex_x[dx]);
                    Wm[2][dx] = with_exist<TOP>(~Kp[2 - dx], ez_m1 & ey[2] & ex_x[dx]);
                    Wm[0][dx] = with_exist<TOP>(~Hp_dn[2 - dx], ez_m1 & ey[0] & ex_x[dx]);
                }
                // in-plane wins of (z+1, y, x)
                wx[2] = with_exist<TOP>(at_offset<+1>(E), ex_p);
                wx[0] = with_exist<TOP>(~E, ex_m);
                wyp[0] = with_exist<TOP>(at_offset<-1>(F[0]), ey_p & ex_m);
                wyp[1] = with_exist<TOP>(F[1], ey_p);
                wyp[2] = with_exist<TOP>(at_offset<+1>(F[2]), ey_p & ex_p);
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) wym[dx] = with_exist<TOP>(~F_dn[2 - dx], ey_m & ex_x[dx]);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    A[k] = B[k];
                    Au[k] = Bu[k];
                }
            }
            end_step();
        }
    }

    if (aborted) {
        // wait (bounded) for the copies still in flight before leaving
        if (tid == 0)
            for (int64_t q = g; q < p_g; ++q) mbar_wait(&bar[q % S], (uint32_t)((q / S) & 1));
        __syncthreads();
    }
    __syncthreads();
    if (a.smem_hist)
        for (int i = tid; i < a.h.nbins; i += NTH) {
            int v = 0;
#pragma unroll
            for (int r = 0; r < HREP; ++r) v += hist[r * a.h.nbins + i];
            if (v) atomicAdd(a.h.acc + i, (unsigned long long)(long long)v);
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
};

constexpr int kWarps2d = 4;

template <typename T>
__device__ __forceinline__ void load_row_words(const unsigned char *row, int64_t row_bytes, int64_t first_byte,
                                               uint32_t *w)
{
    // words covering bytes [first_byte, first_byte + 32*ES) of the row, from
    // the 4-byte aligned address at or below it; 0 where no row byte lies
    using C = Cfg<T>;
    const uintptr_t start = reinterpret_cast<uintptr_t>(row) + first_byte;
    const uintptr_t a0 = start & ~uintptr_t(3);
    const uintptr_t lo = reinterpret_cast<uintptr_t>(row), hi = lo + row_bytes;
#pragma unroll
    for (int i = 0; i <= C::WORDS; ++i) {
        const uintptr_t ad = a0 + 4 * i;
        w[i] = (ad + 4 > lo && ad < hi) ? __ldg(reinterpret_cast<const uint32_t *>(ad)) : 0u;
    }
}

template <typename T>
__device__ __forceinline__ void window_from_words(const uint32_t *w, int sh, uint32_t *planes)
{
    using C = Cfg<T>;
    uint32_t raw[C::WORDS];
#pragma unroll
    for (int i = 0; i < C::WORDS; ++i) raw[i] = __funnelshift_r(w[i], w[i + 1], sh);
    if (C::ES == 1)
        bs::transpose_u8(raw, planes);
    else
        bs::transpose_u16(raw, planes);
}

template <typename T, bool TOP, int HREP>
__global__ void __launch_bounds__(kWarps2d * 32) bs2d_kernel(const Bs2dArgs a)
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
        uint32_t xex = 0;
        {
            const int64_t lo_i = -xw, hi_i = a.nx - xw;
            const int l = lo_i < 0 ? 0 : (lo_i > 32 ? 32 : (int)lo_i);
            const int h = hi_i < 0 ? 0 : (hi_i > 32 ? 32 : (int)hi_i);
            if (h > l) xex = (h - l == 32 ? 0xffffffffu : (((1u << (h - l)) - 1u) << l));
        }
        const uint32_t ex_p = xex >> 1, ex_m = xex << 1;
        const uint32_t ex_x[3] = {ex_m, 0xffffffffu, ex_p};
        const uint32_t out_x = xex & 0x7ffffffeu;
        if (!xex) continue;  // lane past the right edge: nothing to read or emit

        // the byte shift of the window inside its aligned words depends on the
        // row's address (pitches need not be multiples of 4)
        auto fetch = [&](int64_t yy, uint32_t *w, int &sh) {
            if (yy < 0 || yy >= a.ny) {
#pragma unroll
                for (int i = 0; i <= C::WORDS; ++i) w[i] = 0;
                sh = 0;
            } else {
                const unsigned char *row = a.data + yy * a.pitch;
                sh = (int)((reinterpret_cast<uintptr_t>(row) + (uintptr_t)first) & 3u) * 8;
                load_row_words<T>(row, row_bytes, first, w);
            }
        };
        uint32_t wnext[C::WORDS + 1], A[K];
        int sh_next;
        {
            uint32_t w0[C::WORDS + 1];
            int sh0;
            fetch(yb - 1, w0, sh0);
            window_from_words<T>(w0, sh0, A);
        }
        fetch(yb, wnext, sh_next);
        uint32_t wx[3] = {0, 0, 0}, wym[3] = {0, 0, 0};
        for (int64_t y1 = yb; y1 <= ye; ++y1) {
            uint32_t B[K];
            window_from_words<T>(wnext, sh_next, B);
            if (y1 + 1 <= ye) fetch(y1 + 1, wnext, sh_next);  // prefetch the next row
            uint32_t H[3], E;
            {
                uint32_t Ap[K], Am[K], Bp[K], Bm[K];
                shifted<K>(A, Ap, Am);
                shifted<K>(B, Bp, Bm);
                H[0] = beats_later<K, TOP>(Ap, B);  // [x] = A[x+1] vs B[x]
                H[1] = beats_later<K, TOP>(A, B);
                H[2] = beats_later<K, TOP>(Am, B);  // [x] = A[x-1] vs B[x]
                E = beats_later<K, TOP>(Bm, B);     // [x] = B[x-1] vs B[x]
            }
            const int64_t y = y1 - 1;
            const uint32_t ey_p = y1 < a.ny ? 0xffffffffu : 0u;
            const uint32_t ey_m1 = y >= 0 ? 0xffffffffu : 0u;
            if (y >= yb) {
                uint32_t w[3][3];
                w[0][0] = wym[0];
                w[0][1] = wym[1];
                w[0][2] = wym[2];
                w[1][0] = wx[0];
                w[1][1] = 0;
                w[1][2] = wx[2];
                w[2][0] = with_exist<TOP>(at_offset<-1>(H[0]), ey_p & ex_m);
                w[2][1] = with_exist<TOP>(H[1], ey_p);
                w[2][2] = with_exist<TOP>(at_offset<+1>(H[2]), ey_p & ex_p);
                uint32_t F[3], Q[3];
                uint32_t m = bs::kappa2d(w, F, Q) & out_x;
                while (m) {
                    const int i = __ffs(m) - 1;
                    m &= m - 1;
                    const int kap = 1 + bs::bits_at<3>(Q, i) - bs::bits_at<3>(F, i);  // (-1)^2 = +1
                    const int v = bs::bits_at<K>(A, i);  // the voxel's gray level from its bit planes
                    const int bin = v - a.h.lo;
                    if (a.range_check && (unsigned)bin >= (unsigned)a.h.nbins) {
                        atomicOr(a.status, DEV_RANGE);
                        continue;
                    }
                    if (a.smem_hist)
                        atomicAdd(&my_hist[bin], kap);
                    else
                        atomicAdd(a.h.acc + bin, (unsigned long long)(long long)kap);
                }
            }
            // wins of row y+1 for the next step
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) wym[dx] = with_exist<TOP>(~H[2 - dx], ey_m1 & ex_x[dx]);
            wx[2] = with_exist<TOP>(at_offset<+1>(E), ex_p);
            wx[0] = with_exist<TOP>(~E, ex_m);
#pragma unroll
            for (int k = 0; k < K; ++k) A[k] = B[k];
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
}

template <typename T, bool TOP>
cudaError_t launch_2d_t(const Geom &g, int64_t yb, int64_t ye, const HistDst &h, bool range_check,
                        unsigned int *status, int num_sms, cudaStream_t s)
{
    constexpr int HREP = 2;
    Bs2dArgs a{};
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
    if (nyc > (depth + 15) / 16) nyc = (depth + 15) / 16;
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
    return cudaGetLastError();
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
                     unsigned int *status, int num_sms, cudaStream_t s)
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
    const size_t stage_bytes = (size_t)C::S * 32 * BWB + (size_t)C::S * 8;
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
    if (occ_smem != smem || per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, smem);
        if (e != cudaSuccess) return e;
        occ_smem = smem;
    }
    if (per_sm < 1) return cudaErrorNotSupported;
    const int64_t ctas_max = (int64_t)num_sms * per_sm;
    const int64_t cols = (int64_t)a.ntx * a.nty;
    const int64_t depth = ze - zb;
    // z-chunks: enough items for about three per CTA, each chunk >= 8 planes
    int64_t nzc = (3 * ctas_max + cols - 1) / cols;
    if (nzc > (depth + 7) / 8) nzc = (depth + 7) / 8;
    if (nzc < 1) nzc = 1;
    a.zchunk = (int32_t)((depth + nzc - 1) / nzc);
    a.nzc = (int32_t)((depth + a.zchunk - 1) / a.zchunk);
    const int64_t items = cols * a.nzc;
    if (items > 2147483647) return cudaErrorNotSupported;
    a.nitems = (int32_t)items;
    const int64_t ctas = items < ctas_max ? items : ctas_max;
    kern<<<(unsigned)ctas, NW * 32, smem, s>>>(map, a);
    return cudaGetLastError();
}

template <int NW, int HREP>
cudaError_t launch_nw(const Geom &g, int64_t zb, int64_t ze, const HistDst &h, int mode, bool rc, unsigned int *st,
                      int sms, cudaStream_t s)
{
    const bool top = mode == ECC_TOPCELL_MIN;
    if (g.esize == 1)
        return top ? launch_t<unsigned char, NW, true, HREP>(g, zb, ze, h, rc, st, sms, s)
                   : launch_t<unsigned char, NW, false, HREP>(g, zb, ze, h, rc, st, sms, s);
    return top ? launch_t<unsigned short, NW, true, HREP>(g, zb, ze, h, rc, st, sms, s)
               : launch_t<unsigned short, NW, false, HREP>(g, zb, ze, h, rc, st, sms, s);
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

// tune_param: 0 = choose by x-waste; otherwise the windows per CTA (3, 4 or 6).
cudaError_t launch_bitslice(const Geom &g, int64_t outer_begin, int64_t outer_end, const HistDst &h, int mode,
                            bool range_check, unsigned int *status, int num_sms, int tune_param, cudaStream_t s)
{
    if (outer_end <= outer_begin) return cudaSuccess;
    if (!bitslice_supported(g)) return cudaErrorNotSupported;
    if (g.ndim == 2) {
        const bool top = mode == ECC_TOPCELL_MIN;
        if (g.esize == 1)
            return top ? launch_2d_t<unsigned char, true>(g, outer_begin, outer_end, h, range_check, status, num_sms, s)
                       : launch_2d_t<unsigned char, false>(g, outer_begin, outer_end, h, range_check, status, num_sms, s);
        return top ? launch_2d_t<unsigned short, true>(g, outer_begin, outer_end, h, range_check, status, num_sms, s)
                   : launch_2d_t<unsigned short, false>(g, outer_begin, outer_end, h, range_check, status, num_sms, s);
    }
    int nw = tune_param;
    if (nw != 3 && nw != 4 && nw != 6) {
        // fewest wasted columns; ties to the wider tile
        int64_t best = -1;
        for (int cand : {6, 4, 3}) {
            const int64_t w = kOut * cand;
            const int64_t waste = (g.nx + w - 1) / w * w - g.nx;
            if (best < 0 || waste < best) {
                best = waste;
                nw = cand;
            }
        }
    }
    if (nw == 6) return launch_nw<6, 2>(g, outer_begin, outer_end, h, mode, range_check, status, num_sms, s);
    if (nw == 4) return launch_nw<4, 2>(g, outer_begin, outer_end, h, mode, range_check, status, num_sms, s);
    return launch_nw<3, 1>(g, outer_begin, outer_end, h, mode, range_check, status, num_sms, s);
}

}  // namespace ecc
