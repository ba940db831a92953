// ecc_walk.cuh -- warp-level walkers of the bit-sliced stencil (device only).
//
// Shared pieces of the bit-sliced walkers (ecc_walk2.cuh, ecc_walk3.cuh and
// the 4D walker of ecc_nd.cu): lane shuffles, window existence masks, row
// word loads, the gray-range test, histogram bins, and the slice
// comparisons of the 4D walker.  Windows are 32 voxels of one row held as
// bit planes, overlapping by one voxel on each side, so bits 1..30 are
// outputs and the +-1 shifts along x stay in the register (Sec. 2.3 "Faces
// introduced by a voxel"; Algorithm 1 regrouped per voxel).
//
// A voxel's win over a neighbour that precedes it in memory is the negation
// of that neighbour's win over it (ties go to the lower linear index).
#pragma once

#include <stdint.h>

#include "ecc_bitslice.cuh"
#include "ecc_internal.h"

namespace ecc {
namespace walk {

__device__ __forceinline__ uint32_t from_next_lane(uint32_t v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ uint32_t from_prev_lane(uint32_t v) { return __shfl_up_sync(0xffffffffu, v, 1); }

__device__ __forceinline__ uint32_t shl1(uint32_t x) { return x << 1; }
__device__ __forceinline__ uint32_t shr1(uint32_t x) { return x >> 1; }

// r[x] = m[x + dx]
template <int DX>
__device__ __forceinline__ uint32_t at_offset(uint32_t m)
{
    return DX > 0 ? shr1(m) : (DX < 0 ? shl1(m) : m);
}

// A comparison turned into a win: in the vertex complex a missing neighbour
// means the cell does not exist (no win); in the top-cell complex the voxel
// owns the boundary cell alone (a win) -- the paper's +infinity collar.
template <bool TOP>
__device__ __forceinline__ uint32_t with_exist(uint32_t cmp, uint32_t exist)
{
    return TOP ? (cmp | ~exist) : (cmp & exist);
}

// Voxel a beats voxel b that follows it in memory (a wins ties): the max of
// the two for the vertex complex, the min for the top-cell complex.
template <int K, bool TOP>
__device__ __forceinline__ uint32_t beats_later(const uint32_t *a, const uint32_t *b)
{
    return TOP ? bs::ge<K>(b, a) : bs::ge<K>(a, b);
}

// The last carry step of beats_later for one more plane: folds the
// existence plane (ea of the earlier operand, eb of the later one) into a
// comparison taken over the value planes.
template <bool TOP>
__device__ __forceinline__ uint32_t fold_plane(uint32_t c, uint32_t ea, uint32_t eb)
{
    return TOP ? ((eb & ~ea) | ((eb | ~ea) & c)) : ((ea & ~eb) | ((ea | ~eb) & c));
}

template <int K>
__device__ __forceinline__ void shifted(const uint32_t *a, uint32_t *p, uint32_t *m)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        p[k] = shr1(a[k]);  // bit x holds voxel x+1
        m[k] = shl1(a[k]);  // bit x holds voxel x-1
    }
}

// Bits i of a window starting at voxel xw whose voxel lies in [0, nx).
__device__ __forceinline__ uint32_t x_exist_mask(int64_t xw, int64_t nx)
{
    const int64_t lo_i = -xw, hi_i = nx - xw;
    const int l = lo_i < 0 ? 0 : (lo_i > 32 ? 32 : (int)lo_i);
    const int h = hi_i < 0 ? 0 : (hi_i > 32 ? 32 : (int)hi_i);
    if (h <= l) return 0u;
    return h - l == 32 ? 0xffffffffu : (((1u << (h - l)) - 1u) << l);
}

// Aligned 32-bit words covering bytes [first, first + 4*NW) of a row of
// row_bytes bytes, from the aligned address at or below it; a word that holds
// no byte of the row is not read (0 instead), so no access leaves the row's
// 4-byte-aligned extent.  Returns the bit shift of the window in the words.
template <int NW>
__device__ __forceinline__ int load_row_words(const unsigned char *row, int64_t row_bytes, int64_t first, uint32_t *w)
{
    const uintptr_t start = reinterpret_cast<uintptr_t>(row) + (uintptr_t)first;
    const uintptr_t a0 = start & ~uintptr_t(3);
    const uintptr_t lo = reinterpret_cast<uintptr_t>(row), hi = lo + (uintptr_t)row_bytes;
#pragma unroll
    for (int i = 0; i <= NW; ++i) {
        const uintptr_t ad = a0 + 4 * i;
        w[i] = (ad + 4 > lo && ad < hi) ? __ldg(reinterpret_cast<const uint32_t *>(ad)) : 0u;
    }
    return (int)(start & 3u) * 8;
}

// Bit planes of the window held in aligned words w shifted by sh bits.
template <int K>
__device__ __forceinline__ void planes_from_words(const uint32_t *w, int sh, uint32_t *planes)
{
    constexpr int NW = K;  // 32 voxels of K bits = K words
    uint32_t raw[NW];
    if (sh == 0) {
#pragma unroll
        for (int i = 0; i < NW; ++i) raw[i] = w[i];
    } else {
        // (w[i] >> sh) | (w[i+1] << (32 - sh)) as two multiplies (disjoint bits)
        const uint32_t m = bs::kPow2[32 - sh];
#pragma unroll
        for (int i = 0; i < NW; ++i) raw[i] = w[i + 1] * m + __umulhi(w[i], m);
    }
    if (K == 8)
        bs::transpose_u8(raw, planes);
    else
        bs::transpose_u16(raw, planes);
}

// ------------------------------------------------------------------ gray range

// Mask of voxels with lo <= v <= hi over K value planes, the bounds given as
// their bits (bit k of lo_bits / hi_bits is bit k of the bound): two
// bit-serial comparisons with broadcast planes.
template <int K>
__device__ __forceinline__ uint32_t in_range(const uint32_t *v, uint32_t lo_bits, uint32_t hi_bits)
{
    uint32_t cl = v[0] | ((lo_bits & 1u) ? 0u : ~0u);  // v >= lo
    uint32_t ch = ((hi_bits & 1u) ? ~0u : 0u) | ~v[0];  // hi >= v
#pragma unroll
    for (int k = 1; k < K; ++k) {
        const uint32_t l = ((lo_bits >> k) & 1u) ? ~0u : 0u, h = ((hi_bits >> k) & 1u) ? ~0u : 0u;
        cl = (v[k] & ~l) | ((v[k] | ~l) & cl);
        ch = (h & ~v[k]) | ((h | ~v[k]) & ch);
    }
    return cl & ch;
}

// Does [lo, lo + nbins) leave out values of a K-bit type?  Only then can an
// image value fall outside the range, and only then are voxels checked.
__host__ __device__ inline bool range_is_narrow(int lo, int nbins, int esize)
{
    const long long type_max = esize == 1 ? 255 : 65535;
    return lo > 0 || (long long)lo + nbins - 1 < type_max;
}

// ------------------------------------------------------------------ histogram

// One warp's histogram destination: shared int32 bins (flushed per CTA) or,
// when the gray range does not fit shared memory, the int64 global bins.
struct Bins {
    int *hist;                  // shared bins, or null for global
    unsigned long long *acc;    // global bins
    int lo, nbins, range_check;
    unsigned int *status;
    // bin of value v += k; a value outside [lo, lo + nbins) sets DEV_RANGE
    __device__ __forceinline__ void add(int v, int k) const
    {
        const int bin = v - lo;
        if (range_check && (unsigned)bin >= (unsigned)nbins) {
            atomicOr(status, DEV_RANGE);
            return;
        }
        if (hist)
            atomicAdd(&hist[bin], k);
        else
            atomicAdd(acc + bin, (unsigned long long)(long long)k);
    }
};

// ------------------------------------------------------------------ 4D slices

// Wins between slices X and Y, every voxel of X earlier in memory than
// every voxel of Y (X lies at a smaller w, or the same w and a smaller z):
//   f[dy][dx]: X(y, x) beats Y(y+dy-1, x+dx-1)        (when FWD)
//   r[dy][dx]: Y(y, x) beats X(y+dy-1, x+dx-1)        (when REV)
// Nine comparisons per lane: X(y) against Y(y) (R0), X(y-1) against Y(y)
// (G) and X(y+1) against Y(y) (K2), at the three x offsets; the rest are
// neighbouring lanes' results or the complements of shifted ones.
// Warp-collective.
template <int K, bool TOP, bool FWD, bool REV>
__device__ __forceinline__ void slice_pair(const uint32_t *X, const uint32_t *Y, uint32_t f[3][3], uint32_t r[3][3])
{
    constexpr int KP = K + 1;
    uint32_t Yp[KP], Ym[KP], XD[KP], XU[KP];
    shifted<KP>(Y, Yp, Ym);
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        XD[k] = from_prev_lane(X[k]);
        XU[k] = from_next_lane(X[k]);
    }
    // [d] at bit x: against Y(., x+d-1)
    uint32_t R0[3], G[3], K2[3];
    R0[0] = beats_later<KP, TOP>(X, Ym);
    R0[1] = beats_later<KP, TOP>(X, Y);
    R0[2] = beats_later<KP, TOP>(X, Yp);
    G[0] = beats_later<KP, TOP>(XD, Ym);
    G[1] = beats_later<KP, TOP>(XD, Y);
    G[2] = beats_later<KP, TOP>(XD, Yp);
    K2[0] = beats_later<KP, TOP>(XU, Ym);
    K2[1] = beats_later<KP, TOP>(XU, Y);
    K2[2] = beats_later<KP, TOP>(XU, Yp);
    if (FWD) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            f[0][d] = from_prev_lane(K2[d]);   // lane y-1: X(y) vs Y(y-1)
            f[1][d] = R0[d];
            f[2][d] = from_next_lane(G[d]);    // lane y+1: X(y) vs Y(y+1)
        }
    }
    if (REV) {
        r[0][0] = ~at_offset<-1>(G[2]);
        r[0][1] = ~G[1];
        r[0][2] = ~at_offset<+1>(G[0]);
        r[1][0] = ~at_offset<-1>(R0[2]);
        r[1][1] = ~R0[1];
        r[1][2] = ~at_offset<+1>(R0[0]);
        r[2][0] = ~at_offset<-1>(K2[2]);
        r[2][1] = ~K2[1];
        r[2][2] = ~at_offset<+1>(K2[0]);
    }
}

// Wins of the voxels of slice A over their eight neighbours in the slice:
// a[dy][dx]: A(y, x) beats A(y+dy-1, x+dx-1); a[1][1] = 0.  Warp-collective.
template <int K, bool TOP>
__device__ __forceinline__ void in_slice(const uint32_t *A, uint32_t a[3][3])
{
    constexpr int KP = K + 1;
    uint32_t Ap[KP], Am[KP], U[KP];
    shifted<KP>(A, Ap, Am);
#pragma unroll
    for (int k = 0; k < KP; ++k) U[k] = from_next_lane(A[k]);
    // E[x]: A(y, x-1) vs A(y, x); F[d][x]: A(y, x+1-d) vs A(y+1, x)
    const uint32_t E = beats_later<KP, TOP>(Am, A);
    const uint32_t F0 = beats_later<KP, TOP>(Ap, U);
    const uint32_t F1 = beats_later<KP, TOP>(A, U);
    const uint32_t F2 = beats_later<KP, TOP>(Am, U);
    a[1][0] = ~E;
    a[1][1] = 0u;
    a[1][2] = at_offset<+1>(E);
    a[2][0] = at_offset<-1>(F0);
    a[2][1] = F1;
    a[2][2] = at_offset<+1>(F2);
    a[0][0] = ~from_prev_lane(F2);
    a[0][1] = ~from_prev_lane(F1);
    a[0][2] = ~from_prev_lane(F0);
}

}  // namespace walk
}  // namespace ecc
