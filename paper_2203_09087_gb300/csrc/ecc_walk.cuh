// ecc_walk.cuh -- warp-level walkers of the bit-sliced stencil (device only).
//
// A walker holds one warp's sliding state while it walks an image along its
// slowest axis and, at every step, emits the voxels of the previous row or
// plane whose signed cell count is nonzero (Sec. 2.3 "Faces introduced by a
// voxel"; Algorithm 1 regrouped per voxel).  Windows are 32 voxels of one
// row held as bit planes, overlapping by one voxel on each side, so bits
// 1..30 are outputs and the +-1 shifts along x stay in the register.
//
//   Walk3d: lane l holds row y0-1+l (lanes 0 and 31 are the y halo); the warp
//           walks planes z.  Each step compares planes z and z+1 (9 pairs per
//           voxel) and the in-plane pairs of z+1 (4), sharing the pairs with
//           row y-1 through shuffles, so each neighbour pair is compared once.
//   Walk2d: lanes hold consecutive windows of one row; the warp walks rows.
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

// Emission, per lane: the voxels of mask m (bit i: window element i, value
// val_at(i)) have nonzero signed counts.  In smooth images 0.4 % of voxels
// have one and almost all are +-1, so most lanes emit nothing in a step and
// the others one voxel: each lane adds its first +-1 voxel without a loop,
// and only when some lane has more (or a larger count) does the warp run
// the per-lane loop.  Warp-collective (all lanes call it).
//
// 3D: count = T - 5 from the four bit planes of T (negated for the top-cell
// complex, (-1)^3); T = 6 and T = 4 (+1 and -1) need no bit-plane read.
template <bool TOP, class ValAt>
__device__ __forceinline__ void emit_sparse3d(uint32_t m, const uint32_t *T, ValAt &&val_at, const Bins &b)
{
    const uint32_t c = T[2] & ~T[3] & ~T[0];   // T = 4 or 6
    const uint32_t pm = m & c;
    uint32_t rest = (m & ~c) | (pm & (pm - 1u));
    if (pm) {
        const int i = __ffs(pm) - 1;
        const int k = ((T[1] >> i) & 1u) ? 1 : -1;
        b.add(val_at(i), TOP ? -k : k);
    }
    if (__any_sync(0xffffffffu, rest != 0u)) {
        while (rest) {
            const int i = __ffs(rest) - 1;
            rest &= rest - 1;
            const int k = bs::bits_at<4>(T, i) - 5;
            b.add(val_at(i), TOP ? -k : k);
        }
    }
}

// 2D: count = X[0] + X[1] + 2 X[2] - 3 ((-1)^2 = +1 in both complexes).
template <class ValAt>
__device__ __forceinline__ void emit_sparse2d(uint32_t m, const uint32_t *X, ValAt &&val_at, const Bins &b)
{
    while (m) {
        const int i = __ffs(m) - 1;
        m &= m - 1;
        const int k = (int)((X[0] >> i) & 1u) + (int)((X[1] >> i) & 1u) + 2 * (int)((X[2] >> i) & 1u) - 3;
        b.add(val_at(i), k);
    }
}

// ------------------------------------------------------------------ 3D

// One plane's part of a lane: row y as planes P and row y+1 (the next
// lane's P) as U.  Planes 0..K-1 hold the value; plane K is 1 where the
// voxel does not exist (outside the image), which makes a missing voxel
// compare above every real one, the value 2^K.  That is exactly the
// existence rule of both complexes with no masking: in the vertex complex
// a voxel never beats a missing neighbour (the cell does not exist); in the
// top-cell complex, where the min wins, it always does (the +infinity
// collar).  The one-voxel shifts of P are recomputed where needed rather
// than kept, to save registers.
template <int K>
struct Rows3 {
    uint32_t P[K + 1], U[K + 1];
};

// Fill U of a freshly loaded P (all K + 1 planes).  Warp-collective.
template <int K>
__device__ __forceinline__ void complete_rows(Rows3<K> &r)
{
#pragma unroll
    for (int k = 0; k <= K; ++k) r.U[k] = from_next_lane(r.P[k]);
}

template <int K, bool TOP>
struct Walk3d {
    static constexpr int KP = K + 1;               // value planes + existence plane
    uint32_t wx0, wx2, wyp[3], wym[3], Wm[3][3];   // wins of (z, y) known so far

    __device__ __forceinline__ void begin()
    {
        wx0 = wx2 = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            wyp[d] = wym[d] = 0;
            Wm[0][d] = Wm[1][d] = Wm[2][d] = 0;
        }
    }

    // From plane z (rows a) to plane z+1 (rows b).  When `emit_z`
    // (warp-uniform), calls emit(mask, T, a.P) for plane z: output voxels
    // with a nonzero count, count = T - 5 before the top-cell sign.
    // Warp-collective.
    template <class Emit>
    __device__ __forceinline__ void step(const Rows3<K> &a, const Rows3<K> &b, bool emit_z, uint32_t out_x,
                                         Emit &&emit)
    {
        // Plane z against plane z+1 (z earlier):
        //   R0[d][x] = A[x]  vs B[x+d-1]    (z, y)   vs (z+1, y)
        //   G[d][x]  = D[x]  vs B[x+d-1]    (z, y-1) vs (z+1, y)
        //   Gu[d][x] = A[x]  vs Bu[x+d-1]   (z, y)   vs (z+1, y+1)  (lane y+1's G)
        //   K2[d][x] = Au[x] vs B[x+d-1]    (z, y+1) vs (z+1, y)
        // and the in-plane pairs of plane z+1:
        //   E[x] = B[x-1] vs B[x],  F[d][x] = B[x+1-d] vs Bu[x].
        // With 8 planes every shifted operand is a shift of this lane's new
        // row B: G is taken against D = row y-1 of plane z (from the previous
        // lane) and Gu is the next lane's G.  With 16 planes plane z is
        // shifted instead and G is the previous lane's Gu.
        uint32_t R0[3], G[3], Gu[3], K2[3], E, F[3];
        // value planes only; the existence plane is folded in below where
        // some voxel of the two planes is missing (it is zero elsewhere)
        if constexpr (K == 8) {
            uint32_t Bp[K], Bm[K], D[K];
            shifted<K>(b.P, Bp, Bm);
#pragma unroll
            for (int k = 0; k < K; ++k) D[k] = from_prev_lane(a.P[k]);
            R0[0] = beats_later<K, TOP>(a.P, Bm);
            R0[1] = beats_later<K, TOP>(a.P, b.P);
            R0[2] = beats_later<K, TOP>(a.P, Bp);
            G[0] = beats_later<K, TOP>(D, Bm);
            G[1] = beats_later<K, TOP>(D, b.P);
            G[2] = beats_later<K, TOP>(D, Bp);
            K2[0] = beats_later<K, TOP>(a.U, Bm);
            K2[1] = beats_later<K, TOP>(a.U, b.P);
            K2[2] = beats_later<K, TOP>(a.U, Bp);
            E = beats_later<K, TOP>(Bm, b.P);
            F[0] = beats_later<K, TOP>(Bp, b.U);
            F[1] = beats_later<K, TOP>(b.P, b.U);
            F[2] = beats_later<K, TOP>(Bm, b.U);
        } else {
            // 16 planes: shifting plane z costs less than shuffling the 16
            // planes of row y-1 would; Gu is this lane's own comparison with
            // row y+1 and G the previous lane's
            {
                uint32_t Ap[K], Am[K];
                shifted<K>(a.P, Ap, Am);
                R0[0] = at_offset<-1>(beats_later<K, TOP>(Ap, b.P));   // A[x] vs B[x-1]
                R0[1] = beats_later<K, TOP>(a.P, b.P);
                R0[2] = at_offset<+1>(beats_later<K, TOP>(Am, b.P));   // A[x] vs B[x+1]
                Gu[0] = at_offset<-1>(beats_later<K, TOP>(Ap, b.U));
                Gu[1] = beats_later<K, TOP>(a.P, b.U);
                Gu[2] = at_offset<+1>(beats_later<K, TOP>(Am, b.U));
            }
            uint32_t Bp[K], Bm[K];
            shifted<K>(b.P, Bp, Bm);
            K2[0] = beats_later<K, TOP>(a.U, Bm);
            K2[1] = beats_later<K, TOP>(a.U, b.P);
            K2[2] = beats_later<K, TOP>(a.U, Bp);
            E = beats_later<K, TOP>(Bm, b.P);
            F[0] = beats_later<K, TOP>(Bp, b.U);
            F[1] = beats_later<K, TOP>(b.P, b.U);
            F[2] = beats_later<K, TOP>(Bm, b.U);
        }
        if (__any_sync(0xffffffffu, (a.P[K] | b.P[K]) != 0u)) {
            const uint32_t eB = b.P[K], eBp = shr1(eB), eBm = shl1(eB), eA = a.P[K];
            const uint32_t eAu = a.U[K], eBu = b.U[K];
            R0[0] = fold_plane<TOP>(R0[0], eA, eBm);
            R0[1] = fold_plane<TOP>(R0[1], eA, eB);
            R0[2] = fold_plane<TOP>(R0[2], eA, eBp);
            if constexpr (K == 8) {
                const uint32_t eD = from_prev_lane(eA);
                G[0] = fold_plane<TOP>(G[0], eD, eBm);
                G[1] = fold_plane<TOP>(G[1], eD, eB);
                G[2] = fold_plane<TOP>(G[2], eD, eBp);
            } else {
                Gu[0] = fold_plane<TOP>(Gu[0], eA, shl1(eBu));
                Gu[1] = fold_plane<TOP>(Gu[1], eA, eBu);
                Gu[2] = fold_plane<TOP>(Gu[2], eA, shr1(eBu));
            }
            K2[0] = fold_plane<TOP>(K2[0], eAu, eBm);
            K2[1] = fold_plane<TOP>(K2[1], eAu, eB);
            K2[2] = fold_plane<TOP>(K2[2], eAu, eBp);
            E = fold_plane<TOP>(E, eBm, eB);
            F[0] = fold_plane<TOP>(F[0], eBp, eBu);
            F[1] = fold_plane<TOP>(F[1], eB, eBu);
            F[2] = fold_plane<TOP>(F[2], eBm, eBu);
        }
        uint32_t K2_dn[3], F_dn[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if constexpr (K == 8)
                Gu[d] = from_next_lane(G[d]);   // lane y+1's G: (z, y) vs (z+1, y+1)
            else
                G[d] = from_prev_lane(Gu[d]);   // lane y-1's Gu: (z, y-1) vs (z+1, y)
            K2_dn[d] = from_prev_lane(K2[d]);   // lane y-1's K2: (z, y) vs (z+1, y-1)
            F_dn[d] = from_prev_lane(F[d]);
        }
        if (emit_z) {
            uint32_t w[3][3][3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                w[2][1][d] = R0[d];
                w[2][2][d] = Gu[d];
                w[2][0][d] = K2_dn[d];
            }
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) w[0][dy][dx] = Wm[dy][dx];
            w[1][1][0] = wx0;
            w[1][1][1] = 0;
            w[1][1][2] = wx2;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                w[1][0][dx] = wym[dx];
                w[1][2][dx] = wyp[dx];
            }
            uint32_t T[4];
            const uint32_t m = bs::kappa3d(w, T) & out_x;
            emit(m, T, a.P);
        }
        // wins of (z+1, y) over plane z (an earlier neighbour wins ties)
        Wm[1][0] = ~at_offset<-1>(R0[2]);
        Wm[1][1] = ~R0[1];
        Wm[1][2] = ~at_offset<+1>(R0[0]);
        Wm[2][0] = ~at_offset<-1>(K2[2]);
        Wm[2][1] = ~K2[1];
        Wm[2][2] = ~at_offset<+1>(K2[0]);
        Wm[0][0] = ~at_offset<-1>(G[2]);
        Wm[0][1] = ~G[1];
        Wm[0][2] = ~at_offset<+1>(G[0]);
        // in-plane wins of (z+1, y)
        wx2 = at_offset<+1>(E);
        wx0 = ~E;
        wyp[0] = at_offset<-1>(F[0]);
        wyp[1] = F[1];
        wyp[2] = at_offset<+1>(F[2]);
        wym[0] = ~F_dn[2];
        wym[1] = ~F_dn[1];
        wym[2] = ~F_dn[0];
    }
};

// ------------------------------------------------------------------ 2D

template <int K, bool TOP>
struct Walk2d {
    uint32_t A[K];                 // planes of row y
    uint32_t wx0, wx2, wym[3];     // wins of row y known so far
    uint32_t ex_x[3];

    __device__ __forceinline__ void begin(const uint32_t *P, uint32_t xex)
    {
        ex_x[0] = xex << 1;
        ex_x[1] = 0xffffffffu;
        ex_x[2] = xex >> 1;
#pragma unroll
        for (int k = 0; k < K; ++k) A[k] = P[k];
        wx0 = wx2 = 0;
        wym[0] = wym[1] = wym[2] = 0;
    }

    // Advance to row y+1 (window B).  yp: row y+1 exists; y_ok: row y exists.
    // When emit_y, calls emit(mask, X, A) for row y with count = X0 + X1 + 2 X2 - 3.
    template <class Emit>
    __device__ __forceinline__ void step(const uint32_t *B, bool yp, bool y_ok, bool emit_y, uint32_t out_x,
                                         Emit &&emit)
    {
        uint32_t H[3], E;
        {
            uint32_t Ap[K], Am[K], Bp[K], Bm[K];
            shifted<K>(A, Ap, Am);
            shifted<K>(B, Bp, Bm);
            H[0] = beats_later<K, TOP>(Ap, B);  // [x]: A[x+1] vs B[x]
            H[1] = beats_later<K, TOP>(A, B);
            H[2] = beats_later<K, TOP>(Am, B);  // [x]: A[x-1] vs B[x]
            E = beats_later<K, TOP>(Bm, B);     // [x]: B[x-1] vs B[x]
        }
        const uint32_t ey_p = yp ? 0xffffffffu : 0u;
        const uint32_t ey_m1 = y_ok ? 0xffffffffu : 0u;
        if (emit_y) {
            uint32_t w[3][3];
            w[0][0] = wym[0];
            w[0][1] = wym[1];
            w[0][2] = wym[2];
            w[1][0] = wx0;
            w[1][1] = 0;
            w[1][2] = wx2;
            w[2][0] = with_exist<TOP>(at_offset<-1>(H[0]), ey_p & ex_x[0]);
            w[2][1] = with_exist<TOP>(H[1], ey_p);
            w[2][2] = with_exist<TOP>(at_offset<+1>(H[2]), ey_p & ex_x[2]);
            uint32_t X[3];
            const uint32_t m = bs::kappa2d(w, X) & out_x;
            emit(m, X, A);
        }
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) wym[dx] = with_exist<TOP>(~H[2 - dx], ey_m1 & ex_x[dx]);
        wx2 = with_exist<TOP>(at_offset<+1>(E), ex_x[2]);
        wx0 = with_exist<TOP>(~E, ex_x[0]);
#pragma unroll
        for (int k = 0; k < K; ++k) A[k] = B[k];
    }
};

// ------------------------------------------------------------------ 4D
//
// Slices: a 4D image is a stack of 2D (y, x) slices indexed by (w, z); a
// warp holds a slice as lane-packed rows (lane l: row y0-1+l, planes 0..K-1
// the value, plane K set where the voxel is missing).  Comparisons take the
// existence plane as the most significant bit (a missing voxel is 2^K).

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
