// ecc_walk3.cuh -- the 3D bit-sliced walker of the single-volume stencil
// (device only).
//
// The cell logic of Sec. 2.3 "Faces introduced by a voxel" (Algorithm 1
// regrouped per voxel; the 26 signed cell terms as 12 chain bits,
// ecc_bitslice.cuh): each step compares plane z with plane z+1 (9 pairs per
// voxel) and the in-plane pairs of z+1 (4), sharing the pairs with row y-1
// through shuffles, so each neighbour pair is compared once.  Arranged for
// the integer ALU pipe, which bounds this kernel on GB300:
//
//  * every one-bit shift (the x +-1 operands, the walk state) and every shift
//    of the bit-plane transpose is a multiply by a power of two held in a
//    kernel argument (IMAD / IMAD.HI on the FMA pipe), so the ALU pipe only
//    runs the logic operations of the comparisons and the cell count;
//  * the walk state is stored un-negated and negated where it enters the
//    cell count, so the negations fold into the three-input logic
//    operations there;
//  * the comparisons run plane-major with each plane's shifted and shuffled
//    operands made just before use, which keeps the register footprint small
//    enough for 4-5 warps per scheduler.
//
// Lane l holds row y0-1+l of the walked plane (lanes 0 and 31 are the y
// halo); bit i of a plane is voxel xw+i of that row (bits 0 and 31 are the x
// halo).  Planes 0..K-1 hold the value, plane K is 1 where the voxel is
// outside the image (it then compares as 2^K, which is the existence rule
// of both complexes).
#pragma once

#include <stdint.h>

#include "ecc_bitlogic.cuh"
#include "ecc_bitslice.cuh"
#include "ecc_walk.cuh"

namespace ecc {
namespace walk3 {

// One row window of a plane: its K + 1 bit planes.
template <int K>
struct Row {
    uint32_t P[K + 1];
};

// Emission of the voxels in m (bit i: value val_at(i)); the count is T - 5
// (negated for the top-cell complex).  In smooth fields few voxels have a
// nonzero count and almost all are +-1 (T = 6 or 4): each lane adds its
// lowest such voxel in straight-line code (the value read unconditionally
// from a valid index, only the add predicated), and the warp runs the
// general loop only when some lane has more, or a larger count.
// Warp-collective.
template <bool TOP, class ValAt, class Add, class AddIf>
__device__ __forceinline__ void emit3(uint32_t m, const uint32_t *T, ValAt &&val_at, Add &&add, AddIf &&add_if)
{
    const uint32_t c = lop3<0x10u>(T[2], T[3], T[0]);  // T[2] & ~T[3] & ~T[0]: T = 4 or 6
    const uint32_t pm = m & c;
    const uint32_t first = pm & (0u - pm);              // lowest +-1 voxel, 0 if none
    uint32_t rest = lop3<0xBAu>(m, c, pm ^ first);      // (m & ~c) | (pm ^ first)
    const int i = 31 - __clz(first | 1u);
    const int v = val_at(i);
    const int k = (T[1] & first) ? 1 : -1;
    add_if(first != 0u, v, TOP ? -k : k);
    if (__any_sync(0xffffffffu, rest != 0u)) {
        while (rest) {
            const int j = __ffs(rest) - 1;
            rest &= rest - 1u;
            const int kk = bs::bits_at<4>(T, j) - 5;
            add(val_at(j), TOP ? -kk : kk);
        }
    }
}

// Tiles along x (windows) and y (lane rows) of n positions.  A tile holds 32
// consecutive positions from `start`; its outputs are [lo, hi).  Positions
// next to an output must be in the tile -- except beyond the image edge,
// where the neighbour is missing and its comparisons are known (see Fill) --
// so the first tile outputs positions 0..30 (31), inner tiles 30 (their
// positions 1..30), the last tile up to 31 (positions up to 31), and a single
// tile (n <= 32) all n.
__host__ __device__ __forceinline__ int tiles_of(int n)
{
    return n <= 32 ? 1 : 2 + (n - 62 > 0 ? (n - 62 + 29) / 30 : 0);
}

__host__ __device__ __forceinline__ void tile_span(int n, int nt, int t, int &start, int &lo, int &hi)
{
    if (nt == 1) {
        start = 0;
        lo = 0;
        hi = n < 32 ? n : 32;
    } else if (t == 0) {
        start = 0;
        lo = 0;
        hi = 31;
    } else if (t < nt - 1) {
        start = 30 * t;
        lo = 1;
        hi = 31;
    } else {
        start = n - 32;
        lo = 30 * (nt - 1) + 1 - start;
        hi = 32;
    }
}

// What the walk knows about neighbours beyond the image edge of its tile.
// A comparison with a missing voxel has a fixed outcome: in the vertex
// complex a missing voxel beats every real one (it compares as 2^K), in the
// top-cell complex it loses (the voxel owns the boundary cell).  Those
// outcomes are shifted in where a window's bit 0 or 31, or a warp's lane 0
// or 31, takes a neighbour from outside the tile.
struct Fill {
    uint32_t xl, xr;    // 1 / 0x80000000 when the voxel left of bit 0 / right of bit 31 is missing, else 0
    bool yt, yb;        // this lane is lane 0 and row y-1 is missing / lane 31 and row y+1 is missing
    bool edge;          // any of these for the warp (warp-uniform)
};

// The walk: step(a, b) compares plane z (row a) with plane z+1 (row b) and
// the in-plane pairs of plane z+1, and emits plane z.  State between steps:
// the wins of plane z+1 over plane z and over its in-plane neighbours that
// precede it, un-negated (see each field).
//
// The 13 comparisons run plane-major: their carry chains advance together
// and each plane's operands -- the x-shifts of b, and rows y-1 of a and y+1
// of a and b from the neighbouring lanes -- are made just before use, so no
// shifted or shuffled copy of a whole row is held in registers.
template <int K, bool TOP>
struct Walk {
    uint32_t nW[3][3];  // wins of (z, y, x) over (z-1, y+dy-1, x+dx-1) are ~nW[dy][dx]
    uint32_t sE;        // wins over (z, y, x-1): ~sE; over (z, y, x+1): sE >> 1
    uint32_t sF[3];     // wins over (z, y+1, x+dx-1): sF[dx]
    uint32_t sD[3];     // wins over (z, y-1, x+dx-1): ~sD[2-dx]

    __device__ __forceinline__ void begin()
    {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            nW[i][0] = nW[i][1] = nW[i][2] = ~0u;
            sF[i] = 0u;
            sD[i] = ~0u;
        }
        sE = ~0u;
    }

    // emit(mask, T): output voxels of plane z with a nonzero count (mask
    // already restricted to out_x).  Warp-collective.
    template <class Emit>
    __device__ __forceinline__ void step(const Row<K> &a, const Row<K> &b, bool emit_z, uint32_t out_x, const Fill &fl,
                                         const Mul &mu, Emit &&emit)
    {
        // R0[d] = A(y)[x] vs B(y)[x+d-1]; G[d] = A(y-1)[x] vs B(y)[x+d-1];
        // K2[d] = A(y+1)[x] vs B(y)[x+d-1]; E = B(y)[x-1] vs B(y)[x];
        // F[d] = B(y)[x+1-d] vs B(y+1)[x]  (each: the earlier voxel beats the
        // later one).  Plane K, the existence plane, is the last carry step;
        // it is zero wherever every voxel of the two planes exists.
        uint32_t R0[3], G[3], K2[3], E, F[3];
        auto plane = [&](int k, bool first) {
            const uint32_t bP = b.P[k], bp = shr1(bP, mu), bm = shl1(bP, mu), bU = walk::from_next_lane(bP);
            const uint32_t aP = a.P[k], aU = walk::from_next_lane(aP), d = walk::from_prev_lane(aP);
            if (first) {
                R0[0] = cmp0<TOP>(aP, bm);
                R0[1] = cmp0<TOP>(aP, bP);
                R0[2] = cmp0<TOP>(aP, bp);
                G[0] = cmp0<TOP>(d, bm);
                G[1] = cmp0<TOP>(d, bP);
                G[2] = cmp0<TOP>(d, bp);
                K2[0] = cmp0<TOP>(aU, bm);
                K2[1] = cmp0<TOP>(aU, bP);
                K2[2] = cmp0<TOP>(aU, bp);
                E = cmp0<TOP>(bm, bP);
                F[0] = cmp0<TOP>(bp, bU);
                F[1] = cmp0<TOP>(bP, bU);
                F[2] = cmp0<TOP>(bm, bU);
            } else {
                R0[0] = cmpk<TOP>(aP, bm, R0[0]);
                R0[1] = cmpk<TOP>(aP, bP, R0[1]);
                R0[2] = cmpk<TOP>(aP, bp, R0[2]);
                G[0] = cmpk<TOP>(d, bm, G[0]);
                G[1] = cmpk<TOP>(d, bP, G[1]);
                G[2] = cmpk<TOP>(d, bp, G[2]);
                K2[0] = cmpk<TOP>(aU, bm, K2[0]);
                K2[1] = cmpk<TOP>(aU, bP, K2[1]);
                K2[2] = cmpk<TOP>(aU, bp, K2[2]);
                E = cmpk<TOP>(bm, bP, E);
                F[0] = cmpk<TOP>(bp, bU, F[0]);
                F[1] = cmpk<TOP>(bP, bU, F[1]);
                F[2] = cmpk<TOP>(bm, bU, F[2]);
            }
        };
        plane(0, true);
#pragma unroll
        for (int k = 1; k < K; ++k) plane(k, false);
        if (fl.edge || __any_sync(0xffffffffu, (a.P[K] | b.P[K]) != 0u)) {
            // the existence planes, with missing neighbours shifted and
            // shuffled in beyond the image edge
            const uint32_t bP = b.P[K], aP = a.P[K];
            const uint32_t bm = bP * mu.two + fl.xl, bp = umulhi(bP, mu.half) + fl.xr;
            uint32_t bU = walk::from_next_lane(bP), aU = walk::from_next_lane(aP), d = walk::from_prev_lane(aP);
            if (fl.yb) bU = aU = ~0u;
            if (fl.yt) d = ~0u;
            R0[0] = cmpk<TOP>(aP, bm, R0[0]);
            R0[1] = cmpk<TOP>(aP, bP, R0[1]);
            R0[2] = cmpk<TOP>(aP, bp, R0[2]);
            G[0] = cmpk<TOP>(d, bm, G[0]);
            G[1] = cmpk<TOP>(d, bP, G[1]);
            G[2] = cmpk<TOP>(d, bp, G[2]);
            K2[0] = cmpk<TOP>(aU, bm, K2[0]);
            K2[1] = cmpk<TOP>(aU, bP, K2[1]);
            K2[2] = cmpk<TOP>(aU, bp, K2[2]);
            E = cmpk<TOP>(bm, bP, E);
            F[0] = cmpk<TOP>(bp, bU, F[0]);
            F[1] = cmpk<TOP>(bP, bU, F[1]);
            F[2] = cmpk<TOP>(bm, bU, F[2]);
        }
        uint32_t Gu[3], K2d[3], Fd[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Gu[d] = walk::from_next_lane(G[d]);    // lane y+1's G: A(y) vs B(y+1)
            K2d[d] = walk::from_prev_lane(K2[d]);  // lane y-1's K2: A(y) vs B(y-1)
            Fd[d] = walk::from_prev_lane(F[d]);    // lane y-1's F
        }
        if (fl.edge) {
            // rows beyond the image edge: A(y) vs missing B(y+1) or B(y-1),
            // missing B(y-1) vs B(y)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (fl.yb) Gu[d] = TOP ? ~0u : 0u;
                if (fl.yt) {
                    K2d[d] = TOP ? ~0u : 0u;
                    Fd[d] = TOP ? 0u : ~0u;
                }
            }
        }
        if (emit_z) {
            uint32_t up[3][3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                up[1][d] = R0[d];
                up[2][d] = Gu[d];
                up[0][d] = K2d[d];
            }
            uint32_t T[4];
            const uint32_t m = kappa3w(up, nW, sE, umulhi(sE, mu.half) + (TOP ? fl.xr : 0u), sF, sD, out_x, T);
            emit(m, T);
        }
        // the state of plane z+1: its wins over plane z (a neighbour earlier
        // in memory wins ties, so these are negations) and in-plane
        // (shifts bring in a missing neighbour's outcome beyond the image
        // edge: the earlier voxel missing, it beats in the vertex complex;
        // the later one missing, it is beaten in the top-cell complex)
        const uint32_t el = TOP ? 0u : fl.xl, er = TOP ? 0u : fl.xr;  // earlier operand missing
        const uint32_t ll = TOP ? fl.xl : 0u, lr = TOP ? fl.xr : 0u;  // later operand missing
        nW[1][0] = R0[2] * mu.two + el;
        nW[1][1] = R0[1];
        nW[1][2] = umulhi(R0[0], mu.half) + er;
        nW[2][0] = K2[2] * mu.two + el;
        nW[2][1] = K2[1];
        nW[2][2] = umulhi(K2[0], mu.half) + er;
        nW[0][0] = G[2] * mu.two + el;
        nW[0][1] = G[1];
        nW[0][2] = umulhi(G[0], mu.half) + er;
        sE = E;
        sF[0] = F[0] * mu.two + ll;
        sF[1] = F[1];
        sF[2] = umulhi(F[2], mu.half) + lr;
        sD[0] = Fd[0];
        sD[1] = Fd[1];
        sD[2] = Fd[2];
    }
};

}  // namespace walk3
}  // namespace ecc
