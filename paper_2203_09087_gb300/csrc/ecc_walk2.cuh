// ecc_walk2.cuh -- the 2D bit-sliced walker (device only), in the form of
// the 3D walker (ecc_walk3.cuh): explicit three-input logic operations with
// their truth tables, left shifts only on the bit planes (a left shift is a
// multiply, off the ALU pipe; a right shift costs an ALU slot, so the three
// results that need one are shifted instead of eight planes), and an
// existence plane folded in as the most significant carry step only where
// some pixel of the two rows is missing.
//
// A lane holds a window of 32 pixels of one row (bit i: pixel xw + i; bits
// 1..30 are outputs, bits 0 and 31 the x halo) and walks rows; nothing in a
// step is warp-collective, so lanes may walk different rows and images.  A
// pixel's wins over neighbours that precede it in memory are negations of
// their comparisons (ties to the lower linear index), as in Walk2d.
#pragma once

#include <stdint.h>

#include "ecc_bitlogic.cuh"
#include "ecc_walk.cuh"

namespace ecc {
namespace walk2 {

using walk3::cmp0;
using walk3::cmpk;
using walk3::lop3;
using walk3::Mul;

// Aligned 32-bit words covering the window's bytes [first, first + 4 NW) of
// a row of row_bytes bytes, from the aligned address at or below it, then
// shifted into place by byte permutes and transposed into K planes.  Words
// that hold no byte of the row are not read (0 instead); a window wholly
// inside the row (the common case) loads without checks.
template <int K>
__device__ __forceinline__ void load_window(const unsigned char *row, int64_t row_bytes, int64_t first,
                                            uint32_t *P, const Mul &mu)
{
    constexpr int NW = K;  // 32 pixels of K bits = K words
    const uintptr_t start = reinterpret_cast<uintptr_t>(row) + (uintptr_t)first;
    const uintptr_t a0 = start & ~uintptr_t(3);
    const uintptr_t lo = reinterpret_cast<uintptr_t>(row), hi = lo + (uintptr_t)row_bytes;
    uint32_t w[NW + 1];
    if (a0 >= lo && a0 + 4 * (NW + 1) <= hi) {
#pragma unroll
        for (int i = 0; i <= NW; ++i) w[i] = __ldg(reinterpret_cast<const uint32_t *>(a0) + i);
    } else {
#pragma unroll
        for (int i = 0; i <= NW; ++i) {
            const uintptr_t ad = a0 + 4 * i;
            w[i] = (ad + 4 > lo && ad < hi) ? __ldg(reinterpret_cast<const uint32_t *>(ad)) : 0u;
        }
    }
    const uint32_t sh = (uint32_t)(start & 3u);
    const uint32_t sel = sh | ((sh + 1) << 4) | ((sh + 2) << 8) | ((sh + 3) << 12);
    uint32_t r[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) r[i] = __byte_perm(w[i], w[i + 1], sel);
    if (K == 8)
        walk3::transpose_u8(r, P, mu);
    else
        walk3::transpose_u16(r, P, mu);
}

using walk3::kappa2w;

template <int K, bool TOP>
struct Walk {
    uint32_t A[K + 1];   // row y (planes, existence plane K)
    uint32_t Am[K + 1];  // row y shifted: bit x holds pixel x-1
    uint32_t sW[3];      // wins of row y over row y-1, negated (see kappa2w)
    uint32_t sE, sEr;    // wins of row y over (y, x-1): ~sE; over (y, x+1): sEr

    __device__ __forceinline__ void begin(const uint32_t *P, const Mul &mu)
    {
#pragma unroll
        for (int k = 0; k <= K; ++k) {
            A[k] = P[k];
            Am[k] = P[k] * mu.two;
        }
        sW[0] = sW[1] = sW[2] = 0u;
        sE = sEr = 0u;
    }

    // Advance to row y+1 (B, K + 1 planes).  When emit_y (warp-uniform),
    // calls emit(mask, X) for row y: count = X0 + X1 + 2 X2 - 3.
    template <class Emit>
    __device__ __forceinline__ void step(const uint32_t *B, bool emit_y, uint32_t out_x, const Mul &mu, Emit &&emit)
    {
        // H0 = A[x] vs B[x-1], H1 = A[x] vs B[x], H2 = A[x-1] vs B[x],
        // E = B[x-1] vs B[x]  (the earlier pixel beats the later one)
        uint32_t H0, H1, H2, E;
        uint32_t Bm[K + 1];
        auto plane = [&](int k, bool first) {
            const uint32_t b = B[k], bm = b * mu.two, a = A[k], am = Am[k];
            Bm[k] = bm;
            if (first) {
                H0 = cmp0<TOP>(a, bm);
                H1 = cmp0<TOP>(a, b);
                H2 = cmp0<TOP>(am, b);
                E = cmp0<TOP>(bm, b);
            } else {
                H0 = cmpk<TOP>(a, bm, H0);
                H1 = cmpk<TOP>(a, b, H1);
                H2 = cmpk<TOP>(am, b, H2);
                E = cmpk<TOP>(bm, b, E);
            }
        };
        plane(0, true);
#pragma unroll
        for (int k = 1; k < K; ++k) plane(k, false);
        // per lane (lanes of a batch tile walk different rows): no warp-wide vote
        if ((A[K] | B[K]) != 0u)
            plane(K, false);
        else
            Bm[K] = 0u;
        if (emit_y) {
            uint32_t X[3];
            const uint32_t m = kappa2w(sW, sE, sEr, H0, H1, walk3::umulhi(H2, mu.half), out_x, X);
            emit(m, X);
        }
        // state of row y+1: its wins over row y (negated) and in-row
        sW[0] = H2;
        sW[1] = H1;
        sW[2] = walk3::umulhi(H0, mu.half);
        sE = E;
        sEr = walk3::umulhi(E, mu.half);
#pragma unroll
        for (int k = 0; k <= K; ++k) {
            A[k] = B[k];
            Am[k] = Bm[k];
        }
    }
};

}  // namespace walk2
}  // namespace ecc
