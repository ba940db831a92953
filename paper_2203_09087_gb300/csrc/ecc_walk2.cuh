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
// their comparisons (ties to the lower linear index).
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

// A window's aligned 32-bit words as loaded, before alignment: the loads can
// be issued a step ahead of their use (load_raw), and the words shifted and
// transposed once they are needed (unpack).
template <int K>
struct RawWin {
    uint32_t w[K + 1];
    uint32_t sel;  // byte-permute selector of the window's offset in the words
};

// Aligned 32-bit words covering the window's bytes [first, first + 4 K) of a
// row of row_bytes bytes, from the aligned address at or below it.  Words
// that hold no byte of the row are not read (0 instead); a window wholly
// inside the row (the common case) loads without checks.
template <int K>
__device__ __forceinline__ void load_raw(const unsigned char *row, int64_t row_bytes, int64_t first, RawWin<K> &r)
{
    constexpr int NW = K;  // 32 pixels of K bits = K words
    const uintptr_t start = reinterpret_cast<uintptr_t>(row) + (uintptr_t)first;
    const uintptr_t a0 = start & ~uintptr_t(3);
    const uintptr_t lo = reinterpret_cast<uintptr_t>(row), hi = lo + (uintptr_t)row_bytes;
    if (a0 >= lo && a0 + 4 * (NW + 1) <= hi) {
#pragma unroll
        for (int i = 0; i <= NW; ++i) r.w[i] = __ldg(reinterpret_cast<const uint32_t *>(a0) + i);
    } else {
#pragma unroll
        for (int i = 0; i <= NW; ++i) {
            const uintptr_t ad = a0 + 4 * i;
            r.w[i] = (ad + 4 > lo && ad < hi) ? __ldg(reinterpret_cast<const uint32_t *>(ad)) : 0u;
        }
    }
    const uint32_t sh = (uint32_t)(start & 3u);
    r.sel = sh | ((sh + 1) << 4) | ((sh + 2) << 8) | ((sh + 3) << 12);
}

// The window's 32 elements, shifted into place by byte permutes and
// transposed into K planes.
template <int K>
__device__ __forceinline__ void unpack(const RawWin<K> &r, uint32_t *P, const Mul &mu)
{
    uint32_t v[K];
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = __byte_perm(r.w[i], r.w[i + 1], r.sel);
    if (K == 8)
        walk3::transpose_u8(v, P, mu);
    else
        walk3::transpose_u16(v, P, mu);
}

template <int K>
__device__ __forceinline__ void load_window(const unsigned char *row, int64_t row_bytes, int64_t first,
                                            uint32_t *P, const Mul &mu)
{
    RawWin<K> r;
    load_raw<K>(row, row_bytes, first, r);
    unpack<K>(r, P, mu);
}

using walk3::kappa2w;

// Adds +kp (where plus) or -kp for every element of mask pm, U elements per
// iteration, their value loads issued together so that U are in flight at
// once (a lane rarely has more than a few).  Bits are taken from the top
// (one find-leading-one each).
template <int U, class ValAt, class Add>
__device__ __forceinline__ void emit_units(uint32_t pm, uint32_t plus, int kp, ValAt &&val_at, Add &&add)
{
    while (pm) {
        int i[U], v[U];
        uint32_t b[U];
        i[0] = 31 - __clz(pm);  // the loop's own element: always present
        b[0] = 1u << i[0];
        pm ^= b[0];
#pragma unroll
        for (int u = 1; u < U; ++u) {
            i[u] = 31 - __clz(pm | 1u);
            b[u] = pm ? 1u << i[u] : 0u;
            pm ^= b[u];
        }
        v[0] = val_at(i[0]);
#pragma unroll
        for (int u = 1; u < U; ++u) {
            v[u] = 0;
            if (b[u]) v[u] = val_at(i[u]);
        }
        add(v[0], (plus & b[0]) ? kp : -kp);
#pragma unroll
        for (int u = 1; u < U; ++u)
            if (b[u]) add(v[u], (plus & b[u]) ? kp : -kp);
    }
}

// Elements per iteration: measured on the uneven batch, 2 for the 2D
// walker's windows and 3 for the 3D tiles (3 or 4 gave the 2D part nothing,
// the 3D part 8 % more than 2).
constexpr int kEmitUnroll2d = 2, kEmitUnroll3d = 3;

// Emission of one step, per lane: m marks the window's pixels whose cell
// count X0 + X1 + 2 X2 - 3 is nonzero (bit i: element i, value val_at(i));
// add(v, k) adds k to the bin of value v.  The +-1 counts (in smooth images
// nearly all) go first, their sign read from one plane; then the rest
// (-2, -3) with the full count.
template <class ValAt, class Add>
__device__ __forceinline__ void emit2(uint32_t m, const uint32_t *X, ValAt &&val_at, Add &&add)
{
    uint32_t pm, plus;
    walk3::split_pm1_2d(X, pm, plus);
    pm &= m;
    uint32_t rest = m & ~pm;
    emit_units<kEmitUnroll2d>(pm, plus, 1, val_at, add);
    while (rest) {
        const int i = 31 - __clz(rest);
        rest ^= 1u << i;
        const int k = (int)((X[0] >> i) & 1u) + (int)((X[1] >> i) & 1u) + 2 * (int)((X[2] >> i) & 1u) - 3;
        add(val_at(i), k);
    }
}

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
