// ecc_bitlogic.cuh -- bit logic of the 3D walker (ecc_walk3.cuh) as
// host + device functions, so the CPU tests can check it against the plain
// forms in ecc_bitslice.cuh (tests/test_bitslice_core.py).
//
// On the device every logic operation is one explicit three-input LOP3 with
// its truth table, and every shift is a multiply by a power of two held in a
// run-time value (IMAD on the FMA pipe): the compiler then keeps negations
// inside the logic operations and the integer ALU pipe, which bounds the
// walker, runs nothing but the logic.  On the host the same functions are
// plain C++.
#pragma once

#include <stdint.h>

#include "ecc_bitslice.cuh"

namespace ecc {
namespace walk3 {

// One three-input logic operation with truth table LUT: bit (4a + 2b + c)
// of LUT is the result for input bits a, b, c (a = 0xF0, b = 0xCC, c = 0xAA
// in the usual notation).
template <uint32_t LUT>
BS_HD uint32_t lop3(uint32_t a, uint32_t b, uint32_t c)
{
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
#else
    uint32_t d = 0;
    for (int m = 0; m < 8; ++m)
        if ((LUT >> m) & 1u) d |= ((m & 4) ? a : ~a) & ((m & 2) ? b : ~b) & ((m & 1) ? c : ~c);
    return d;
#endif
}

// The same with an immediate third operand.
template <uint32_t LUT, uint32_t C>
BS_HD uint32_t lop3i(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "n"(C), "n"(LUT));
    return d;
#else
    return lop3<LUT>(a, b, C);
#endif
}

BS_HD uint32_t umulhi(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Powers of two as run-time values, so the compiler cannot turn the
// multiplies back into shifts (which run on the ALU pipe).
struct Mul {
    uint32_t two;     // 2:    x * two         == x << 1
    uint32_t half;    // 2^31: umulhi(x, half) == x >> 1
    uint32_t up[4];   // 2, 4, 16, 256:            x << d for the transpose stages d = 1, 2, 4, 8
    uint32_t dn[4];   // 2^31, 2^30, 2^28, 2^24:   x >> d
};

BS_HD Mul make_mul()
{
    Mul m{};
    m.two = 2u;
    m.half = 1u << 31;
    const int d[4] = {1, 2, 4, 8};
    for (int i = 0; i < 4; ++i) {
        m.up[i] = 1u << d[i];
        m.dn[i] = 1u << (32 - d[i]);
    }
    return m;
}

BS_HD uint32_t shl1(uint32_t x, const Mul &mu) { return x * mu.two; }
BS_HD uint32_t shr1(uint32_t x, const Mul &mu) { return umulhi(x, mu.half); }

// r[x] = m[x + DX]
template <int DX>
BS_HD uint32_t at_offset(uint32_t m, const Mul &mu)
{
    return DX > 0 ? shr1(m, mu) : (DX < 0 ? shl1(m, mu) : m);
}

// Delta swap of index bit s between registers lo/hi (they differ in register
// bit s) and position bit s inside the registers (M: positions with bit s
// set), the shifts by d = 2^s as multiplies.
// Each half is one select (c ? b : a, truth table 0xD8) by the mask.
template <uint32_t M>
BS_HD void swap_bit(uint32_t &lo, uint32_t &hi, uint32_t up, uint32_t dn)
{
    const uint32_t a = lo, b = hi;
    lo = lop3i<0xD8u, M>(a, b * up);
    hi = lop3i<0xD8u, M>(umulhi(a, dn), b);
}

// 32 uint8 voxels (byte j of r[q] is voxel 4q+j) -> 8 planes (bit x of p[k] =
// bit k of voxel x).  The byte permutes make the register number (j0, j1,
// q0) and the byte position (q1, q2); three delta-swap stages exchange the
// sub-byte position bits with the register number.
BS_HD void transpose_u8(const uint32_t r[8], uint32_t p[8], const Mul &mu)
{
#pragma unroll
    for (int q0 = 0; q0 < 2; ++q0) {
        const uint32_t t01 = bs::byte_perm(r[q0], r[q0 + 2], 0x5140u);
        const uint32_t t23 = bs::byte_perm(r[q0], r[q0 + 2], 0x7362u);
        const uint32_t u01 = bs::byte_perm(r[q0 + 4], r[q0 + 6], 0x5140u);
        const uint32_t u23 = bs::byte_perm(r[q0 + 4], r[q0 + 6], 0x7362u);
        p[0 + 4 * q0] = bs::byte_perm(t01, u01, 0x5410u);
        p[1 + 4 * q0] = bs::byte_perm(t01, u01, 0x7632u);
        p[2 + 4 * q0] = bs::byte_perm(t23, u23, 0x5410u);
        p[3 + 4 * q0] = bs::byte_perm(t23, u23, 0x7632u);
    }
#pragma unroll
    for (int k = 0; k < 8; k += 2) swap_bit<0xAAAAAAAAu>(p[k], p[k + 1], mu.up[0], mu.dn[0]);
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (!(k & 2)) swap_bit<0xCCCCCCCCu>(p[k], p[k + 2], mu.up[1], mu.dn[1]);
#pragma unroll
    for (int k = 0; k < 4; ++k) swap_bit<0xF0F0F0F0u>(p[k], p[k + 4], mu.up[2], mu.dn[2]);
}

// 32 uint16 voxels (halfword j of r[q] is voxel 2q+j) -> 16 planes.
BS_HD void transpose_u16(const uint32_t r[16], uint32_t p[16], const Mul &mu)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        p[2 * i + 0] = bs::byte_perm(r[i], r[i + 8], 0x5410u);
        p[2 * i + 1] = bs::byte_perm(r[i], r[i + 8], 0x7632u);
    }
#pragma unroll
    for (int k = 0; k < 16; k += 2) swap_bit<0xAAAAAAAAu>(p[k], p[k + 1], mu.up[0], mu.dn[0]);
#pragma unroll
    for (int k = 0; k < 16; ++k)
        if (!(k & 2)) swap_bit<0xCCCCCCCCu>(p[k], p[k + 2], mu.up[1], mu.dn[1]);
#pragma unroll
    for (int k = 0; k < 16; ++k)
        if (!(k & 4)) swap_bit<0xF0F0F0F0u>(p[k], p[k + 4], mu.up[2], mu.dn[2]);
#pragma unroll
    for (int k = 0; k < 8; ++k) swap_bit<0xFF00FF00u>(p[k], p[k + 8], mu.up[3], mu.dn[3]);
}

// Mask of voxels with a >= b over K planes: the carry of a - b, one
// majority(a_k, ~b_k, c) per plane (truth table 0xB2), a_0 | ~b_0 (0xF3)
// for the first.
template <int K>
BS_HD uint32_t ge(const uint32_t *a, const uint32_t *b)
{
    uint32_t c = lop3<0xF3u>(a[0], b[0], 0u);
#pragma unroll
    for (int k = 1; k < K; ++k) c = lop3<0xB2u>(a[k], b[k], c);
    return c;
}

// a beats b that follows it in memory (ties to a): max for the vertex
// complex, min for the top-cell complex.
template <int K, bool TOP>
BS_HD uint32_t beats_later(const uint32_t *a, const uint32_t *b)
{
    return TOP ? ge<K>(b, a) : ge<K>(a, b);
}

// One plane of beats_later: the first (cmp0) and each further plane's
// carry step (cmpk).
template <bool TOP>
BS_HD uint32_t cmp0(uint32_t a, uint32_t b)
{
    return TOP ? lop3<0xF3u>(b, a, 0u) : lop3<0xF3u>(a, b, 0u);
}
template <bool TOP>
BS_HD uint32_t cmpk(uint32_t a, uint32_t b, uint32_t c)
{
    return TOP ? lop3<0xB2u>(b, a, c) : lop3<0xB2u>(a, b, c);
}

// Three-input AND with each input optionally negated (the negations inside
// the one logic operation).
template <bool NA, bool NB, bool NC>
BS_HD uint32_t and3(uint32_t a, uint32_t b, uint32_t c)
{
    constexpr uint32_t A = NA ? 0x0Fu : 0xF0u, B = NB ? 0x33u : 0xCCu, C = NC ? 0x55u : 0xAAu;
    return lop3<A & B & C>(a, b, c);
}

// Per-voxel sum of 12 one-bit inputs as four bit planes: a carry-save tree
// of full adders (sum 0x96, carry 0xE8) and half adders.
BS_HD void count12(const uint32_t x[12], uint32_t o[4])
{
    auto fa = [](uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &cy) {
        s = lop3<0x96u>(a, b, c);
        cy = lop3<0xE8u>(a, b, c);
    };
    uint32_t s0, s1, s2, s3, s4, c0, c1, c2, c3, c4, c5, s5, s6, d0, d1, d2;
    fa(x[0], x[1], x[2], s0, c0);
    fa(x[3], x[4], x[5], s1, c1);
    fa(x[6], x[7], x[8], s2, c2);
    fa(x[9], x[10], x[11], s3, c3);
    fa(s0, s1, s2, s4, c4);
    o[0] = lop3<0x3Cu>(s4, s3, 0u);  // s4 ^ s3
    c5 = lop3<0xC0u>(s4, s3, 0u);    // s4 & s3
    fa(c0, c1, c2, s5, d0);
    fa(c3, c4, c5, s6, d1);
    o[1] = lop3<0x3Cu>(s5, s6, 0u);
    d2 = lop3<0xC0u>(s5, s6, 0u);
    fa(d0, d1, d2, o[2], o[3]);
}

// The signed cell count of the walk's voxels (bs::kappa3d's chain form,
// kappa = T - 5), from the wins in the polarity the walk keeps them in:
//   up[dy][dx]: wins over (z+1, y+dy-1, x+dx-1), positive;
//   nW[dy][dx]: wins over (z-1, ...) are ~nW, negative;
//   sE: wins over (z, y, x-1) are ~sE; xp: wins over (z, y, x+1), positive;
//   sF[dx]: wins over (z, y+1, x+dx-1), positive; sD: over (z, y-1, x+dx-1)
//   are ~sD[2-dx].
// Returns the mask of voxels with T != 5 within out_x, and T's planes.
BS_HD uint32_t kappa3w(const uint32_t up[3][3], const uint32_t nW[3][3], uint32_t sE,
                                            uint32_t xp, const uint32_t sF[3], const uint32_t sD[3], uint32_t out_x,
                                            uint32_t T[4])
{
    // faces: ex0 = ~sE, ex1 = xp, ey0 = ~sD[1], ey1 = sF[1], ez0 = ~nW[1][1], ez1 = up[1][1]
    // squares (side a along the first axis, side b along the second)
    const uint32_t sxy00 = and3<true, true, true>(sD[1], sE, sD[2]);      // ey0 ex0 w(y-1,x-1)
    const uint32_t sxy01 = and3<true, false, true>(sD[1], xp, sD[0]);     // ey0 ex1 w(y-1,x+1)
    const uint32_t sxy10 = and3<false, true, false>(sF[1], sE, sF[0]);    // ey1 ex0 w(y+1,x-1)
    const uint32_t sxy11 = and3<false, false, false>(sF[1], xp, sF[2]);   // ey1 ex1 w(y+1,x+1)
    const uint32_t sxz00 = and3<true, true, true>(nW[1][1], sE, nW[1][0]);
    const uint32_t sxz01 = and3<true, false, true>(nW[1][1], xp, nW[1][2]);
    const uint32_t sxz10 = and3<false, true, false>(up[1][1], sE, up[1][0]);
    const uint32_t sxz11 = and3<false, false, false>(up[1][1], xp, up[1][2]);
    const uint32_t syz00 = and3<true, true, true>(nW[1][1], sD[1], nW[0][1]);
    const uint32_t syz01 = and3<true, false, true>(nW[1][1], sF[1], nW[2][1]);
    const uint32_t syz10 = and3<false, true, false>(up[1][1], sD[1], up[0][1]);
    const uint32_t syz11 = and3<false, false, false>(up[1][1], sF[1], up[2][1]);
    // chains: (1 - f) + s - c = ~f | (s & ~c), with c = s & (rest of the cube)
    uint32_t t[12];
    t[0] = lop3<0xF4u>(sE, sxy00, and3<false, false, true>(sxz00, syz00, nW[0][0]));            // -x, cube (0,0,0)
    t[1] = lop3<0x4Fu>(xp, sxy11, and3<false, false, true>(sxz01, syz01, nW[2][2]));            // +x, cube (1,1,0)
    t[2] = lop3<0xF4u>(sD[1], syz10, and3<false, false, false>(sxy00, sxz10, up[0][0]));        // -y, cube (0,0,1)
    t[3] = lop3<0x4Fu>(sF[1], syz01, and3<false, false, true>(sxy10, sxz00, nW[2][0]));         // +y, cube (0,1,0)
    t[4] = lop3<0xF4u>(nW[1][1], sxz01, and3<false, false, true>(sxy01, syz00, nW[0][2]));      // -z, cube (1,0,0)
    t[5] = lop3<0x4Fu>(up[1][1], sxz11, and3<false, false, false>(sxy11, syz11, up[2][2]));     // +z, cube (1,1,1)
    t[6] = lop3<0x30u>(sxy10, and3<false, false, false>(sxz10, syz11, up[2][0]), 0u);           // cube (0,1,1)
    t[7] = lop3<0x30u>(sxy01, and3<false, false, false>(sxz11, syz10, up[0][2]), 0u);           // cube (1,0,1)
    t[8] = sxz00;
    t[9] = sxz10;
    t[10] = syz00;
    t[11] = syz11;
    count12(t, T);
    // T != 5 (0b0101) within out_x
    return lop3<0xA8u>(lop3<0xDFu>(T[0], T[1], T[2]), T[3], out_x);
}

// The signed cell count of the pixels of row y (kappa = X0 + X1 + 2 X2 - 3,
// bs::kappa2d's chain form: four face/square chains), from the wins in the
// polarity the walk keeps them:
//   wins over row y-1 at x-1, x, x+1 are ~sW[0], ~sW[1], ~sW[2];
//   over (y, x-1): ~sE; over (y, x+1): sEr;
//   over row y+1 at x-1, x, x+1: H0, H1, H2r.
// Returns the mask of nonzero counts within out_x and X.
BS_HD uint32_t kappa2w(const uint32_t sW[3], uint32_t sE, uint32_t sEr, uint32_t H0,
                                            uint32_t H1, uint32_t H2r, uint32_t out_x, uint32_t X[3])
{
    // ex0 = ~sE, ex1 = sEr, ey0 = ~sW[1], ey1 = H1
    const uint32_t b0 = lop3<0xF1u>(sE, sW[1], sW[0]);   // ~ex0 | (ey0 & w(y-1, x-1))
    const uint32_t b1 = lop3<0x8Fu>(sEr, H1, H2r);       // ~ex1 | (ey1 & w(y+1, x+1))
    const uint32_t b2 = lop3<0xF4u>(sW[1], sEr, sW[2]);  // ~ey0 | (ex1 & w(y-1, x+1))
    const uint32_t b3 = lop3<0x2Fu>(H1, sE, H0);         // ~ey1 | (ex0 & w(y+1, x-1))
    X[0] = lop3<0x96u>(b0, b1, b2);
    X[2] = lop3<0xE8u>(b0, b1, b2);
    X[1] = b3;
    // sum == 3 iff X2 and exactly one of X0, X1
    return lop3<0x9Fu>(X[2], X[0], X[1]) & out_x;
}

// Counts of +-1, which are nearly all the nonzero counts of smooth images,
// so the emission can take their sign from one plane.  2D (count X0 + X1 +
// 2 X2 - 3): pm marks the +-1 (X2 ? X0 == X1 : X0 & X1), plus the +1 among
// them (X2 & X0).
BS_HD void split_pm1_2d(const uint32_t X[3], uint32_t &pm, uint32_t &plus)
{
    pm = lop3<0xC2u>(X[0], X[1], X[2]);
    plus = X[2] & X[0];
}

// 3D (count T - 5, T = T0 + 2 T1 + 4 T2 + 8 T3): T = 4 or 6 (T2 & ~T3 & ~T0),
// the +1 where T1.
BS_HD void split_pm1_3d(const uint32_t T[4], uint32_t &pm, uint32_t &plus)
{
    pm = lop3<0x10u>(T[2], T[3], T[0]);
    plus = T[1];
}

}  // namespace walk3
}  // namespace ecc
