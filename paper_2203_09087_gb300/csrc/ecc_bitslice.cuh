// ecc_bitslice.cuh -- bit-sliced building blocks of the stencil (host+device).
//
// A "window" is 32 consecutive voxels of one image row.  Bit-slicing turns
// it into K = 8*sizeof(T) bit planes: plane k holds bit k of every voxel, bit
// i of a plane belongs to voxel i of the window.  All comparisons and all
// cell-counting logic then run on 32 voxels per 32-bit operation.
//
// These functions are plain C++ so the tests can check them on the CPU
// against naive per-voxel code (tests/test_bitslice_core.py).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define BS_HD __host__ __device__ __forceinline__
#else
#define BS_HD inline
#endif

namespace ecc {
namespace bs {

#if defined(__CUDACC__)
// Powers of two in constant memory, for the byte alignment of a window read
// at an arbitrary offset: (w0 >> s) | (w1 << (32 - s)) as two multiplies by
// 2^(32-s) (the high and low words), which issue on the FMA pipe instead of
// the integer pipe that the bit logic keeps busy.  (Plain shifts stay plain:
// moving all of them to multiplies measured slower.)
static __constant__ uint32_t kPow2[33] = {
    1u << 0,  1u << 1,  1u << 2,  1u << 3,  1u << 4,  1u << 5,  1u << 6,  1u << 7,  1u << 8,
    1u << 9,  1u << 10, 1u << 11, 1u << 12, 1u << 13, 1u << 14, 1u << 15, 1u << 16, 1u << 17,
    1u << 18, 1u << 19, 1u << 20, 1u << 21, 1u << 22, 1u << 23, 1u << 24, 1u << 25, 1u << 26,
    1u << 27, 1u << 28, 1u << 29, 1u << 30, 1u << 31, 0u};
#endif

// Byte permute: result byte i = byte (s >> 4i) & 7 of the 8 bytes {a, b}.
BS_HD uint32_t byte_perm(uint32_t a, uint32_t b, uint32_t s)
{
#if defined(__CUDA_ARCH__)
    return __byte_perm(a, b, s);
#else
    const uint64_t x = ((uint64_t)b << 32) | a;
    uint32_t r = 0;
    for (int i = 0; i < 4; ++i) r |= (uint32_t)((x >> (8 * ((s >> (4 * i)) & 7))) & 0xffu) << (8 * i);
    return r;
#endif
}

// Exchange index bit s of the register number with bit s of the position
// inside the register, for the register pair (lo, hi) that differ in
// register bit s (delta swap; M = positions whose bit s is set).
BS_HD void swap_bit(uint32_t &lo, uint32_t &hi, int d, uint32_t M)
{
    const uint32_t a = lo, b = hi;
    lo = (a & ~M) | ((b << d) & M);
    hi = ((a >> d) & ~M) | (b & M);
}

// 32 uint8 voxels in r[0..7] (little-endian: byte j of r[q] is voxel 4q+j)
// -> planes p[0..7], bit x of p[k] = bit k of voxel x.
// Step 1 (byte permutes) makes the register number (j0, j1, q0) and the byte
// position (q1, q2); step 2 swaps the three sub-byte position bits with the
// register number, giving register k and position x.
BS_HD void transpose_u8(const uint32_t r[8], uint32_t p[8])
{
    uint32_t q[8];
#pragma unroll
    for (int q0 = 0; q0 < 2; ++q0) {
        const uint32_t t01 = byte_perm(r[q0], r[q0 + 2], 0x5140u);
        const uint32_t t23 = byte_perm(r[q0], r[q0 + 2], 0x7362u);
        const uint32_t u01 = byte_perm(r[q0 + 4], r[q0 + 6], 0x5140u);
        const uint32_t u23 = byte_perm(r[q0 + 4], r[q0 + 6], 0x7362u);
        q[0 + 4 * q0] = byte_perm(t01, u01, 0x5410u);
        q[1 + 4 * q0] = byte_perm(t01, u01, 0x7632u);
        q[2 + 4 * q0] = byte_perm(t23, u23, 0x5410u);
        q[3 + 4 * q0] = byte_perm(t23, u23, 0x7632u);
    }
    const uint32_t M[3] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u};
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (!(k & (1 << s))) swap_bit(q[k], q[k | (1 << s)], 1 << s, M[s]);
#pragma unroll
    for (int k = 0; k < 8; ++k) p[k] = q[k];
}

// 32 uint16 voxels in r[0..15] (halfword j of r[q] is voxel 2q+j) -> 16 planes.
BS_HD void transpose_u16(const uint32_t r[16], uint32_t p[16])
{
    uint32_t q[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        q[2 * i + 0] = byte_perm(r[i], r[i + 8], 0x5410u);
        q[2 * i + 1] = byte_perm(r[i], r[i + 8], 0x7632u);
    }
    const uint32_t M[4] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u};
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (!(k & (1 << s))) swap_bit(q[k], q[k | (1 << s)], 1 << s, M[s]);
#pragma unroll
    for (int k = 0; k < 16; ++k) p[k] = q[k];
}

// Mask of voxels with a >= b (bit-serial from the least significant plane:
// the carry of a - b, one majority function per plane).
template <int K>
BS_HD uint32_t ge(const uint32_t *a, const uint32_t *b)
{
    uint32_t c = a[0] | ~b[0];
#pragma unroll
    for (int k = 1; k < K; ++k) c = (a[k] & ~b[k]) | ((a[k] | ~b[k]) & c);
    return c;
}

BS_HD void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &carry)
{
    s = a ^ b ^ c;
    carry = (a & b) | (a & c) | (b & c);
}

BS_HD void half_add(uint32_t a, uint32_t b, uint32_t &s, uint32_t &carry)
{
    s = a ^ b;
    carry = a & b;
}

// Per-voxel count of 4 one-bit inputs as three bit planes (max 4).
BS_HD void count4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t o[3])
{
    uint32_t s, c1, c2;
    full_add(a, b, c, s, c1);
    half_add(s, d, o[0], c2);
    half_add(c1, c2, o[1], o[2]);
}

// Value of a bit-sliced field at bit i.
template <int K>
BS_HD int bits_at(const uint32_t *x, int i)
{
    int v = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) v |= (int)((x[k] >> i) & 1u) << k;
    return v;
}

// ---------------------------------------------------------------- 3D cells
//
// Wins of a voxel over its 26 neighbours, as masks over the window.
// Index [dz+1][dy+1][dx+1]; the centre entry is unused.  A win means the
// voxel beats the neighbour (the neighbour, if it exists, is not the
// voxel's rival for any cell they share).
//
// kappa = sum over cells containing the voxel that it introduces of
// (-1)^dim = 1 - F + S - C with F faces (6), S squares (12), C cubes (8).
// Equivalently kappa = T - 13 where T counts the 26 one-bit terms
// {squares} + {not face} + {not cube} (since 1 - F - C = (6 - F) + (8 - C) - 13).
// Returns the nonzero mask (T != 13) and the five bit planes of T.

// Per-voxel count of 26 one-bit inputs as five bit planes (max 26).
BS_HD void count26(const uint32_t x[26], uint32_t o[5])
{
    uint32_t s[8], c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) full_add(x[3 * i], x[3 * i + 1], x[3 * i + 2], s[i], c[i]);
    // weight 1: s[0..7], x[24], x[25]
    uint32_t a0, a1, a2, d0, d1, d2, b0, e0, e1;
    full_add(s[0], s[1], s[2], a0, d0);
    full_add(s[3], s[4], s[5], a1, d1);
    full_add(s[6], s[7], x[24], a2, d2);
    full_add(a0, a1, a2, b0, e0);
    half_add(b0, x[25], o[0], e1);
    // weight 2: c[0..7], d0, d1, d2, e0, e1 (13 terms)
    uint32_t f[4], g[4];
    full_add(c[0], c[1], c[2], f[0], g[0]);
    full_add(c[3], c[4], c[5], f[1], g[1]);
    full_add(c[6], c[7], d0, f[2], g[2]);
    full_add(d1, d2, e0, f[3], g[3]);
    uint32_t h0, k0, k1;
    full_add(f[0], f[1], f[2], h0, k0);
    full_add(f[3], e1, h0, o[1], k1);
    // weight 4: g[0..3], k0, k1 (6 terms)
    uint32_t m0, n0, m1, n1, n2;
    full_add(g[0], g[1], g[2], m0, n0);
    full_add(g[3], k0, k1, m1, n1);
    half_add(m0, m1, o[2], n2);
    // weight 8: n0, n1, n2
    full_add(n0, n1, n2, o[3], o[4]);
}

BS_HD uint32_t kappa3d(const uint32_t w[3][3][3], uint32_t T[5])
{
    const uint32_t ex[2] = {w[1][1][0], w[1][1][2]};
    const uint32_t ey[2] = {w[1][0][1], w[1][2][1]};
    const uint32_t ez[2] = {w[0][1][1], w[2][1][1]};
    uint32_t t[26];
    uint32_t sxy[2][2], sxz[2][2], syz[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            sxy[a][b] = ey[a] & ex[b] & w[1][2 * a][2 * b];   // y side a, x side b
            sxz[a][b] = ez[a] & ex[b] & w[2 * a][1][2 * b];   // z side a, x side b
            syz[a][b] = ez[a] & ey[b] & w[2 * a][2 * b][1];   // z side a, y side b
            t[0 + 2 * a + b] = sxy[a][b];
            t[4 + 2 * a + b] = sxz[a][b];
            t[8 + 2 * a + b] = syz[a][b];
        }
    t[12] = ~ex[0];
    t[13] = ~ex[1];
    t[14] = ~ey[0];
    t[15] = ~ey[1];
    t[16] = ~ez[0];
    t[17] = ~ez[1];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)   // cube on z side c, y side b, x side a
                t[18 + 4 * c + 2 * b + a] = ~(sxy[b][a] & sxz[c][a] & syz[c][b] & w[2 * c][2 * b][2 * a]);
    count26(t, T);
    // T == 13 = 0b01101
    return ~(T[0] & ~T[1] & T[2] & T[3] & ~T[4]);
}

// 2D: w[dy+1][dx+1]; kappa = 1 - faces + squares.  Returns the nonzero mask
// and the planes of F (faces, max 4) and Q (squares, max 4).
BS_HD uint32_t kappa2d(const uint32_t w[3][3], uint32_t F[3], uint32_t Q[3])
{
    const uint32_t ex0 = w[1][0], ex1 = w[1][2], ey0 = w[0][1], ey1 = w[2][1];
    count4(ex0, ex1, ey0, ey1, F);
    count4(ey0 & ex0 & w[0][0], ey0 & ex1 & w[0][2], ey1 & ex0 & w[2][0], ey1 & ex1 & w[2][2], Q);
    // nonzero iff 1 + Q != F (both at most 4, three planes)
    const uint32_t p0 = ~Q[0], c0 = Q[0];
    const uint32_t p1 = Q[1] ^ c0, c1 = Q[1] & c0;
    const uint32_t p2 = Q[2] ^ c1;
    return (p0 ^ F[0]) | (p1 ^ F[1]) | (p2 ^ F[2]);
}

}  // namespace bs
}  // namespace ecc
