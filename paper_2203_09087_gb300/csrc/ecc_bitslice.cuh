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

// Per-voxel count of 12 one-bit inputs as four bit planes (max 12).
BS_HD void count12(const uint32_t x[12], uint32_t o[4])
{
    uint32_t a[4], b[4];
    full_add(x[0], x[1], x[2], a[0], b[0]);
    full_add(x[3], x[4], x[5], a[1], b[1]);
    full_add(x[6], x[7], x[8], a[2], b[2]);
    full_add(x[9], x[10], x[11], a[3], b[3]);
    uint32_t c1, d2, e2;
    full_add(a[0], a[1], a[2], c1, d2);
    half_add(c1, a[3], o[0], e2);                  // weight 1 done
    uint32_t f2, g4, f2b, g4b, h4;
    full_add(b[0], b[1], b[2], f2, g4);
    full_add(b[3], d2, e2, f2b, g4b);
    half_add(f2, f2b, o[1], h4);                   // weight 2 done
    full_add(g4, g4b, h4, o[2], o[3]);             // weights 4 and 8
}

// Per-voxel count of 14 one-bit inputs as four bit planes (max 14).
BS_HD void count14(const uint32_t x[14], uint32_t o[4])
{
    uint32_t a[4], b[4];
    full_add(x[0], x[1], x[2], a[0], b[0]);
    full_add(x[3], x[4], x[5], a[1], b[1]);
    full_add(x[6], x[7], x[8], a[2], b[2]);
    full_add(x[9], x[10], x[11], a[3], b[3]);
    uint32_t s1, c1, s2, c2, c3;
    full_add(a[0], a[1], a[2], s1, c1);
    full_add(a[3], x[12], x[13], s2, c2);
    half_add(s1, s2, o[0], c3);                    // weight 1 done; weight 2: b[0..3], c1, c2, c3
    uint32_t t1, u1, t2, u2, u3;
    full_add(b[0], b[1], b[2], t1, u1);
    full_add(b[3], c1, c2, t2, u2);
    uint32_t t3;
    full_add(t1, t2, c3, o[1], u3);                // weight 2 done; weight 4: u1, u2, u3
    full_add(u1, u2, u3, o[2], o[3]);
    (void)t3;
}

// Per-voxel count of 4 one-bit inputs as three bit planes (max 4).
BS_HD void count4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t o[3])
{
    uint32_t s, c1, c2;
    full_add(a, b, c, s, c1);
    half_add(s, d, o[0], c2);
    half_add(c1, c2, o[1], o[2]);
}

// Mask of voxels where the 4-bit value x + 1 differs from the 4-bit value n.
BS_HD uint32_t plus_one_differs(const uint32_t x[4], const uint32_t n[4])
{
    const uint32_t p0 = ~x[0];
    const uint32_t c0 = x[0];
    const uint32_t p1 = x[1] ^ c0;
    const uint32_t c1 = x[1] & c0;
    const uint32_t p2 = x[2] ^ c1;
    const uint32_t c2 = x[2] & c1;
    const uint32_t p3 = x[3] ^ c2;
    return (p0 ^ n[0]) | (p1 ^ n[1]) | (p2 ^ n[2]) | (p3 ^ n[3]);
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
// (-1)^dim = 1 - faces + squares - cubes.  Returns the nonzero mask and the
// bit planes of S = squares and N = faces + cubes (kappa = 1 + S - N).
BS_HD uint32_t kappa3d(const uint32_t w[3][3][3], uint32_t S[4], uint32_t N[4])
{
    const uint32_t ex[2] = {w[1][1][0], w[1][1][2]};
    const uint32_t ey[2] = {w[1][0][1], w[1][2][1]};
    const uint32_t ez[2] = {w[0][1][1], w[2][1][1]};
    uint32_t sq[12];
    uint32_t sxy[2][2], sxz[2][2], syz[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            sxy[a][b] = ey[a] & ex[b] & w[1][2 * a][2 * b];   // y side a, x side b
            sxz[a][b] = ez[a] & ex[b] & w[2 * a][1][2 * b];   // z side a, x side b
            syz[a][b] = ez[a] & ey[b] & w[2 * a][2 * b][1];   // z side a, y side b
            sq[0 + 2 * a + b] = sxy[a][b];
            sq[4 + 2 * a + b] = sxz[a][b];
            sq[8 + 2 * a + b] = syz[a][b];
        }
    uint32_t n[14];
    n[0] = ex[0];
    n[1] = ex[1];
    n[2] = ey[0];
    n[3] = ey[1];
    n[4] = ez[0];
    n[5] = ez[1];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)   // cube on z side c, y side b, x side a
                n[6 + 4 * c + 2 * b + a] = sxy[b][a] & sxz[c][a] & syz[c][b] & w[2 * c][2 * b][2 * a];
    count12(sq, S);
    count14(n, N);
    return plus_one_differs(S, N);
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
