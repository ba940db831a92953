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
// (-1)^dim = 1 - F + S - C with F faces won (of 6), S squares (of 12) and C
// cubes (of 8).  A cell is won when all its edges at the voxel and all its
// other vertices are, so a cube won implies each of its three squares at
// the voxel, and a square its two faces.  The 26 signed terms therefore
// group into chains whose partial sums are single bits:
//   (1 - f) + s - c  with c => s => f   is  ~f | (s & ~c)    (6 chains)
//   s - c            with c => s        is  s & ~c           (2 chains)
//   s                                                        (4 squares)
// pairing every face, cube and square once (a matching of the cube/square
// and square/face incidences), so kappa = T - 5 with T the sum of 12 bits,
// 0 <= T <= 12.  The chain bits cost two logic operations each and T a
// 12-input carry-save count.

// Per-voxel count of 12 one-bit inputs as four bit planes (max 12).
BS_HD void count12(const uint32_t x[12], uint32_t o[4])
{
    uint32_t s0, s1, s2, s3, s4, c0, c1, c2, c3, c4, c5;
    full_add(x[0], x[1], x[2], s0, c0);
    full_add(x[3], x[4], x[5], s1, c1);
    full_add(x[6], x[7], x[8], s2, c2);
    full_add(x[9], x[10], x[11], s3, c3);
    full_add(s0, s1, s2, s4, c4);
    half_add(s4, s3, o[0], c5);
    // weight 2: c0..c5
    uint32_t s5, s6, d0, d1, d2;
    full_add(c0, c1, c2, s5, d0);
    full_add(c3, c4, c5, s6, d1);
    half_add(s5, s6, o[1], d2);
    // weight 4: d0, d1, d2
    full_add(d0, d1, d2, o[2], o[3]);
}

// Returns the nonzero mask (T != 5) and the four bit planes of T.
BS_HD uint32_t kappa3d(const uint32_t w[3][3][3], uint32_t T[4])
{
    const uint32_t ex0 = w[1][1][0], ex1 = w[1][1][2];
    const uint32_t ey0 = w[1][0][1], ey1 = w[1][2][1];
    const uint32_t ez0 = w[0][1][1], ez1 = w[2][1][1];
    // squares sAB[a][b]: side a along the first axis, side b along the second
    uint32_t sxy[2][2], sxz[2][2], syz[2][2];
    const uint32_t ey[2] = {ey0, ey1}, ex[2] = {ex0, ex1}, ez[2] = {ez0, ez1};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            sxy[a][b] = ey[a] & ex[b] & w[1][2 * a][2 * b];
            sxz[a][b] = ez[a] & ex[b] & w[2 * a][1][2 * b];
            syz[a][b] = ez[a] & ey[b] & w[2 * a][2 * b][1];
        }
    // cube (x side a, y side b, z side c) = sxy[b][a] & sxz[c][a] & syz[c][b] & corner;
    // each chain's cube is its square AND the rest (r) of the cube's condition
    uint32_t t[12];
    t[0] = ~ex0 | (sxy[0][0] & ~(sxz[0][0] & syz[0][0] & w[0][0][0]));    // -x, cube (0,0,0)
    t[1] = ~ex1 | (sxy[1][1] & ~(sxz[0][1] & syz[0][1] & w[0][2][2]));    // +x, cube (1,1,0)
    t[2] = ~ey0 | (syz[1][0] & ~(sxy[0][0] & sxz[1][0] & w[2][0][0]));    // -y, cube (0,0,1)
    t[3] = ~ey1 | (syz[0][1] & ~(sxy[1][0] & sxz[0][0] & w[0][2][0]));    // +y, cube (0,1,0)
    t[4] = ~ez0 | (sxz[0][1] & ~(sxy[0][1] & syz[0][0] & w[0][0][2]));    // -z, cube (1,0,0)
    t[5] = ~ez1 | (sxz[1][1] & ~(sxy[1][1] & syz[1][1] & w[2][2][2]));    // +z, cube (1,1,1)
    t[6] = sxy[1][0] & ~(sxz[1][0] & syz[1][1] & w[2][2][0]);             // cube (0,1,1)
    t[7] = sxy[0][1] & ~(sxz[1][1] & syz[1][0] & w[2][0][2]);             // cube (1,0,1)
    t[8] = sxz[0][0];
    t[9] = sxz[1][0];
    t[10] = syz[0][0];
    t[11] = syz[1][1];
    count12(t, T);
    // T == 5 = 0b0101
    return ~T[0] | T[1] | ~T[2] | T[3];
}

// ---------------------------------------------------------------- 4D cells
//
// Wins over the 80 neighbours as masks w[dw+1][dz+1][dy+1][dx+1] (centre
// unused).  The star of the voxel splits along w: the cells of its own
// hyperplane (count kappa3d of the in-hyperplane wins W0), and each such cell
// extended to w+1 (or w-1), one dimension higher, which the voxel wins when
// it beats its w-neighbour (b+) and the cell's vertices in both hyperplanes
// (W0 & W+).  Hence
//   kappa4 = k3(W0) - b+ k3(W0 & W+) - b- k3(W0 & W-),   k3 = T - 5,
// and kappa4 != 0 iff X != Y with X = T0 + 5 (b+ + b-) and
// Y = b+ T+ + b- T- + 5 (both at most 32, six bit planes).

// x + y over n-bit planes (carry out dropped: callers keep sums in range).
template <int N>
BS_HD void add_planes(const uint32_t *x, const uint32_t *y, uint32_t *out)
{
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const uint32_t a = x[k], b = y[k];
        out[k] = a ^ b ^ c;
        c = (a & b) | (a & c) | (b & c);
    }
}

// Nonzero mask of kappa4 from the chain counts T0 = T(W0), Tp = T(W0 & W+),
// Tm = T(W0 & W-) (four planes each) and the w-wins bp = b+, bm = b-.
BS_HD uint32_t kappa4_nonzero(const uint32_t *T0, const uint32_t *Tp, const uint32_t *Tm, uint32_t bp, uint32_t bm)
{
    // X = T0 + 5 (bp + bm); 5 (bp + bm) is 0, 5 or 10: planes (one, both, one, both)
    const uint32_t both = bp & bm, one = bp ^ bm;
    const uint32_t f[6] = {one, both, one, both, 0u, 0u};
    const uint32_t t0[6] = {T0[0], T0[1], T0[2], T0[3], 0u, 0u};
    uint32_t X[6];
    add_planes<6>(t0, f, X);
    // Y = (bp & Tp) + (bm & Tm) + 5
    const uint32_t p[6] = {bp & Tp[0], bp & Tp[1], bp & Tp[2], bp & Tp[3], 0u, 0u};
    const uint32_t q[6] = {bm & Tm[0], bm & Tm[1], bm & Tm[2], bm & Tm[3], 0u, 0u};
    uint32_t pq[6], Y[6];
    add_planes<6>(p, q, pq);
    const uint32_t five[6] = {~0u, 0u, ~0u, 0u, 0u, 0u};
    add_planes<6>(pq, five, Y);
    uint32_t nz = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) nz |= X[k] ^ Y[k];
    return nz;
}

// All 80 wins at once (w[1][1][1][1] unused).  Returns the nonzero mask and
// the planes kappa4_at needs.
BS_HD uint32_t kappa4d(const uint32_t w[3][3][3][3], uint32_t T0[4], uint32_t Tp[4], uint32_t Tm[4], uint32_t &bp,
                       uint32_t &bm)
{
    uint32_t a[3][3][3];
#pragma unroll
    for (int i = 0; i < 27; ++i) (&a[0][0][0])[i] = (&w[1][0][0][0])[i];
    kappa3d(a, T0);
#pragma unroll
    for (int i = 0; i < 27; ++i) (&a[0][0][0])[i] = (&w[1][0][0][0])[i] & (&w[2][0][0][0])[i];
    kappa3d(a, Tp);
#pragma unroll
    for (int i = 0; i < 27; ++i) (&a[0][0][0])[i] = (&w[1][0][0][0])[i] & (&w[0][0][0][0])[i];
    kappa3d(a, Tm);
    bp = w[2][1][1][1];
    bm = w[0][1][1][1];
    return kappa4_nonzero(T0, Tp, Tm, bp, bm);
}

// kappa4 of the voxel at bit i from kappa4d's planes.
BS_HD int kappa4_at(const uint32_t *T0, const uint32_t *Tp, const uint32_t *Tm, uint32_t bp, uint32_t bm, int i)
{
    const int k0 = bits_at<4>(T0, i) - 5, kp = bits_at<4>(Tp, i) - 5, km = bits_at<4>(Tm, i) - 5;
    return k0 - (int)((bp >> i) & 1u) * kp - (int)((bm >> i) & 1u) * km;
}

// 2D: w[dy+1][dx+1]; kappa = 1 - F + Q with F faces (of 4) and Q squares
// (of 4).  Each face pairs with a square containing it: (1 - f) + q with
// q => f is the bit ~f | q, so kappa = X[0] + X[1] + 2 X[2] - 3 where
// X[0] + X[1] + 2 X[2] is the sum of the four chain bits.  Returns the
// nonzero mask and X.
BS_HD uint32_t kappa2d(const uint32_t w[3][3], uint32_t X[3])
{
    const uint32_t ex0 = w[1][0], ex1 = w[1][2], ey0 = w[0][1], ey1 = w[2][1];
    // square (y side a, x side b) = ey[a] & ex[b] & w[2a][2b]
    const uint32_t b0 = ~ex0 | (ey0 & w[0][0]);   // -x with square (0,0)
    const uint32_t b1 = ~ex1 | (ey1 & w[2][2]);   // +x with square (1,1)
    const uint32_t b2 = ~ey0 | (ex1 & w[0][2]);   // -y with square (0,1)
    const uint32_t b3 = ~ey1 | (ex0 & w[2][0]);   // +y with square (1,0)
    full_add(b0, b1, b2, X[0], X[2]);
    X[1] = b3;
    // sum == 3 iff X[2] and exactly one of X[0], X[1] (X[0] + X[1] <= 2)
    return ~(X[2] & (X[0] ^ X[1]));
}

}  // namespace bs
}  // namespace ecc
