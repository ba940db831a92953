// Host harness exposing the bit-sliced helpers of the CUDA path to the CPU
// tests (tests/test_bitslice_core.py).  Built with g++; no CUDA needed.
#include <stdint.h>

#include "ecc_bitlogic.cuh"
#include "ecc_bitslice.cuh"

using namespace ecc::bs;

extern "C" {

void h_transpose_u8(const uint32_t *r, uint32_t *p) { transpose_u8(r, p); }
void h_transpose_u16(const uint32_t *r, uint32_t *p) { transpose_u16(r, p); }
uint32_t h_ge8(const uint32_t *a, const uint32_t *b) { return ge<8>(a, b); }
uint32_t h_ge16(const uint32_t *a, const uint32_t *b) { return ge<16>(a, b); }

// w: 27 masks in [dz][dy][dx] order; writes T[4] (kappa = T - 5); returns nonzero mask
uint32_t h_kappa3d(const uint32_t *w27, uint32_t *T)
{
    uint32_t w[3][3][3];
    for (int i = 0; i < 27; ++i) w[i / 9][(i / 3) % 3][i % 3] = w27[i];
    return kappa3d(w, T);
}

// n words per input: w27[i * n + j] is input i of word j; T[k * n + j], nz[j]
void h_kappa3d_many(const uint32_t *w27, int64_t n, uint32_t *T, uint32_t *nz)
{
    for (int64_t j = 0; j < n; ++j) {
        uint32_t w[3][3][3], t[4];
        for (int i = 0; i < 27; ++i) w[i / 9][(i / 3) % 3][i % 3] = w27[i * n + j];
        nz[j] = kappa3d(w, t);
        for (int k = 0; k < 4; ++k) T[k * n + j] = t[k];
    }
}

// w81: 81 masks in [dw][dz][dy][dx] order; writes kappa4 of each of the 32 voxels; returns nonzero mask
uint32_t h_kappa4d(const uint32_t *w81, int32_t *kappa)
{
    uint32_t w[3][3][3][3], T0[4], Tp[4], Tm[4], bp, bm;
    for (int i = 0; i < 81; ++i) (&w[0][0][0][0])[i] = w81[i];
    const uint32_t nz = kappa4d(w, T0, Tp, Tm, bp, bm);
    for (int i = 0; i < 32; ++i) kappa[i] = kappa4_at(T0, Tp, Tm, bp, bm, i);
    return nz;
}

// kappa4_nonzero for 32 voxels given as per-voxel counts (T0, Tp, Tm in
// 0..12) and w-wins; returns the nonzero mask
uint32_t h_kappa4_nonzero(const int32_t *t0, const int32_t *tp, const int32_t *tm, const int32_t *bp,
                          const int32_t *bm)
{
    uint32_t T0[4] = {0, 0, 0, 0}, Tp[4] = {0, 0, 0, 0}, Tm[4] = {0, 0, 0, 0}, P = 0, M = 0;
    for (int i = 0; i < 32; ++i) {
        for (int k = 0; k < 4; ++k) {
            T0[k] |= (uint32_t)((t0[i] >> k) & 1) << i;
            Tp[k] |= (uint32_t)((tp[i] >> k) & 1) << i;
            Tm[k] |= (uint32_t)((tm[i] >> k) & 1) << i;
        }
        P |= (uint32_t)(bp[i] & 1) << i;
        M |= (uint32_t)(bm[i] & 1) << i;
    }
    return kappa4_nonzero(T0, Tp, Tm, P, M);
}

void h_count12(const uint32_t *x, uint32_t *o) { count12(x, o); }

// w: 9 masks in [dy][dx] order; writes X[3] (kappa = X0 + X1 + 2 X2 - 3); returns nonzero mask
uint32_t h_kappa2d(const uint32_t *w9, uint32_t *X)
{
    uint32_t w[3][3];
    for (int i = 0; i < 9; ++i) w[i / 3][i % 3] = w9[i];
    return kappa2d(w, X);
}


// ---- the 3D walker's bit logic (ecc_bitlogic.cuh) with multiply shifts and
// explicit three-input operations

void h_w3_transpose_u8(const uint32_t *r, uint32_t *p) { ecc::walk3::transpose_u8(r, p, ecc::walk3::make_mul()); }
void h_w3_transpose_u16(const uint32_t *r, uint32_t *p) { ecc::walk3::transpose_u16(r, p, ecc::walk3::make_mul()); }
uint32_t h_w3_ge8(const uint32_t *a, const uint32_t *b) { return ecc::walk3::ge<8>(a, b); }
uint32_t h_w3_ge16(const uint32_t *a, const uint32_t *b) { return ecc::walk3::ge<16>(a, b); }
void h_w3_count12(const uint32_t *x, uint32_t *o) { ecc::walk3::count12(x, o); }

// The walker's cell count from the 27 wins w[dz][dy][dx] (the centre unused),
// handed over in the walker's polarities; returns the nonzero mask, writes T.
uint32_t h_w3_kappa3(const uint32_t *w27, uint32_t out_x, uint32_t *T)
{
    uint32_t w[3][3][3];
    for (int i = 0; i < 27; ++i) w[i / 9][(i / 3) % 3][i % 3] = w27[i];
    uint32_t up[3][3], nW[3][3], sF[3], sD[3];
    for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx) {
            up[dy][dx] = w[2][dy][dx];
            nW[dy][dx] = ~w[0][dy][dx];
        }
    for (int dx = 0; dx < 3; ++dx) {
        sF[dx] = w[1][2][dx];
        sD[2 - dx] = ~w[1][0][dx];
    }
    return ecc::walk3::kappa3w(up, nW, ~w[1][1][0], w[1][1][2], sF, sD, out_x, T);
}

// The 2D walker's cell count from the 9 wins w[dy][dx] (centre unused), in
// the walker's polarities; returns the nonzero mask, writes X.
uint32_t h_w2_kappa2(const uint32_t *w9, uint32_t out_x, uint32_t *X)
{
    uint32_t w[3][3];
    for (int i = 0; i < 9; ++i) w[i / 3][i % 3] = w9[i];
    const uint32_t sW[3] = {~w[0][0], ~w[0][1], ~w[0][2]};
    return ecc::walk3::kappa2w(sW, ~w[1][0], w[1][2], w[2][0], w[2][1], w[2][2], out_x, X);
}

// The +-1 split of the emission: out[0] = pm, out[1] = plus
void h_split_pm1_2d(const uint32_t *X, uint32_t *out) { ecc::walk3::split_pm1_2d(X, out[0], out[1]); }
void h_split_pm1_3d(const uint32_t *T, uint32_t *out) { ecc::walk3::split_pm1_3d(T, out[0], out[1]); }
}
