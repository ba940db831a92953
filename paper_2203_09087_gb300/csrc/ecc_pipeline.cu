// ecc_pipeline.cu -- the paper's GPU-only pipeline (Sec. 4, Table 2): an
// image resident in device memory goes through `iterations` rounds of
// (1) its ECC at given thresholds and (2) a separable smoothing filter, and
// never leaves the device.
//
// The filter is a discrete convolution, one pass per axis (last axis first),
// with the caller's taps (the paper uses a 13-tap Gaussian) and half-sample
// symmetric reflection at the borders.  Every output is the taps' products
// summed in tap order with float32 rounding after each multiply and each add
// (no fused multiply-add), so the result is reproducible bit for bit by any
// implementation that follows the same order.
//
// 2D images with at most 255 levels take one fused kernel per round (below:
// the image read once and written once per round).  Otherwise the ECC step
// is ecc_compute_levels (quantize to level indices, stencil, scan) and the
// smoothing ping-pongs between the image and a float32 buffer of the plan.
// Everything is enqueued on one stream; nothing waits on the host.
#include <cuda_runtime.h>

#include <algorithm>

#include "ecc_bitslice.cuh"
#include "ecc_internal.h"
#include "ecc_levels.cuh"
#include "ecc_plan.h"
#include "ecc_scan_block.cuh"
#include "ecc_walk.cuh"
#include "ecc_walk2.cuh"

namespace ecc {
ecc_status levels_prepare(ecc_plan_s *p, const ecc_image *img, int32_t m, Geom *g);
cudaError_t levels_enqueue(ecc_plan_s *p, const Geom &g, const float *d_levels, int32_t m, cudaStream_t s);
}  // namespace ecc

namespace ecc {
namespace {

constexpr int kMaxTaps = 33;
constexpr int kBlurThreads = 256;

struct Taps {
    float w[kMaxTaps];
    int32_t n;  // odd
};

struct BlurArgs {
    const float *in;
    float *out;
    int64_t nx, ny, nz;
    int64_t in_sy, in_sz;    // element strides
    int64_t out_sy, out_sz;
    int32_t axis;            // 0 = x, 1 = y, 2 = z
};

// Half-sample symmetric reflection into [0, n) (rarely taken: borders only).
__device__ __forceinline__ int64_t reflect(int64_t j, int64_t n)
{
    int64_t p = j % (2 * n);
    if (p < 0) p += 2 * n;
    return p >= n ? 2 * n - 1 - p : p;
}

// One pass along `axis`: threads over x, one row (y, z) per block row, so no
// per-element index division; interior outputs read their taps directly.
__global__ void __launch_bounds__(kBlurThreads) blur_kernel(const BlurArgs a, const Taps t)
{
    const int r = t.n / 2;
    const int64_t n_axis = a.axis == 0 ? a.nx : (a.axis == 1 ? a.ny : a.nz);
    const int64_t stride = a.axis == 0 ? 1 : (a.axis == 1 ? a.in_sy : a.in_sz);
    const int64_t rows = a.ny * a.nz;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const int64_t z = row / a.ny, y = row - z * a.ny;
        for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.nx;
             x += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c = a.axis == 0 ? x : (a.axis == 1 ? y : z);
            const float *base = a.in + z * a.in_sz + y * a.in_sy + x - c * stride;   // coordinate 0 of the axis
            float acc = 0.0f;
            if (c >= r && c + r < n_axis) {
                const float *q = base + (c - r) * stride;
                for (int k = 0; k < t.n; ++k) acc = __fadd_rn(acc, __fmul_rn(t.w[k], __ldg(q + k * stride)));
            } else {
                for (int k = -r; k <= r; ++k)
                    acc = __fadd_rn(acc, __fmul_rn(t.w[k + r], __ldg(base + reflect(c + k, n_axis) * stride)));
            }
            a.out[z * a.out_sz + y * a.out_sy + x] = acc;
        }
    }
}

// Copies the round's ECC (m entries of stage) into row *row of out and
// advances the row counter; one block, so the counter moves after the copy.
__global__ void __launch_bounds__(256) store_row(const long long *stage, int64_t *out, int32_t m, int *row)
{
    const int64_t r = *row;
    for (int i = threadIdx.x; i < m; i += blockDim.x) out[r * m + i] = stage[i];
    __syncthreads();
    if (threadIdx.x == 0) *row = (int)(r + 1);
}

// ---------------------------------------------------------------- fused 2D round
//
// One kernel per round for 2D images with at most 255 levels: every CTA
// reads a float32 tile of the current image once, with the filter's halo
// (r pixels, at least 1 for the stencil) reflected at the image border, and
// from shared memory
//   * maps the tile and a one-pixel ring to level indices (the Eytzinger
//     search of ecc_levels.cuh) and counts the cells each pixel introduces
//     with the bit-sliced 2D walker (one warp: 4 windows of 30 columns x 8
//     chunks of 8 rows), into shared int32 bins flushed once per CTA;
//   * runs the filter's x pass over the tile's rows plus r above and below,
//     then the y pass, with the same tap order and rounding as blur_kernel,
//     and writes the smoothed tile (the next round's image) to the other
//     buffer.
// The last CTA scans the bins (ecc_scan_block.cuh), stores the round's ECC
// row and advances the round counter, which also tells every CTA of the
// next round which buffer holds its image.  HBM traffic per round: the
// image read once plus the halo, and written once.
constexpr int kFTX = 120;             // output columns per tile (4 windows of 30)
constexpr int kFTYBig = 64;           // output rows per tile (images that fill the GPU)
constexpr int kFTYSmall = 32;         // output rows per tile when 64-row tiles leave SMs idle
constexpr int kFusedThreads = 256;
constexpr int kStencilWarps = 2;                         // warps counting cells while the others filter

struct FusedArgs {
    float *img, *tmp;                 // the image and the plan's scratch image
    int64_t img_sy, tmp_sy;           // row pitches (elements)
    int32_t nx, ny;
    const float *levels;
    int32_t m;                        // levels (at most 255)
    int32_t nbins;                    // the plan's bins (>= m + 1)
    unsigned long long *acc;
    long long *stage;                 // the scanned ECC (nbins)
    int64_t *out;                     // [iterations][m]
    int *round;                       // rounds done (device)
    unsigned int *done;               // finished CTAs of this launch (zero between launches)
    unsigned int *status;
    int32_t tiles_x;
};

// Index j reflected into [0, n) (half-sample symmetric), for j in range
// returned as is; 32-bit (images of the fused path are below 2^30 a side).
__device__ __forceinline__ int reflect32(int j, int n)
{
    if (j >= 0 && j < n) return j;
    int p = j % (2 * n);
    if (p < 0) p += 2 * n;
    return p >= n ? 2 * n - 1 - p : p;
}

// acc = sum over taps k of w[k] * q[k * stride], in tap order, float32
// rounding after every product and sum (as blur_kernel); NT > 0: NT taps
// known at compile time (unrolled), NT = 0: t.n taps.
template <int NT>
__device__ __forceinline__ float tap_sum(const Taps &t, const float *q, int stride)
{
    float acc = 0.0f;
    if constexpr (NT > 0) {
#pragma unroll
        for (int k = 0; k < NT; ++k) acc = __fadd_rn(acc, __fmul_rn(t.w[k], q[k * stride]));
    } else {
        for (int k = 0; k < t.n; ++k) acc = __fadd_rn(acc, __fmul_rn(t.w[k], q[k * stride]));
    }
    return acc;
}

template <bool TOP, int NT, int kFTY>
__global__ void __launch_bounds__(kFusedThreads) fused_round2d_kernel(const FusedArgs a, const Taps t)
{
    constexpr int kChunkRows = kFTY / (8 * kStencilWarps);  // rows a stencil lane walks (4 windows x chunks)
    extern __shared__ __align__(16) unsigned char fsm[];
    const int r = (NT > 0 ? NT : t.n) / 2, R = r > 0 ? r : 1;  // filter radius, tile halo
    const int FW = kFTX + 2 * R, FH = kFTY + 2 * R;  // float tile with halo
    float *ftile = reinterpret_cast<float *>(fsm);                   // [FH][FW]
    float *hbuf = ftile + FH * FW;                                   // [kFTY + 2r][kFTX]
    unsigned char *qbuf = reinterpret_cast<unsigned char *>(hbuf + (kFTY + 2 * r) * kFTX);  // [kFTY + 2][4][32]
    float *tree = reinterpret_cast<float *>(qbuf + (kFTY + 2) * 128);  // 255 nodes
    int *hist = reinterpret_cast<int *>(tree + 256);                  // [nbins]
    __shared__ int s_round, s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) s_round = *a.round;
    for (int k = tid; k < 255; k += kFusedThreads) tree[k] = lv::padded_level(a.levels, a.m, lv::eytz_rank_of_node<8>(k));
    for (int i = tid; i < a.nbins; i += kFusedThreads) hist[i] = 0;
    if (blockIdx.x == 0)
        for (int i = tid + 1; i < a.m; i += kFusedThreads)
            if (!(a.levels[i - 1] <= a.levels[i])) atomicOr(a.status, DEV_LEVELS);
    __syncthreads();
    const bool odd = s_round & 1;
    const float *src = odd ? a.tmp : a.img;
    float *dst = odd ? a.img : a.tmp;
    const int64_t src_sy = odd ? a.tmp_sy : a.img_sy, dst_sy = odd ? a.img_sy : a.tmp_sy;
    const int x0 = (int)(blockIdx.x % a.tiles_x) * kFTX, y0 = (int)(blockIdx.x / a.tiles_x) * kFTY;

    // 1. the float tile, reflected at the image border (Sec. 4's filter):
    //    a warp per four rows, lanes along them, every load of the four rows
    //    issued before the first store (FW <= 152: at most 5 per row)
    constexpr int kRowsIn = 4;
    for (int ty = kRowsIn * warp; ty < FH; ty += kRowsIn * (kFusedThreads / 32)) {
        float v[kRowsIn][5];
#pragma unroll
        for (int h = 0; h < kRowsIn; ++h) {
            const int yy = ty + h < FH ? ty + h : ty;
            const float *srow = src + (int64_t)reflect32(y0 - R + yy, a.ny) * src_sy;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const int tx = lane + 32 * j;
                v[h][j] = tx < FW ? __ldg(srow + reflect32(x0 - R + tx, a.nx)) : 0.0f;
            }
        }
#pragma unroll
        for (int h = 0; h < kRowsIn; ++h)
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const int tx = lane + 32 * j;
                if (ty + h < FH && tx < FW) ftile[(ty + h) * FW + tx] = v[h][j];
            }
    }
    __syncthreads();
    // 2. level indices of the tile and a one-pixel ring, laid out per window
    //    (window w holds tile columns 30w-1 .. 30w+30) so a lane reads its
    //    window with two aligned 16-byte loads; pixels outside the image are
    //    missing to the walker, their index is never read as a value
    //    (four searches per thread at a time: each is a chain of 8
    //    dependent shared loads, so independent chains hide one another)
    constexpr int kQ = (kFTY + 2) * 128, kQU = 4;
    for (int i0 = tid; i0 < kQ; i0 += kQU * kFusedThreads) {
        float v[kQU];
#pragma unroll
        for (int u = 0; u < kQU; ++u) {
            const int i = i0 + u * kFusedThreads;
            const int qy = i >> 7, w = (i >> 5) & 3, j = i & 31;
            v[u] = i < kQ ? ftile[(qy - 1 + R) * FW + 30 * w - 1 + j + R] : 0.0f;
        }
        int q[kQU];
#pragma unroll
        for (int u = 0; u < kQU; ++u) q[u] = lv::lower_bound_count<8, false>(tree, a.m, v[u]);
#pragma unroll
        for (int u = 0; u < kQU; ++u)
            if (i0 + u * kFusedThreads < kQ) qbuf[i0 + u * kFusedThreads] = (unsigned char)q[u];
    }
    // 3. the x pass over rows -r .. kFTY + r - 1 of the tile; with the taps
    //    known, a thread makes 4 neighbouring outputs from 3 + NT loaded
    //    values (the same sums, in the same order)
    if constexpr (NT > 0) {
        constexpr int NX = 4, NV = NX + NT - 1;
        for (int i = tid; i < (kFTY + 2 * r) * (kFTX / NX); i += kFusedThreads) {
            const int hy = i / (kFTX / NX), hx = (i - hy * (kFTX / NX)) * NX;
            const float *q = ftile + (hy + R - r) * FW + hx + R - r;
            float v[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) v[j] = q[j];
#pragma unroll
            for (int o = 0; o < NX; ++o) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < NT; ++k) acc = __fadd_rn(acc, __fmul_rn(t.w[k], v[o + k]));
                hbuf[hy * kFTX + hx + o] = acc;
            }
        }
    } else {
        for (int i = tid; i < (kFTY + 2 * r) * kFTX; i += kFusedThreads) {
            const int hy = i / kFTX, hx = i - hy * kFTX;
            hbuf[i] = tap_sum<NT>(t, ftile + (hy + R - r) * FW + hx + R - r, 1);
        }
    }
    __syncthreads();
    if (warp < kStencilWarps) {
        // 4. the cell count of this round's image (the first kStencilWarps
        //    warps; lane l of them walks window l mod 4 of row chunk l / 4)
        const int w = lane & 3, c = (warp * 32 + lane) >> 2;
        const int64_t xw = (int64_t)x0 + 30 * w - 1;          // image column of window bit 0
        const uint32_t xex = walk::x_exist_mask(xw, a.nx);
        const uint32_t out_x = xex & 0x7ffffffeu;
        const int yb = y0 + kChunkRows * c, ye = yb + kChunkRows;  // output rows [yb, ye)
        const walk::Bins bins{hist, a.acc, 0, a.nbins, 0, a.status};
        const walk3::Mul mu = walk3::make_mul();
        // row gy as 8 planes and the existence plane (rows outside the
        // image all missing)
        auto planes = [&](int gy, uint32_t *P) {
            const uint4 *q = reinterpret_cast<const uint4 *>(qbuf + ((gy - y0 + 1) * 4 + w) * 32);
            const uint4 q0 = q[0], q1 = q[1];
            const uint32_t raw[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
            walk3::transpose_u8(raw, P, mu);
            P[8] = gy >= 0 && gy < a.ny ? ~xex : 0xffffffffu;
        };
        uint32_t P[9];
        planes(yb - 1, P);
        walk2::Walk<8, TOP> wk;
        wk.begin(P, mu);
        for (int y1 = yb; y1 <= ye; ++y1) {
            uint32_t B[9];
            planes(y1, B);
            const unsigned char *vrow = qbuf + ((y1 - 1 - y0 + 1) * 4 + w) * 32;
            wk.step(B, y1 - 1 >= yb && y1 - 1 < a.ny, out_x, mu, [&](uint32_t mm, const uint32_t *X) {
                walk2::emit2(mm, X, [&](int i) { return (int)vrow[i]; }, [&](int v, int k) { bins.add(v, k); });
            });
        }
    } else {
        // 5. the y pass, written to the other buffer (the other warps); with the
        //    taps known, 4 outputs down a column per thread
        if constexpr (NT > 0) {
            constexpr int NY = 4, NV = NY + NT - 1;
            for (int i = tid - 32 * kStencilWarps; i < (kFTY / NY) * kFTX; i += kFusedThreads - 32 * kStencilWarps) {
                const int oy = (i / kFTX) * NY, ox = i - (i / kFTX) * kFTX;
                const int gx = x0 + ox;
                const float *q = hbuf + oy * kFTX + ox;
                float v[NV];
#pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = q[j * kFTX];
#pragma unroll
                for (int o = 0; o < NY; ++o) {
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k < NT; ++k) acc = __fadd_rn(acc, __fmul_rn(t.w[k], v[o + k]));
                    const int gy = y0 + oy + o;
                    if (gy < a.ny && gx < a.nx) dst[gy * dst_sy + gx] = acc;
                }
            }
        } else {
            for (int i = tid - 32 * kStencilWarps; i < kFTY * kFTX; i += kFusedThreads - 32 * kStencilWarps) {
                const int oy = i / kFTX, ox = i - oy * kFTX;
                const int gy = y0 + oy, gx = x0 + ox;
                if (gy >= a.ny || gx >= a.nx) continue;
                dst[gy * dst_sy + gx] = tap_sum<NT>(t, hbuf + oy * kFTX + ox, kFTX);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < a.nbins; i += kFusedThreads)
        if (hist[i]) atomicAdd(a.acc + i, (unsigned long long)(long long)hist[i]);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
        if (s_last) {
            *a.done = 0u;
            __threadfence();
        }
    }
    __syncthreads();
    if (s_last) {
        scan_bins<kFusedThreads>(a.acc, a.stage, nullptr, a.nbins, tid);
        __syncthreads();
        int64_t *row = a.out + (int64_t)s_round * a.m;
        for (int i = tid; i < a.m; i += kFusedThreads) row[i] = a.stage[i];
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            *a.round = s_round + 1;
        }
    }
}

size_t fused_smem(int ntaps, int nbins, int kFTY)
{
    const int r = ntaps / 2, R = r > 0 ? r : 1;
    return sizeof(float) * (size_t)((kFTY + 2 * R) * (kFTX + 2 * R) + (kFTY + 2 * r) * kFTX) +
           (size_t)(kFTY + 2) * 128 + sizeof(float) * 256 + sizeof(int) * (size_t)nbins;
}

cudaError_t blur_pass(const float *in, int64_t in_sy, int64_t in_sz, float *out, int64_t out_sy, int64_t out_sz,
                      const Geom &g, int axis, const Taps &t, cudaStream_t s)
{
    BlurArgs a{in, out, g.nx, g.ny, g.nz, in_sy, in_sz, out_sy, out_sz, axis};
    const int64_t bx = std::min<int64_t>((g.nx + kBlurThreads - 1) / kBlurThreads, 64);
    const int64_t by = std::min<int64_t>(g.ny * g.nz, 65535);
    blur_kernel<<<dim3((unsigned)bx, (unsigned)by), kBlurThreads, 0, s>>>(a, t);
    return cudaGetLastError();
}

}  // namespace
}  // namespace ecc

using namespace ecc;

extern "C" ecc_status ecc_pipeline_gaussian(ecc_plan_t p, const ecc_image *img, const float *h_taps, int32_t ntaps,
                                            int32_t iterations, const float *d_levels, int32_t m, int64_t *d_ecc,
                                            void *stream)
{
    if (!p) return invalid("ecc_pipeline_gaussian: NULL plan");
    if (!h_taps || ntaps < 1 || ntaps > kMaxTaps || ntaps % 2 == 0)
        return invalid("ecc_pipeline_gaussian: need an odd number of taps, at most 33");
    if (iterations < 0) return invalid("ecc_pipeline_gaussian: negative iteration count");
    if (!img || img->dtype != ECC_F32) return invalid("ecc_pipeline_gaussian: the image must be ECC_F32");
    if (!d_levels || (!d_ecc && iterations > 0)) return invalid("ecc_pipeline_gaussian: NULL levels or output");
    Geom g;
    ecc_status st = levels_prepare(p, img, m, &g);
    if (st != ECC_OK) return st;
    const int64_t nvox = g.nx * g.ny * g.nz;
    // scratch image plus the round counter
    st = p->ensure_aux(nvox * (int64_t)sizeof(float) + 256);
    if (st != ECC_OK) return st;
    if (iterations == 0) return ECC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Taps t{};
    t.n = ntaps;
    for (int i = 0; i < ntaps; ++i) t.w[i] = h_taps[i];

    float *im = const_cast<float *>(reinterpret_cast<const float *>(g.data));
    const int64_t im_sy = g.pitch_y / 4, im_sz = g.pitch_z / 4;
    float *tmp = reinterpret_cast<float *>(p->aux);
    int *row = reinterpret_cast<int *>(static_cast<unsigned char *>(p->aux) + (nvox * sizeof(float) + 255) / 256 * 256);
    const int64_t t_sy = g.nx, t_sz = g.nx * g.ny;
    const int axes = g.ndim;  // passes: x, y (, z)

    // 2D images with at most 255 levels: one fused kernel per round (the
    // image read once and written once); otherwise the round is the
    // float-threshold path and one filter kernel per axis.
    // tile height: 64 rows, or 32 when 64-row tiles would leave SMs idle
    // (a round is then as long as one CTA's chain of steps)
    const int fty = (int64_t)((g.nx + kFTX - 1) / kFTX) * ((g.ny + kFTYBig - 1) / kFTYBig) < 2 * (int64_t)p->num_sms
                        ? kFTYSmall
                        : kFTYBig;
    const size_t fsmem = fused_smem(ntaps, p->nbins, fty);
    const bool fused = g.ndim == 2 && m <= 255 && p->nbins <= 4096 && fsmem <= 220 * 1024 &&
                       g.nx <= (int64_t(1) << 30) && g.ny <= (int64_t(1) << 30);
    FusedArgs fa{};
    const bool top = p->d.complex_mode == ECC_TOPCELL_MIN;
    if (fused) {
        fa.img = im;
        fa.tmp = tmp;
        fa.img_sy = im_sy;
        fa.tmp_sy = t_sy;
        fa.nx = (int32_t)g.nx;
        fa.ny = (int32_t)g.ny;
        fa.levels = d_levels;
        fa.m = m;
        fa.nbins = p->nbins;
        fa.acc = p->acc;
        fa.stage = p->stage_ecc;
        fa.out = d_ecc;
        fa.round = row;
        fa.done = p->sched + 3;   // a word of the plan's scheduling block no stencil uses here
        fa.status = p->status;
        fa.tiles_x = (int32_t)((g.nx + kFTX - 1) / kFTX);
        if (fsmem > 48 * 1024) {
            const void *fns[8] = {(const void *)fused_round2d_kernel<false, 0, kFTYBig>,
                                  (const void *)fused_round2d_kernel<true, 0, kFTYBig>,
                                  (const void *)fused_round2d_kernel<false, 13, kFTYBig>,
                                  (const void *)fused_round2d_kernel<true, 13, kFTYBig>,
                                  (const void *)fused_round2d_kernel<false, 0, kFTYSmall>,
                                  (const void *)fused_round2d_kernel<true, 0, kFTYSmall>,
                                  (const void *)fused_round2d_kernel<false, 13, kFTYSmall>,
                                  (const void *)fused_round2d_kernel<true, 13, kFTYSmall>};
            for (const void *fn : fns) {
                cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
                if (e != cudaSuccess) return cuda_fail(e, "ecc_pipeline_gaussian: fused kernel attributes");
            }
        }
    }
    const int64_t fused_tiles = fused ? (int64_t)fa.tiles_x * ((g.ny + fty - 1) / fty) : 0;

    // One round -- ECC at the levels, its row stored, the filter passes --
    // captured once on the plan's side stream and launched `iterations`
    // times on the caller's stream (a round is six or more short kernels;
    // launched one by one they would be bound by host launch cost).
    auto round = [&](cudaStream_t cs) -> cudaError_t {
        if (fused) {
            // the paper's 13-tap filter with its taps unrolled, any other width looped
            const dim3 grid((unsigned)fused_tiles);
            auto go = [&](auto kern) { kern<<<grid, kFusedThreads, fsmem, cs>>>(fa, t); };
            if (fty == kFTYBig) {
                if (ntaps == 13)
                    top ? go(fused_round2d_kernel<true, 13, kFTYBig>) : go(fused_round2d_kernel<false, 13, kFTYBig>);
                else
                    top ? go(fused_round2d_kernel<true, 0, kFTYBig>) : go(fused_round2d_kernel<false, 0, kFTYBig>);
            } else {
                if (ntaps == 13)
                    top ? go(fused_round2d_kernel<true, 13, kFTYSmall>) : go(fused_round2d_kernel<false, 13, kFTYSmall>);
                else
                    top ? go(fused_round2d_kernel<true, 0, kFTYSmall>) : go(fused_round2d_kernel<false, 0, kFTYSmall>);
            }
            p->last_launches = 1;
            return cudaGetLastError();
        }
        cudaError_t e = levels_enqueue(p, g, d_levels, m, cs);
        if (e == cudaSuccess) {
            store_row<<<1, 256, 0, cs>>>(p->stage_ecc, d_ecc, m, row);
            e = cudaGetLastError();
        }
        // passes alternate image -> tmp -> image ...; an odd count ends with a copy back
        for (int ax = 0; ax < axes && e == cudaSuccess; ++ax) {
            if (ax % 2 == 0)
                e = blur_pass(im, im_sy, im_sz, tmp, t_sy, t_sz, g, ax, t, cs);
            else
                e = blur_pass(tmp, t_sy, t_sz, im, im_sy, im_sz, g, ax, t, cs);
        }
        if (e == cudaSuccess && axes % 2 == 1) {
            if (g.pitch_z == g.ny * g.pitch_y)   // slices contiguous: one copy of all rows
                e = cudaMemcpy2DAsync(im, g.pitch_y, tmp, g.nx * 4, g.nx * 4, g.ny * g.nz,
                                      cudaMemcpyDeviceToDevice, cs);
            else                                 // pitched slices: never touch the gaps between them
                for (int64_t z = 0; z < g.nz && e == cudaSuccess; ++z)
                    e = cudaMemcpy2DAsync(im + z * im_sz, g.pitch_y, tmp + z * t_sz, g.nx * 4, g.nx * 4, g.ny,
                                          cudaMemcpyDeviceToDevice, cs);
        }
        return e;
    };

    // the fused rounds alternate image -> scratch -> image ...: after an odd
    // number of them the result is in the scratch image
    auto finish = [&]() -> cudaError_t {
        if (!fused || iterations % 2 == 0) return cudaSuccess;
        return cudaMemcpy2DAsync(im, g.pitch_y, tmp, g.nx * 4, g.nx * 4, g.ny, cudaMemcpyDeviceToDevice, s);
    };
    cudaError_t e = cudaMemsetAsync(row, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_pipeline_gaussian");
    if (iterations < 4) {   // too few rounds to pay for a capture
        for (int32_t it = 0; it < iterations && e == cudaSuccess; ++it) e = round(s);
        if (e == cudaSuccess) e = finish();
        if (e != cudaSuccess) return cuda_fail(e, "ecc_pipeline_gaussian");
        return ECC_OK;
    }
    // the executable graph of the previous call must have finished before it goes
    if (p->pipe_exec) {
        e = cudaEventSynchronize(p->pipe_done);
        cudaGraphExecDestroy(p->pipe_exec);
        p->pipe_exec = nullptr;
        if (e != cudaSuccess) return cuda_fail(e, "ecc_pipeline_gaussian: previous run");
    }
    cudaStream_t cs = p->copy_stream;
    cudaGraph_t graph = nullptr;
    // events recorded by graph nodes cannot be timed: the captured round
    // leaves ECC_FLAG_TIME_KERNELS out
    const uint32_t flags = p->d.flags;
    p->d.flags &= ~(uint32_t)ECC_FLAG_TIME_KERNELS;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        const cudaError_t er = round(cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (er != cudaSuccess) e = er;
    }
    p->d.flags = flags;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->pipe_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess && !p->pipe_done) e = cudaEventCreateWithFlags(&p->pipe_done, cudaEventDisableTiming);
    for (int32_t it = 0; it < iterations && e == cudaSuccess; ++it) e = cudaGraphLaunch(p->pipe_exec, s);
    if (e == cudaSuccess) e = finish();
    if (e == cudaSuccess) e = cudaEventRecord(p->pipe_done, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "ecc_pipeline_gaussian: graph");
    }
    return ECC_OK;
}
