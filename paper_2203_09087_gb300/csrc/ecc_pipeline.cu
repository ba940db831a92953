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
// The ECC step is ecc_compute_levels (quantize to level indices, stencil,
// scan); the smoothing ping-pongs between the image and a float32 buffer of
// the plan.  Everything is enqueued on one stream; nothing waits on the host.
#include <cuda_runtime.h>

#include <algorithm>

#include "ecc_internal.h"
#include "ecc_plan.h"

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

    // One round -- ECC at the levels, its row stored, the filter passes --
    // captured once on the plan's side stream and launched `iterations`
    // times on the caller's stream (a round is six or more short kernels;
    // launched one by one they would be bound by host launch cost).
    auto round = [&](cudaStream_t cs) -> cudaError_t {
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

    cudaError_t e = cudaMemsetAsync(row, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_pipeline_gaussian");
    if (iterations < 4) {   // too few rounds to pay for a capture
        for (int32_t it = 0; it < iterations && e == cudaSuccess; ++it) e = round(s);
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
    if (e == cudaSuccess) e = cudaEventRecord(p->pipe_done, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "ecc_pipeline_gaussian: graph");
    }
    return ECC_OK;
}
