// ecc_levels.cu -- float32 images at given thresholds (Eq. 1 with the t_i
// given): ECC_i = chi(K_{<= t_i}) for ascending levels t_0 <= ... <= t_{m-1}.
//
// The paper's datasets are float32 and its kernel bins voxel values as
// integers (Algorithm 2).  Here every voxel is mapped to the number of levels
// strictly below its value (its lower bound in the level list; NaN maps to m,
// above every level).  The map is monotone, so it commutes with the max over
// a cell's vertices (vertex complex) and the min over its cofaces (top-cell
// complex): a cell lies in K_{<= t_i} exactly when its mapped value is <= i.
// The integer stencil and scan then give the ECC at every threshold; mapped
// value m (above every level) is counted in a bin that is not returned.
//
// The quantize kernel is a streaming pass (4 bytes read, 1 or 2 written per
// voxel) with an unrolled fixed-step lower-bound search, the same on every
// lane, over the levels laid out as a breadth-first search tree in shared
// memory up to 16383 levels, over the sorted global level array (reads past
// m taken as +infinity) beyond.  Its output is a dense copy with rows padded
// to 16 bytes, so the stencil takes the TMA path.
#include <cuda_runtime.h>

#include <algorithm>

#include "ecc_internal.h"
#include "ecc_levels.cuh"
#include "ecc_plan.h"

namespace ecc {
namespace {

constexpr int kQuantThreads = 256;
constexpr int kInFlight = 8;  // voxels a lane searches at once

struct QuantArgs {
    const unsigned char *src;
    int64_t nx, rows, ny;          // rows = nz * ny
    int64_t sp_y, sp_z;            // source pitches (bytes)
    const float *levels;
    int32_t m;
    unsigned char *dst;
    int64_t dp_y, dp_z;            // destination pitches (bytes)
    unsigned int *status;
};

using lv::eytz_rank_of_node;
using lv::lower_bound_count;
using lv::padded_level;

template <typename OutT, int L, bool GLOBAL>
__global__ void __launch_bounds__(kQuantThreads, 4) quantize_kernel(const QuantArgs a)
{
    extern __shared__ float tree_s[];
    const float *lv = a.levels;
    if (!GLOBAL) {
        constexpr int N = (1 << L) - 1;
        for (int k = threadIdx.x; k < N; k += blockDim.x) tree_s[k] = padded_level(a.levels, a.m, eytz_rank_of_node<L>(k));
        __syncthreads();
        lv = tree_s;
    }
    // the first block checks that the levels ascend
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x + 1; i < a.m; i += blockDim.x)
            if (!(a.levels[i - 1] <= a.levels[i])) atomicOr(a.status, DEV_LEVELS);
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < a.rows; r += nwarps) {
        const int64_t z = r / a.ny, y = r - z * a.ny;
        const float *row = reinterpret_cast<const float *>(a.src + z * a.sp_z + y * a.sp_y);
        OutT *out = reinterpret_cast<OutT *>(a.dst + z * a.dp_z + y * a.dp_y);
        int x = lane;
        const int nx = (int)a.nx;
        // kInFlight voxels per lane at once: their loads and their searches
        // (chains of L dependent shared loads) overlap
        for (; x + 32 * (kInFlight - 1) < nx; x += 32 * kInFlight) {
            float v[kInFlight];
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) v[u] = __ldg(row + x + 32 * u);
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) out[x + 32 * u] = (OutT)lower_bound_count<L, GLOBAL>(lv, a.m, v[u]);
        }
        for (; x < nx; x += 32) out[x] = (OutT)lower_bound_count<L, GLOBAL>(lv, a.m, __ldg(row + x));
    }
}

template <typename OutT, int LOG, bool GLOBAL>
cudaError_t launch_quantize(const QuantArgs &a, int64_t blocks, cudaStream_t s)
{
    const size_t smem = GLOBAL ? 0 : sizeof(float) * (size_t)((1 << LOG) - 1);
    auto k = quantize_kernel<OutT, LOG, GLOBAL>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)blocks, kQuantThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// The smallest tree (2^LOG - 1 >= m) among LOG = 8, 11, 14 in shared memory;
// LOG = 16 walks the sorted global array by the same node-to-rank map.
template <typename OutT>
cudaError_t launch_quantize_any(const QuantArgs &a, int64_t blocks, cudaStream_t s)
{
    if (a.m <= 255) return launch_quantize<OutT, 8, false>(a, blocks, s);
    if (a.m <= 2047) return launch_quantize<OutT, 11, false>(a, blocks, s);
    if (a.m <= 16383) return launch_quantize<OutT, 14, false>(a, blocks, s);
    return launch_quantize<OutT, 16, true>(a, blocks, s);
}

}  // namespace
}  // namespace ecc

namespace ecc {

// Checks a float32 image and level count against the plan and sizes the
// staging copy; on success fills the image's geometry.
ecc_status levels_prepare(ecc_plan_s *p, const ecc_image *img, int32_t m, Geom *g)
{
    if (m < 1 || m > 65535) return invalid("ecc_compute_levels: the number of levels must be in [1, 65535]");
    if (p->d.lo != 0 || p->d.hi < m)
        return invalid("ecc_compute_levels: the plan must cover levels [0, m] (lo = 0, hi >= m)");
    int64_t nvox = 0;
    ecc_status st = image_geom(img, ECC_F32, p->d.max_voxels, g, &nvox, false);
    if (st != ECC_OK) return st;
    if (reinterpret_cast<uintptr_t>(g->data) % 4 || g->pitch_y % 4 || g->pitch_z % 4)
        return invalid("ecc_compute_levels: float32 image must be 4-byte aligned");
    const int es = p->d.dtype == ECC_U16 ? 2 : 1;
    const int64_t dp_y = (g->nx * es + 15) / 16 * 16;
    return p->ensure_stage(g->nz * g->ny * dp_y);
}

// Quantize, stencil and scan; the ECC (nbins entries) is left in the plan's
// stage_ecc.  Only stream operations (capturable into a graph).
cudaError_t levels_enqueue(ecc_plan_s *p, const Geom &g, const float *d_levels, int32_t m, cudaStream_t s)
{
    const int es = p->d.dtype == ECC_U16 ? 2 : 1;
    const int64_t dp_y = (g.nx * es + 15) / 16 * 16;
    const int64_t dp_z = g.ny * dp_y;
    QuantArgs a{};
    a.src = g.data;
    a.nx = g.nx;
    a.ny = g.ny;
    a.rows = g.nz * g.ny;
    a.sp_y = g.pitch_y;
    a.sp_z = g.pitch_z;
    a.levels = d_levels;
    a.m = m;
    a.dst = p->stage;
    a.dp_y = dp_y;
    a.dp_z = dp_z;
    a.status = p->status;
    const int64_t rows_per_block = kQuantThreads / 32;
    const int64_t blocks = std::min<int64_t>((a.rows + rows_per_block - 1) / rows_per_block,
                                             (int64_t)p->num_sms * 8);
    cudaError_t e = es == 1 ? launch_quantize_any<unsigned char>(a, blocks, s)
                            : launch_quantize_any<unsigned short>(a, blocks, s);
    p->last_launches = 1;
    Geom dg = g;
    dg.data = p->stage;
    dg.esize = es;
    dg.pitch_y = dp_y;
    dg.pitch_z = dp_z;
    HistDst h{p->acc, 0, p->nbins};
    if (p->d.flags & ECC_FLAG_COUNT_EMITTED) h.emitted = p->emitted;
    // the stencil's last CTA scans small histograms itself (fs.done)
    FusedScan fs{p->stage_ecc, nullptr, false};
    if (e == cudaSuccess) e = launch_stencil(p, dg, 0, g.ndim == 3 ? g.nz : g.ny, h, s, &fs);
    if (e == cudaSuccess && !fs.done) {
        e = launch_scan(p->acc, p->stage_ecc, nullptr, 1, p->nbins, p->scan_ws(), p->status, s);
        ++p->last_launches;
    }
    return e;
}

}  // namespace ecc

using namespace ecc;

extern "C" ecc_status ecc_compute_levels(ecc_plan_t p, const ecc_image *img, const float *d_levels, int32_t m,
                                         int64_t *d_ecc, void *stream)
{
    if (!p) return invalid("ecc_compute_levels: NULL plan");
    if (!d_levels || !d_ecc) return invalid("ecc_compute_levels: NULL levels or output");
    Geom g;
    ecc_status st = levels_prepare(p, img, m, &g);
    if (st != ECC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = levels_enqueue(p, g, d_levels, m, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ecc, p->stage_ecc, sizeof(int64_t) * (size_t)m, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_levels");
    return ECC_OK;
}
