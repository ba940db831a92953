// ecc_nd.cu -- images of up to four dimensions (d > 3: the paper's texture
// path stops at three, Sec. 5).  ecc_compute_nd forwards 2D and 3D images to
// ecc_compute; 4D images take the bit-sliced walker below.
//
// The per-voxel rule is the one of every other kernel here (Sec. 2.3,
// Algorithm 1 regrouped per voxel): a voxel p introduces a cell containing
// it when it beats every other vertex of the cell, and adds (-1)^dim of each
// such cell to the bin of its value.  In four dimensions the cells
// containing p are p + sum over a in A of {0, s_a e_a} for an axis subset A
// and signs s_A: 1 vertex, 8 edges, 24 squares, 32 cubes and 16 tesseracts.
// Ties go to the lower linear index (a neighbour later in memory is beaten
// on >=, an earlier one on >).  Vertex complex: a missing neighbour is never
// beaten (the cell does not exist).  Top-cell complex: comparisons reversed,
// a missing neighbour always beaten (the +infinity collar), and the count
// multiplied by (-1)^4 = +1.
#include <cuda_runtime.h>

#include <algorithm>

#include "ecc_bitslice.cuh"
#include "ecc_internal.h"
#include "ecc_plan.h"
#include "ecc_walk.cuh"

namespace ecc {
namespace {

// ------------------------------------------------------------ bit-sliced walker
//
// The star of a voxel splits along w into the cells of its own hyperplane
// and those cells extended to w+1 or w-1, so its count is
//   kappa4 = k3(W0) - b+ k3(W0 & W+) - b- k3(W0 & W-)
// with W0, W+, W- its wins over hyperplanes w, w+1, w-1, b+- its wins over
// its two w-neighbours and k3 the 3D count (bs::kappa4_nonzero).  Each warp
// takes one (z, 30-row tile, 30-column window) column over a chunk of w
// (or several partial tiles side by side): it holds slices (w, z-1..z+1),
// loads (w+1, z-1..z+1) at every step, and
// compares slices in blocks of nine directions (walk::slice_pair), each
// pair of voxels at most once per warp.  The wins over hyperplane w-1 are
// the complements carried from the step before.
constexpr int kWalk4Warps = 4;

struct Walk4Args {
    const unsigned char *data;
    int64_t n[4];        // w, z, y, x
    int64_t pitch[3];    // bytes: w, z, y
    int64_t items;       // w chunks x per_chunk
    int64_t chunk;       // hyperplanes per item
    int64_t per_chunk;   // items per w chunk: full_items, then the packed ones
    int64_t full_items;  // nz x full row tiles x windows
    int32_t ntx;         // windows of 30 columns
    int32_t nty_full;    // tiles of 30 rows
    int32_t remy;        // rows left below the full tiles (0..29)
    int32_t pack;        // partial tiles (remy rows + 2 halo lanes) per warp
    HistDst h;
    int32_t smem_hist, range_check;
    unsigned int *status;
};

template <typename T, bool TOP>
__global__ void __launch_bounds__(kWalk4Warps * 32) walk4d_kernel(const Walk4Args a)
{
    constexpr int K = 8 * sizeof(T), KP = K + 1;
    extern __shared__ int hist4w[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.smem_hist)
        for (int i = threadIdx.x; i < a.h.nbins; i += blockDim.x) hist4w[i] = 0;
    __syncthreads();
    const walk::Bins bins{a.smem_hist ? hist4w : nullptr, a.h.acc, a.h.lo, a.h.nbins, a.range_check, a.status};
    const int64_t nw = a.n[0], nz = a.n[1], ny = a.n[2], nx = a.n[3];
    const int64_t row_bytes = nx * (int64_t)sizeof(T);
    unsigned n_emitted = 0;
    for (int64_t item = (int64_t)blockIdx.x * kWalk4Warps + warp; item < a.items;
         item += (int64_t)gridDim.x * kWalk4Warps) {
        // Full items: lane l holds row 30 ty - 1 + l of column (z, tx).  Packed
        // items: the last remy rows of `pack` columns side by side, remy + 2
        // lanes each (a halo lane on either side), so a partial tile does not
        // take a whole warp.
        const int64_t ci = item / a.per_chunk;
        int64_t r = item - ci * a.per_chunk;
        const int64_t w0 = ci * a.chunk, w1 = w0 + a.chunk < nw ? w0 + a.chunk : nw;
        int64_t z, y;
        int tx;
        bool lane_out;
        if (r < a.full_items) {
            tx = (int)(r % a.ntx);
            r /= a.ntx;
            const int ty = (int)(r % a.nty_full);
            z = r / a.nty_full;
            y = (int64_t)ty * 30 - 1 + lane;
            lane_out = lane >= 1 && lane <= 30;
        } else {
            const int seg_len = a.remy + 2, seg = lane / seg_len, j = lane - seg * seg_len;
            const int64_t c = (r - a.full_items) * a.pack + seg;
            const bool valid = seg < a.pack && c < nz * a.ntx;
            z = valid ? c / a.ntx : 0;
            tx = valid ? (int)(c % a.ntx) : 0;
            y = valid ? (int64_t)a.nty_full * 30 - 1 + j : -2;   // -2: no row
            lane_out = valid && j >= 1 && j <= a.remy;
        }
        const int64_t xw = (int64_t)tx * 30 - 1;   // voxel of bit 0
        const uint32_t xm = walk::x_exist_mask(xw, nx);
        const uint32_t out = lane_out ? (xm & 0x7ffffffeu) : 0u;
        // this lane's row of slice (w, zz); a row outside the image is all missing
        auto load = [&](int64_t w, int64_t zz, uint32_t *P) {
            if ((uint64_t)w < (uint64_t)nw && (uint64_t)zz < (uint64_t)nz && (uint64_t)y < (uint64_t)ny) {
                const unsigned char *row = a.data + w * a.pitch[0] + zz * a.pitch[1] + y * a.pitch[2];
                uint32_t words[K + 1];
                const int sh = walk::load_row_words<K>(row, row_bytes, xw * (int64_t)sizeof(T), words);
                walk::planes_from_words<K>(words, sh, P);
                P[K] = ~xm;
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) P[k] = 0u;
                P[K] = 0xffffffffu;
            }
        };
        uint32_t Am[KP], A0[KP], Ap[KP];
        uint32_t C[3][3][3];   // wins of slice (w, z) over hyperplane w-1
        uint32_t unused[3][3];
        {
            uint32_t B0[KP];
            load(w0 - 1, z - 1, Am);
            load(w0 - 1, z, A0);
            load(w0 - 1, z + 1, Ap);
            load(w0, z, B0);
            walk::slice_pair<K, TOP, false, true>(Am, B0, unused, C[0]);
            walk::slice_pair<K, TOP, false, true>(A0, B0, unused, C[1]);
            walk::slice_pair<K, TOP, false, true>(Ap, B0, unused, C[2]);
#pragma unroll
            for (int k = 0; k < KP; ++k) A0[k] = B0[k];
            load(w0, z - 1, Am);
            load(w0, z + 1, Ap);
        }
        for (int64_t w = w0; w < w1; ++w) {
            // W0: wins of slice (w, z) in its hyperplane, as [dz][dy][dx]
            uint32_t W[3][3][3];
            walk::slice_pair<K, TOP, false, true>(Am, A0, unused, W[0]);
            walk::in_slice<K, TOP>(A0, W[1]);
            walk::slice_pair<K, TOP, true, false>(A0, Ap, W[2], unused);
            uint32_t T0[4], Tm[4], Tp[4];
            bs::kappa3d(W, T0);
            const uint32_t bm = C[1][1][1];
#pragma unroll
            for (int i = 0; i < 27; ++i) (&C[0][0][0])[i] &= (&W[0][0][0])[i];
            bs::kappa3d(C, Tm);
            // hyperplane w+1: W becomes W0 & W+, C the wins of (w+1, z) over w
            uint32_t B0[KP], Bm[KP], Bp[KP], fw[3][3];
            load(w + 1, z, B0);
            walk::slice_pair<K, TOP, true, true>(A0, B0, fw, C[1]);
            const uint32_t bp = fw[1][1];
#pragma unroll
            for (int i = 0; i < 9; ++i) (&W[1][0][0])[i] &= (&fw[0][0])[i];
            load(w + 1, z - 1, Bm);
            walk::slice_pair<K, TOP, true, false>(A0, Bm, fw, unused);
#pragma unroll
            for (int i = 0; i < 9; ++i) (&W[0][0][0])[i] &= (&fw[0][0])[i];
            load(w + 1, z + 1, Bp);
            walk::slice_pair<K, TOP, true, false>(A0, Bp, fw, unused);
#pragma unroll
            for (int i = 0; i < 9; ++i) (&W[2][0][0])[i] &= (&fw[0][0])[i];
            bs::kappa3d(W, Tp);
            walk::slice_pair<K, TOP, false, true>(Am, B0, unused, C[0]);
            walk::slice_pair<K, TOP, false, true>(Ap, B0, unused, C[2]);
            uint32_t m = bs::kappa4_nonzero(T0, Tp, Tm, bp, bm) & ~A0[K] & out;
            if (a.h.emitted) n_emitted += __popc(m);
            while (m) {
                const int i = __ffs(m) - 1;
                m &= m - 1u;
                // (-1)^4 = +1: the same sign in both complexes
                bins.add(bs::bits_at<K>(A0, i), bs::kappa4_at(T0, Tp, Tm, bp, bm, i));
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                Am[k] = Bm[k];
                A0[k] = B0[k];
                Ap[k] = Bp[k];
            }
        }
    }
    if (a.h.emitted) {
        const unsigned n = __reduce_add_sync(0xffffffffu, n_emitted);
        if (lane == 0 && n) atomicAdd(a.h.emitted, (unsigned long long)n);
    }
    __syncthreads();
    if (a.smem_hist)
        for (int i = threadIdx.x; i < a.h.nbins; i += blockDim.x)
            if (hist4w[i]) atomicAdd(a.h.acc + i, (unsigned long long)(long long)hist4w[i]);
}

template <typename T, bool TOP>
cudaError_t launch_walk4(Walk4Args a, int num_sms, size_t smem, cudaStream_t s)
{
    auto k = walk4d_kernel<T, TOP>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWalk4Warps * 32, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    // w chunks of c hyperplanes: an item costs c + 1 steps (one to fill the
    // state), each warp runs ceil(items / resident warps) items; take the c
    // with the least of (rounds x steps), the longest any warp runs.
    a.ntx = (int32_t)((a.n[3] + 29) / 30);
    a.nty_full = (int32_t)(a.n[2] / 30);
    a.remy = (int32_t)(a.n[2] % 30);
    a.pack = 32 / (a.remy + 2);
    a.full_items = a.n[1] * a.nty_full * a.ntx;
    a.per_chunk = a.full_items + (a.remy ? (a.n[1] * a.ntx + a.pack - 1) / a.pack : 0);
    const int64_t base = a.per_chunk;
    const int64_t resident = (int64_t)num_sms * per_sm * kWalk4Warps;
    int64_t best_c = a.n[0], best_cost = -1;
    // chunk counts k = 1, 2, ... until there are far more items than warps
    for (int64_t k = 1; k <= a.n[0]; ++k) {
        const int64_t c = (a.n[0] + k - 1) / k;
        const int64_t chunks = (a.n[0] + c - 1) / c;
        const int64_t rounds = (chunks * base + resident - 1) / resident;
        const int64_t cost = rounds * (c + 1);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_c = c;
        }
        if (chunks * base > 64 * resident) break;
    }
    a.chunk = best_c;
    a.items = ((a.n[0] + best_c - 1) / best_c) * base;
    const int64_t blocks =
        std::min<int64_t>((a.items + kWalk4Warps - 1) / kWalk4Warps, (int64_t)num_sms * per_sm);
    k<<<(unsigned)blocks, kWalk4Warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace
}  // namespace ecc

using namespace ecc;

extern "C" ecc_status ecc_compute_nd(ecc_plan_t p, const ecc_image_nd *img, int64_t *d_ecc, int64_t *d_vcec,
                                     void *stream)
{
    if (!p) return invalid("ecc_compute_nd: NULL plan");
    if (!img || !img->data) return invalid("ecc_compute_nd: NULL image");
    if (img->ndim < 2 || img->ndim > 4) return invalid("ecc_compute_nd: ndim must be 2, 3 or 4");
    if (img->ndim < 4) {
        ecc_image im{};
        im.data = img->data;
        im.ndim = img->ndim;
        im.dtype = img->dtype;
        for (int a = 0; a < img->ndim; ++a) im.dims[a] = img->dims[a];
        im.row_pitch = img->pitches[img->ndim - 2];
        im.slice_pitch = img->ndim == 3 ? img->pitches[0] : 0;
        return ecc_compute(p, &im, d_ecc, d_vcec, stream);
    }
    if (!d_ecc) return invalid("ecc_compute_nd: NULL output");
    if (img->dtype != p->d.dtype) return invalid("ecc_compute_nd: image dtype differs from the plan's dtype");
    const int es = img->dtype == ECC_U16 ? 2 : 1;
    Walk4Args a{};
    a.data = static_cast<const unsigned char *>(img->data);
    int64_t nvox = 1;
    for (int ax = 0; ax < 4; ++ax) {
        if (img->dims[ax] < 1 || img->dims[ax] > (int64_t(1) << 31)) return invalid("ecc_compute_nd: bad dim");
        a.n[ax] = img->dims[ax];
        nvox *= img->dims[ax];
        if (nvox > (int64_t(1) << 40)) return invalid("ecc_compute_nd: image too large");
    }
    if (nvox > p->d.max_voxels) {
        set_error("ecc_compute_nd: image has more voxels than the plan's max_voxels");
        return ECC_E_BUSY;
    }
    // dense strides by default; given pitches must hold the inner extent
    const int64_t dense[3] = {a.n[1] * a.n[2] * a.n[3] * es, a.n[2] * a.n[3] * es, a.n[3] * es};
    for (int ax = 0; ax < 3; ++ax) {
        a.pitch[ax] = img->pitches[ax] ? img->pitches[ax] : dense[ax];
        if (a.pitch[ax] % es) return invalid("ecc_compute_nd: pitch not a multiple of the element size");
    }
    if (a.pitch[2] < a.n[3] * es || a.pitch[1] < (a.n[2] - 1) * a.pitch[2] + a.n[3] * es ||
        a.pitch[0] < (a.n[1] - 1) * a.pitch[1] + (a.n[2] - 1) * a.pitch[2] + a.n[3] * es)
        return invalid("ecc_compute_nd: pitches smaller than the extents they span");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    a.h = HistDst{p->acc, p->d.lo, p->nbins};
    if (p->d.flags & ECC_FLAG_COUNT_EMITTED) a.h.emitted = p->emitted;
    a.range_check = !(p->d.flags & ECC_FLAG_NO_RANGE_CHECK);
    a.status = p->status;
    a.smem_hist = p->nbins <= kSmemBinsMax;
    const size_t smem = a.smem_hist ? sizeof(int) * (size_t)p->nbins : 0;
    const bool top = p->d.complex_mode == ECC_TOPCELL_MIN;
    cudaError_t e = es == 1 ? (top ? launch_walk4<unsigned char, true>(a, p->num_sms, smem, s)
                                   : launch_walk4<unsigned char, false>(a, p->num_sms, smem, s))
                            : (top ? launch_walk4<unsigned short, true>(a, p->num_sms, smem, s)
                                   : launch_walk4<unsigned short, false>(a, p->num_sms, smem, s));
    p->last_launches = 1;
    if (e == cudaSuccess) {
        e = launch_scan(p->acc, reinterpret_cast<long long *>(d_ecc), reinterpret_cast<long long *>(d_vcec), 1,
                        p->nbins, p->scan_ws(), p->status, s);
        ++p->last_launches;
    }
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_nd");
    return ECC_OK;
}
