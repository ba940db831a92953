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
#include "ecc_scan_block.cuh"
#include "ecc_walk.cuh"

namespace ecc {
namespace {

// ------------------------------------------------------------ bit-sliced walker
//
// The star of a voxel splits along w into the cells of its own hyperplane
// and those cells extended to w+1 or w-1, so its count is
//   kappa4 = k3(W0) - b+ k3(W0 & W+) - b- k3(W0 & W-)
// with W0, W+, W- its wins over hyperplanes w, w+1, w-1, b+- its wins over
// its two w-neighbours and k3 the 3D count (bs::kappa4_nonzero).
//
// A CTA of kZ warps takes kZ consecutive z over one (30-row tile,
// 30-column window) column and a chunk of w (or several partial row tiles
// side by side); warp i holds z0 + i, lanes hold the rows (the 3D walker's
// layout).  At every step the CTA loads hyperplane w+1 (its kZ slices and
// the two halo slices z0-1, z0+kZ) into shared memory once, and each pair
// of neighbouring slices is compared once (walk::slice_pair, nine
// directions per block): warp i compares its slice (w, z) with (w+1, z-1),
// (w+1, z), (w+1, z+1) and slice (w+1, z) with (w+1, z+1); the reverse
// halves it does not need itself go through shared memory to the warps of
// z-1 and z+1, which read them at the next step (one __syncthreads a step;
// slices triple-buffered, exchanged wins double-buffered, by step).  The
// three halo pairs go to warps 1-3 (1 and 2 when kZ = 4); warps 0 and kZ-1
// load the halo slices.  kZ = 4 for 8-bit images (4 and 6 measured alike,
// 8 slower); 16-bit ones, at about 230 registers a thread, fit 8 warps per
// SM either way and take kZ = 8 (fewer halo loads and pairs per output:
// 209 against 245 us at 64^4).
template <typename T>
__host__ __device__ constexpr int z_group() { return sizeof(T) == 1 ? 4 : 8; }

struct Walk4Args {
    const unsigned char *data;
    int64_t n[4];        // w, z, y, x
    int64_t pitch[3];    // bytes: w, z, y
    int64_t items;       // w chunks x per_chunk
    int64_t chunk;       // hyperplanes per item
    int64_t per_chunk;   // items per w chunk: full_items, then the packed ones
    int64_t full_items;  // z groups x full row tiles x windows
    int64_t ngz;         // groups of z_group<T>() consecutive z
    int32_t ntx;         // windows of 30 columns
    int32_t nty_full;    // tiles of 30 rows
    int32_t remy;        // rows left below the full tiles (0..29)
    int32_t pack;        // partial tiles (remy rows + 2 halo lanes) per warp
    HistDst h;
    int32_t smem_hist, range_check;  // range_check: the bins are guarded (range narrower than the type)
    int32_t check_all;               // every output voxel is compared with [lo, hi]
    uint32_t lo_bits, hi_bits;
    unsigned int *status;
    long long *ecc_out;    // non-null: the last CTA also scans the bins (at most kFusedScanMaxBins)
    long long *vcec_out;
    unsigned int *done;    // finished-CTA count for that scan (zero between launches)
};

// Shared-memory words before the histogram: slices of three hyperplanes
// (kZ + 2 each, KP planes) and three double-buffered win exchanges.
__host__ __device__ constexpr int walk4_slice_words(int kZ, int KP) { return 3 * (kZ + 2) * KP * 32; }
__host__ __device__ constexpr int walk4_xchg_words(int kZ) { return 2 * kZ * 9 * 32; }
__host__ __device__ constexpr int walk4_words(int kZ, int KP)
{
    return walk4_slice_words(kZ, KP) + 3 * walk4_xchg_words(kZ);
}

template <typename T, bool TOP>
__global__ void __launch_bounds__(z_group<T>() * 32) walk4d_kernel(const Walk4Args a)
{
    constexpr int K = 8 * sizeof(T), KP = K + 1, kZ = z_group<T>();
    extern __shared__ uint32_t smem4[];
    uint32_t *const SL = smem4;                                   // [3][kZ + 2][KP][32]
    uint32_t *const MZ = SL + walk4_slice_words(kZ, KP);          // [2][kZ][9][32]
    uint32_t *const CM = MZ + walk4_xchg_words(kZ);
    uint32_t *const CP = CM + walk4_xchg_words(kZ);
    int *const hist = reinterpret_cast<int *>(CP + walk4_xchg_words(kZ));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.smem_hist)
        for (int i = threadIdx.x; i < a.h.nbins; i += blockDim.x) hist[i] = 0;
    const walk::Bins bins{a.smem_hist ? hist : nullptr, a.h.acc, a.h.lo, a.h.nbins, a.range_check, a.status};
    const int64_t nw = a.n[0], nz = a.n[1], ny = a.n[2], nx = a.n[3];
    const int64_t row_bytes = nx * (int64_t)sizeof(T);
    unsigned n_emitted = 0;
    uint32_t bad = 0;  // output voxels outside [lo, hi] (when checked)

    // slot j of hyperplane buffer h holds slice z0 - 1 + j; plane k at [k * 32]
    auto slot = [&](int h, int j) { return SL + (h * (kZ + 2) + j) * KP * 32 + lane; };
    auto put_slice = [&](int h, int j, const uint32_t *P) {
        uint32_t *d = slot(h, j);
#pragma unroll
        for (int k = 0; k < KP; ++k) d[k * 32] = P[k];
    };
    auto get_slice = [&](int h, int j, uint32_t *P) {
        const uint32_t *d = slot(h, j);
#pragma unroll
        for (int k = 0; k < KP; ++k) P[k] = d[k * 32];
    };
    auto xchg = [&](uint32_t *base, int par, int i) { return base + (par * kZ + i) * 9 * 32 + lane; };
    auto put9 = [&](uint32_t *d, const uint32_t m[3][3]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i * 32] = (&m[0][0])[i];
    };
    auto get9 = [&](const uint32_t *d, uint32_t m[3][3]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) (&m[0][0])[i] = d[i * 32];
    };

    for (int64_t item = blockIdx.x; item < a.items; item += gridDim.x) {
        // Full items: lane l holds row 30 ty - 1 + l of column (z group,
        // window).  Packed items: the last remy rows of `pack` columns side
        // by side, remy + 2 lanes each (a halo lane on either side).
        const int64_t ci = item / a.per_chunk;
        int64_t r = item - ci * a.per_chunk;
        const int64_t w0 = ci * a.chunk, w1 = w0 + a.chunk < nw ? w0 + a.chunk : nw;
        int64_t z0, y;
        int tx;
        bool lane_out;
        if (r < a.full_items) {
            tx = (int)(r % a.ntx);
            r /= a.ntx;
            const int ty = (int)(r % a.nty_full);
            z0 = (r / a.nty_full) * kZ;
            y = (int64_t)ty * 30 - 1 + lane;
            lane_out = lane >= 1 && lane <= 30;
        } else {
            const int seg_len = a.remy + 2, seg = lane / seg_len, j = lane - seg * seg_len;
            const int64_t c = (r - a.full_items) * a.pack + seg;
            const bool valid = seg < a.pack && c < a.ngz * a.ntx;
            z0 = valid ? (c / a.ntx) * kZ : 0;
            tx = valid ? (int)(c % a.ntx) : 0;
            y = valid ? (int64_t)a.nty_full * 30 - 1 + j : -2;   // -2: no row
            lane_out = valid && j >= 1 && j <= a.remy;
        }
        const int64_t z = z0 + warp;
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
        // hyperplane slots of this CTA's z range, halos from warps 0 and kZ-1
        auto load_hyperplane = [&](int64_t w, int h, uint32_t *own) {
            load(w, z, own);
            put_slice(h, warp + 1, own);
            if (warp == 0 || warp == kZ - 1) {
                uint32_t H[KP];
                const int j = warp == 0 ? 0 : kZ + 1;
                load(w, z0 - 1 + j, H);
                put_slice(h, j, H);
            }
        };

        __syncthreads();   // the previous item's readers are done with every buffer
        uint32_t A0[KP];
        load_hyperplane(w0 - 1, 0, A0);
        uint32_t W2[3][3], C1[3][3];   // carried: W0 layer z+1 and W- layer z of the next output
        int hA = 0;
        for (int64_t w = w0 - 1; w < w1; ++w) {
            const int hB = hA == 2 ? 0 : hA + 1;
            const int par = (int)((w - w0 + 1) & 1), prv = par ^ 1;
            uint32_t B0[KP];
            load_hyperplane(w + 1, hB, B0);
            if (a.check_all && w + 1 < w1 && z < nz) bad |= ~walk::in_range<K>(B0, a.lo_bits, a.hi_bits) & out;
            __syncthreads();
            const bool emit_step = w >= w0;   // the first step only fills the carried state
            uint32_t W[3][3][3], T0[4], Tm[4], Tp[4], bm = 0, bp = 0;
            if (emit_step) {
                // W0 of slice (w, z), then its wins over hyperplane w-1
                get9(xchg(MZ, prv, warp), W[0]);
                walk::in_slice<K, TOP>(A0, W[1]);
#pragma unroll
                for (int i = 0; i < 9; ++i) (&W[2][0][0])[i] = (&W2[0][0])[i];
                bs::kappa3d(W, T0);
                uint32_t C[3][3][3];
                get9(xchg(CM, prv, warp), C[0]);
                get9(xchg(CP, prv, warp), C[2]);
#pragma unroll
                for (int i = 0; i < 9; ++i) (&C[1][0][0])[i] = (&C1[0][0])[i];
                bm = C[1][1][1];
#pragma unroll
                for (int i = 0; i < 27; ++i) (&C[0][0][0])[i] &= (&W[0][0][0])[i];
                bs::kappa3d(C, Tm);
            }
            uint32_t fw[3][3], rv[3][3];
            {
                // (w, z) against (w+1, z-1): W+ layer z-1; the reverse is W- layer z+1 of warp z-1
                uint32_t Bm[KP];
                get_slice(hB, warp, Bm);
                walk::slice_pair<K, TOP, true, true>(A0, Bm, fw, rv);
                if (warp > 0) put9(xchg(CP, par, warp - 1), rv);
                if (emit_step)
#pragma unroll
                    for (int i = 0; i < 9; ++i) (&W[0][0][0])[i] &= (&fw[0][0])[i];
            }
            // (w, z) against (w+1, z): W+ layer z and this warp's next W- layer z
            walk::slice_pair<K, TOP, true, true>(A0, B0, fw, C1);
            bp = fw[1][1];
            if (emit_step)
#pragma unroll
                for (int i = 0; i < 9; ++i) (&W[1][0][0])[i] &= (&fw[0][0])[i];
            {
                uint32_t Bp[KP];
                get_slice(hB, warp + 2, Bp);
                // (w, z) against (w+1, z+1): W+ layer z+1; the reverse is W- layer z-1 of warp z+1
                walk::slice_pair<K, TOP, true, true>(A0, Bp, fw, rv);
                if (warp < kZ - 1) put9(xchg(CM, par, warp + 1), rv);
                if (emit_step)
#pragma unroll
                    for (int i = 0; i < 9; ++i) (&W[2][0][0])[i] &= (&fw[0][0])[i];
                // (w+1, z) against (w+1, z+1): next W0 layer z+1; the reverse is warp z+1's layer z-1
                walk::slice_pair<K, TOP, true, true>(B0, Bp, W2, rv);
                if (warp < kZ - 1) put9(xchg(MZ, par, warp + 1), rv);
            }
            // the halo pairs of warps 0 and kZ-1 (kZ = 4: warp 2 takes two)
            if (warp == 1) {
                uint32_t X[KP], Y[KP];
                get_slice(hB, 0, X);
                get_slice(hB, 1, Y);
                walk::slice_pair<K, TOP, false, true>(X, Y, fw, rv);
                put9(xchg(MZ, par, 0), rv);
            } else if (warp == 2) {
                uint32_t X[KP], Y[KP];
                get_slice(hA, 0, X);
                get_slice(hB, 1, Y);
                walk::slice_pair<K, TOP, false, true>(X, Y, fw, rv);
                put9(xchg(CM, par, 0), rv);
            }
            if (warp == (kZ > 4 ? 3 : 2)) {
                uint32_t X[KP], Y[KP];
                get_slice(hA, kZ + 1, X);
                get_slice(hB, kZ, Y);
                walk::slice_pair<K, TOP, false, true>(X, Y, fw, rv);
                put9(xchg(CP, par, kZ - 1), rv);
            }
            if (emit_step) {
                bs::kappa3d(W, Tp);
                uint32_t m = bs::kappa4_nonzero(T0, Tp, Tm, bp, bm) & ~A0[K] & out;
                if (a.h.emitted) n_emitted += __popc(m);
                while (m) {
                    const int i = __ffs(m) - 1;
                    m &= m - 1u;
                    // (-1)^4 = +1: the same sign in both complexes
                    bins.add(bs::bits_at<K>(A0, i), bs::kappa4_at(T0, Tp, Tm, bp, bm, i));
                }
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) A0[k] = B0[k];
            hA = hB;
        }
    }
    if (a.h.emitted) {
        const unsigned n = __reduce_add_sync(0xffffffffu, n_emitted);
        if (lane == 0 && n) atomicAdd(a.h.emitted, (unsigned long long)n);
    }
    if (a.check_all && __any_sync(0xffffffffu, bad != 0u) && lane == 0) atomicOr(a.status, DEV_RANGE);
    __syncthreads();
    if (a.smem_hist)
        for (int i = threadIdx.x; i < a.h.nbins; i += blockDim.x)
            if (hist[i]) atomicAdd(a.h.acc + i, (unsigned long long)(long long)hist[i]);
    if (a.ecc_out) {
        // the last CTA to finish scans the bins (as the 2D and 3D stencils do)
        __shared__ int s_last;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
            if (s_last) {
                *a.done = 0u;
                __threadfence();
            }
        }
        __syncthreads();
        if (s_last) scan_bins<kZ * 32>(a.h.acc, a.ecc_out, a.vcec_out, a.h.nbins, threadIdx.x);
    }
}

template <typename T, bool TOP>
cudaError_t launch_walk4(Walk4Args a, int num_sms, cudaStream_t s, FusedScan *fs)
{
    const bool fuse = fs && fs->ecc && a.done && a.h.nbins <= kFusedScanMaxBins;
    a.ecc_out = fuse ? fs->ecc : nullptr;
    a.vcec_out = fuse ? fs->vcec : nullptr;
    constexpr int KP = 8 * sizeof(T) + 1, kZ = z_group<T>();
    auto k = walk4d_kernel<T, TOP>;
    const size_t smem =
        sizeof(uint32_t) * (size_t)walk4_words(kZ, KP) + (a.smem_hist ? sizeof(int) * (size_t)a.h.nbins : 0);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kZ * 32, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    a.ntx = (int32_t)((a.n[3] + 29) / 30);
    a.nty_full = (int32_t)(a.n[2] / 30);
    a.remy = (int32_t)(a.n[2] % 30);
    a.pack = 32 / (a.remy + 2);
    a.ngz = (a.n[1] + kZ - 1) / kZ;
    a.full_items = a.ngz * a.nty_full * a.ntx;
    a.per_chunk = a.full_items + (a.remy ? (a.ngz * a.ntx + a.pack - 1) / a.pack : 0);
    // w chunks of c hyperplanes: an item costs c + 1 steps (one to fill the
    // state), each CTA runs ceil(items / resident CTAs) items; take the c
    // with the least of (rounds x steps), the longest any CTA runs.
    const int64_t base = a.per_chunk;
    const int64_t resident = (int64_t)num_sms * per_sm;
    int64_t best_c = a.n[0], best_cost = -1;
    for (int64_t kc = 1; kc <= a.n[0]; ++kc) {   // chunk counts, until items far outnumber CTAs
        const int64_t c = (a.n[0] + kc - 1) / kc;
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
    const int64_t blocks = std::min<int64_t>(a.items, resident);
    k<<<(unsigned)blocks, kZ * 32, smem, s>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess && fuse) fs->done = true;
    return e;
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
    // the bins are guarded whenever values can fall outside them; every
    // output voxel is compared with the bounds unless the plan opted out
    a.range_check = walk::range_is_narrow(p->d.lo, p->nbins, es);
    a.check_all = a.range_check && !(p->d.flags & ECC_FLAG_NO_RANGE_CHECK);
    a.lo_bits = (uint32_t)p->d.lo;
    a.hi_bits = (uint32_t)(p->d.hi);
    a.status = p->status;
    a.smem_hist = p->nbins <= kSmemBinsMax;
    const bool top = p->d.complex_mode == ECC_TOPCELL_MIN;
    // the walker's last CTA scans small histograms itself; its finished-CTA
    // count is a word of the plan's scheduling block the stencils leave free
    a.done = p->sched + 3;
    FusedScan fs{reinterpret_cast<long long *>(d_ecc), reinterpret_cast<long long *>(d_vcec), false};
    cudaError_t e = es == 1 ? (top ? launch_walk4<unsigned char, true>(a, p->num_sms, s, &fs)
                                   : launch_walk4<unsigned char, false>(a, p->num_sms, s, &fs))
                            : (top ? launch_walk4<unsigned short, true>(a, p->num_sms, s, &fs)
                                   : launch_walk4<unsigned short, false>(a, p->num_sms, s, &fs));
    p->last_launches = 1;
    if (e == cudaSuccess && !fs.done) {
        e = launch_scan(p->acc, reinterpret_cast<long long *>(d_ecc), reinterpret_cast<long long *>(d_vcec), 1,
                        p->nbins, p->scan_ws(), p->status, s);
        ++p->last_launches;
    }
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_nd");
    return ECC_OK;
}
