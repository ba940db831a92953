// ecc_nd.cu -- images of up to four dimensions (d > 3: the paper's texture
// path stops at three, Sec. 5).  ecc_compute_nd forwards 2D and 3D images to
// ecc_compute; 4D images take a one-thread-per-voxel kernel.
//
// The per-voxel rule is the one of every other kernel here (Sec. 2.3,
// Algorithm 1 regrouped per voxel): a voxel p introduces a cell containing
// it when it beats every other vertex of the cell, and adds (-1)^dim of each
// such cell to the bin of its value.  In four dimensions the cells
// containing p are p + sum over a in A of {0, s_a e_a} for an axis subset A
// and signs s_A: 1 vertex, 8 edges, 24 squares, 32 cubes and 16 tesseracts.
// The kernel compares p with its 80 neighbours (ties go to the lower linear
// index: a neighbour later in memory is beaten on >=, an earlier one on >),
// keeps the wins as an 81-bit mask, and counts the 81 cells against
// precomputed masks of the neighbours each cell needs.  Vertex complex: a
// missing neighbour is never beaten (the cell does not exist).  Top-cell
// complex: comparisons reversed, a missing neighbour always beaten (the
// +infinity collar), and the count multiplied by (-1)^4 = +1.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ecc_internal.h"
#include "ecc_plan.h"

namespace ecc {
namespace {

constexpr int kNdThreads = 256;
constexpr int kCells4 = 81;

// Cell c needs the neighbours in bits of kCellMask[c][0..2] (neighbour index
// (dw+1)*27 + (dz+1)*9 + (dy+1)*3 + (dx+1); 40 is the voxel itself) and
// counts kCellSign[c] = (-1)^dim.
__constant__ uint32_t kCellMask[kCells4][3];
__constant__ int kCellSign[kCells4];

struct Nd4Args {
    const unsigned char *data;
    int64_t n[4];        // dims, slowest first: w, z, y, x
    int64_t pitch[3];    // bytes: w, z, y
    HistDst h;
    int32_t smem_hist, range_check;
    unsigned int *status;
};

template <typename T, bool TOP>
__global__ void __launch_bounds__(kNdThreads) direct4d_kernel(const Nd4Args a)
{
    extern __shared__ int hist4[];
    if (a.smem_hist)
        for (int i = threadIdx.x; i < a.h.nbins; i += blockDim.x) hist4[i] = 0;
    __syncthreads();
    const int64_t total = a.n[0] * a.n[1] * a.n[2] * a.n[3];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t c[4];
        int64_t r = i;
        for (int ax = 3; ax >= 0; --ax) {
            c[ax] = r % a.n[ax];
            r /= a.n[ax];
        }
        const unsigned char *pp = a.data + c[0] * a.pitch[0] + c[1] * a.pitch[1] + c[2] * a.pitch[2] + c[3] * sizeof(T);
        const int v = (int)*reinterpret_cast<const T *>(pp);
        // neighbour (dw, dz, dy, dx) has index k = (dw+1)*27 + (dz+1)*9 + (dy+1)*3 + (dx+1);
        // addresses and "inside the image" flags are built axis by axis
        bool lo_ok[4], hi_ok[4];
#pragma unroll
        for (int ax = 0; ax < 4; ++ax) {
            lo_ok[ax] = c[ax] > 0;
            hi_ok[ax] = c[ax] + 1 < a.n[ax];
        }
        uint32_t win[3] = {0u, 0u, 0u};
#pragma unroll
        for (int dw = -1; dw <= 1; ++dw) {
            const unsigned char *pw = pp + dw * a.pitch[0];
            const bool okw = dw < 0 ? lo_ok[0] : (dw > 0 ? hi_ok[0] : true);
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz) {
                const unsigned char *pz = pw + dz * a.pitch[1];
                const bool okz = okw && (dz < 0 ? lo_ok[1] : (dz > 0 ? hi_ok[1] : true));
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    const unsigned char *py = pz + dy * a.pitch[2];
                    const bool oky = okz && (dy < 0 ? lo_ok[2] : (dy > 0 ? hi_ok[2] : true));
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int k = (dw + 1) * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                        if (k == 40) continue;
                        const bool ok = oky && (dx < 0 ? lo_ok[3] : (dx > 0 ? hi_ok[3] : true));
                        // a neighbour later in memory: its first nonzero offset is positive
                        const bool later = k > 40;
                        bool beats = TOP;
                        if (ok) {
                            const int u = (int)__ldg(reinterpret_cast<const T *>(py) + dx);
                            beats = TOP ? (later ? v <= u : v < u) : (later ? v >= u : v > u);
                        }
                        if (beats) win[k >> 5] |= 1u << (k & 31);
                    }
                }
            }
        }
        int kappa = 0;
#pragma unroll
        for (int cell = 0; cell < kCells4; ++cell) {
            const bool won = (win[0] & kCellMask[cell][0]) == kCellMask[cell][0] &&
                             (win[1] & kCellMask[cell][1]) == kCellMask[cell][1] &&
                             (win[2] & kCellMask[cell][2]) == kCellMask[cell][2];
            kappa += won ? kCellSign[cell] : 0;
        }
        {
            const int bin = v - a.h.lo;
            const bool bad = kappa && a.range_check && (unsigned)bin >= (unsigned)a.h.nbins;
            if (bad) atomicOr(a.status, DEV_RANGE);
            const bool add = kappa && !bad;
            // lanes adding to the same bin combine first (neighbouring voxels of
            // a smooth field often share a gray level)
            const unsigned act = __activemask();
            const unsigned grp = __match_any_sync(act, add ? bin : -1 - (int)(threadIdx.x & 31));
            const int sum = __reduce_add_sync(grp, kappa);
            if (add && (int)(threadIdx.x & 31) == __ffs(grp) - 1 && sum) {
                if (a.smem_hist)
                    atomicAdd(&hist4[bin], sum);
                else
                    atomicAdd(a.h.acc + bin, (unsigned long long)(long long)sum);
            }
        }
    }
    __syncthreads();
    if (a.smem_hist)
        for (int i = threadIdx.x; i < a.h.nbins; i += blockDim.x)
            if (hist4[i]) atomicAdd(a.h.acc + i, (unsigned long long)(long long)hist4[i]);
}

// The 81 cells of four dimensions containing the voxel: axis subset A and a
// side per axis of A; the neighbours are the nonempty sub-sums.
void cell_tables(uint32_t mask[kCells4][3], int sign[kCells4])
{
    int c = 0;
    for (int A = 0; A < 16; ++A) {
        int axes[4], k = 0;
        for (int ax = 0; ax < 4; ++ax)
            if (A & (1 << ax)) axes[k++] = ax;
        for (int s = 0; s < (1 << k); ++s) {
            uint32_t m[3] = {0, 0, 0};
            for (int B = 1; B < (1 << k); ++B) {
                int d[4] = {0, 0, 0, 0};
                for (int j = 0; j < k; ++j)
                    if (B & (1 << j)) d[axes[j]] = (s & (1 << j)) ? 1 : -1;
                const int idx = (d[0] + 1) * 27 + (d[1] + 1) * 9 + (d[2] + 1) * 3 + (d[3] + 1);
                m[idx >> 5] |= 1u << (idx & 31);
            }
            mask[c][0] = m[0];
            mask[c][1] = m[1];
            mask[c][2] = m[2];
            sign[c] = (k % 2 == 0) ? 1 : -1;
            ++c;
        }
    }
}

cudaError_t upload_tables()
{
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        uint32_t mask[kCells4][3];
        int sign[kCells4];
        cell_tables(mask, sign);
        err = cudaMemcpyToSymbol(kCellMask, mask, sizeof(mask));
        if (err == cudaSuccess) err = cudaMemcpyToSymbol(kCellSign, sign, sizeof(sign));
    });
    return err;
}

template <typename T, bool TOP>
cudaError_t launch4(const Nd4Args &a, int num_sms, size_t smem, cudaStream_t s)
{
    auto k = direct4d_kernel<T, TOP>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t total = a.n[0] * a.n[1] * a.n[2] * a.n[3];
    const int64_t blocks = std::min<int64_t>((total + kNdThreads - 1) / kNdThreads, (int64_t)num_sms * 8);
    k<<<(unsigned)blocks, kNdThreads, smem, s>>>(a);
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
    Nd4Args a{};
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
    cudaError_t e = upload_tables();
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_nd: cell tables");
    a.h = HistDst{p->acc, p->d.lo, p->nbins};
    if (p->d.flags & ECC_FLAG_COUNT_EMITTED) a.h.emitted = p->emitted;
    a.range_check = !(p->d.flags & ECC_FLAG_NO_RANGE_CHECK);
    a.status = p->status;
    a.smem_hist = p->nbins <= kSmemBinsMax;
    const size_t smem = a.smem_hist ? sizeof(int) * (size_t)p->nbins : 0;
    const bool top = p->d.complex_mode == ECC_TOPCELL_MIN;
    e = es == 1 ? (top ? launch4<unsigned char, true>(a, p->num_sms, smem, s)
                       : launch4<unsigned char, false>(a, p->num_sms, smem, s))
                : (top ? launch4<unsigned short, true>(a, p->num_sms, smem, s)
                       : launch4<unsigned short, false>(a, p->num_sms, smem, s));
    p->last_launches = 1;
    if (e == cudaSuccess) {
        e = launch_scan(p->acc, reinterpret_cast<long long *>(d_ecc), reinterpret_cast<long long *>(d_vcec), 1,
                        p->nbins, p->scan_ws(), p->status, s);
        ++p->last_launches;
    }
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_nd");
    return ECC_OK;
}
