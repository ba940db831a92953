// ecc_direct.cu -- one-thread-per-voxel stencil + shared-memory histogram.
//
// This is the straightforward form of the per-voxel computation of Sec. 3.2
// (each thread realizes the inner loop of Algorithm 1 for one voxel): the
// thread compares its voxel with the 8 (2D) or 26 (3D) neighbours, counts
// the cells the voxel introduces with sign (-1)^dim, and adds that count to
// a block-private histogram (Sec. 3.3 "Using registers", "Shared memory",
// "Parallel initialization and finalization"), which is flushed once per
// block into the int64 global VCEC.  Threads walk the slowest axis with a
// register window of 3 planes (3D) or 3 rows (2D), so each voxel is fetched
// from memory once per thread-column instead of 9 or 27 times.
//
// It serves as the general kernel: any pitch, any alignment, both complexes,
// both element types; the bit-sliced kernel is the fast path where it applies.
#include "ecc_internal.h"

namespace ecc {
namespace {

constexpr int kBX = 32, kBY = 8;

struct DirectArgs {
    Geom g;
    int64_t outer_begin, outer_end;  // outer axis = z (3D) or y (2D)
    int64_t chunk;                   // outer indices per thread column
    HistDst h;
    unsigned int *status;
    int smem_hist;
    int range_check;  // the bins are guarded (range narrower than the type)
    int check_all;    // every voxel is compared with [lo, hi]
};

template <typename T>
__device__ __forceinline__ int ld(const unsigned char *p)
{
    return (int)__ldg(reinterpret_cast<const T *>(p));
}

// Does the centre voxel c "beat" neighbour q (offset d), i.e. introduce the
// cells they share as far as this pair is concerned?  Vertex complex: c is
// the max, ties to the lower linear index (a later neighbour loses ties).
// Top-cell complex: c is the min, ties to the lower linear index.  A missing
// neighbour means the cell does not exist (vertex) or is owned by c alone
// (top-cell: the paper's +infinity collar).
template <bool TOP>
__device__ __forceinline__ bool beats(int c, int q, bool later, bool exists)
{
    if (TOP) return !exists || (later ? c <= q : c < q);
    return exists && (later ? c >= q : c > q);
}

// Adds each thread's voxel count to its bin, aggregated per warp: the
// lanes of a warp are 32 consecutive voxels of a row, which in smooth data
// often share a gray level, so lanes adding to the same bin in this step
// are grouped with __match_any_sync and one of them adds the group's sum
// (__reduce_add_sync).  Called by every thread that walks a voxel (the
// active threads of a warp are converged here).
__device__ __forceinline__ void add_bin(const DirectArgs &a, int *s_hist, int value, int kappa)
{
    const unsigned active = __activemask();
    int bin = value - a.h.lo;
    const bool bad = a.range_check && (unsigned)bin >= (unsigned)a.h.nbins;
    // a voxel outside [lo, hi] is reported when every voxel is checked, or
    // when it would have contributed; it never reaches the bins
    const unsigned report = __ballot_sync(active, bad && (a.check_all || kappa));
    if (report && (int)(threadIdx.x & 31) == __ffs(active) - 1) atomicOr(a.status, DEV_RANGE);
    if (bad || !kappa) bin = -1;
    if (a.h.emitted) {
        const unsigned nz = __ballot_sync(active, kappa != 0);
        if (nz && (int)(threadIdx.x & 31) == __ffs(active) - 1) atomicAdd(a.h.emitted, (unsigned long long)__popc(nz));
    }
    if (!__any_sync(active, bin >= 0)) return;
    const unsigned peers = __match_any_sync(active, bin);
    const int sum = __reduce_add_sync(peers, bin >= 0 ? kappa : 0);
    if (bin < 0 || sum == 0 || (int)(threadIdx.x & 31) != __ffs(peers) - 1) return;
    if (a.smem_hist)
        atomicAdd(&s_hist[bin], sum);
    else
        atomicAdd(a.h.acc + bin, (unsigned long long)(long long)sum);
}

template <typename T, bool TOP>
__global__ void __launch_bounds__(kBX * kBY) direct3d_kernel(DirectArgs a)
{
    extern __shared__ int s_hist[];
    const int tid = threadIdx.y * kBX + threadIdx.x;
    if (a.smem_hist)
        for (int i = tid; i < a.h.nbins; i += kBX * kBY) s_hist[i] = 0;
    __syncthreads();

    const Geom &g = a.g;
    const int64_t x = (int64_t)blockIdx.x * kBX + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * kBY + threadIdx.y;
    const int64_t zb = a.outer_begin + (int64_t)blockIdx.z * a.chunk;
    const int64_t ze = min(zb + a.chunk, a.outer_end);
    if (x < g.nx && y < g.ny && zb < ze) {
        const bool hx[3] = {x > 0, true, x + 1 < g.nx};
        const bool hy[3] = {y > 0, true, y + 1 < g.ny};
        const int64_t ox[3] = {(hx[0] ? x - 1 : x) * g.esize, x * g.esize, (hx[2] ? x + 1 : x) * g.esize};
        const int64_t oy[3] = {(hy[0] ? y - 1 : y) * g.pitch_y, y * g.pitch_y,
                               (hy[2] ? y + 1 : y) * g.pitch_y};
        int v[3][3][3];  // [dz+1][dy+1][dx+1]
        auto load_plane = [&](int slot, int64_t zz) {
            zz = zz < 0 ? 0 : (zz >= g.nz ? g.nz - 1 : zz);
            const unsigned char *p = g.data + zz * g.pitch_z;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) v[slot][dy][dx] = ld<T>(p + oy[dy] + ox[dx]);
        };
        load_plane(0, zb - 1);
        load_plane(1, zb);
        for (int64_t z = zb; z < ze; ++z) {
            load_plane(2, z + 1);
            const bool hz[3] = {z > 0, true, z + 1 < g.nz};
            const int c = v[1][1][1];
            bool w[3][3][3];
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const bool later = dz > 1 || (dz == 1 && (dy > 1 || (dy == 1 && dx > 1)));
                        w[dz][dy][dx] = beats<TOP>(c, v[dz][dy][dx], later, hz[dz] && hy[dy] && hx[dx]);
                    }
            // kappa = sum over cells containing the voxel that it introduces
            // of (-1)^dim: 1 vertex, 6 edges, 12 squares, 8 cubes.
            int kappa = 1;
            kappa -= w[0][1][1] + w[2][1][1] + w[1][0][1] + w[1][2][1] + w[1][1][0] + w[1][1][2];
#pragma unroll
            for (int a1 = 0; a1 < 3; a1 += 2)
#pragma unroll
                for (int b1 = 0; b1 < 3; b1 += 2) {
                    kappa += w[1][a1][1] & w[1][1][b1] & w[1][a1][b1];  // xy squares
                    kappa += w[a1][1][1] & w[1][1][b1] & w[a1][1][b1];  // xz squares
                    kappa += w[a1][1][1] & w[1][b1][1] & w[a1][b1][1];  // yz squares
                }
#pragma unroll
            for (int sz = 0; sz < 3; sz += 2)
#pragma unroll
                for (int sy = 0; sy < 3; sy += 2)
#pragma unroll
                    for (int sx = 0; sx < 3; sx += 2)
                        kappa -= w[sz][1][1] & w[1][sy][1] & w[1][1][sx] & w[sz][sy][1] & w[sz][1][sx] &
                                 w[1][sy][sx] & w[sz][sy][sx];
            if (TOP) kappa = -kappa;  // (-1)^d with d = 3: voxels are the 3-cells
            add_bin(a, s_hist, c, kappa);
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    v[0][dy][dx] = v[1][dy][dx];
                    v[1][dy][dx] = v[2][dy][dx];
                }
        }
    }
    __syncthreads();
    if (a.smem_hist)
        for (int i = tid; i < a.h.nbins; i += kBX * kBY)
            if (s_hist[i]) atomicAdd(a.h.acc + i, (unsigned long long)(long long)s_hist[i]);
}

template <typename T, bool TOP>
__global__ void __launch_bounds__(kBX * kBY) direct2d_kernel(DirectArgs a)
{
    extern __shared__ int s_hist[];
    const int tid = threadIdx.y * kBX + threadIdx.x;
    if (a.smem_hist)
        for (int i = tid; i < a.h.nbins; i += kBX * kBY) s_hist[i] = 0;
    __syncthreads();

    const Geom &g = a.g;
    const int64_t x = (int64_t)blockIdx.x * kBX + threadIdx.x;
    const int64_t col = (int64_t)blockIdx.y * kBY + threadIdx.y;
    const int64_t yb = a.outer_begin + col * a.chunk;
    const int64_t ye = min(yb + a.chunk, a.outer_end);
    if (x < g.nx && yb < ye) {
        const bool hx[3] = {x > 0, true, x + 1 < g.nx};
        const int64_t ox[3] = {(hx[0] ? x - 1 : x) * g.esize, x * g.esize, (hx[2] ? x + 1 : x) * g.esize};
        int v[3][3];  // [dy+1][dx+1]
        auto load_row = [&](int slot, int64_t yy) {
            yy = yy < 0 ? 0 : (yy >= g.ny ? g.ny - 1 : yy);
            const unsigned char *p = g.data + yy * g.pitch_y;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) v[slot][dx] = ld<T>(p + ox[dx]);
        };
        load_row(0, yb - 1);
        load_row(1, yb);
        for (int64_t y = yb; y < ye; ++y) {
            load_row(2, y + 1);
            const bool hy[3] = {y > 0, true, y + 1 < g.ny};
            const int c = v[1][1];
            bool w[3][3];
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const bool later = dy > 1 || (dy == 1 && dx > 1);
                    w[dy][dx] = beats<TOP>(c, v[dy][dx], later, hy[dy] && hx[dx]);
                }
            // 1 vertex, 4 edges, 4 squares; (-1)^d = +1 for top cells in 2D.
            int kappa = 1 - (w[0][1] + w[2][1] + w[1][0] + w[1][2]);
#pragma unroll
            for (int sy = 0; sy < 3; sy += 2)
#pragma unroll
                for (int sx = 0; sx < 3; sx += 2) kappa += w[sy][1] & w[1][sx] & w[sy][sx];
            add_bin(a, s_hist, c, kappa);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                v[0][dx] = v[1][dx];
                v[1][dx] = v[2][dx];
            }
        }
    }
    __syncthreads();
    if (a.smem_hist)
        for (int i = tid; i < a.h.nbins; i += kBX * kBY)
            if (s_hist[i]) atomicAdd(a.h.acc + i, (unsigned long long)(long long)s_hist[i]);
}

template <typename T, bool TOP>
cudaError_t launch_typed(const DirectArgs &a0, int num_sms, cudaStream_t s)
{
    DirectArgs a = a0;
    const int64_t outer = a.outer_end - a.outer_begin;
    const size_t smem = a.smem_hist ? (size_t)a.h.nbins * sizeof(int) : 0;
    if (a.g.ndim == 3) {
        const int64_t gx = (a.g.nx + kBX - 1) / kBX, gy = (a.g.ny + kBY - 1) / kBY;
        // enough thread columns to fill the GPU a few times, each walking >= 8 planes
        int64_t want = (int64_t)num_sms * 8;
        int64_t chunks = (want + gx * gy - 1) / (gx * gy);
        chunks = chunks < 1 ? 1 : chunks;
        a.chunk = (outer + chunks - 1) / chunks;
        if (a.chunk < 8) a.chunk = 8;
        const int64_t gz = (outer + a.chunk - 1) / a.chunk;
        if (gx > 2147483647 || gy > 65535 || gz > 65535) return cudaErrorInvalidConfiguration;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(direct3d_kernel<T, TOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        direct3d_kernel<T, TOP><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), dim3(kBX, kBY), smem, s>>>(a);
    } else {
        const int64_t gx = (a.g.nx + kBX - 1) / kBX;
        int64_t want = (int64_t)num_sms * 8 * kBY;
        int64_t cols = (want + gx - 1) / gx;
        cols = cols < 1 ? 1 : cols;
        a.chunk = (outer + cols - 1) / cols;
        if (a.chunk < 8) a.chunk = 8;
        const int64_t ncol = (outer + a.chunk - 1) / a.chunk;
        const int64_t gy = (ncol + kBY - 1) / kBY;
        if (gx > 2147483647 || gy > 65535) return cudaErrorInvalidConfiguration;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(direct2d_kernel<T, TOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        direct2d_kernel<T, TOP><<<dim3((unsigned)gx, (unsigned)gy), dim3(kBX, kBY), smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

// Loads (under lazy module loading) every one-thread-per-voxel kernel.
cudaError_t preload_direct()
{
    const void *fns[] = {
        (const void *)direct3d_kernel<unsigned char, false>, (const void *)direct3d_kernel<unsigned char, true>,
        (const void *)direct3d_kernel<unsigned short, false>, (const void *)direct3d_kernel<unsigned short, true>,
        (const void *)direct2d_kernel<unsigned char, false>, (const void *)direct2d_kernel<unsigned char, true>,
        (const void *)direct2d_kernel<unsigned short, false>, (const void *)direct2d_kernel<unsigned short, true>};
    cudaFuncAttributes fa;
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_direct(const Geom &g, int64_t outer_begin, int64_t outer_end, const HistDst &h,
                          int complex_mode, bool range_check, unsigned int *status, int num_sms,
                          cudaStream_t s)
{
    if (outer_end <= outer_begin) return cudaSuccess;
    DirectArgs a{};
    a.g = g;
    a.outer_begin = outer_begin;
    a.outer_end = outer_end;
    a.h = h;
    a.status = status;
    a.smem_hist = h.nbins <= 4096;
    a.range_check = (g.esize == 1 ? 255 : 65535) > (int64_t)h.lo + h.nbins - 1 || h.lo > 0;
    a.check_all = range_check && a.range_check;
    const bool top = complex_mode == ECC_TOPCELL_MIN;
    if (g.esize == 1)
        return top ? launch_typed<unsigned char, true>(a, num_sms, s)
                   : launch_typed<unsigned char, false>(a, num_sms, s);
    return top ? launch_typed<unsigned short, true>(a, num_sms, s)
               : launch_typed<unsigned short, false>(a, num_sms, s);
}

}  // namespace ecc
