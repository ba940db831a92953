// ecc_present.cu -- Eq. 1's thresholds of a float32 image found on the
// device: the values present in it, distinct and ascending (t_1 < ... < t_n,
// Sec. 2.2).  ecc_compute_levels at these levels is the paper's ECC
// sequence.
//
// A NaN voxel is in no sublevel set, so it defines no threshold; -0.0
// compares equal to 0.0, so they are one threshold (reported as +0.0).
//
//  1. collect_kernel: every voxel's value becomes a 32-bit key whose
//     unsigned order is the float order.  A lane walks 4 consecutive
//     voxels of each 128 of a row and inserts a key into a CTA-private
//     open-addressing table in shared memory only where it differs from the
//     last key the lane inserted (runs of one value cost one probe).  At the
//     end the CTA flushes its distinct keys into one global table.  Images
//     have few distinct values compared with their voxels (the paper's
//     datasets have 11-1024), so the global table sees a few thousand
//     inserts per CTA at most.  A CTA whose shared table passes half full
//     sends the rest straight to the global one.
//  2. compact_kernel: the global table's keys are gathered into a list
//     (any order), and the slots are reset for the next call.
//  3. rank_kernel: each key's rank is the number of smaller keys (keys are
//     distinct, so ranks are too).  It is counted over the whole list in
//     shared-memory tiles, and levels[rank] is the key's value.
//
// Every probe loop is bounded by its table size.  A global table that fills
// (more distinct values than the caller allowed) is reported through the
// count and not waited out.
#include <cuda_runtime.h>

#include "ecc.h"
#include "ecc_internal.h"
#include "ecc_plan.h"

namespace ecc {
namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;  // above every key (+infinity is 0xFF800000)
constexpr int kCollectThreads = 1024;  // large CTAs: fewer flushes of the same keys into the global table
constexpr int kSmemSlots = 4096;          // per-CTA table, 16 KB
constexpr int kSmemFill = kSmemSlots / 2;  // inserts after which the CTA goes global
constexpr int kRankThreads = 256;
constexpr int kRankTile = 2048;

// Order-preserving key of a non-NaN float (-0.0 taken as 0.0): negative
// values flip every bit, the others set the sign bit.
__device__ __forceinline__ uint32_t key_of(float f)
{
    uint32_t b = __float_as_uint(f);
    if (b == 0x80000000u) b = 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float value_of(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ uint32_t slot_of(uint32_t k, uint32_t mask)
{
    return (k * 0x9E3779B1u) & mask;  // Fibonacci hashing; mask = size - 1
}

// Inserts k into a table of mask + 1 slots by linear probing: 1 if k was
// new, 0 if present, -1 if no free slot was found in a full sweep.
__device__ __forceinline__ int table_insert(uint32_t *tab, uint32_t mask, uint32_t k)
{
    uint32_t h = slot_of(k, mask);
    for (uint32_t p = 0; p <= mask; ++p) {
        const uint32_t cur = *reinterpret_cast<volatile uint32_t *>(tab + h);
        if (cur == k) return 0;
        if (cur == kEmpty) {
            const uint32_t prev = atomicCAS(tab + h, kEmpty, k);
            if (prev == kEmpty) return 1;
            if (prev == k) return 0;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

struct CollectArgs {
    const unsigned char *src;
    int64_t nx, rows, ny;  // rows = nz * ny
    int64_t sp_y, sp_z;    // source pitches (bytes)
    uint32_t *gtab;        // global table, gmask + 1 slots, all kEmpty on entry
    uint32_t gmask;
};

__global__ void __launch_bounds__(kCollectThreads) collect_kernel(const CollectArgs a)
{
    __shared__ uint32_t stab[kSmemSlots];
    __shared__ unsigned int s_n;
    for (int i = threadIdx.x; i < kSmemSlots; i += kCollectThreads) stab[i] = kEmpty;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * kCollectThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kCollectThreads) >> 5;
    auto insert = [&](uint32_t k) {
        if (*reinterpret_cast<volatile unsigned int *>(&s_n) < kSmemFill) {
            if (table_insert(stab, kSmemSlots - 1, k) == 1) atomicAdd(&s_n, 1u);
        } else {
            table_insert(a.gtab, a.gmask, k);
        }
    };
    // rows r = warp, warp + nwarps, ... as (z, y) stepped without a division
    int64_t z = warp / a.ny, y = warp - z * a.ny;
    const int64_t dz = nwarps / a.ny, dy = nwarps - dz * a.ny;
    uint32_t last = kEmpty;  // the key this lane inserted last: equal keys in a row skip the table
    for (int64_t r = warp; r < a.rows; r += nwarps) {
        const float *row = reinterpret_cast<const float *>(a.src + z * a.sp_z + y * a.sp_y);
        // a lane takes 4 consecutive voxels of each 128, so in a smooth image
        // a lane sees runs of one value and probes the table once per run
        for (int64_t x = 4 * lane; x < a.nx; x += 128) {
            float v[4];
            if (x + 3 < a.nx && (reinterpret_cast<uintptr_t>(row + x) & 15) == 0) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(row + x));
                v[0] = q.x;
                v[1] = q.y;
                v[2] = q.z;
                v[3] = q.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = x + u < a.nx ? __ldg(row + x + u) : __int_as_float(0x7fc00000);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (v[u] != v[u]) continue;  // NaN (or past the row): no threshold
                const uint32_t k = key_of(v[u]);
                if (k == last) continue;
                last = k;
                insert(k);
            }
        }
        y += dy;
        z += dz;
        if (y >= a.ny) {
            y -= a.ny;
            ++z;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSmemSlots; i += kCollectThreads) {
        const uint32_t k = stab[i];
        if (k != kEmpty) table_insert(a.gtab, a.gmask, k);
    }
}

// Gathers the global table's keys into keys[] (at most max_keys kept; the
// count is exact either way) and empties the table for the next call.
__global__ void __launch_bounds__(256) compact_kernel(uint32_t *gtab, uint32_t nslots, uint32_t *keys,
                                                      unsigned int *nkeys, uint32_t max_keys)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += gridDim.x * blockDim.x) {
        const uint32_t k = gtab[i];
        if (k == kEmpty) continue;
        gtab[i] = kEmpty;
        const unsigned int j = atomicAdd(nkeys, 1u);
        if (j < max_keys) keys[j] = k;
    }
}

// levels[rank of key i] = value of key i, the rank counted over all n keys
// in shared-memory tiles; *d_count = n, or max_levels + 1 when n is larger
// (levels then untouched).  Blocks past n leave at once (block-uniform).
__global__ void __launch_bounds__(kRankThreads) rank_kernel(const uint32_t *keys, const unsigned int *nkeys,
                                                            float *levels, int32_t *d_count, int32_t max_levels)
{
    __shared__ uint32_t tile[kRankTile];
    const unsigned int n = *nkeys;
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_count = n > (unsigned)max_levels ? max_levels + 1 : (int32_t)n;
    if (n > (unsigned)max_levels || blockIdx.x * kRankThreads >= n) return;
    const unsigned int i = blockIdx.x * kRankThreads + threadIdx.x;
    const uint32_t mine = i < n ? keys[i] : kEmpty;
    unsigned int rank = 0;
    for (unsigned int t0 = 0; t0 < n; t0 += kRankTile) {
        const unsigned int len = n - t0 < (unsigned)kRankTile ? n - t0 : (unsigned)kRankTile;
        __syncthreads();
        for (unsigned int j = threadIdx.x; j < len; j += kRankThreads) tile[j] = keys[t0 + j];
        __syncthreads();
        for (unsigned int j = 0; j < len; ++j) rank += tile[j] < mine ? 1u : 0u;
    }
    if (i < n) levels[rank] = value_of(mine);
}

// Workspace layout in the plan's present buffer: the table (nslots words),
// the key list (max_levels words), four words (the key count, the count of
// ecc_compute_present, two spare).
uint32_t table_slots(int32_t max_levels)
{
    uint32_t s = 1024;
    while (s < 2u * ((uint32_t)max_levels + 1u)) s <<= 1;
    return s;
}

}  // namespace
}  // namespace ecc

namespace ecc {
namespace {

// The three launches of ecc_levels_present.  With d_count null the count
// goes to the workspace's own word, returned in *count_word.
ecc_status levels_present(ecc_plan_s *p, const ecc_image *img, float *d_levels, int32_t max_levels,
                          int32_t *d_count, cudaStream_t s, int32_t **count_word)
{
    if (max_levels < 1 || max_levels > 65536) return invalid("ecc_levels_present: max_levels must be in 1..65536");
    if (img->dtype != ECC_F32) return invalid("ecc_levels_present: image dtype must be ECC_F32");
    Geom g;
    ecc_status st = image_geom(img, ECC_F32, p->d.max_voxels, &g, nullptr, false);
    if (st != ECC_OK) return st;
    if (g.pitch_y % 4 || (g.ndim == 3 && g.pitch_z % 4) || reinterpret_cast<uintptr_t>(g.data) % 4)
        return invalid("ecc_levels_present: pitches and data must be 4-byte aligned");
    const uint32_t nslots = table_slots(max_levels);
    const size_t tab_bytes = sizeof(uint32_t) * nslots;
    const size_t key_bytes = sizeof(uint32_t) * (size_t)max_levels;
    st = p->ensure_present((int64_t)(tab_bytes + key_bytes + 4 * sizeof(unsigned int)));
    if (st != ECC_OK) return st;
    uint32_t *gtab = static_cast<uint32_t *>(p->present);
    uint32_t *keys = gtab + nslots;
    unsigned int *nkeys = reinterpret_cast<unsigned int *>(keys + max_levels);
    int32_t *own_count = reinterpret_cast<int32_t *>(nkeys + 1);
    if (!d_count) d_count = own_count;
    if (count_word) *count_word = d_count;
    // the table starts empty (compact_kernel empties it again after use;
    // cleared here too so that an interrupted call leaves nothing behind)
    cudaError_t e = cudaMemsetAsync(gtab, 0xFF, tab_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(nkeys, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_levels_present: clear");

    CollectArgs a{};
    a.src = g.data;
    a.nx = g.nx;
    a.ny = g.ny;
    a.rows = (g.ndim == 3 ? g.nz : 1) * g.ny;
    a.sp_y = g.pitch_y;
    a.sp_z = g.ndim == 3 ? g.pitch_z : g.pitch_y * g.ny;
    a.gtab = gtab;
    a.gmask = nslots - 1;
    // one warp per row, at most 2 CTAs of 32 warps per SM (each CTA flushes
    // its distinct keys into the global table once, so fewer, larger CTAs
    // mean fewer probes of the same global slots)
    int64_t ctas = (a.rows + kCollectThreads / 32 - 1) / (kCollectThreads / 32);
    const int64_t ctas_max = (int64_t)p->num_sms * 2;
    if (ctas > ctas_max) ctas = ctas_max;
    if (ctas < 1) ctas = 1;
    collect_kernel<<<(unsigned)ctas, kCollectThreads, 0, s>>>(a);
    const unsigned compact_ctas = (nslots + 255) / 256 < 1024u ? (nslots + 255) / 256 : 1024u;
    compact_kernel<<<compact_ctas, 256, 0, s>>>(gtab, nslots, keys, nkeys, (uint32_t)max_levels);
    rank_kernel<<<(unsigned)((max_levels + kRankThreads - 1) / kRankThreads), kRankThreads, 0, s>>>(
        keys, nkeys, d_levels, d_count, max_levels);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ecc_levels_present: launch");
    p->last_launches = 3;
    return ECC_OK;
}

}  // namespace
}  // namespace ecc

using namespace ecc;

extern "C" ecc_status ecc_levels_present(ecc_plan_t p, const ecc_image *img, float *d_levels, int32_t max_levels,
                                         int32_t *d_count, void *stream)
{
    if (!p) return invalid("ecc_levels_present: NULL plan");
    if (!img || !d_levels || !d_count) return invalid("ecc_levels_present: NULL argument");
    return levels_present(p, img, d_levels, max_levels, d_count, static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" ecc_status ecc_compute_present(ecc_plan_t p, const ecc_image *img, float *d_levels, int32_t max_levels,
                                          int32_t *h_count, int64_t *d_ecc, void *stream)
{
    if (!p) return invalid("ecc_compute_present: NULL plan");
    if (!img || !d_levels || !h_count || !d_ecc) return invalid("ecc_compute_present: NULL argument");
    *h_count = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *d_count = nullptr;
    ecc_status st = levels_present(p, img, d_levels, max_levels, nullptr, s, &d_count);
    if (st != ECC_OK) return st;
    int32_t n = 0;
    cudaError_t e = cudaMemcpyAsync(&n, d_count, sizeof(n), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_present: count read");
    *h_count = n;
    if (n > max_levels) {
        set_error("ecc_compute_present: the image holds more distinct values than max_levels");
        return ECC_E_BUSY;
    }
    if (n == 0) return ECC_OK;  // every voxel NaN: no threshold
    if (p->d.lo != 0 || n > p->d.hi) {
        set_error("ecc_compute_present: the plan's levels [0, hi] do not cover the image's distinct values");
        return ECC_E_BUSY;
    }
    return ecc_compute_levels(p, img, d_levels, n, d_ecc, stream);
}
