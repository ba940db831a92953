// ecc_bs3d.cu -- the bit-sliced stencil + histogram of one 3D volume (sm_103a).
//
// The per-voxel rule is the paper's (Sec. 2.3, Algorithm 1; Sec. 3.2-3.3): a
// voxel introduces the cells it wins against every other member of, and adds
// (-1)^dim of each to the histogram bin of its gray level.  The mapping onto
// GB300:
//
//  * Bit-slicing (ecc_walk3.cuh).  A lane holds a window of 32 voxels of one
//    row as bit planes; lanes are 32 consecutive rows.  Windows and lane
//    rows overlap their neighbours by one voxel on each side, so an inner
//    warp owns a 30x30 column of the volume (31 along an axis where its tile
//    touches the image edge: the missing neighbour there needs no halo) and
//    walks it along z.  Each of the 13 neighbour directions is compared once
//    per voxel pair.
//  * Independent warps.  Each warp streams its own column through a private
//    ring of S shared-memory stages, one TMA copy (cp.async.bulk.tensor.3d)
//    of D planes x 32 rows x 48 (uint8) or 80 (uint16) bytes per stage,
//    completed on an mbarrier.  The warp refills a stage itself once it has
//    read it, so warps never wait for one another and there is no producer
//    warp.  The box starts on the 16-byte boundary at or below the window and
//    is an odd number of 16-byte units wide, so the lanes' 16-byte shared
//    loads are free of bank conflicts.
//  * Work list.  A warp claims (x-window, y-tile, z-chunk) items from a
//    global counter one item ahead of its walk, so the ring stays full across
//    item boundaries.
//  * Histogram.  Only voxels with a nonzero signed count are emitted (0.4 %
//    in smooth fields), into shared int32 bins flushed once per CTA into the
//    int64 accumulator, or into global int64 bins when the gray range does
//    not fit shared memory.  The last CTA to finish may also scan the bins
//    (ecc_scan_block.cuh), so a whole volume is one launch.
//  * Gray range.  When [lo, hi] is narrower than the element type, every
//    output voxel is compared with both bounds (bit-sliced) and a voxel
//    outside sets DEV_RANGE; the full range needs no check.
//  * Every mbarrier wait is bounded by %globaltimer (DEV_TIMEOUT); a warp
//    that gives up waits (bounded) for its copies in flight before leaving.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>

#include "ecc_bitslice.cuh"
#include "ecc_internal.h"
#include "ecc_scan_block.cuh"
#include "ecc_sync.cuh"
#include "ecc_walk.cuh"
#include "ecc_walk3.cuh"

namespace ecc {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn();  // ecc_bitslice.cu

namespace {

// Ring shape per element type and warps per CTA: D planes per stage (one TMA
// copy), S stages per warp.  A stage is refilled once the step after its
// last plane has run, so S - 1 stages are in flight ahead of the walk.
template <typename T, int NWARP>
struct C3 {
    static constexpr int ES = (int)sizeof(T);
    static constexpr int K = 8 * ES;                    // value bit planes
    static constexpr int WORDS = 8 * ES;                // 32-bit words of a 32-voxel window
    static constexpr int CHUNKS = 2 * ES + 1;           // 16-byte loads covering a window at any offset
    static constexpr int ROWB = 16 * CHUNKS;            // bytes of a staged row (odd number of 16-byte units)
    static constexpr int D = 2;                         // uint16: 2 x 2 measured 2 % faster than 1 x 4
    static constexpr int S = ES == 1 ? 3 : 2;
    static constexpr int PLANE = 32 * ROWB;
    static constexpr int STAGE = D * PLANE;             // multiple of 128 bytes
};

struct Bs3Args {
    unsigned int *sched;     // [0] next item, [1] finished CTAs (both reset by the last CTA)
    int32_t nx, ny, nz;
    int32_t z_begin, z_end;  // output planes [z_begin, z_end)
    int32_t ntx, nty, zchunk, nitems;
    int32_t smem_hist;
    int32_t check_range;     // compare every output voxel with [lo, hi] (only when narrower than the type)
    uint32_t lo_bits, hi_bits;
    HistDst h;
    unsigned int *status;
    long long *ecc_out;      // non-null: the last CTA also scans the bins (whole image, small histogram)
    long long *vcec_out;
    walk3::Mul mu;
};

using sync::mbar_arrive;
using sync::mbar_expect_tx;
using sync::mbar_init;
using sync::mbar_wait;
using sync::smem_u32;

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// This lane's 32-voxel window, starting `off` bytes into its staged row
// (0 <= off < 16), transposed into planes P[0..K-1].
template <typename T>
__device__ __forceinline__ void load_window(const unsigned char *row, int off, uint32_t *P, const walk3::Mul &mu)
{
    using C = C3<T, 4>;
    uint32_t v[4 * C::CHUNKS];
#pragma unroll
    for (int c = 0; c < C::CHUNKS; ++c) {
        const uint4 q = *reinterpret_cast<const uint4 *>(row + 16 * c);
        v[4 * c + 0] = q.x;
        v[4 * c + 1] = q.y;
        v[4 * c + 2] = q.z;
        v[4 * c + 3] = q.w;
    }
    uint32_t r[C::WORDS];
    const uint32_t sh = (uint32_t)(off & 3);
    // the byte shift as one byte permute per word: bytes sh..sh+3 of the pair
    // (a right shift would cost the same ALU slot, and a multiply pair more)
    const uint32_t sel = sh | ((sh + 1) << 4) | ((sh + 2) << 8) | ((sh + 3) << 12);
    // word offset (warp-uniform) by a switch
    switch (off >> 2) {
#define ECC_WIN(W)                                                                \
    case W:                                                                       \
        if (sh == 0) {                                                            \
            _Pragma("unroll") for (int i = 0; i < C::WORDS; ++i) r[i] = v[i + W]; \
        } else {                                                                  \
            _Pragma("unroll") for (int i = 0; i < C::WORDS; ++i) r[i] =           \
                __byte_perm(v[i + W], v[i + W + 1], sel);                         \
        }                                                                         \
        break;
        ECC_WIN(0)
        ECC_WIN(1)
        ECC_WIN(2)
        ECC_WIN(3)
#undef ECC_WIN
    }
    if (C::ES == 1)
        walk3::transpose_u8(r, P, mu);
    else
        walk3::transpose_u16(r, P, mu);
}

template <typename T, int NWARP>
constexpr int bs3_min_blocks()
{
    return sizeof(T) == 1 ? (NWARP == 4 ? 5 : 3) : (NWARP == 4 ? 4 : 2);
}

// The TMA side of one warp's ring, kept in shared memory and used by lane 0
// only (no registers in the other lanes): what changes per stage in one
// 16-byte word, the item's box origin in another.
struct __align__(16) LoadCursor {
    int st, nst;   // next stage of the item, and its number of stages
    int slot;      // ring slot of the next stage
    int issued;    // stages issued so far
    int item;      // item being loaded; -1 once the work list is exhausted, -2 before the first
    int bx, y0, z0;
};

template <typename T, int NWARP, bool TOP, bool NARROW, bool SMEM, bool COUNT>
__global__ void __launch_bounds__(NWARP * 32, bs3_min_blocks<T, NWARP>())
    bs3_kernel(const __grid_constant__ CUtensorMap tmap, const Bs3Args a)
{
    using C = C3<T, NWARP>;
    constexpr int K = C::K, S = C::S, D = C::D, ES = C::ES, ROWB = C::ROWB, PLANE = C::PLANE, STAGE = C::STAGE;
    constexpr int NTH = NWARP * 32;
    constexpr int ALIGN_EL = 16 / ES;
    constexpr int RING = NWARP * S * STAGE;

    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ring = warp * S * STAGE;  // byte offset of this warp's ring in smem
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + RING) + warp * S;
    int *tag = reinterpret_cast<int *>(smem + RING + NWARP * S * 8) + warp * S;
    int *hist = reinterpret_cast<int *>(smem + RING + NWARP * S * 12);
    __shared__ LoadCursor s_cur[NWARP];
    __shared__ int s_last;

    if (SMEM)
        for (int i = tid; i < a.h.nbins; i += NTH) hist[i] = 0;
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_cur[warp] = LoadCursor{0, 0, 0, 0, -2, 0, 0, 0};
    }
    __syncthreads();

    const walk3::Mul &mu = a.mu;

    // ------------------------------------------------ loads (lane 0)
    // Issue the next stage of the warp's walk into the next ring slot: claim
    // the next item when the current one has no stages left; once the work
    // list is exhausted, a stage is a plain arrival tagged -1.
    auto issue = [&]() {
        if (lane != 0) return;
        LoadCursor c;
        *reinterpret_cast<int4 *>(&c.st) = *reinterpret_cast<const int4 *>(&s_cur[warp].st);
        *reinterpret_cast<int4 *>(&c.item) = *reinterpret_cast<const int4 *>(&s_cur[warp].item);
        if (c.st >= c.nst) {
            if (c.item != -1) {
                const unsigned int it = atomicAdd(a.sched, 1u);
                c.item = it < (unsigned int)a.nitems ? (int)it : -1;  // unsigned: never a negative item
            }
            if (c.item >= 0) {
                const int xi = c.item % a.ntx, r = c.item / a.ntx;
                const int yt = r % a.nty, zc = r / a.nty;
                int xw, ylo, yhi;
                walk3::tile_span(a.nx, a.ntx, xi, xw, ylo, yhi);
                c.bx = xw / ALIGN_EL * ALIGN_EL;
                walk3::tile_span(a.ny, a.nty, yt, c.y0, ylo, yhi);
                const int zb = a.z_begin + zc * a.zchunk;
                const int ze = zb + a.zchunk < a.z_end ? zb + a.zchunk : a.z_end;
                c.z0 = zb - 1;
                c.nst = (ze - zb + 1 + D) / D;
            } else {
                c.nst = 0;
            }
            c.st = 0;
            *reinterpret_cast<int4 *>(&s_cur[warp].item) = *reinterpret_cast<const int4 *>(&c.item);
        }
        tag[c.slot] = c.item;
        if (c.item >= 0) {
            mbar_expect_tx(&full[c.slot], STAGE);
            tma_load_3d(smem + ring + c.slot * STAGE, &tmap, c.bx, c.y0, c.z0 + D * c.st, &full[c.slot]);
        } else {
            mbar_arrive(&full[c.slot]);
        }
        ++c.st;
        ++c.issued;
        if (++c.slot == S) c.slot = 0;
        *reinterpret_cast<int4 *>(&s_cur[warp].st) = *reinterpret_cast<const int4 *>(&c.st);
    };

    // ------------------------------------------------ walk
    int c_slot = 0;
    uint32_t c_phase = 0;
    int consumed = 0;
    bool ok = true;
    auto wait_stage = [&]() -> bool {
        if (__any_sync(0xffffffffu, mbar_wait(&full[c_slot], c_phase))) return true;
        if (lane == 0) atomicOr(a.status, DEV_TIMEOUT);
        ok = false;
        return false;
    };
    auto next_stage = [&]() {
        ++consumed;
        if (++c_slot == S) {
            c_slot = 0;
            c_phase ^= 1u;
        }
    };
    unsigned n_emitted = 0;  // ECC_FLAG_COUNT_EMITTED
    // bin of value v += k; with a range narrower than the type, a value
    // outside it never reaches the bins and sets DEV_RANGE
    auto add = [&](int v, int k) {
        if (COUNT) ++n_emitted;
        const int bin = v - a.h.lo;
        if (NARROW && (unsigned)bin >= (unsigned)a.h.nbins) {
            atomicOr(a.status, DEV_RANGE);
            return;
        }
        if (SMEM)
            atomicAdd(&hist[bin], k);
        else
            atomicAdd(a.h.acc + bin, (unsigned long long)(long long)k);
    };
    // the common single +-1 add of a lane, predicated instead of branched
    // (full range and shared bins only: nothing to check)
    auto add_if = [&](bool p, int v, int k) {
        if constexpr (SMEM && !NARROW && !COUNT) {
            const uint32_t addr = sync::smem_u32(hist + (v - a.h.lo));
            asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q red.shared.add.s32 [%1], %2;\n}\n"
                         ::"r"((uint32_t)p), "r"(addr), "r"(k) : "memory");
        } else {
            if (p) add(v, k);
        }
    };

    for (int i = 0; i < S; ++i) issue();
    __syncwarp();

    while (ok) {
        if (!wait_stage()) break;
        const int item = tag[c_slot];
        if (item < 0) {
            next_stage();
            break;
        }
        const int xi = item % a.ntx, rr = item / a.ntx;
        const int yt = rr % a.nty, zc = rr / a.nty;
        int xw, xlo, xhi, y0, ylo, yhi;  // window bit 0 is voxel xw, lane 0 is row y0
        walk3::tile_span(a.nx, a.ntx, xi, xw, xlo, xhi);
        walk3::tile_span(a.ny, a.nty, yt, y0, ylo, yhi);
        const int bx = xw / ALIGN_EL * ALIGN_EL;
        const int off = (xw - bx) * ES;
        const int y = y0 + lane;
        const int zb = a.z_begin + zc * a.zchunk;
        const int ze = zb + a.zchunk < a.z_end ? zb + a.zchunk : a.z_end;
        const int n = ze - zb + 2;  // planes zb-1 .. ze
        const uint32_t xex = walk::x_exist_mask(xw, a.nx);
        const bool lane_out = lane >= ylo && lane < yhi && y < a.ny;
        const uint32_t xmask = (xhi == 32 ? 0xffffffffu : (1u << xhi) - 1u) & ~((1u << xlo) - 1u);
        const uint32_t out_x = lane_out ? (xex & xmask) : 0u;
        const uint32_t e_row = y < a.ny ? ~xex : 0xffffffffu;
        walk3::Fill fill;
        fill.xl = xw == 0 ? 1u : 0u;
        fill.xr = xw + 32 >= a.nx ? 0x80000000u : 0u;
        fill.yt = lane == 0 && y0 == 0;
        fill.yb = lane == 31 && y0 + 32 >= a.ny;
        fill.edge = xw == 0 || xw + 32 >= a.nx || y0 == 0 || y0 + 32 >= a.ny;
        int vals = 0;  // smem offset of the emitted plane's window in this lane's row
        auto emit = [&](uint32_t m, const uint32_t *T) {
            walk3::emit3<TOP>(
                m, T,
                [&](int i) {
                    return ES == 1 ? (int)smem[vals + i]
                                   : (int)reinterpret_cast<const unsigned short *>(smem + vals)[i];
                },
                add, add_if);
        };
        // load plane z (this lane's row at smem offset `row`) into r
        auto load = [&](walk3::Row<K> &r, int row, int z) {
            load_window<T>(smem + row, off, r.P, mu);
            const bool exists = z >= 0 && z < a.nz;
            r.P[K] = exists ? e_row : 0xffffffffu;
            if (NARROW && a.check_range && z >= zb && z < ze) {
                const uint32_t bad = ~walk::in_range<K>(r.P, a.lo_bits, a.hi_bits) & out_x;
                if (__any_sync(0xffffffffu, bad != 0u) && lane == 0) atomicOr(a.status, DEV_RANGE);
            }
        };

        walk3::Walk<K, TOP> wk;
        wk.begin();
        // one step per plane: plane p (in rB) against plane p-1 (rA), which
        // it emits from p = 2 on; one loop body keeps the register footprint
        // small (two unrolled steps cost 16 registers more), at the price of
        // a copy of the row
        walk3::Row<K> rA, rB;
#pragma unroll 1
        for (int p = 0; p < n; ++p) {
            const int d = p % D;  // plane of the stage
            if (d == 0 && p > 0 && !wait_stage()) break;
            const int row = ring + c_slot * STAGE + lane * ROWB + d * PLANE;
            load(rB, row, zb - 1 + p);
            if (p > 0) {
                wk.step(rA, rB, p >= 2, out_x, fill, mu, emit);
                if (d == 0) {
                    __syncwarp();
                    issue();  // the previous stage (plane p-1) is free
                }
            }
            vals = row + off;
#pragma unroll
            for (int k = 0; k <= K; ++k) rA.P[k] = rB.P[k];
            if (d == D - 1 || p == n - 1) next_stage();
        }
        if (!ok) break;
        __syncwarp();
        issue();  // the item's last stage is free
    }
    __syncwarp();
    if (!ok && lane == 0) {
        // copies still in flight target this warp's ring: wait (bounded)
        // for them before the CTA can leave
        for (int q = consumed; q < s_cur[warp].issued; ++q) mbar_wait(&full[q % S], (uint32_t)((q / S) & 1));
    }
    if (COUNT) {
        const unsigned nn = __reduce_add_sync(0xffffffffu, n_emitted);
        if (lane == 0 && nn) atomicAdd(a.h.emitted, (unsigned long long)nn);
    }

    __syncthreads();
    if (SMEM)
        for (int i = tid; i < a.h.nbins; i += NTH) {
            const int v = hist[i];
            if (v) atomicAdd(a.h.acc + i, (unsigned long long)(long long)v);
        }
    // The last CTA to finish resets the work counter for the next launch and,
    // when asked, scans the bins: the CTA's adds to acc (ordered before thread
    // 0 by the barrier) are made visible device-wide by its fence before the
    // CTA counts itself finished.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(a.sched + 1, 1u) == gridDim.x - 1;
        if (s_last) {
            a.sched[0] = 0u;
            a.sched[1] = 0u;
            __threadfence();
        }
    }
    if (a.ecc_out) {
        __syncthreads();
        if (s_last) scan_bins<NTH>(a.h.acc, a.ecc_out, a.vcec_out, a.h.nbins, tid);
    }
}

template <typename T, int NWARP, bool TOP, bool NARROW, bool SMEM, bool COUNT>
cudaError_t launch_t(const Geom &g, int64_t zb, int64_t ze, const HistDst &h, bool range_check,
                     unsigned int *status, unsigned int *sched, int num_sms, cudaStream_t s, FusedScan *fs)
{
    using C = C3<T, NWARP>;
    auto encode = encode_fn();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch_y, (cuuint64_t)g.pitch_z};
    const cuuint32_t box[3] = {(cuuint32_t)(C::ROWB / C::ES), 32u, (cuuint32_t)C::D};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = encode(&map, C::ES == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                        const_cast<unsigned char *>(g.data), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorNotSupported;

    Bs3Args a{};
    a.sched = sched;
    a.nx = (int32_t)g.nx;
    a.ny = (int32_t)g.ny;
    a.nz = (int32_t)g.nz;
    a.z_begin = (int32_t)zb;
    a.z_end = (int32_t)ze;
    a.ntx = walk3::tiles_of((int)g.nx);
    a.nty = walk3::tiles_of((int)g.ny);
    a.h = h;
    a.check_range = NARROW && range_check;
    a.lo_bits = (uint32_t)h.lo;
    a.hi_bits = (uint32_t)(h.lo + h.nbins - 1);
    a.status = status;
    a.mu = walk3::make_mul();
    const bool fuse = fs && fs->ecc && zb == 0 && ze == g.nz && h.nbins <= kFusedScanMaxBins;
    a.ecc_out = fuse ? fs->ecc : nullptr;
    a.vcec_out = fuse ? fs->vcec : nullptr;
    const size_t ring_bytes = (size_t)NWARP * C::S * (C::STAGE + 12);
    a.smem_hist = SMEM;
    const size_t smem = ring_bytes + (SMEM ? (size_t)h.nbins * 4 : 0);
    auto kern = bs3_kernel<T, NWARP, TOP, NARROW, SMEM, COUNT>;
    static size_t attr_smem = 48 * 1024;  // per instantiation: dynamic smem allowed so far
    static size_t occ_smem = 0;
    static int per_sm = 0;
    if (smem > attr_smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cudaErrorNotSupported;
        }
        attr_smem = smem;
    }
    static bool carveout = false;
    if (!carveout) {  // let the rings of several CTAs share an SM
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaGetLastError();
        carveout = true;
    }
    if (occ_smem != smem || per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NWARP * 32, smem);
        if (e != cudaSuccess) return e;
        occ_smem = smem;
    }
    if (per_sm < 1) return cudaErrorNotSupported;
    const int64_t ctas_max = (int64_t)num_sms * per_sm;
    const int64_t slots = ctas_max * NWARP;  // resident warps
    const int64_t cols = (int64_t)a.ntx * a.nty;
    const int64_t depth = ze - zb;
    // z-chunks.  An item costs its planes plus two (the plane below and the
    // step that emits nothing).  Warps take items dynamically, so the launch
    // costs about (waves of `slots` items) x (item cost), a partial last wave
    // costing a whole one; a single wave is charged 10 % more (nothing hides
    // the start-up).  ECC_ZCHUNK overrides the choice (sweeps).
    int64_t zchunk = depth;
    {
        double best = -1.0;
        for (int64_t k = 1; k <= 64; ++k) {
            int64_t nc = k * slots / cols;
            if (nc < 1) nc = 1;
            const int64_t zc = (depth + nc - 1) / nc;
            nc = (depth + zc - 1) / zc;
            if (zc < 8 && k > 1) break;
            const int64_t waves = (cols * nc + slots - 1) / slots;
            const double cost = (double)waves * (double)(zc + 2) * (waves == 1 ? 1.1 : 1.0);
            if (best < 0.0 || cost < best) {
                best = cost;
                zchunk = zc;
            }
        }
        static const int64_t forced = [] {
            const char *e = std::getenv("ECC_ZCHUNK");
            return e ? (int64_t)std::atoll(e) : (int64_t)0;
        }();
        if (forced > 0) zchunk = forced < depth ? forced : depth;
    }
    a.zchunk = (int32_t)zchunk;
    const int64_t nzc = (depth + zchunk - 1) / zchunk;
    const int64_t items = cols * nzc;
    if (items > 2147483647) return cudaErrorNotSupported;
    a.nitems = (int32_t)items;
    int64_t ctas = (items + NWARP - 1) / NWARP;
    if (ctas > ctas_max) ctas = ctas_max;
    kern<<<(unsigned)ctas, NWARP * 32, smem, s>>>(map, a);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && fuse) fs->done = true;
    return e;
}

// Shared-memory bins when the range fits next to the rings.
template <typename T, int NWARP>
bool smem_bins(int nbins)
{
    return (size_t)nbins * 4 + (size_t)NWARP * C3<T, NWARP>::S * (C3<T, NWARP>::STAGE + 12) <= 160 * 1024;
}

template <typename T, int NWARP, bool TOP, bool NARROW>
cudaError_t launch_b(const Geom &g, int64_t zb, int64_t ze, const HistDst &h, bool rc, unsigned int *st,
                     unsigned int *sched, int sms, cudaStream_t s, FusedScan *fs)
{
    const bool count = h.emitted != nullptr;
    if constexpr (sizeof(T) == 1) {  // at most 256 bins: always shared
        return count ? launch_t<T, NWARP, TOP, NARROW, true, true>(g, zb, ze, h, rc, st, sched, sms, s, fs)
                     : launch_t<T, NWARP, TOP, NARROW, true, false>(g, zb, ze, h, rc, st, sched, sms, s, fs);
    } else {
        if (smem_bins<T, NWARP>(h.nbins))
            return count ? launch_t<T, NWARP, TOP, NARROW, true, true>(g, zb, ze, h, rc, st, sched, sms, s, fs)
                         : launch_t<T, NWARP, TOP, NARROW, true, false>(g, zb, ze, h, rc, st, sched, sms, s, fs);
        return count ? launch_t<T, NWARP, TOP, NARROW, false, true>(g, zb, ze, h, rc, st, sched, sms, s, fs)
                     : launch_t<T, NWARP, TOP, NARROW, false, false>(g, zb, ze, h, rc, st, sched, sms, s, fs);
    }
}

template <typename T, int NWARP>
cudaError_t launch_w(const Geom &g, int64_t zb, int64_t ze, const HistDst &h, int mode, bool rc,
                     unsigned int *st, unsigned int *sched, int sms, cudaStream_t s, FusedScan *fs)
{
    const bool top = mode == ECC_TOPCELL_MIN;
    const bool narrow = walk::range_is_narrow(h.lo, h.nbins, (int)sizeof(T));
    if (narrow)
        return top ? launch_b<T, NWARP, true, true>(g, zb, ze, h, rc, st, sched, sms, s, fs)
                   : launch_b<T, NWARP, false, true>(g, zb, ze, h, rc, st, sched, sms, s, fs);
    return top ? launch_b<T, NWARP, true, false>(g, zb, ze, h, rc, st, sched, sms, s, fs)
               : launch_b<T, NWARP, false, false>(g, zb, ze, h, rc, st, sched, sms, s, fs);
}

}  // namespace

// Loads (under lazy module loading) every 3D kernel a plan-free call with the
// default tile can launch.
cudaError_t preload_bs3d()
{
    const void *fns[] = {
        (const void *)bs3_kernel<unsigned char, 8, false, false, true, false>,
        (const void *)bs3_kernel<unsigned char, 8, true, false, true, false>,
        (const void *)bs3_kernel<unsigned char, 8, false, true, true, false>,
        (const void *)bs3_kernel<unsigned char, 8, true, true, true, false>,
        (const void *)bs3_kernel<unsigned short, 8, false, false, true, false>,
        (const void *)bs3_kernel<unsigned short, 8, true, false, true, false>,
        (const void *)bs3_kernel<unsigned short, 8, false, true, true, false>,
        (const void *)bs3_kernel<unsigned short, 8, true, true, true, false>,
        (const void *)bs3_kernel<unsigned short, 8, false, false, false, false>,
        (const void *)bs3_kernel<unsigned short, 8, true, false, false, false>,
        (const void *)bs3_kernel<unsigned short, 8, false, true, false, false>,
        (const void *)bs3_kernel<unsigned short, 8, true, true, false, false>,
    };
    cudaFuncAttributes fa;
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// tune: warps per CTA (4 or 8); anything else picks 8.
cudaError_t launch_bs3d(const Geom &g, int64_t zb, int64_t ze, const HistDst &h, int mode, bool range_check,
                        unsigned int *status, unsigned int *sched, int num_sms, int tune, cudaStream_t s,
                        FusedScan *fs)
{
    if (g.nx > 2147483647 - 64 || g.ny > 2147483647 - 64 || g.nz > 2147483647 - 64) return cudaErrorNotSupported;
    if (g.esize == 1)
        return tune == 4 ? launch_w<unsigned char, 4>(g, zb, ze, h, mode, range_check, status, sched, num_sms, s, fs)
                         : launch_w<unsigned char, 8>(g, zb, ze, h, mode, range_check, status, sched, num_sms, s, fs);
    return tune == 4 ? launch_w<unsigned short, 4>(g, zb, ze, h, mode, range_check, status, sched, num_sms, s, fs)
                     : launch_w<unsigned short, 8>(g, zb, ze, h, mode, range_check, status, sched, num_sms, s, fs);
}

}  // namespace ecc
