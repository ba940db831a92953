// ecc_scan.cu -- VCEC -> ECC: single-pass segmented inclusive prefix sum.
//
// Sec. 2.3: ECC_i = sum_{j <= i} VCEC_j; the paper notes that a log(m)
// parallel scan is a practical alternative on GPUs and itself finishes on the
// CPU.  Here the scan stays on the device: one pass, decoupled look-back
// (each tile publishes its aggregate, then its inclusive prefix, and a tile
// waits only for its predecessors' published values), segmented so that a
// batch of images (segment i = bins of image i) is scanned in one launch.
// Tiles take their index from an atomic counter, so a tile only ever waits
// on tiles that already started; every wait is bounded by %globaltimer and
// reports DEV_TIMEOUT instead of hanging.  The scan also copies the VCEC
// out if asked and zeroes the accumulator, and the last tile resets the
// look-back state, so the workspace is clean for the next call.
#include "ecc_internal.h"
#include "ecc_sync.cuh"

namespace ecc {
namespace {

// Segmented-scan operator on (flag, value): a then b.
__device__ __forceinline__ void seg_combine(bool af, long long av, bool &bf, long long &bv)
{
    if (!bf) bv += av;
    bf = bf || af;
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(ScanArgs a)
{
    constexpr int kWarps = kScanThreads / 32;
    __shared__ unsigned int s_tile;
    __shared__ long long s_wv[kWarps];
    __shared__ int s_wf[kWarps];
    __shared__ long long s_carry;
    __shared__ int s_last;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.n_seg_dev) a.n = (int64_t)(*a.n_seg_dev) * a.nbins;
    if (threadIdx.x == 0) s_tile = atomicAdd(a.ws.tile_counter, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    // The counter starts at zero (plan creation, and every scan's last tile
    // resets it), so the index is below the grid; if the state was ever not
    // clean, report it and touch nothing rather than write past the arrays.
    if (tile >= (int64_t)gridDim.x) {
        if (threadIdx.x == 0) atomicOr(a.status, DEV_STATE);
        return;
    }
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;

    long long v[kScanItems], orig[kScanItems];
    bool f[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + i;
        const bool in = idx < a.n;
        orig[i] = in ? (long long)a.acc[idx] : 0;
        v[i] = orig[i];
        f[i] = in && (idx % a.nbins == 0);
    }
    // thread-local segmented inclusive scan
#pragma unroll
    for (int i = 1; i < kScanItems; ++i)
        if (!f[i]) v[i] += v[i - 1];
    bool tf = false;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) tf = tf || f[i];
    long long tv = v[kScanItems - 1];

    // warp-level inclusive scan of the thread aggregates
    bool wf = tf;
    long long wv = tv;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long pv = __shfl_up_sync(0xffffffffu, wv, off);
        const int pf = __shfl_up_sync(0xffffffffu, (int)wf, off);
        if (lane >= off) seg_combine(pf != 0, pv, wf, wv);
    }
    if (lane == 31) {
        s_wv[warp] = wv;
        s_wf[warp] = wf;
    }
    __syncthreads();
    if (warp == 0) {
        bool xf = lane < kWarps ? s_wf[lane] != 0 : false;
        long long xv = lane < kWarps ? s_wv[lane] : 0;
#pragma unroll
        for (int off = 1; off < kWarps; off <<= 1) {
            const long long pv = __shfl_up_sync(0xffffffffu, xv, off);
            const int pf = __shfl_up_sync(0xffffffffu, (int)xf, off);
            if (lane >= off) seg_combine(pf != 0, pv, xf, xv);
        }
        if (lane < kWarps) {
            s_wv[lane] = xv;  // inclusive over warps
            s_wf[lane] = xf;
        }
    }
    __syncthreads();
    // exclusive prefix of this thread inside the tile
    long long ev = __shfl_up_sync(0xffffffffu, wv, 1);
    int ef = __shfl_up_sync(0xffffffffu, (int)wf, 1);
    if (lane == 0) {
        ev = 0;
        ef = 0;
    }
    if (warp > 0) {
        // prefix from earlier warps, then this warp's earlier lanes
        bool pf = s_wf[warp - 1] != 0;
        long long pv = s_wv[warp - 1];
        bool cf = ef != 0;
        long long cv = ev;
        if (lane == 0) {
            cf = pf;
            cv = pv;
        } else {
            seg_combine(pf, pv, cf, cv);
        }
        ef = cf;
        ev = cv;
    }
    const bool tile_f = s_wf[kWarps - 1] != 0;
    const long long tile_v = s_wv[kWarps - 1];

    // decoupled look-back (one thread).  Each tile owns two value slots: its
    // aggregate (published with status 1, never rewritten) and its inclusive
    // prefix (published with status 2), so a reader never sees a value that
    // does not match the status it read.
    if (threadIdx.x == 0) {
        volatile int *st = a.ws.tile_status;
        volatile long long *agg = a.ws.tile_value;
        volatile long long *incl = a.ws.tile_value + a.ws.max_tiles;
        if (tile_f) {  // the tile's inclusive prefix is known right away
            incl[tile] = tile_v;
            __threadfence();
            st[tile] = 2;
        } else {
            agg[tile] = tile_v;
            __threadfence();
            st[tile] = 1;
        }
        long long carry = 0;
        // tiles past the data (a graph launched for more images than this
        // call has) need nothing from their predecessors
        const bool needs_carry = (tile * kScanTile) % a.nbins != 0 && tile * kScanTile < a.n;
        if (needs_carry) {
            int64_t j = tile - 1;
            while (j >= 0) {
                const int s = sync::flag_wait(st + j);
                if (s == 0) {
                    atomicOr(a.status, DEV_TIMEOUT);
                    break;
                }
                __threadfence();
                if (s == 2) {
                    carry += incl[j];
                    break;
                }
                carry += agg[j];
                --j;
            }
        }
        if (!tile_f) {
            incl[tile] = carry + tile_v;
            __threadfence();
            st[tile] = 2;
        }
        s_carry = carry;
    }
    __syncthreads();
    const long long carry = s_carry;

    // v[i] restarts at every segment start inside this thread; before the
    // thread's first start it needs the thread's exclusive prefix ev, and,
    // when no start precedes the thread in the tile either, the carry.
    bool start_in_thread = false;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        start_in_thread = start_in_thread || f[i];
        long long out = v[i];
        if (!start_in_thread) out += ev + (ef ? 0 : carry);
        const int64_t idx = base + i;
        if (idx < a.n) {
            a.ecc[idx] = out;
            if (a.vcec) a.vcec[idx] = orig[i];
            a.acc[idx] = 0ull;
        }
    }

    // the last tile to finish resets the look-back state
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(a.ws.done_counter, 1u);
        s_last = (done == gridDim.x - 1u);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int i = threadIdx.x; i < (int)gridDim.x; i += kScanThreads) a.ws.tile_status[i] = 0;
        if (threadIdx.x == 0) {
            *a.ws.tile_counter = 0u;
            *a.ws.done_counter = 0u;
        }
    }
}

}  // namespace

const void *scan_kernel_entry() { return reinterpret_cast<const void *>(scan_kernel); }

int64_t scan_tiles(int64_t n_seg, int32_t nbins)
{
    const int64_t n = n_seg * (int64_t)nbins;
    return (n + kScanTile - 1) / kScanTile;
}

// Loads (under lazy module loading) the scan kernel.
cudaError_t preload_scan()
{
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, (const void *)scan_kernel);
}

cudaError_t launch_scan(unsigned long long *acc, long long *ecc, long long *vcec, int64_t n_seg,
                        int32_t nbins, const ScanWs &ws, unsigned int *status, cudaStream_t s)
{
    ScanArgs a{};
    a.acc = acc;
    a.ecc = ecc;
    a.vcec = vcec;
    a.n = n_seg * (int64_t)nbins;
    a.nbins = nbins;
    const int64_t nt = scan_tiles(n_seg, nbins);
    if (nt > ws.max_tiles || nt > 2147483647) return cudaErrorInvalidValue;
    a.ntiles = (int32_t)nt;
    a.ws = ws;
    a.status = status;
    a.n_seg_dev = nullptr;
    scan_kernel<<<(unsigned)nt, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ecc
