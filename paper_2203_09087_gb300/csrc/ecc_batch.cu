// ecc_batch.cu -- ecc_compute_batch: thousands of images of uneven shapes.
//
// Table 3 of the paper shows per-image GPU overhead amortizing over many
// files; Sec. 3.4 reassigns free blocks to new chunks.  Here the whole batch
// is one persistent kernel:
//
//  1. the host packs one descriptor per image into pinned staging memory;
//  2. a one-CTA kernel turns the descriptors into a device-side work list:
//     per image, its number of tiles (2D: 32 pairs of a 30-column window and
//     a `chunk`-row range, one per lane, so narrow images still fill a warp;
//     3D: 30x30 voxels x `chunk` planes) and the exclusive prefix of the
//     counts;
//  3. the persistent kernel's warps pull tiles from an atomic counter, find
//     their image by binary search over the prefix, and walk the tile with the
//     bit-sliced walkers (ecc_walk.cuh), reading rows straight from global
//     memory (any pitch, any alignment); each warp accumulates into its own
//     shared-memory histogram, flushed into image i's bins (offset i*nbins)
//     whenever the warp moves to another image;
//  4. one segmented scan turns all histograms into ECCs.
//
// Steps 1-4 are captured once per plan into a CUDA graph whose parameters
// live in device memory; each call updates the copy and scan nodes (source
// staging buffer, number of images, output pointer) and relaunches the graph.
// ECC_FLAG_BATCH_PER_IMAGE keeps the plain one-launch-per-image path for
// comparison.
#include <cuda_runtime.h>

#include <vector>

#include "ecc_plan.h"
#include "ecc_walk.cuh"
#include "ecc_walk2.cuh"
#include "ecc_walk3.cuh"

namespace ecc {

struct BatchImage {  // 64 bytes
    const unsigned char *data;
    int64_t nx, ny, nz;
    int64_t pitch_y, pitch_z;
    int32_t ndim, esize;
};

struct BatchHeader {
    int32_t n;
    int32_t chunk2d, chunk3d;  // chunk lengths of this call, chosen by the work-list kernel
    int32_t pad;
};

// A batch of at least this many voxels fills the GPU many times over: tail
// imbalance matters less than halo re-reads there, so it takes long chunks
// (2D rows 32, 3D planes 24: 4 % faster than 16 x 16 on the 4352-image,
// 1.96 G-voxel batch); smaller batches take the plan's tuned lengths.
constexpr long long kBigBatchVoxels = 1ll << 29;

struct BatchState {
    int32_t cap = 0;
    // device: header + descriptors, work-list prefix [cap + 1] and order [cap], counter
    unsigned char *d_desc = nullptr;
    long long *d_start = nullptr;
    int *d_order = nullptr;
    unsigned int *d_counter = nullptr;
    // pinned staging (double-buffered) and the event of each buffer's last use
    unsigned char *h_stage[2] = {nullptr, nullptr};
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    int next = 0;
    // the captured graph and the nodes updated per call
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy_node = nullptr, scan_node = nullptr;
    ScanArgs scan{};            // kernel arguments of the scan node (output set per call)
    void *scan_argv[1] = {nullptr};
    unsigned scan_grid = 0;
    int persistent_ctas = 0;
    int chunk2d = 32, chunk3d = 24;
    // the persistent kernel and its shared memory, for single-image launches
    void *fn = nullptr;
    size_t smem = 0;
    bool smem_hist = false;
};

namespace {

constexpr int kBatchWarps = 4;

struct BatchArgs {
    const BatchHeader *hdr;
    const BatchImage *img;
    long long *start;  // [n + 1] exclusive prefix of tile counts, in list order
    int *order;        // [n] image index at each list position
    unsigned int *counter;
    unsigned long long *acc;
    int32_t lo, nbins;
    int32_t chunk2d, chunk3d;
    int32_t smem_hist, range_check;  // range_check: the bins are guarded (range narrower than the type)
    int32_t check_all;               // every output voxel is compared with [lo, hi]
    uint32_t lo_bits, hi_bits;
    walk3::Mul mu;
    unsigned int *status;
};

__device__ __forceinline__ long long tiles_of(const BatchImage &im, int chunk2d, int chunk3d)
{
    if (im.ndim == 2) {
        // 32 (window, row-chunk) pairs per tile, one per lane
        const long long nwin = (im.nx + 29) / 30;
        const long long ty = (im.ny + chunk2d - 1) / chunk2d;
        return (nwin * ty + 31) / 32;
    }
    const long long tx = walk3::tiles_of((int)im.nx);
    const long long ty = walk3::tiles_of((int)im.ny);
    const long long tz = (im.nz + chunk3d - 1) / chunk3d;
    return tx * ty * tz;
}

// Inclusive prefix of x over the 1024 threads of the CTA, plus *carry (the
// sum of earlier chunks), which it then advances by this chunk's sum.
__device__ __forceinline__ long long cta_prefix(long long x, long long *s_part, long long *carry)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_part[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long p = s_part[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, p, off);
            if (lane >= off) p += y;
        }
        s_part[lane] = p;
    }
    __syncthreads();
    const long long incl = x + (warp ? s_part[warp - 1] : 0) + *carry;
    __syncthreads();
    if (tid == 1023) *carry = incl;
    __syncthreads();
    return incl;
}

// Work list (one CTA of 1024): the images in list order -- every 3D image
// first, then every 2D image, each group in the caller's order -- in
// order[], and the exclusive prefix of their tile counts in start[].  A 3D
// tile walks a z-chunk of planes and costs about twice a 2D tile, so putting
// the 2D tiles last leaves short tiles for the end of the run, when warps
// run out of work at different times.
__global__ void __launch_bounds__(1024) build_worklist(BatchArgs a)
{
    __shared__ long long s_part[32];
    __shared__ long long s_carry;
    const int n = a.hdr->n;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_carry = 0;
        *a.counter = 0u;
    }
    __syncthreads();
    // 3D images: position = number of 3D images before them (kept in start[])
    for (int base = 0; base < n; base += 1024) {
        const int i = base + tid;
        const long long f = i < n && a.img[i].ndim == 3 ? 1 : 0;
        const long long incl = cta_prefix(f, s_part, &s_carry);
        if (i < n) {
            a.start[i] = incl - f;
            if (f) a.order[incl - f] = i;
        }
    }
    const long long n3 = s_carry;
    __syncthreads();
    // 2D images: after the 3D ones
    for (int i = tid; i < n; i += 1024)
        if (a.img[i].ndim != 3) a.order[n3 + (i - a.start[i])] = i;
    __syncthreads();
    // the batch's voxels decide the chunk lengths of this call
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + tid;
        const BatchImage *im = a.img + (i < n ? i : 0);
        cta_prefix(i < n ? im->nx * im->ny * (im->ndim == 3 ? im->nz : 1) : 0, s_part, &s_carry);
    }
    const bool big = s_carry >= kBigBatchVoxels;
    const int c2 = big ? 32 : a.chunk2d, c3 = big ? 24 : a.chunk3d;
    if (tid == 0) {
        BatchHeader *hdr = const_cast<BatchHeader *>(a.hdr);
        hdr->chunk2d = c2;
        hdr->chunk3d = c3;
    }
    __syncthreads();
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int k = base + tid;
        const long long c = k < n ? tiles_of(a.img[a.order[k]], c2, c3) : 0;
        const long long incl = cta_prefix(c, s_part, &s_carry);
        if (k < n) a.start[k] = incl - c;
    }
    if (tid == 0) a.start[n] = s_carry;
}

template <int K, bool TOP, int ND>
__device__ void run_tile(const BatchArgs &a, int chunk2d, int chunk3d, const BatchImage &im, long long local,
                         const walk::Bins &em,
                         int lane)
{
    constexpr bool PF = K == 8;  // loads issued a step ahead
    const int64_t row_bytes = im.nx * (K / 8);
    if (ND == 2) {
        // Lane l walks pair q = 32 local + l: window q mod nwin of row chunk
        // q / nwin.  The 2D walker needs nothing from other lanes (each
        // window carries its own one-voxel halo), so lanes may walk
        // different rows and narrow images still fill the warp.
        const long long nwin = (im.nx + 29) / 30;
        const long long ty = (im.ny + chunk2d - 1) / chunk2d;
        const long long q = 32 * local + lane;
        if (q >= nwin * ty) return;
        const int64_t yc = q / nwin, xt = q - yc * nwin;
        const int64_t yb = yc * chunk2d;
        const int64_t ye = yb + chunk2d < im.ny ? yb + chunk2d : im.ny;
        const int64_t xw = 30 * xt - 1;
        const int64_t first = xw * (K / 8);
        const uint32_t xex = walk::x_exist_mask(xw, im.nx);
        const uint32_t out_x = xex & 0x7ffffffeu;
        // 8-bit rows: a row's words are loaded one step ahead of their use
        // (issue), so the loads are in flight while the walker works on the
        // row before; 16-bit rows load just before use (twice the words
        // held across a step would spill)
        walk2::RawWin<K> raw;
        bool raw_ok = false;
        auto issue = [&](int64_t y) {
            raw_ok = y >= 0 && y < im.ny && xex;
            if (raw_ok) walk2::load_raw<K>(im.data + y * im.pitch_y, row_bytes, first, raw);
        };
        auto finish = [&](uint32_t *P) {
            if (!raw_ok) {
#pragma unroll
                for (int i = 0; i < K; ++i) P[i] = 0u;
                P[K] = 0xffffffffu;
                return;
            }
            walk2::unpack<K>(raw, P, a.mu);
            P[K] = ~xex;
        };
        uint32_t P[K + 1];
        issue(yb - 1);
        finish(P);
        walk2::Walk<K, TOP> wk;
        wk.begin(P, a.mu);
        if (PF) issue(yb);
        for (int64_t y1 = yb; y1 <= ye; ++y1) {
            uint32_t B[K + 1];
            if (!PF) issue(y1);
            finish(B);
            if (PF && y1 < ye) issue(y1 + 1);
            if (a.check_all && y1 < ye && (~walk::in_range<K>(B, a.lo_bits, a.hi_bits) & out_x))
                atomicOr(a.status, DEV_RANGE);
            wk.step(B, y1 - 1 >= yb, out_x, a.mu,
                    [&](uint32_t m, const uint32_t *X) {
                        // values of row y1-1, just read (cached)
                        const unsigned char *row = im.data + (y1 - 1) * im.pitch_y + xw * (K / 8);
                        walk2::emit2(
                            m, X,
                            [&](int i) {
                                return K == 8 ? (int)__ldg(row + i)
                                              : (int)__ldg(reinterpret_cast<const unsigned short *>(row) + i);
                            },
                            [&](int v, int k) { em.add(v, k); });
                    });
        }
    } else {
        // 3D: the single-volume walker (ecc_walk3.cuh) over a tile of 32
        // rows x 32-voxel windows (inner tiles 30 x 30 outputs, 31 along an
        // axis at the image edge), rows read from global memory
        const int ntx = walk3::tiles_of((int)im.nx), nty = walk3::tiles_of((int)im.ny);
        const int xt = (int)(local % ntx);
        const int64_t r = local / ntx;
        const int yt = (int)(r % nty);
        const int64_t zc = r / nty;
        const int64_t zb = zc * chunk3d;
        const int64_t ze = zb + chunk3d < im.nz ? zb + chunk3d : im.nz;
        int xw, xlo, xhi, y0, ylo, yhi;
        walk3::tile_span((int)im.nx, ntx, xt, xw, xlo, xhi);
        walk3::tile_span((int)im.ny, nty, yt, y0, ylo, yhi);
        const int64_t y = y0 + lane;
        const int64_t first = (int64_t)xw * (K / 8);
        const uint32_t xex = walk::x_exist_mask(xw, im.nx);
        const bool row_ok = y < im.ny;
        const uint32_t xmask = (xhi == 32 ? 0xffffffffu : (1u << xhi) - 1u) & ~((1u << xlo) - 1u);
        const uint32_t out_x = (lane >= ylo && lane < yhi && row_ok) ? (xex & xmask) : 0u;
        const uint32_t e_row = row_ok ? ~xex : 0xffffffffu;  // existence plane of this lane's window
        walk3::Fill fill;
        fill.xl = xw == 0 ? 1u : 0u;
        fill.xr = xw + 32 >= im.nx ? 0x80000000u : 0u;
        fill.yt = lane == 0 && y0 == 0;
        fill.yb = lane == 31 && y0 + 32 >= im.ny;
        fill.edge = xw == 0 || xw + 32 >= im.nx || y0 == 0 || y0 + 32 >= im.ny;
        // 8-bit rows: a plane's words are loaded one step ahead of their use
        walk2::RawWin<K> raw;
        bool raw_ok = false;
        const unsigned char *row0 = im.data + (row_ok ? y : 0) * im.pitch_y;
        auto issue = [&](int64_t z) {
            raw_ok = z >= 0 && z < im.nz && row_ok;
            if (raw_ok) walk2::load_raw<K>(row0 + z * im.pitch_z, row_bytes, first, raw);
        };
        auto finish = [&](walk3::Row<K> &rw) {
            if (!raw_ok) {
#pragma unroll
                for (int i = 0; i < K; ++i) rw.P[i] = 0u;
                rw.P[K] = 0xffffffffu;
                return;
            }
            walk2::unpack<K>(raw, rw.P, a.mu);
            rw.P[K] = e_row;
        };
        // values of the plane being emitted: this lane's window in global
        // memory (just read, so cached)
        const unsigned char *vals = im.data;
        auto val_at = [&](int i) {
            return K == 8 ? (int)__ldg(vals + i) : (int)__ldg(reinterpret_cast<const unsigned short *>(vals) + i);
        };
        // Batch images are often rough (smoothing widths from 1 voxel), with
        // a nonzero count at several percent of the voxels: the +-1 counts
        // go through a loop of their own with the sign read from one plane,
        // several per iteration (their value loads in flight together), then
        // the rest with the full count T - 5.
        auto emit = [&](uint32_t m, const uint32_t *Tc) {
            uint32_t pm, plus;
            walk3::split_pm1_3d(Tc, pm, plus);
            pm &= m;
            uint32_t rest = m & ~pm;
            // +1 where plus (negated for the top-cell complex, (-1)^3)
            walk2::emit_units<walk2::kEmitUnroll3d>(pm, plus, TOP ? -1 : 1, val_at,
                                                  [&](int v, int k) { em.add(v, k); });
            while (rest) {
                const int i = 31 - __clz(rest);
                rest ^= 1u << i;
                const int k = bs::bits_at<4>(Tc, i) - 5;
                em.add(val_at(i), TOP ? -k : k);
            }
        };
        walk3::Walk<K, TOP> wk;
        wk.begin();
        walk3::Row<K> rA, rB;
        issue(zb - 1);
        finish(rA);
        if (PF) issue(zb);
        uint32_t bad = 0;  // output voxels outside [lo, hi] (when checked)
        for (int64_t z1 = zb; z1 <= ze; ++z1) {
            if (!PF) issue(z1);
            finish(rB);
            if (PF && z1 < ze) issue(z1 + 1);
            if (a.check_all && z1 < ze) bad |= ~walk::in_range<K>(rB.P, a.lo_bits, a.hi_bits) & out_x;
            vals = im.data + (z1 - 1) * im.pitch_z + (row_ok ? y : 0) * im.pitch_y + first;
            wk.step(rA, rB, z1 - 1 >= zb, out_x, fill, a.mu, emit);
#pragma unroll
            for (int k = 0; k <= K; ++k) rA.P[k] = rB.P[k];
        }
        if (a.check_all && __any_sync(0xffffffffu, bad != 0u) && lane == 0) atomicOr(a.status, DEV_RANGE);
    }
}

template <int K, bool TOP>
__global__ void __launch_bounds__(kBatchWarps * 32, 4) batch_kernel(BatchArgs a)
{
    extern __shared__ __align__(16) int bhist[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int *hist = a.smem_hist ? bhist + warp * a.nbins : nullptr;
    if (hist)
        for (int i = lane; i < a.nbins; i += 32) hist[i] = 0;
    __syncwarp();
    const int n = a.hdr->n;
    const int chunk2d = a.hdr->chunk2d, chunk3d = a.hdr->chunk3d;  // as the work-list kernel chose them
    const long long total = a.start[n];
    int cur = -1;      // list position of the image whose bins this warp's shared histogram holds
    int cur_img = -1;  // that image's index
    long long cur_begin = 0, cur_end = 0;  // its tile range
    auto flush = [&]() {
        if (hist && cur >= 0) {
            __syncwarp();
            unsigned long long *dst = a.acc + (size_t)cur_img * a.nbins;
            for (int i = lane; i < a.nbins; i += 32) {
                const int v = hist[i];
                if (v) {
                    atomicAdd(dst + i, (unsigned long long)(long long)v);
                    hist[i] = 0;
                }
            }
            __syncwarp();
        }
    };
    for (;;) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(a.counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        // list position owning this tile: last k with start[k] <= item (tiles
        // are handed out in list order, so it is usually the warp's last one)
        int lo = 0, hi = n - 1;
        if (cur >= 0 && item >= cur_begin && item < cur_end) {
            lo = hi = cur;
        } else if (cur >= 0 && item >= cur_end) {
            lo = cur + 1;
        }
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.start[mid] <= item)
                lo = mid;
            else
                hi = mid - 1;
        }
        if (lo != cur) {
            flush();
            cur = lo;
            cur_img = a.order[lo];
            cur_begin = a.start[lo];
            cur_end = a.start[lo + 1];
        }
        const BatchImage im = a.img[cur_img];
        const walk::Bins em{hist, a.acc + (size_t)cur_img * a.nbins, a.lo, a.nbins, a.range_check, a.status};
        if (im.ndim == 2)
            run_tile<K, TOP, 2>(a, chunk2d, chunk3d, im, item - a.start[lo], em, lane);
        else
            run_tile<K, TOP, 3>(a, chunk2d, chunk3d, im, item - a.start[lo], em, lane);
    }
    flush();
}

// The bins are guarded whenever the plan's range leaves out values of its
// type; every output voxel is compared with the bounds unless the plan opted
// out (ECC_FLAG_NO_RANGE_CHECK).
void set_range(BatchArgs &args, const ecc_plan_s *p)
{
    args.range_check = walk::range_is_narrow(args.lo, args.nbins, p->d.dtype == ECC_U16 ? 2 : 1);
    args.check_all = args.range_check && !(p->d.flags & ECC_FLAG_NO_RANGE_CHECK);
    args.lo_bits = (uint32_t)args.lo;
    args.hi_bits = (uint32_t)(args.lo + args.nbins - 1);
    args.mu = walk3::make_mul();
}

template <int K, bool TOP>
cudaError_t batch_instance(void **fn, size_t smem, int *per_sm)
{
    auto kern = batch_kernel<K, TOP>;
    *fn = reinterpret_cast<void *>(kern);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, kBatchWarps * 32, smem);
}

cudaError_t capture_graph(ecc_plan_s *p, BatchState *b)
{
    const bool top = p->d.complex_mode == ECC_TOPCELL_MIN;
    const int K = p->d.dtype == ECC_U16 ? 16 : 8;
    const bool smem_hist = (size_t)kBatchWarps * p->nbins * 4 <= 96 * 1024;
    const size_t smem = smem_hist ? (size_t)kBatchWarps * p->nbins * 4 : 0;
    void *fn = nullptr;
    int per_sm = 0;
    cudaError_t e = K == 8 ? (top ? batch_instance<8, true>(&fn, smem, &per_sm) : batch_instance<8, false>(&fn, smem, &per_sm))
                           : (top ? batch_instance<16, true>(&fn, smem, &per_sm) : batch_instance<16, false>(&fn, smem, &per_sm));
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    b->persistent_ctas = p->num_sms * per_sm;
    b->fn = fn;
    b->smem = smem;
    b->smem_hist = smem_hist;

    BatchArgs args{};  // the kernel nodes copy their arguments at creation
    args.hdr = reinterpret_cast<const BatchHeader *>(b->d_desc);
    args.img = reinterpret_cast<const BatchImage *>(b->d_desc + sizeof(BatchHeader));
    args.start = b->d_start;
    args.order = b->d_order;
    args.counter = b->d_counter;
    args.acc = p->acc;
    args.lo = p->d.lo;
    args.nbins = p->nbins;
    args.chunk2d = b->chunk2d;
    args.chunk3d = b->chunk3d;
    args.smem_hist = smem_hist;
    set_range(args, p);
    args.status = p->status;

    e = cudaGraphCreate(&b->graph, 0);
    if (e != cudaSuccess) return e;
    // copy node: staging -> device descriptors (parameters replaced per call)
    cudaMemcpy3DParms cp{};
    cp.srcPtr = make_cudaPitchedPtr(b->h_stage[0], 64, 64, 1);
    cp.dstPtr = make_cudaPitchedPtr(b->d_desc, 64, 64, 1);
    cp.extent = make_cudaExtent(64, 1, 1);
    cp.kind = cudaMemcpyHostToDevice;
    e = cudaGraphAddMemcpyNode(&b->copy_node, b->graph, nullptr, 0, &cp);
    if (e != cudaSuccess) return e;
    // work-list kernel
    cudaGraphNode_t build_node, batch_node;
    void *bargs[] = {&args};
    cudaKernelNodeParams kp{};
    kp.func = reinterpret_cast<void *>(build_worklist);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1024);
    kp.kernelParams = bargs;
    e = cudaGraphAddKernelNode(&build_node, b->graph, &b->copy_node, 1, &kp);
    if (e != cudaSuccess) return e;
    // persistent kernel
    kp.func = fn;
    kp.gridDim = dim3((unsigned)b->persistent_ctas);
    kp.blockDim = dim3(kBatchWarps * 32);
    kp.sharedMemBytes = (unsigned)smem;
    e = cudaGraphAddKernelNode(&batch_node, b->graph, &build_node, 1, &kp);
    if (e != cudaSuccess) return e;
    // segmented scan (output pointer set per call; image count read on the device)
    b->scan = ScanArgs{};
    b->scan.acc = p->acc;
    b->scan.nbins = p->nbins;
    b->scan.n = (int64_t)p->d.max_images * p->nbins;
    b->scan.ws = p->scan_ws();
    b->scan.status = p->status;
    b->scan.n_seg_dev = reinterpret_cast<const int *>(b->d_desc);  // BatchHeader::n
    b->scan_grid = (unsigned)scan_tiles(p->d.max_images, p->nbins);
    b->scan.ntiles = (int32_t)b->scan_grid;
    b->scan_argv[0] = &b->scan;
    kp = cudaKernelNodeParams{};
    kp.func = const_cast<void *>(scan_kernel_entry());
    kp.gridDim = dim3(b->scan_grid);
    kp.blockDim = dim3(kScanThreads);
    kp.kernelParams = b->scan_argv;
    e = cudaGraphAddKernelNode(&b->scan_node, b->graph, &batch_node, 1, &kp);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    return e;
}

ecc_status ensure_batch(ecc_plan_s *p)
{
    if (p->batch) return ECC_OK;
    auto *b = new BatchState();
    b->cap = p->d.max_images;
    b->chunk2d = p->tuned_batch[0] > 0 ? p->tuned_batch[0] : 32;
    b->chunk3d = p->tuned_batch[1] > 0 ? p->tuned_batch[1] : 24;
    const size_t desc_bytes = sizeof(BatchHeader) + sizeof(BatchImage) * (size_t)b->cap;
    cudaError_t e = cudaMalloc(&b->d_desc, desc_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_start, sizeof(long long) * ((size_t)b->cap + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int) * (size_t)b->cap);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 256);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMallocHost(&b->h_stage[i], desc_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->stage_ev[i], cudaEventDisableTiming);
    }
    p->batch = b;
    if (e == cudaSuccess) e = capture_graph(p, b);
    if (e != cudaSuccess) {
        release_batch(p);
        return cuda_fail(e, "ecc_compute_batch: batch state set-up");
    }
    return ECC_OK;
}

}  // namespace

namespace {

// The work list of one image, written on the device from a by-value
// descriptor (no host staging, so a single-image call never waits).
__global__ void init_single(BatchArgs a, BatchImage im)
{
    BatchHeader *hdr = const_cast<BatchHeader *>(a.hdr);
    hdr->n = 1;
    const_cast<BatchImage *>(a.img)[0] = im;
    hdr->chunk2d = a.chunk2d;
    hdr->chunk3d = a.chunk3d;
    a.order[0] = 0;
    a.start[0] = 0;
    a.start[1] = tiles_of(im, a.chunk2d, a.chunk3d);
    *a.counter = 0u;
}

}  // namespace

// One whole 3D image through the persistent batch kernel (any pitch: rows
// come from aligned 32-bit global loads): the path for images whose row
// pitch rules out the TMA kernel.  Two stream launches (work list, kernel);
// accumulates into h.acc like the other stencils.
cudaError_t launch_batch_single(ecc_plan_s *p, const Geom &g, const HistDst &h, cudaStream_t s)
{
    if (ensure_batch(p) != ECC_OK) return cudaErrorMemoryAllocation;
    BatchState *b = p->batch;
    BatchArgs args{};
    args.hdr = reinterpret_cast<const BatchHeader *>(b->d_desc);
    args.img = reinterpret_cast<const BatchImage *>(b->d_desc + sizeof(BatchHeader));
    args.start = b->d_start;
    args.order = b->d_order;
    args.counter = b->d_counter;
    args.acc = h.acc;
    args.lo = h.lo;
    args.nbins = h.nbins;
    args.chunk2d = b->chunk2d;
    args.chunk3d = b->chunk3d;
    args.smem_hist = b->smem_hist;
    set_range(args, p);
    args.status = p->status;
    const BatchImage im{g.data, g.nx, g.ny, g.nz, g.pitch_y, g.pitch_z, g.ndim, g.esize};
    init_single<<<1, 1, 0, s>>>(args, im);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        void *argv[] = {&args};
        e = cudaLaunchKernel(b->fn, dim3((unsigned)b->persistent_ctas), dim3(kBatchWarps * 32), argv, b->smem, s);
    }
    return e;
}

// launch_batch_single without a plan, for ecc_compute_noalloc: the one-image
// work list lives in kBatchSingleWsBytes of the caller's scratch (8-byte
// aligned; nothing allocated), and the grid comes from an occupancy query.
cudaError_t launch_batch_single_ws(const Geom &g, const HistDst &h, int complex_mode, bool check_values, void *ws,
                                   unsigned int *status, int num_sms, cudaStream_t s)
{
    const bool top = complex_mode == ECC_TOPCELL_MIN;
    const bool wide = g.esize == 2;
    const bool smem_hist = (size_t)kBatchWarps * h.nbins * 4 <= 96 * 1024;
    const size_t smem = smem_hist ? (size_t)kBatchWarps * h.nbins * 4 : 0;
    void *fn = nullptr;
    int per_sm = 0;
    cudaError_t e = wide ? (top ? batch_instance<16, true>(&fn, smem, &per_sm) : batch_instance<16, false>(&fn, smem, &per_sm))
                         : (top ? batch_instance<8, true>(&fn, smem, &per_sm) : batch_instance<8, false>(&fn, smem, &per_sm));
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    unsigned char *w = static_cast<unsigned char *>(ws);
    BatchArgs args{};
    args.hdr = reinterpret_cast<const BatchHeader *>(w);         // 16 bytes
    args.img = reinterpret_cast<const BatchImage *>(w + 16);     // 64 bytes
    args.start = reinterpret_cast<long long *>(w + 80);          // 2 words
    args.order = reinterpret_cast<int *>(w + 96);
    args.counter = reinterpret_cast<unsigned int *>(w + 100);
    args.acc = h.acc;
    args.lo = h.lo;
    args.nbins = h.nbins;
    args.chunk2d = 32;
    args.chunk3d = 24;
    args.smem_hist = smem_hist;
    args.range_check = walk::range_is_narrow(h.lo, h.nbins, g.esize);
    args.check_all = args.range_check && check_values;
    args.lo_bits = (uint32_t)h.lo;
    args.hi_bits = (uint32_t)(h.lo + h.nbins - 1);
    args.mu = walk3::make_mul();
    args.status = status;
    const BatchImage im{g.data, g.nx, g.ny, g.nz, g.pitch_y, g.pitch_z, g.ndim, g.esize};
    init_single<<<1, 1, 0, s>>>(args, im);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        void *argv[] = {&args};
        e = cudaLaunchKernel(fn, dim3((unsigned)(num_sms * per_sm)), dim3(kBatchWarps * 32), argv, smem, s);
    }
    return e;
}

cudaError_t preload_batch()
{
    const void *fns[] = {(const void *)batch_kernel<8, false>, (const void *)batch_kernel<8, true>,
                         (const void *)batch_kernel<16, false>, (const void *)batch_kernel<16, true>,
                         (const void *)init_single};
    cudaFuncAttributes fa;
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The batch state of a plan (work-list buffers, staging, the captured
// graph) made ahead of its first batched call.
ecc_status prepare_batch(ecc_plan_s *p) { return ensure_batch(p); }

void release_batch(ecc_plan_s *p)
{
    BatchState *b = p->batch;
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (int i = 0; i < 2; ++i) {
        if (b->stage_ev[i]) cudaEventDestroy(b->stage_ev[i]);
        if (b->h_stage[i]) cudaFreeHost(b->h_stage[i]);
    }
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_start) cudaFree(b->d_start);
    if (b->d_order) cudaFree(b->d_order);
    if (b->d_counter) cudaFree(b->d_counter);
    delete b;
    p->batch = nullptr;
}

}  // namespace ecc

using namespace ecc;

extern "C" ecc_status ecc_compute_batch(ecc_plan_t p, int32_t n, const ecc_image *descs, int64_t *d_ecc,
                                        void *stream)
{
    if (!p) {
        set_error("ecc_compute_batch: NULL plan");
        return ECC_E_INVALID;
    }
    if (n < 1 || !descs || !d_ecc) {
        set_error("ecc_compute_batch: need n >= 1, descriptors and an output");
        return ECC_E_INVALID;
    }
    if (n > p->d.max_images) {
        set_error("ecc_compute_batch: more images than the plan's max_images");
        return ECC_E_BUSY;
    }
    std::vector<Geom> geoms(n);
    int64_t total = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t nv = 0;
        ecc_status st = image_geom(&descs[i], p->d.dtype, 0, &geoms[i], &nv, false);
        if (st != ECC_OK) return st;
        total += nv;
    }
    if (total > p->d.max_voxels) {
        set_error("ecc_compute_batch: total voxels exceed the plan's max_voxels");
        return ECC_E_BUSY;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->last_launches = 0;

    if (p->d.flags & ECC_FLAG_BATCH_PER_IMAGE) {
        for (int32_t i = 0; i < n; ++i) {
            const Geom &g = geoms[i];
            HistDst h{p->acc + (size_t)i * p->nbins, p->d.lo, p->nbins};
            cudaError_t e = launch_stencil(p, g, 0, g.ndim == 3 ? g.nz : g.ny, h, s);
            if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_batch: stencil launch");
        }
        cudaError_t e = launch_scan(p->acc, reinterpret_cast<long long *>(d_ecc), nullptr, n, p->nbins,
                                    p->scan_ws(), p->status, s);
        ++p->last_launches;
        if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_batch: scan launch");
        return ECC_OK;
    }

    ecc_status st = ensure_batch(p);
    if (st != ECC_OK) return st;
    BatchState *b = p->batch;
    // the staging buffer used two calls ago must be free before rewriting it
    const int buf = b->next;
    b->next ^= 1;
    cudaError_t e = cudaEventSynchronize(b->stage_ev[buf]);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_batch: staging wait");
    BatchHeader *hh = reinterpret_cast<BatchHeader *>(b->h_stage[buf]);
    BatchImage *hi = reinterpret_cast<BatchImage *>(b->h_stage[buf] + sizeof(BatchHeader));
    hh->n = n;
    for (int32_t i = 0; i < n; ++i) {
        const Geom &g = geoms[i];
        hi[i] = BatchImage{g.data, g.nx, g.ny, g.nz, g.pitch_y, g.pitch_z, g.ndim, g.esize};
    }
    const size_t bytes = sizeof(BatchHeader) + sizeof(BatchImage) * (size_t)n;
    cudaMemcpy3DParms cp{};
    cp.srcPtr = make_cudaPitchedPtr(b->h_stage[buf], bytes, bytes, 1);
    cp.dstPtr = make_cudaPitchedPtr(b->d_desc, bytes, bytes, 1);
    cp.extent = make_cudaExtent(bytes, 1, 1);
    cp.kind = cudaMemcpyHostToDevice;
    e = cudaGraphExecMemcpyNodeSetParams(b->exec, b->copy_node, &cp);
    if (e == cudaSuccess) {
        b->scan.ecc = reinterpret_cast<long long *>(d_ecc);
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void *>(scan_kernel_entry());
        kp.gridDim = dim3(b->scan_grid);
        kp.blockDim = dim3(kScanThreads);
        kp.kernelParams = b->scan_argv;
        e = cudaGraphExecKernelNodeSetParams(b->exec, b->scan_node, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->stage_ev[buf], s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_batch: graph launch");
    p->last_launches = 3;  // work list, persistent kernel, scan
    return ECC_OK;
}
