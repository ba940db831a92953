/*
 * ecc.h -- C ABI of the GB300 (sm_103a) Euler characteristic curve library.
 *
 * Problem (Wang, Wagner, Chen, "GPU Computation of the Euler Characteristic
 * Curve for Imaging Data", SoCG 2022, Sec. 2): given a 2D or 3D integer
 * grayscale image and a gray-level range [lo, hi], return the integer vector
 *
 *     ECC[g] = chi(K_{<= lo+g}) = sum_j (-1)^j c_j(K_{<= lo+g}),  g = 0..hi-lo
 *
 * (Sec. 2.2, Eq. 1), computed as the prefix sum (Sec. 2.3) of the vector of
 * changes VCEC, where each voxel adds (-1)^dim for every cell it introduces
 * (Sec. 2.3 "Faces introduced by a voxel", Algorithm 1).  The paper indexes
 * the ECC by the values present in the image (t_i in Eq. 1); this library
 * returns every level in [lo, hi], of which the paper's sequence is the
 * subsequence at present values.
 *
 * Two cubical complexes are supported (ecc_complex):
 *   ECC_VERTEX_MAX   voxels are the VERTICES of the cubical grid; a cell
 *                    (vertex, edge, square, cube) exists when all its vertices
 *                    are in the image and enters at the MAX of its vertex
 *                    values.  Each voxel introduces the cells it is the
 *                    maximum of, ties going to the lowest linear index.
 *   ECC_TOPCELL_MIN  voxels are the TOP-dimensional cells (Sec. 2.1); every
 *                    lower cell takes the MIN over its top-dimensional
 *                    cofaces, ties going to the lowest linear index
 *                    (Sec. 2.3); the image boundary behaves like the paper's
 *                    +infinity collar (Sec. 3.3 "Branching").
 *
 * Conventions (all entry points):
 *  - Every call returns an ecc_status; no C++ exception crosses this ABI.
 *    On failure ecc_last_error() returns a message for the calling thread.
 *  - Image and ECC buffers passed to ecc_compute / ecc_compute_batch are
 *    DEVICE pointers owned by the caller, who keeps them alive until the
 *    work queued on `stream` has finished.  `stream` is a cudaStream_t
 *    passed as void* (NULL = the legacy default stream).
 *  - Layout: row-major, dims[0] slowest (the paper's chunking cuts along
 *    dims[0], Sec. 3.4).  Pitches are in bytes; 0 means dense.
 *  - Results are exact int64; there is no floating point anywhere.
 *  - Values outside [lo, hi] are reported on the device (ECC_E_RANGE from
 *    ecc_status_get): when [lo, hi] leaves out values of the element type,
 *    every voxel is compared with both bounds.  A plan whose range is the
 *    type's whole range (0..255 for ECC_U8, 0..65535 for ECC_U16) cannot
 *    meet such a value and checks nothing.  ECC_FLAG_NO_RANGE_CHECK skips
 *    the comparison of every voxel; an offending voxel whose signed cell
 *    count is nonzero is then still reported.  Offending voxels never reach
 *    the histogram.
 *  - A plan is used by one host thread at a time and by one stream at a
 *    time (calls on a plan are ordered on the stream they are issued to).
 *    The server (ecc_server_*) is thread-safe.
 *  - Everything runs on the CUDA device that is current when the plan or
 *    server is created.
 */
#ifndef ECC_GB300_ECC_H
#define ECC_GB300_ECC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ECC_OK = 0,
    ECC_E_INVALID = 1,    /* bad argument: ndim, dims, pitch, range, dtype, null pointer */
    ECC_E_RANGE = 2,      /* the device saw an image value outside [lo, hi] */
    ECC_E_NOMEM = 3,      /* device or pinned-host allocation failed, or over the HBM budget */
    ECC_E_CUDA = 4,       /* a CUDA runtime call failed (message in ecc_last_error) */
    ECC_E_TIMEOUT = 5,    /* a bounded device wait or a host wait ran out */
    ECC_E_BUSY = 6,       /* the object is in use (e.g. a batch larger than the plan) */
    ECC_E_SHUTDOWN = 7,   /* the server is shutting down */
    ECC_E_CANCELLED = 8   /* the job was cancelled before it ran */
} ecc_status;

/* ECC_F32: float32 images, accepted only by ecc_compute_levels (plans are
 * ECC_U8 or ECC_U16). */
typedef enum { ECC_U8 = 1, ECC_U16 = 2, ECC_F32 = 3 } ecc_dtype;

typedef enum { ECC_VERTEX_MAX = 0, ECC_TOPCELL_MIN = 1 } ecc_complex;

/* One image or volume.  data: device pointer (host pointer only where an
 * entry point says so).  ndim: 2 or 3.  dims[0..ndim-1] >= 1, dims[0]
 * slowest.  row_pitch: bytes between consecutive rows (steps of
 * dims[ndim-2]); slice_pitch: bytes between consecutive slices (3D only,
 * steps of dims[0]).  0 = dense.  Pitches must be multiples of the element
 * size and at least the dense extent. */
typedef struct ecc_image {
    const void *data;
    int32_t ndim;
    int32_t dtype;          /* ecc_dtype */
    int64_t dims[3];
    int64_t row_pitch;
    int64_t slice_pitch;
} ecc_image;

/* An image of 2 to 4 dimensions (ecc_compute_nd).  dims[0..ndim-1] >= 1,
 * dims[0] slowest.  pitches[a] (a = 0 .. ndim-2): bytes between
 * consecutive indices of axis a; 0 = dense.  Pitches must be multiples of
 * the element size and hold the extent of the axes inside them. */
typedef struct ecc_image_nd {
    const void *data;
    int32_t ndim;
    int32_t dtype;          /* ECC_U8 or ECC_U16 */
    int64_t dims[4];
    int64_t pitches[3];
} ecc_image_nd;

/* Plan flags. */
#define ECC_FLAG_NO_RANGE_CHECK   0x1u  /* caller guarantees lo <= value <= hi: skip the per-voxel check */
#define ECC_FLAG_NO_AUTOTUNE      0x2u  /* use built-in tile defaults, never time candidates */
#define ECC_FLAG_KERNEL_DIRECT    0x10u /* force the one-thread-per-voxel stencil kernel */
#define ECC_FLAG_KERNEL_BITSLICE  0x20u /* force the bit-sliced stencil kernel (where it applies) */
#define ECC_FLAG_BATCH_PER_IMAGE  0x40u /* ecc_compute_batch: one stencil launch per image (baseline) */
#define ECC_FLAG_TIME_KERNELS     0x80u /* record CUDA events around every stencil launch */
#define ECC_FLAG_COUNT_EMITTED    0x100u /* single-image stencils count voxels with a nonzero count */

typedef struct ecc_plan_desc {
    int32_t dtype;          /* ecc_dtype of every image computed with this plan */
    int32_t lo, hi;         /* gray-level range; nbins = hi - lo + 1, 1 <= nbins <= 65536 */
    int32_t complex_mode;   /* ecc_complex */
    int32_t max_images;     /* largest batch (ecc_compute_batch); >= 1 */
    int32_t reserved;       /* must be 0 */
    int64_t max_voxels;     /* largest total voxel count of one call (sum over a batch) */
    uint32_t flags;         /* ECC_FLAG_* */
    uint32_t reserved2;     /* must be 0 */
} ecc_plan_desc;

typedef struct ecc_plan_s *ecc_plan_t;

/* Create a plan: validates the description, picks the kernel variant and its
 * tile shape (autotuned on first use per GPU model unless
 * ECC_FLAG_NO_AUTOTUNE), and allocates the plan's device workspace (the
 * int64 VCEC accumulators, scan flags and a status word) and its pinned
 * staging buffers.  Ownership: the caller owns *out and frees it with
 * ecc_plan_destroy.  Errors: ECC_E_INVALID, ECC_E_NOMEM, ECC_E_CUDA. */
ecc_status ecc_plan(ecc_plan_t *out, const ecc_plan_desc *desc);

/* Synchronizes the plan's pending work and frees the plan. */
ecc_status ecc_plan_destroy(ecc_plan_t plan);

/* Number of bins (hi - lo + 1) of a plan, or -1 for an invalid handle. */
int32_t ecc_plan_nbins(ecc_plan_t plan);

/* ECC of one image, asynchronously on `stream` (Sec. 2.3: per-voxel
 * contributions into a histogram over gray levels, then the prefix sum).
 *   img       device image; img->dtype must equal the plan's dtype and its
 *             voxel count must not exceed max_voxels.
 *   d_ecc     device int64[nbins], written: ECC[g] = chi(K_{<= lo+g}).
 *   d_vcec    optional device int64[nbins] (NULL to skip), written with the
 *             VCEC (per-level change of the Euler characteristic).
 * No host synchronization; device-detected errors are read with
 * ecc_status_get.  Errors returned directly: ECC_E_INVALID, ECC_E_CUDA. */
ecc_status ecc_compute(ecc_plan_t plan, const ecc_image *img, int64_t *d_ecc,
                       int64_t *d_vcec, void *stream);

/* Same as ecc_compute, but the image and the ECC live in HOST memory: the
 * image is copied to the device in chunks along dims[0] on the plan's copy
 * stream while earlier chunks are processed (the paper's streaming with a
 * one-voxel collar and copy/compute overlap, Sec. 3.4), and the ECC is
 * copied back.  Synchronous: returns when h_ecc is written.  Pinned host
 * memory gives the fastest copies; pageable memory works.  Errors as
 * ecc_compute plus ECC_E_RANGE (device errors are checked before return). */
ecc_status ecc_compute_host(ecc_plan_t plan, const ecc_image *h_img, int64_t *h_ecc, void *stream);

/* ECC of a float32 image at m given thresholds (Eq. 1 with the t_i given:
 * ECC_i = chi(K_{<= t_i})), asynchronously on `stream`.  The paper's
 * datasets are float32 and its kernel bins values as integers (Algorithm
 * 2); here each voxel is mapped to the number of levels strictly below it
 * (NaN: above every level) -- a monotone map, so a cell is in K_{<= t_i}
 * exactly when its mapped value is <= i -- into a copy in the plan's
 * staging memory, and the integer stencil and scan follow.
 *   plan      ECC_U8 (m <= 255) or ECC_U16 plan with lo = 0 and hi >= m;
 *             its max_voxels bounds the image; the copy is 1 (ECC_U8) or 2
 *             bytes per voxel, allocated on first use.
 *   img       device image, dtype ECC_F32, 4-byte aligned pitches.
 *   d_levels  device float[m], ascending (ties allowed; the order is
 *             checked on the device).
 *   d_ecc     device int64[m], written: d_ecc[i] = chi(K_{<= d_levels[i]}).
 * No host synchronization.  Errors returned directly: ECC_E_INVALID,
 * ECC_E_BUSY (more voxels than max_voxels), ECC_E_NOMEM, ECC_E_CUDA;
 * through ecc_status_get: ECC_E_INVALID (levels not ascending),
 * ECC_E_TIMEOUT. */
ecc_status ecc_compute_levels(ecc_plan_t plan, const ecc_image *img, const float *d_levels, int32_t m,
                              int64_t *d_ecc, void *stream);

/* Eq. 1's thresholds of a float32 image, found on the device: the values
 * present in it, distinct and ascending, t_1 < ... < t_n (Sec. 2.2: the
 * paper's ECC is indexed by them).  ecc_compute_levels at these n levels is
 * then the paper's ECC sequence.  A NaN voxel is in no sublevel set and
 * defines no threshold; -0.0 is the value 0.0 and is reported as +0.0.
 *   plan        any plan; its max_voxels bounds the image.  A hash table of
 *               about 8 * max_levels bytes is allocated in it on first use.
 *   img         device image, dtype ECC_F32, 4-byte aligned pitches.
 *   d_levels    device float[max_levels], written with the n levels in
 *               ascending order when n <= max_levels (untouched otherwise).
 *   max_levels  1..65536.
 *   d_count     device int32, written n, or max_levels + 1 when the image
 *               holds more distinct values than that.
 * Asynchronous on `stream` (three launches; the caller reads d_count to
 * learn n).  Errors returned directly: ECC_E_INVALID, ECC_E_BUSY (more
 * voxels than max_voxels), ECC_E_NOMEM, ECC_E_CUDA. */
ecc_status ecc_levels_present(ecc_plan_t plan, const ecc_image *img, float *d_levels, int32_t max_levels,
                              int32_t *d_count, void *stream);

/* The paper's ECC sequence of a float32 image (Eq. 1 at its present values):
 * ecc_levels_present, then ecc_compute_levels at the n levels found.
 *   plan        as for ecc_compute_levels, with hi >= the number of
 *               distinct values (an ECC_U16 plan with hi = 65535 takes any).
 *   d_levels    device float[max_levels]: the levels (first n entries).
 *   h_count     host int32, written n (max_levels + 1 when there are more).
 *   d_ecc       device int64[max_levels]: d_ecc[i] = chi(K_{<= d_levels[i]})
 *               for i < n.
 * Synchronizes `stream` once, to read n.  Errors as ecc_levels_present and
 * ecc_compute_levels, plus ECC_E_BUSY (nothing computed) when n >
 * max_levels or when the plan does not cover n levels (lo = 0, hi >= n). */
ecc_status ecc_compute_present(ecc_plan_t plan, const ecc_image *img, float *d_levels, int32_t max_levels,
                               int32_t *h_count, int64_t *d_ecc, void *stream);

/* The paper's GPU-only pipeline (Sec. 4 "GPU-only pipeline", Table 2): a
 * float32 image resident on the device goes through `iterations` rounds of
 * (1) its ECC at the m thresholds d_levels (exactly ecc_compute_levels) and
 * (2) a separable smoothing filter applied in place, one pass per axis,
 * last axis first, with the given taps (the paper uses a 13-tap Gaussian):
 * out[x] = sum over k = -r..r, in that order, of taps[k + r] * in[x + k]
 * along the axis, with half-sample symmetric reflection at the borders
 * (in[-1] = in[0], in[n] = in[n-1]) and float32 rounding after every
 * multiply and every add (no fused multiply-add), so any implementation
 * with the same order reproduces it bit for bit.
 *   plan       as for ecc_compute_levels; also holds a float32 scratch
 *              copy of the image (allocated on first use).
 *   img        device ECC_F32 image, smoothed in place: on return it has
 *              been filtered `iterations` times.
 *   h_taps     host float[ntaps], ntaps odd, at most 33 (copied).
 *   d_ecc      device int64[iterations][m]: row i is the ECC of the image
 *              after i filter rounds.
 * Asynchronous on `stream`.  Errors as ecc_compute_levels. */
ecc_status ecc_pipeline_gaussian(ecc_plan_t plan, const ecc_image *img, const float *h_taps, int32_t ntaps,
                                 int32_t iterations, const float *d_levels, int32_t m, int64_t *d_ecc,
                                 void *stream);

/* ECC of a 2D, 3D or 4D device image (d > 3: the paper's method in any
 * dimension, Sec. 2.1-2.3; its texture-based kernel stops at three, Sec. 5).
 * 2D and 3D images go to ecc_compute.  A 4D image takes a bit-sliced
 * walker: the wins over the 80 neighbours (ties to the lower linear index)
 * give the signed count of the 81 cells containing the voxel (1 vertex, 8
 * edges, 24 squares, 32 cubes, 16 tesseracts) as three 3D counts, both
 * complexes, the same histogram and scan.  Arguments and errors as ecc_compute; the image's voxel count must not
 * exceed max_voxels. */
ecc_status ecc_compute_nd(ecc_plan_t plan, const ecc_image_nd *img, int64_t *d_ecc, int64_t *d_vcec,
                          void *stream);

/* Out-of-core ECC of a HOST image of any size (Sec. 3.4, Fig. 5: the
 * streaming that lets the paper process volumes larger than device memory).
 * The image is cut along dims[0] into chunks; each chunk travels with a
 * one-slab collar on each side that exists into one of three device
 * buffers taken from the plan (allocated on first use, kept until
 * ecc_plan_destroy), so the device holds at most device_budget_bytes of
 * image data (0 = 1 GiB) whatever the image size.  The copy of a chunk (on
 * the plan's copy stream) overlaps the stencil of the previous one (on
 * `stream`); the stencil of a chunk emits only its own slabs and reads the
 * collar as neighbours, so the result equals ecc_compute on the whole
 * image.
 *   h_img     host image; may exceed the plan's max_voxels and the device
 *             memory.  Pinned memory gives overlapped copies.
 *   h_ecc     host int64[nbins], written before return.
 * Synchronous: returns when h_ecc is written.  Errors: ECC_E_INVALID
 * (including a budget below three buffers of three slabs, one slab being
 * dims[1] rows in 3D or one row in 2D, rows padded to 16 bytes),
 * ECC_E_NOMEM (the chunk buffers could not be allocated), ECC_E_RANGE,
 * ECC_E_TIMEOUT, ECC_E_CUDA. */
ecc_status ecc_compute_stream(ecc_plan_t plan, const ecc_image *h_img, int64_t *h_ecc,
                              int64_t device_budget_bytes, void *stream);

/* ECC of n images of arbitrary, uneven shapes in ONE persistent kernel that
 * walks a device-side tile work list (per-image histogram offsets), launched
 * through a CUDA graph captured once per plan, followed by one segmented
 * scan.  Table 3 of the paper motivates batching: per-image overhead
 * amortizes over many images.
 *   host_descs  host array of n image descriptors (device data pointers, all
 *               of the plan's dtype, ndim 2 or 3 mixed freely).
 *   d_ecc       device int64[n][nbins]; row i is the ECC of image i.
 * Asynchronous on `stream`; the descriptor array is copied before return.
 * Errors: ECC_E_INVALID, ECC_E_BUSY (n > max_images or total voxels >
 * max_voxels), ECC_E_CUDA. */
ecc_status ecc_compute_batch(ecc_plan_t plan, int32_t n, const ecc_image *host_descs,
                             int64_t *d_ecc, void *stream);

/* ECC of one image without allocating anything: for callers that cannot
 * allocate device memory once running -- a real-time pipeline whose device
 * memory budget is fixed at start-up, code running inside another
 * framework's memory pool or allocator callback, or a process whose device
 * memory that pool has fully reserved.  A plan allocates its workspace with
 * cudaMalloc; this call instead uses one fixed scratch array of the library
 * (an int64 accumulator of 65536 levels plus scan state, about 513 KiB),
 * which every GPU that loads the library holds until the process exits.
 * The paper has no counterpart: it is a deployment variant of ecc_compute.
 *   img, d_ecc, d_vcec   as in ecc_compute (device buffers owned by the caller)
 *   lo, hi, complex_mode as in ecc_plan_desc; hi - lo + 1 must be <= 65536
 *   flags                ECC_FLAG_NO_RANGE_CHECK and ECC_FLAG_KERNEL_DIRECT honoured
 * Calls no cudaMalloc, cudaFree or allocating library routine.  The first
 * call on a device looks the scratch array up, clears it, and has the CUDA
 * runtime load every kernel this call may launch (CUDA loads modules lazily
 * by default, and loading one can take device memory): make that first
 * call at start-up, before any memory pool reserves the device's memory and
 * before any stream capture, or run with CUDA_MODULE_LOADING=EAGER.  A 3D
 * image whose row pitch is not a multiple of 16 bytes takes the batch
 * kernel, its one-image work list kept in the same array, as ecc_compute
 * runs it from a plan.  Each call clears what must start
 * at zero; all calls on a device share the array, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race and corrupt
 * each other's results.  Synchronous: returns after the work on `stream`
 * finished, with device-detected errors (ECC_E_RANGE, ECC_E_TIMEOUT).
 * Errors: ECC_E_INVALID (including more than 65536 levels), ECC_E_CUDA. */
ecc_status ecc_compute_noalloc(const ecc_image *img, int32_t lo, int32_t hi, int32_t complex_mode,
                               uint32_t flags, int64_t *d_ecc, int64_t *d_vcec, void *stream);

/* Waits for the plan's work on `stream`, then returns and clears the device
 * status word: ECC_OK, ECC_E_RANGE (a value outside [lo, hi] was seen) or
 * ECC_E_TIMEOUT (a bounded device-side wait gave up). */
ecc_status ecc_status_get(ecc_plan_t plan, void *stream);

/* Number of kernels the last ecc_compute / ecc_compute_batch call enqueued
 * (for launch accounting); -1 for an invalid handle. */
int32_t ecc_plan_last_launches(ecc_plan_t plan);

/* With ECC_FLAG_TIME_KERNELS: total device time in ms of the stencil
 * launches recorded since the previous call (measured with CUDA events on
 * the launching stream; the paper's "exec (kernel)" column of Table 1), and
 * how many launches that covers.  Waits for the recorded events; resets the
 * record.  Errors: ECC_E_INVALID (flag not set), ECC_E_CUDA. */
ecc_status ecc_plan_kernel_time(ecc_plan_t plan, double *ms, int64_t *launches);

/* With ECC_FLAG_COUNT_EMITTED: number of voxels whose signed cell count
 * kappa (Sec. 2.3, the terms of Algorithm 1 regrouped per voxel) was nonzero
 * in the ecc_compute / ecc_compute_host calls since the previous call, i.e.
 * the histogram insertions the stencil made.  Counted by the single-image
 * stencil kernels only (not by ecc_compute_batch).  Synchronizes `stream`,
 * then resets the count.  Errors: ECC_E_INVALID (NULL argument, flag not
 * set), ECC_E_CUDA. */
ecc_status ecc_plan_emitted(ecc_plan_t plan, int64_t *count, void *stream);

/* Failure-detection self-test: launches one warp that waits on a device flag
 * nothing sets (the scan's look-back pattern) and then on an mbarrier nothing
 * arrives on (the TMA ring's pattern), each bounded by limit_us; every such
 * wait in the library gives up the same way and reports ECC_E_TIMEOUT through
 * the device status word instead of hanging.  gave_up[0..1] = 1 for each wait
 * that ran out.  Expected result: ECC_E_TIMEOUT with both set; the CUDA
 * context stays usable.  The paper has no counterpart.
 * Errors: ECC_E_INVALID (limit_us outside [1, 1e7]), ECC_E_CUDA. */
ecc_status ecc_selftest_wait_timeout(int64_t limit_us, int32_t *gave_up, void *stream);

/* Thread-local message describing the last failure of this thread. */
const char *ecc_last_error(void);

/* ------------------------------------------------------------------ serving
 * A request loop for mixed-size, mixed-dtype ECC jobs (continuous batching).
 * Jobs are admitted against an HBM budget (input copy + histogram +
 * workspace); admitted jobs are packed into batched persistent launches on
 * one of n_streams streams as slots free up, so jobs arriving while others
 * run join the next launch.  Not in the paper; it composes the batched path
 * above with the copy/compute overlap of Sec. 3.4.
 */
typedef struct ecc_server_s *ecc_server_t;

typedef void (*ecc_done_fn)(uint64_t ticket, ecc_status status, void *user);

typedef struct ecc_server_desc {
    int64_t hbm_budget_bytes;  /* total device bytes the server may hold for jobs */
    int32_t n_streams;         /* concurrent batch launches (>= 1) */
    int32_t max_batch;         /* most jobs packed into one launch (>= 1) */
    int64_t max_job_voxels;    /* largest single job accepted */
    uint32_t flags;            /* ECC_FLAG_NO_RANGE_CHECK honoured */
    uint32_t reserved;
} ecc_server_desc;

/* Creates the server and its scheduler thread on the current device. */
ecc_status ecc_server_create(ecc_server_t *out, const ecc_server_desc *desc);

/* Makes, on every stream slot, the plan for one job key (dtype, gray range,
 * complex) with its batch state: workspace allocation, the autotuner's
 * timing runs and the captured batch graph, which the first job of that key
 * would otherwise wait for.  Call it at start-up for the keys expected (a
 * slot busy with a launch is waited for).  Thread-safe.
 * Errors: ECC_E_INVALID, ECC_E_NOMEM, ECC_E_CUDA, ECC_E_SHUTDOWN. */
ecc_status ecc_server_prepare(ecc_server_t server, int32_t dtype, int32_t lo, int32_t hi, int32_t complex_mode);

/* Submits one job; thread-safe; returns immediately with *ticket_out.
 *   img   image descriptor; data is a HOST pointer (the server copies it into
 *         a budgeted device buffer at admission) when `host_input` is non-zero,
 *         else a DEVICE pointer the caller keeps alive until completion.
 *   lo, hi, complex_mode  as in ecc_plan_desc (nbins <= 65536).
 *   out_ecc  host int64[nbins] written at completion (NULL to skip; then
 *            read it with ecc_server_result before ecc_release).
 *   done  optional callback run on the server's completion thread.
 * Errors: ECC_E_INVALID, ECC_E_NOMEM (the job alone exceeds the budget),
 * ECC_E_SHUTDOWN. */
ecc_status ecc_submit(ecc_server_t server, const ecc_image *img, int32_t host_input,
                      int32_t lo, int32_t hi, int32_t complex_mode, int64_t *out_ecc,
                      ecc_done_fn done, void *user, uint64_t *ticket_out);

/* Blocks until the job finishes or timeout_us elapses (< 0: no limit).
 * Returns the job's status, or ECC_E_TIMEOUT. */
ecc_status ecc_wait(ecc_server_t server, uint64_t ticket, int64_t timeout_us);

/* Latency/throughput counters since creation (or the last reset).
 *   out[0] jobs completed, out[1] voxels completed, out[2] p50 latency (us),
 *   out[3] p99 latency (us), out[4] max latency (us), out[5] batch launches,
 *   out[6] busy wall time (us), out[7] peak budget bytes in use.
 * Latency = completion - submission.  n_out <= 8 values are written. */
ecc_status ecc_server_stats(ecc_server_t server, double *out, int32_t n_out, int32_t reset);

/* Stops accepting jobs, drains (or cancels, if cancel != 0) queued jobs,
 * joins the threads and frees everything. */
ecc_status ecc_server_destroy(ecc_server_t server, int32_t cancel);

#ifdef __cplusplus
}
#endif

#endif /* ECC_GB300_ECC_H */
