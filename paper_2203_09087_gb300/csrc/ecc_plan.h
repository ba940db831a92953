// ecc_plan.h -- the plan object behind ecc_plan_t (internal).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "ecc.h"
#include "ecc_internal.h"

namespace ecc {

constexpr int kMaxChunkEvents = 16;
constexpr int kRing = 3;  // device chunk buffers of the out-of-core path

struct BatchState;  // ecc_batch.cu

}  // namespace ecc

struct ecc_plan_s {
    ecc_plan_desc d{};
    int device = 0;
    int num_sms = 0;
    int32_t nbins = 0;
    int last_launches = 0;

    // one device allocation: accumulators, status word, scan state
    void *ws = nullptr;
    size_t ws_bytes = 0;
    unsigned long long *acc = nullptr;   // [max_images * nbins] int64, kept zero between calls
    unsigned int *status = nullptr;      // device status word (ecc::DEV_*)
    unsigned int *scan_counters = nullptr;
    unsigned int *sched = nullptr;       // stencil work counter (2 words, self-resetting)
    unsigned long long *emitted = nullptr;  // ECC_FLAG_COUNT_EMITTED counter
    int *tile_status = nullptr;
    long long *tile_value = nullptr;
    int32_t max_tiles = 0;

    // host-input streaming (ecc_compute_host), allocated on first use
    unsigned char *stage = nullptr;
    size_t stage_bytes = 0;
    long long *stage_ecc = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t chunk_ev[ecc::kMaxChunkEvents] = {};

    // out-of-core streaming (ecc_compute_stream): one allocation split into
    // kRing chunk buffers, with "copied" and "consumed" events per buffer
    unsigned char *ring = nullptr;
    size_t ring_bytes = 0;
    cudaEvent_t ring_copied[ecc::kRing] = {};
    cudaEvent_t ring_done[ecc::kRing] = {};

    // float32 scratch image of the smoothing pipeline, allocated on first use
    void *aux = nullptr;
    size_t aux_bytes = 0;
    // present-value thresholds (ecc_levels_present): hash table, key list
    // and counters, allocated on first use
    void *present = nullptr;
    size_t present_bytes = 0;
    // the smoothing pipeline's captured round (kept until its launches finish)
    cudaGraphExec_t pipe_exec = nullptr;
    cudaEvent_t pipe_done = nullptr;

    // tile parameter per (ndim, esize) key chosen by the autotuner
    int tuned[4] = {0, 0, 0, 0};
    // batch path: rows per 2D tile, planes per 3D tile (0 = default)
    int tuned_batch[2] = {0, 0};

    ecc::BatchState *batch = nullptr;

    // ECC_FLAG_TIME_KERNELS: event pairs around stencil launches
    std::vector<cudaEvent_t> time_ev;
    size_t time_used = 0;

    ecc_status allocate();
    void release();
    void autotune();
    ecc_status ensure_stage(int64_t bytes);
    ecc_status ensure_ring(int64_t bytes);
    ecc_status ensure_aux(int64_t bytes);
    ecc_status ensure_present(int64_t bytes);
    int tune_param(const ecc::Geom &g) const;
    ecc::ScanWs scan_ws() const
    {
        return ecc::ScanWs{scan_counters, scan_counters + 1, tile_status, tile_value, max_tiles};
    }
};

namespace ecc {

ecc_status image_geom(const ecc_image *img, int32_t want_dtype, int64_t max_voxels, Geom *g, int64_t *voxels,
                      bool allow_null_data);
cudaError_t launch_stencil(ecc_plan_s *p, const Geom &g, int64_t ob, int64_t oe, const HistDst &h,
                           cudaStream_t s, FusedScan *fs = nullptr);
void release_batch(ecc_plan_s *p);
ecc_status prepare_batch(ecc_plan_s *p);
// One 3D image through the batch kernel with its work list in caller scratch
// of kBatchSingleWsBytes (no plan, no allocation); check_values: compare
// every voxel with [lo, hi] when the range is narrower than the type.
constexpr size_t kBatchSingleWsBytes = 128;
cudaError_t launch_batch_single_ws(const Geom &g, const HistDst &h, int complex_mode, bool check_values, void *ws,
                                   unsigned int *status, int num_sms, cudaStream_t s);
cudaError_t preload_batch();
cudaError_t launch_batch_single(ecc_plan_s *p, const Geom &g, const HistDst &h, cudaStream_t s);

}  // namespace ecc
