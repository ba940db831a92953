// ecc_plan.cu -- plan workspace allocation and release.
#include <cuda_runtime.h>

#include <cstring>

#include "ecc_plan.h"

using namespace ecc;

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

cudaError_t ecc::clear_device_now(void *p, size_t bytes)
{
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (s) cudaStreamDestroy(s);
    return e;
}

ecc_status ecc_plan_s::allocate()
{
    const int64_t max_seg = d.max_images;
    max_tiles = (int32_t)scan_tiles(max_seg, nbins);
    const size_t acc_bytes = align_up(sizeof(unsigned long long) * (size_t)max_seg * nbins, 256);
    const size_t status_bytes = 256;
    const size_t counters_bytes = 256;
    const size_t tstat_bytes = align_up(sizeof(int) * (size_t)max_tiles, 256);
    const size_t tval_bytes = align_up(sizeof(long long) * 2 * (size_t)max_tiles, 256);
    ws_bytes = acc_bytes + status_bytes + counters_bytes + tstat_bytes + tval_bytes;
    cudaError_t e = cudaMalloc(&ws, ws_bytes);
    if (e != cudaSuccess) {
        ws = nullptr;
        cudaGetLastError();
        set_error("ecc_plan: cudaMalloc of the workspace failed");
        return ECC_E_NOMEM;
    }
    // the histogram, status and scan workspace start at zero before any
    // stream, the caller's non-blocking ones included, can use them
    e = clear_device_now(ws, ws_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_plan: workspace clear");
    unsigned char *b = static_cast<unsigned char *>(ws);
    acc = reinterpret_cast<unsigned long long *>(b);
    b += acc_bytes;
    status = reinterpret_cast<unsigned int *>(b);
    b += status_bytes;
    scan_counters = reinterpret_cast<unsigned int *>(b);
    sched = scan_counters + 16;  // same 256-byte block, separate words
    emitted = reinterpret_cast<unsigned long long *>(scan_counters + 32);
    b += counters_bytes;
    tile_status = reinterpret_cast<int *>(b);
    b += tstat_bytes;
    tile_value = reinterpret_cast<long long *>(b);
    return ECC_OK;
}

ecc_status ecc_plan_s::ensure_stage(int64_t bytes)
{
    if (!copy_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking);
        for (int i = 0; i < kMaxChunkEvents && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&chunk_ev[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&stage_ecc, sizeof(long long) * nbins);
        if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_host: stream/event setup");
    }
    if ((size_t)bytes > stage_bytes) {
        if (stage) cudaFree(stage);
        stage = nullptr;
        stage_bytes = 0;
        cudaError_t e = cudaMalloc(&stage, (size_t)bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("ecc_compute_host: device staging allocation failed");
            return ECC_E_NOMEM;
        }
        stage_bytes = (size_t)bytes;
    }
    return ECC_OK;
}

ecc_status ecc_plan_s::ensure_ring(int64_t bytes)
{
    // the streams, events and ECC staging of the host-input path come first
    ecc_status st = ensure_stage(0);
    if (st != ECC_OK) return st;
    if (!ring_copied[0]) {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < kRing && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&ring_copied[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ring_done[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_stream: event setup");
    }
    if ((size_t)bytes > ring_bytes) {
        if (ring) cudaFree(ring);
        ring = nullptr;
        ring_bytes = 0;
        cudaError_t e = cudaMalloc(&ring, (size_t)bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("ecc_compute_stream: device chunk buffers allocation failed");
            return ECC_E_NOMEM;
        }
        ring_bytes = (size_t)bytes;
    }
    return ECC_OK;
}

ecc_status ecc_plan_s::ensure_aux(int64_t bytes)
{
    if ((size_t)bytes > aux_bytes) {
        if (aux) cudaFree(aux);
        aux = nullptr;
        aux_bytes = 0;
        cudaError_t e = cudaMalloc(&aux, (size_t)bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("ecc_pipeline_gaussian: scratch image allocation failed");
            return ECC_E_NOMEM;
        }
        aux_bytes = (size_t)bytes;
    }
    return ECC_OK;
}

ecc_status ecc_plan_s::ensure_present(int64_t bytes)
{
    if ((size_t)bytes > present_bytes) {
        if (present) cudaFree(present);
        present = nullptr;
        present_bytes = 0;
        cudaError_t e = cudaMalloc(&present, (size_t)bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("ecc_levels_present: table allocation failed");
            return ECC_E_NOMEM;
        }
        present_bytes = (size_t)bytes;
    }
    return ECC_OK;
}

void ecc_plan_s::release()
{
    if (pipe_exec) {
        if (pipe_done) cudaEventSynchronize(pipe_done);
        cudaGraphExecDestroy(pipe_exec);
        pipe_exec = nullptr;
    }
    if (pipe_done) cudaEventDestroy(pipe_done);
    pipe_done = nullptr;
    if (batch) release_batch(this);
    if (ws) cudaFree(ws);
    if (stage) cudaFree(stage);
    if (ring) cudaFree(ring);
    if (aux) cudaFree(aux);
    if (present) cudaFree(present);
    if (stage_ecc) cudaFree(stage_ecc);
    for (int i = 0; i < kRing; ++i) {
        if (ring_copied[i]) cudaEventDestroy(ring_copied[i]);
        if (ring_done[i]) cudaEventDestroy(ring_done[i]);
        ring_copied[i] = ring_done[i] = nullptr;
    }
    for (int i = 0; i < kMaxChunkEvents; ++i)
        if (chunk_ev[i]) cudaEventDestroy(chunk_ev[i]);
    for (cudaEvent_t ev : time_ev) cudaEventDestroy(ev);
    time_ev.clear();
    if (copy_stream) cudaStreamDestroy(copy_stream);
    ws = nullptr;
    stage = nullptr;
    ring = nullptr;
    ring_bytes = 0;
    aux = nullptr;
    aux_bytes = 0;
    present = nullptr;
    present_bytes = 0;
    stage_ecc = nullptr;
    copy_stream = nullptr;
}
