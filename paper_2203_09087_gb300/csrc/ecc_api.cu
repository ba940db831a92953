// ecc_api.cu -- the C ABI of include/ecc.h: plans, validation, launches,
// device status, and the host-buffer streaming path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ecc.h"
#include "ecc_internal.h"
#include "ecc_plan.h"

namespace ecc {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

ecc_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return ECC_E_CUDA;
}

ecc_status invalid(const std::string &msg)
{
    set_error(msg);
    return ECC_E_INVALID;
}

ecc_status image_geom(const ecc_image *img, int32_t want_dtype, int64_t max_voxels, Geom *g, int64_t *voxels,
                      bool allow_null_data)
{
    if (!img) return invalid("image descriptor is NULL");
    if (!img->data && !allow_null_data) return invalid("image data pointer is NULL");
    if (img->ndim != 2 && img->ndim != 3) return invalid("ndim must be 2 or 3");
    if (img->dtype != ECC_U8 && img->dtype != ECC_U16 && !(img->dtype == ECC_F32 && want_dtype == ECC_F32))
        return invalid("dtype must be ECC_U8 or ECC_U16 (ECC_F32 only through ecc_compute_levels)");
    if (want_dtype && img->dtype != want_dtype) return invalid("image dtype differs from the plan's dtype");
    int64_t n = 1;
    for (int a = 0; a < img->ndim; ++a) {
        if (img->dims[a] < 1) return invalid("every dim must be >= 1");
        if (img->dims[a] > (int64_t(1) << 31)) return invalid("dim too large");
        n *= img->dims[a];
        if (n > (int64_t(1) << 40)) return invalid("image too large");
    }
    const int es = img->dtype == ECC_F32 ? 4 : (img->dtype == ECC_U16 ? 2 : 1);
    Geom r{};
    r.data = static_cast<const unsigned char *>(img->data);
    r.ndim = img->ndim;
    r.esize = es;
    if (img->ndim == 3) {
        r.nz = img->dims[0];
        r.ny = img->dims[1];
        r.nx = img->dims[2];
    } else {
        r.nz = 1;
        r.ny = img->dims[0];
        r.nx = img->dims[1];
    }
    r.pitch_y = img->row_pitch ? img->row_pitch : r.nx * es;
    if (r.pitch_y < r.nx * es || r.pitch_y % es) return invalid("row_pitch smaller than a row or not a multiple of the element size");
    if (img->ndim == 3) {
        r.pitch_z = img->slice_pitch ? img->slice_pitch : r.ny * r.pitch_y;
        if (r.pitch_z < (r.ny - 1) * r.pitch_y + r.nx * es || r.pitch_z % es)
            return invalid("slice_pitch smaller than a slice or not a multiple of the element size");
    } else {
        if (img->slice_pitch) return invalid("slice_pitch must be 0 for a 2D image");
        r.pitch_z = r.ny * r.pitch_y;
    }
    if (max_voxels > 0 && n > max_voxels) {
        set_error("image has more voxels than the plan's max_voxels");
        return ECC_E_BUSY;
    }
    *g = r;
    if (voxels) *voxels = n;
    return ECC_OK;
}

// Launch the stencil+histogram pass of one image over outer indices
// [ob, oe) into the histogram h.
static cudaError_t launch_stencil_untimed(ecc_plan_s *p, const Geom &g, int64_t ob, int64_t oe, const HistDst &h,
                                         cudaStream_t s, FusedScan *fs);

cudaError_t launch_stencil(ecc_plan_s *p, const Geom &g, int64_t ob, int64_t oe, const HistDst &h, cudaStream_t s,
                           FusedScan *fs)
{
    if (!(p->d.flags & ECC_FLAG_TIME_KERNELS)) return launch_stencil_untimed(p, g, ob, oe, h, s, fs);
    while (p->time_ev.size() < p->time_used + 2) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        p->time_ev.push_back(ev);
    }
    cudaEvent_t t0 = p->time_ev[p->time_used], t1 = p->time_ev[p->time_used + 1];
    p->time_used += 2;
    cudaError_t e = cudaEventRecord(t0, s);
    if (e == cudaSuccess) e = launch_stencil_untimed(p, g, ob, oe, h, s, fs);
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    return e;
}

static cudaError_t launch_stencil_untimed(ecc_plan_s *p, const Geom &g, int64_t ob, int64_t oe, const HistDst &h,
                                         cudaStream_t s, FusedScan *fs)
{
    const bool range = !(p->d.flags & ECC_FLAG_NO_RANGE_CHECK);
    const bool want_bitslice = !(p->d.flags & ECC_FLAG_KERNEL_DIRECT);
    if (want_bitslice && bitslice_supported(g)) {
        const int tp = p->tune_param(g);
        cudaError_t e =
            launch_bitslice(g, ob, oe, h, p->d.complex_mode, range, p->status, p->sched, p->num_sms, tp, s, fs);
        if (e != cudaErrorNotSupported) {
            ++p->last_launches;
            return e;
        }
    }
    // a whole 3D image whose rows the TMA cannot address (pitch not a multiple
    // of 16 bytes): the persistent batch kernel walks it with global loads
    if (want_bitslice && g.ndim == 3 && ob == 0 && oe == g.nz && !h.emitted) {
        cudaError_t e = launch_batch_single(p, g, h, s);
        p->last_launches += 2;
        return e;
    }
    ++p->last_launches;
    return launch_direct(g, ob, oe, h, p->d.complex_mode, range, p->status, p->num_sms, s);
}

}  // namespace ecc

int ecc_plan_s::tune_param(const ecc::Geom &g) const
{
    const int key = (g.ndim == 3 ? 1 : 0) | (g.esize == 2 ? 2 : 0);
    return tuned[key];
}

using namespace ecc;

extern "C" {

const char *ecc_last_error(void) { return g_last_error.c_str(); }

ecc_status ecc_plan(ecc_plan_t *out, const ecc_plan_desc *d)
{
    if (!out || !d) return invalid("ecc_plan: NULL argument");
    *out = nullptr;
    if (d->dtype != ECC_U8 && d->dtype != ECC_U16) return invalid("plan dtype must be ECC_U8 or ECC_U16");
    const int64_t maxval = d->dtype == ECC_U8 ? 255 : 65535;
    if (d->hi < d->lo) return invalid("hi < lo");
    if (d->lo < 0 || d->hi > maxval) return invalid("[lo, hi] outside the dtype's range");
    if ((int64_t)d->hi - d->lo + 1 > 65536) return invalid("more than 65536 bins");
    if (d->complex_mode != ECC_VERTEX_MAX && d->complex_mode != ECC_TOPCELL_MIN)
        return invalid("complex_mode must be ECC_VERTEX_MAX or ECC_TOPCELL_MIN");
    if (d->max_images < 1) return invalid("max_images must be >= 1");
    if (d->max_voxels < 1) return invalid("max_voxels must be >= 1");
    if (d->reserved || d->reserved2) return invalid("reserved fields must be 0");
    if ((d->flags & ECC_FLAG_KERNEL_DIRECT) && (d->flags & ECC_FLAG_KERNEL_BITSLICE))
        return invalid("ECC_FLAG_KERNEL_DIRECT and ECC_FLAG_KERNEL_BITSLICE are exclusive");

    ecc_plan_s *p = new (std::nothrow) ecc_plan_s();
    if (!p) {
        set_error("host allocation failed");
        return ECC_E_NOMEM;
    }
    p->d = *d;
    p->nbins = d->hi - d->lo + 1;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "ecc_plan: device query");
    }
    ecc_status st = p->allocate();
    if (st != ECC_OK) {
        delete p;
        return st;
    }
    p->autotune();
    *out = p;
    return ECC_OK;
}

ecc_status ecc_plan_destroy(ecc_plan_t p)
{
    if (!p) return invalid("ecc_plan_destroy: NULL plan");
    cudaDeviceSynchronize();
    p->release();
    delete p;
    return ECC_OK;
}

int32_t ecc_plan_nbins(ecc_plan_t p) { return p ? p->nbins : -1; }

int32_t ecc_plan_last_launches(ecc_plan_t p) { return p ? p->last_launches : -1; }

ecc_status ecc_plan_kernel_time(ecc_plan_t p, double *ms, int64_t *launches)
{
    if (!p || !ms || !launches) return invalid("ecc_plan_kernel_time: NULL argument");
    if (!(p->d.flags & ECC_FLAG_TIME_KERNELS)) return invalid("ecc_plan_kernel_time: plan lacks ECC_FLAG_TIME_KERNELS");
    double total = 0.0;
    for (size_t i = 0; i + 1 < p->time_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(p->time_ev[i + 1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p->time_ev[i], p->time_ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "ecc_plan_kernel_time");
        total += t;
    }
    *ms = total;
    *launches = (int64_t)(p->time_used / 2);
    p->time_used = 0;
    return ECC_OK;
}

ecc_status ecc_plan_emitted(ecc_plan_t p, int64_t *count, void *stream)
{
    if (!p || !count) return invalid("ecc_plan_emitted: NULL argument");
    if (!(p->d.flags & ECC_FLAG_COUNT_EMITTED)) return invalid("ecc_plan_emitted: plan lacks ECC_FLAG_COUNT_EMITTED");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, p->emitted, sizeof(v), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->emitted, 0, sizeof(v), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_plan_emitted");
    *count = (int64_t)v;
    return ECC_OK;
}

ecc_status ecc_compute(ecc_plan_t p, const ecc_image *img, int64_t *d_ecc, int64_t *d_vcec, void *stream)
{
    if (!p) return invalid("ecc_compute: NULL plan");
    if (!d_ecc) return invalid("ecc_compute: NULL output");
    Geom g;
    ecc_status st = image_geom(img, p->d.dtype, p->d.max_voxels, &g, nullptr, false);
    if (st != ECC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->last_launches = 0;
    HistDst h{p->acc, p->d.lo, p->nbins};
    if (p->d.flags & ECC_FLAG_COUNT_EMITTED) h.emitted = p->emitted;
    const int64_t outer = g.ndim == 3 ? g.nz : g.ny;
    // the 3D stencil's last CTA scans small histograms itself (fs.done)
    FusedScan fs{reinterpret_cast<long long *>(d_ecc), reinterpret_cast<long long *>(d_vcec), false};
    cudaError_t e = launch_stencil(p, g, 0, outer, h, s, &fs);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute: stencil launch");
    if (fs.done) return ECC_OK;
    e = launch_scan(p->acc, reinterpret_cast<long long *>(d_ecc), reinterpret_cast<long long *>(d_vcec), 1,
                    p->nbins, p->scan_ws(), p->status, s);
    ++p->last_launches;
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute: scan launch");
    return ECC_OK;
}

ecc_status ecc_status_get(ecc_plan_t p, void *stream)
{
    if (!p) return invalid("ecc_status_get: NULL plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, p->status, sizeof(word), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && word) {
        e = cudaMemsetAsync(p->status, 0, sizeof(word), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "ecc_status_get");
    if (word & DEV_TIMEOUT) {
        set_error("a bounded device-side wait gave up");
        return ECC_E_TIMEOUT;
    }
    if (word & DEV_RANGE) {
        set_error("an image value lies outside [lo, hi]");
        return ECC_E_RANGE;
    }
    if (word & DEV_STATE) {
        set_error("the scan's look-back state was not clean (plan workspace corrupted)");
        return ECC_E_CUDA;
    }
    if (word & DEV_LEVELS) {
        set_error("the threshold levels are not in ascending order");
        return ECC_E_INVALID;
    }
    return ECC_OK;
}

ecc_status ecc_compute_host(ecc_plan_t p, const ecc_image *h_img, int64_t *h_ecc, void *stream)
{
    if (!p) return invalid("ecc_compute_host: NULL plan");
    if (!h_ecc) return invalid("ecc_compute_host: NULL output");
    Geom hg;
    int64_t nvox = 0;
    ecc_status st = image_geom(h_img, p->d.dtype, p->d.max_voxels, &hg, &nvox, false);
    if (st != ECC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = p->ensure_stage((hg.ndim == 3 ? hg.nz : 1) * hg.ny * ((hg.nx * hg.esize + 15) / 16 * 16));
    if (st != ECC_OK) return st;

    // Dense device copy of the image, filled chunk by chunk along the outer
    // axis (Sec. 3.4): chunk k is processed once chunk k+1 -- which holds
    // its one-voxel collar -- has arrived, so copies overlap the kernels.
    // rows padded to 16 bytes: every chunk takes the TMA kernel
    Geom dg = hg;
    dg.data = p->stage;
    dg.pitch_y = (hg.nx * hg.esize + 15) / 16 * 16;
    dg.pitch_z = hg.ny * dg.pitch_y;
    const int64_t outer = hg.ndim == 3 ? hg.nz : hg.ny;
    const int64_t outer_bytes = hg.ndim == 3 ? dg.pitch_z : dg.pitch_y;
    // the first copy and the last stencil overlap nothing, so chunks are
    // small (8 MiB, up to 32 of them; the host link, ~207 GB/s measured, is
    // the bound, whatever the number of copy streams)
    const int64_t target_chunk_bytes = int64_t(8) << 20;
    int64_t nchunks = std::min<int64_t>(std::max<int64_t>(1, (outer * outer_bytes) / target_chunk_bytes), 32);
    nchunks = std::min(nchunks, outer);
    std::vector<int64_t> cut(nchunks + 1);
    for (int64_t k = 0; k <= nchunks; ++k) cut[k] = outer * k / nchunks;

    p->last_launches = 0;
    cudaError_t e = cudaSuccess;
    HistDst h{p->acc, p->d.lo, p->nbins};
    if (p->d.flags & ECC_FLAG_COUNT_EMITTED) h.emitted = p->emitted;
    for (int64_t k = 0; k < nchunks && e == cudaSuccess; ++k) {
        const int64_t a = cut[k], b = cut[k + 1];
        unsigned char *dst = p->stage + a * outer_bytes;
        const unsigned char *src = static_cast<const unsigned char *>(h_img->data);
        if (hg.ndim == 3) {
            if (hg.pitch_z == hg.ny * hg.pitch_y) {   // host slices contiguous: one 2D copy of all rows
                e = cudaMemcpy2DAsync(dst, dg.pitch_y, src + a * hg.pitch_z, hg.pitch_y, hg.nx * hg.esize,
                                      (b - a) * hg.ny, cudaMemcpyHostToDevice, p->copy_stream);
            } else {
                for (int64_t z = a; z < b && e == cudaSuccess; ++z)
                    e = cudaMemcpy2DAsync(p->stage + z * dg.pitch_z, dg.pitch_y, src + z * hg.pitch_z, hg.pitch_y,
                                          hg.nx * hg.esize, hg.ny, cudaMemcpyHostToDevice, p->copy_stream);
            }
        } else {
            e = cudaMemcpy2DAsync(dst, dg.pitch_y, src + a * hg.pitch_y, hg.pitch_y, hg.nx * hg.esize, b - a,
                                  cudaMemcpyHostToDevice, p->copy_stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(p->chunk_ev[k % kMaxChunkEvents], p->copy_stream);
        // process the previous chunk once this one (its collar) has landed
        if (e == cudaSuccess && k > 0) {
            e = cudaStreamWaitEvent(s, p->chunk_ev[k % kMaxChunkEvents], 0);
            if (e == cudaSuccess) e = launch_stencil(p, dg, cut[k - 1], cut[k], h, s);
        }
    }
    if (e == cudaSuccess) {
        e = cudaStreamWaitEvent(s, p->chunk_ev[(nchunks - 1) % kMaxChunkEvents], 0);
        if (e == cudaSuccess) e = launch_stencil(p, dg, cut[nchunks - 1], cut[nchunks], h, s);
    }
    if (e == cudaSuccess) {
        e = launch_scan(p->acc, p->stage_ecc, nullptr, 1, p->nbins, p->scan_ws(), p->status, s);
        ++p->last_launches;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_ecc, p->stage_ecc, sizeof(int64_t) * p->nbins, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_host");
    return ecc_status_get(p, stream);
}

ecc_status ecc_compute_stream(ecc_plan_t p, const ecc_image *h_img, int64_t *h_ecc, int64_t device_budget_bytes,
                              void *stream)
{
    if (!p) return invalid("ecc_compute_stream: NULL plan");
    if (!h_ecc) return invalid("ecc_compute_stream: NULL output");
    if (device_budget_bytes < 0) return invalid("ecc_compute_stream: negative device budget");
    Geom hg;
    int64_t nvox = 0;
    // any size: the image never has to fit the device or the plan's max_voxels
    ecc_status st = image_geom(h_img, p->d.dtype, 0, &hg, &nvox, false);
    if (st != ECC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t budget = device_budget_bytes ? device_budget_bytes : (int64_t(1) << 30);

    // Chunks along the outer axis (Sec. 3.4, Fig. 5).  A chunk of C outer
    // slabs travels with a one-slab collar on each side that exists, into
    // one of kRing device buffers; the stencil of chunk k emits only its own
    // slabs and reads the collar as real neighbours, while the image's own
    // boundary stays a boundary.  Device rows are padded to 16 bytes so
    // every chunk takes the TMA kernel.
    const int64_t dpitch_y = (hg.nx * hg.esize + 15) / 16 * 16;
    const int64_t outer = hg.ndim == 3 ? hg.nz : hg.ny;
    const int64_t slab = hg.ndim == 3 ? hg.ny * dpitch_y : dpitch_y;   // bytes of one outer slab
    const int64_t per_buf = budget / kRing / 256 * 256;
    if (per_buf / slab < 3) {
        set_error("ecc_compute_stream: device budget below three buffers of three slabs (one slab plus collar)");
        return ECC_E_INVALID;
    }
    const int64_t C = std::min<int64_t>(per_buf / slab - 2, outer);
    const int64_t buf_bytes = (C + 2) * slab;
    const int64_t buf_stride = (buf_bytes + 255) / 256 * 256;
    st = p->ensure_ring(buf_stride * kRing);
    if (st != ECC_OK) return st;

    p->last_launches = 0;
    cudaError_t e = cudaSuccess;
    HistDst h{p->acc, p->d.lo, p->nbins};
    if (p->d.flags & ECC_FLAG_COUNT_EMITTED) h.emitted = p->emitted;
    const unsigned char *src = static_cast<const unsigned char *>(h_img->data);
    const int64_t nchunks = (outer + C - 1) / C;
    for (int64_t k = 0; k < nchunks && e == cudaSuccess; ++k) {
        const int64_t c0 = k * C, c1 = std::min(c0 + C, outer);
        const int64_t base = c0 > 0 ? c0 - 1 : 0, top = c1 < outer ? c1 + 1 : outer;
        const int b = (int)(k % kRing);
        unsigned char *buf = p->ring + b * buf_stride;
        // the buffer is free once the stencil that last read it has run
        if (k >= kRing) e = cudaStreamWaitEvent(p->copy_stream, p->ring_done[b], 0);
        if (e == cudaSuccess) {
            if (hg.ndim == 3 && hg.pitch_z == hg.ny * hg.pitch_y)   // slabs contiguous: one copy
                e = cudaMemcpy2DAsync(buf, dpitch_y, src + base * hg.pitch_z, hg.pitch_y, hg.nx * hg.esize,
                                      (top - base) * hg.ny, cudaMemcpyHostToDevice, p->copy_stream);
            else if (hg.ndim == 3)
                for (int64_t z = base; z < top && e == cudaSuccess; ++z)
                    e = cudaMemcpy2DAsync(buf + (z - base) * slab, dpitch_y, src + z * hg.pitch_z, hg.pitch_y,
                                          hg.nx * hg.esize, hg.ny, cudaMemcpyHostToDevice, p->copy_stream);
            else
                e = cudaMemcpy2DAsync(buf, dpitch_y, src + base * hg.pitch_y, hg.pitch_y, hg.nx * hg.esize,
                                      top - base, cudaMemcpyHostToDevice, p->copy_stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(p->ring_copied[b], p->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ring_copied[b], 0);
        if (e == cudaSuccess) {
            Geom v = hg;
            v.data = buf;
            v.pitch_y = dpitch_y;
            if (hg.ndim == 3) {
                v.nz = top - base;
                v.pitch_z = slab;
            } else {
                v.ny = top - base;
                v.pitch_z = v.ny * dpitch_y;
            }
            e = launch_stencil(p, v, c0 - base, c1 - base, h, s);
        }
        if (e == cudaSuccess) e = cudaEventRecord(p->ring_done[b], s);
    }
    if (e == cudaSuccess) {
        e = launch_scan(p->acc, p->stage_ecc, nullptr, 1, p->nbins, p->scan_ws(), p->status, s);
        ++p->last_launches;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_ecc, p->stage_ecc, sizeof(int64_t) * p->nbins, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_compute_stream");
    return ecc_status_get(p, stream);
}

}  // extern "C"
