// ecc_batch.cu -- ecc_compute_batch: many images of uneven shapes.
#include <cuda_runtime.h>

#include <vector>

#include "ecc_plan.h"

namespace ecc {

struct BatchState {
    int unused = 0;
};

void release_batch(ecc_plan_s *p)
{
    delete p->batch;
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
