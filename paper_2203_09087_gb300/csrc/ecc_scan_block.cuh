// ecc_scan_block.cuh -- the scan of a small histogram by one CTA, for the
// stencil kernels whose last CTA to finish scans the bins itself (device
// only).
#pragma once

#include <stdint.h>

namespace ecc {

// Inclusive scan of the accumulated bins by one CTA of NTH threads, the
// fused form of the scan kernel for small histograms (Sec. 2.3: the ECC is
// the prefix sum of the VCEC): ecc[i] = acc[0] + ... + acc[i], vcec[i] =
// acc[i] if asked, and acc is left zero for the next call.  Each thread takes
// a contiguous run of bins; the runs' sums are scanned across the CTA.
template <int NTH>
__device__ void scan_bins(unsigned long long *acc, long long *ecc, long long *vcec, int nbins, int tid)
{
    __shared__ long long s_warp[NTH / 32];
    const int lane = tid & 31, warp = tid >> 5;
    const int per = (nbins + NTH - 1) / NTH;
    const int b0 = tid * per < nbins ? tid * per : nbins;
    const int b1 = b0 + per < nbins ? b0 + per : nbins;
    long long sum = 0;
    for (int i = b0; i < b1; ++i) sum += (long long)__ldcg(acc + i);
    long long x = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    long long run = x - sum;   // this thread's exclusive prefix
    for (int w = 0; w < warp; ++w) run += s_warp[w];
    for (int i = b0; i < b1; ++i) {
        const long long v = (long long)__ldcg(acc + i);
        run += v;
        ecc[i] = run;
        if (vcec) vcec[i] = v;
        acc[i] = 0ull;
    }
}

}  // namespace ecc
