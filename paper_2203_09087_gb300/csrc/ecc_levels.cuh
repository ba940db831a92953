// ecc_levels.cuh -- the level search of the float-threshold path (device
// only), shared by the quantize kernel (ecc_levels.cu) and the fused
// smoothing round (ecc_pipeline.cu).
//
// Every voxel maps to the number of levels strictly below its value (NaN:
// m, above every level): Eq. 1 with the t_i given, as a monotone map that
// commutes with the max / min a cell takes over its voxels.
#pragma once

#include <math_constants.h>

namespace ecc {
namespace lv {

// The levels padded with +infinity to 2^L - 1 entries form a complete binary
// search tree, stored in breadth-first (Eytzinger) order: node k has
// children 2k+1 and 2k+2, and node k at depth d, position p within the depth,
// holds the padded level of sorted rank (2p + 1) 2^(L-1-d) - 1.  A search
// takes L steps k <- 2k + 1 + (node k < v), the same on every lane; at the
// end k - (2^L - 1) is the number of levels below v.  The nodes of one depth
// are contiguous, so lanes on different paths read different banks (in
// sorted order, every candidate of a step would sit in the same bank).
__device__ __forceinline__ float padded_level(const float *levels, int m, int j)
{
    return j < m ? levels[j] : CUDART_INF_F;
}

template <int L>
__device__ __forceinline__ int eytz_rank_of_node(int k)
{
    const int d = 31 - __clz(k + 1);     // depth
    const int p = k + 1 - (1 << d);      // position within the depth
    return ((2 * p + 1) << (L - 1 - d)) - 1;
}

// Number of levels strictly below v (NaN: m).
template <int L, bool GLOBAL>
__device__ __forceinline__ int lower_bound_count(const float *tree, int m, float v)
{
    int k = 0;
#pragma unroll
    for (int d = 0; d < L; ++d) {
        const float t = GLOBAL ? padded_level(tree, m, eytz_rank_of_node<L>(k)) : tree[k];
        k = 2 * k + 1 + (t < v ? 1 : 0);
    }
    return v != v ? m : k - ((1 << L) - 1);
}

}  // namespace lv
}  // namespace ecc
