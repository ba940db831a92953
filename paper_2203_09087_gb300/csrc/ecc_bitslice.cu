// ecc_bitslice.cu -- bit-sliced stencil kernel (placeholder until written).
#include "ecc_internal.h"

namespace ecc {

bool bitslice_supported(const Geom &) { return false; }

cudaError_t launch_bitslice(const Geom &, int64_t, int64_t, const HistDst &, int, bool, unsigned int *, int, int,
                            cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace ecc
