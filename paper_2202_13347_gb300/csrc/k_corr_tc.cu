// tcgen05 BF16 implicit-GEMM correlation (placeholder until the kernel lands).
#include "internal.h"

namespace sfoc {

size_t corr_tc_smem_bytes(int, int) { return 0; }

cudaError_t launch_corr_tc(const Cube&, const Cube&, const int32_t*, int, int, int, const PointStat*, float*, int*,
                           cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace sfoc
