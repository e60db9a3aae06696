// Tensor-core (tcgen05) complex GEMM for stem steps whose branch is large
// enough to make the step a dense contraction.
#include <cuda_runtime.h>

#include "kernels.h"

namespace tn {

bool tc_gemm_supported(int k, int n) {
    (void)k;
    (void)n;
    return false;
}

cudaError_t launch_tc_stem_gemm(const float2 *, float2 *, int64_t, int, int, int64_t, int64_t,
                                const DevBranch *, const float2 *, BatchArgs, tn_precision,
                                cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace tn
