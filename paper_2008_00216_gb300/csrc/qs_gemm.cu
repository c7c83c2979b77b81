// Dense k in {5, 6} gates on the tensor cores (tcgen05).  Not built yet:
// the planner only selects this pass when a split-precision mode is asked
// for, and the executor then reports QS_ERR_UNSUPPORTED.
#include "qs_internal.h"

namespace qsgb {

cudaError_t launch_gemm(void*, int, int, const int*, const void*, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace qsgb
