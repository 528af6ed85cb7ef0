// k_tc.cu -- tensor-core (tcgen05) label step for the reduced-precision paths.
#include "dpmm_internal.cuh"

namespace dpmm {

bool tc_supported(const dpmm_ctx*) { return false; }
cudaError_t tc_prepare(dpmm_ctx*) { return cudaSuccess; }
cudaError_t launch_labels_tc(dpmm_ctx*, uint64_t) { return cudaErrorNotSupported; }

}  // namespace dpmm
