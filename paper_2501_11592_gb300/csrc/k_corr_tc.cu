// K1: bf16 tensor-core correlation (tcgen05 + TMA) -- not built yet.
#include "cs_internal.cuh"

namespace cs {

bool corr_tc_supported(int, int) { return false; }

cudaError_t launch_corr_tc(const IterArgs&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace cs
