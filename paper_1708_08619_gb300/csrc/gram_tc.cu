// Tensor-core banded Gram path (tcgen05).  Placeholder until the kernel lands:
// every tensor-core method reports TCORR_EUNSUPPORTED.
#include "tcorr_internal.cuh"

namespace tcorr {

__device__ unsigned int g_status;   // device status word (TCORR_OK or an error)

size_t gram_workspace_size(int64_t, int64_t, int64_t, int64_t, int) { return 0; }

int gram_run(int, const float *, int64_t, int64_t, int64_t, int64_t, int, double *, void *, size_t,
             cudaStream_t) {
    return TCORR_EUNSUPPORTED;
}

bool gram_method_available(int) { return false; }

int status_poll_and_clear(cudaStream_t st) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return TCORR_ECUDA;
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof(v)) != cudaSuccess) return TCORR_ECUDA;
    const unsigned int zero = 0;
    if (cudaMemcpyToSymbol(g_status, &zero, sizeof(zero)) != cudaSuccess) return TCORR_ECUDA;
    return static_cast<int>(v);
}

}  // namespace tcorr
