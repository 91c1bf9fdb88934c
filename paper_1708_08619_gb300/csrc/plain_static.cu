// Plain-path entry point that allocates nothing: its scratch (the per-item
// FP64 partial sums that tcorr_msd / tcorr_acf keep in the caller's
// workspace) lives in one fixed array in device memory owned by this file.
//
// It exists for callers that cannot allocate device memory themselves, for
// example an analysis hook running inside a simulation engine that owns all
// device memory through its own pool, or a host that must not call
// cudaMalloc because that call synchronises the device and would stall the
// engine's streams.
//
// The array is a file-scope __device__ object: the host-side name is only a
// stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress (the first call on a device does this, with that
// device current) and passed to the kernels.  Every call on a device uses the
// same array and it keeps the last call's contents; nothing has to start at
// zero because every partial the reduction reads is written earlier in the
// same call.  Calls whose work overlaps on the GPU (different streams, no
// ordering) race on the array.
#include <mutex>

#include "tcorr_internal.cuh"

namespace tcorr {

BandPlan plain_band_plan(int64_t T, int64_t N, int64_t tau_max, int64_t s);
bool corr_sizes_valid(int64_t T, int64_t N, int64_t tau_max, int64_t s);

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_plain_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of this device's scratch array (looked up once per device).
int scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TCORR_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return TCORR_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_plain_scratch) != cudaSuccess || p == nullptr) return TCORR_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TCORR_OK;
}

}  // namespace
}  // namespace tcorr

using namespace tcorr;

extern "C" int tcorr_plain_static(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max,
                                  int64_t stride, double *d_out, void *stream) {
    if ((kind != 0 && kind != 1) || !d_x || !d_out) return TCORR_EINVAL;
    if (!corr_sizes_valid(T, N, tau_max, stride)) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_x) & 3u) || (reinterpret_cast<uintptr_t>(d_out) & 7u))
        return TCORR_EALIGN;
    const BandPlan p = plain_band_plan(T, N, tau_max, stride);
    const size_t need = sizeof(double) * static_cast<size_t>(p.n_items) * p.WP;
    if (need > kStaticScratchBytes) return TCORR_EWORKSPACE;   // shape needs more than the fixed array
    void *scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != TCORR_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *partial = static_cast<double *>(scratch);
    if (launch_plain_tiles(kind, d_x, p, partial, st) != cudaSuccess) return TCORR_ECUDA;
    FinalizeArgs fa{0, nullptr, 0};
    if (launch_lag_reduce(p, partial, fa, d_out, st) != cudaSuccess) return TCORR_ECUDA;
    return TCORR_OK;
}
