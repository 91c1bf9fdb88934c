// Diagnostics: CUDA events recorded on the launching stream around each
// launch of the dominant kernel (the tensor-core band / polyphase kernel, or
// the plain tile kernel), so that a caller can time that kernel alone while
// the library enqueues several kernels per call.  Off unless enabled; when on,
// every recorded launch creates two events (host-side objects, no device
// memory), released when read.
#include <mutex>
#include <vector>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

struct Rec {
    int kind;
    cudaEvent_t a, b;
};

std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<Rec> g_recs;
thread_local Rec g_open{-1, nullptr, nullptr};

}  // namespace

void prof_begin(int kind, cudaStream_t st) {
    {
        std::lock_guard<std::mutex> lock(g_prof_mu);
        if (!g_prof_on) return;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    Rec r{kind, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) {
        cudaEventDestroy(r.a);
        return;
    }
    cudaEventRecord(r.a, st);
    g_open = r;
}

void prof_end(cudaStream_t st) {
    if (g_open.a == nullptr) return;
    cudaEventRecord(g_open.b, st);
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_recs.push_back(g_open);
    g_open = Rec{-1, nullptr, nullptr};
}

}  // namespace tcorr

using namespace tcorr;

extern "C" int tcorr_profile_enable(int on) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    g_prof_on = on != 0;
    return TCORR_OK;
}

extern "C" int tcorr_profile_read(int kind, double *total_ms, int *launches) {
    if (!total_ms || !launches) return TCORR_EINVAL;
    std::lock_guard<std::mutex> lock(g_prof_mu);
    double sum = 0.0;
    int n = 0;
    std::vector<Rec> keep;
    for (const Rec &r : g_recs) {
        if (r.kind != kind) {
            keep.push_back(r);
            continue;
        }
        if (cudaEventSynchronize(r.b) != cudaSuccess) return TCORR_ECUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return TCORR_ECUDA;
        sum += ms;
        ++n;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.swap(keep);
    *total_ms = sum;
    *launches = n;
    return TCORR_OK;
}
