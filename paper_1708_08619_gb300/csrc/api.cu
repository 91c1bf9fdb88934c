// C ABI of libtcorr.so (declared in include/tcorr.h): argument validation,
// work planning, workspace carving and dispatch to the kernels.
#include <cstdint>
#include <cstring>

#include "tcorr_internal.cuh"

namespace tcorr {

// Blocks to aim for per launch of the band kernels: enough waves on a
// 152-SM part at two resident blocks per SM to keep the tail short.
constexpr int64_t kMinItems = 16 * 152;
// K elements per FP32 run of a pair sum before its diagonal is flushed to FP64.
constexpr int64_t kPlainKseg = 256;

int plain_tile_bo();
int plain_tile_bf();
int plain_tile_wp();

// Tensor-core path (gram_tc.cu).
size_t gram_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t s, int method);
int gram_run(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s,
             int method, double *d_out, void *d_ws, size_t ws_bytes, cudaStream_t st);
bool gram_method_available(int method);
int status_poll_and_clear(cudaStream_t st);

BandPlan make_band_plan(int64_t T, int64_t N, int64_t tau_max, int64_t s, int BO, int BF,
                        int64_t kseg, int64_t min_items) {
    BandPlan p;
    p.T = T;
    p.N = N;
    p.K = 3 * N;
    p.tau_max = tau_max;
    p.s = s;
    p.n_orig = (T - 1) / s + 1;
    p.n_res = s < tau_max + 1 ? s : tau_max + 1;
    p.m_max0 = tau_max / s;
    p.BO = BO;
    p.BF = BF;
    p.WP = static_cast<int>(ceil_div(BO + BF - 1, 64) * 64);
    p.n_rows = ceil_div(p.n_orig, BO);
    p.n_cols = ceil_div(BO + p.m_max0, BF);
    p.kseg = kseg;
    const int64_t n_seg = ceil_div(p.K, kseg);
    const int64_t tiles = p.n_res * p.n_rows * p.n_cols;
    int64_t want_groups = ceil_div(min_items, tiles);
    if (want_groups > n_seg) want_groups = n_seg;
    if (want_groups < 1) want_groups = 1;
    p.segs_per_item = ceil_div(n_seg, want_groups);
    p.n_groups = ceil_div(n_seg, p.segs_per_item);
    p.n_items = p.n_groups * tiles;
    return p;
}

namespace {

bool valid_sizes(int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    if (T < 1 || N < 1 || s < 1 || tau_max < 0 || tau_max > T - 1) return false;
    // keep T * 3N and the padded forms far from int64 overflow
    if (N > (int64_t(1) << 40) || T > (int64_t(1) << 40)) return false;
    if (static_cast<double>(T) * static_cast<double>(N) * 3.0 > 9.0e15) return false;
    return true;
}

bool known_method(int m) { return m >= TCORR_PLAIN && m <= TCORR_AUTO; }

size_t plain_workspace(int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    const BandPlan p = make_band_plan(T, N, tau_max, s, plain_tile_bo(), plain_tile_bf(), kPlainKseg,
                                      kMinItems);
    return align256(sizeof(double) * static_cast<size_t>(p.n_items) * p.WP);
}

int resolve_method(int method, int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    (void)T;
    (void)N;
    (void)tau_max;
    (void)s;
    if (method != TCORR_AUTO) return method;
    return gram_method_available(TCORR_TC_FP16X3) ? TCORR_TC_FP16X3 : TCORR_PLAIN;
}

int run_corr(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s,
             int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    if (!d_x || !d_out) return TCORR_EINVAL;
    if (!valid_sizes(T, N, tau_max, s) || !known_method(method)) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_x) & 3u) || (reinterpret_cast<uintptr_t>(d_out) & 7u) ||
        (reinterpret_cast<uintptr_t>(d_ws) & 255u))
        return TCORR_EALIGN;
    const int m = resolve_method(method, T, N, tau_max, s);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m != TCORR_PLAIN)
        return gram_run(kind, d_x, T, N, tau_max, s, m, d_out, d_ws, ws_bytes, st);

    const BandPlan p = make_band_plan(T, N, tau_max, s, plain_tile_bo(), plain_tile_bf(), kPlainKseg,
                                      kMinItems);
    const size_t need = align256(sizeof(double) * static_cast<size_t>(p.n_items) * p.WP);
    if (ws_bytes < need || (need > 0 && !d_ws)) return TCORR_EWORKSPACE;
    double *partial = static_cast<double *>(d_ws);
    cudaError_t e = launch_plain_tiles(kind, d_x, p, partial, st);
    if (e != cudaSuccess) return cuda_fail(e, "plain_tile_kernel launch");
    FinalizeArgs fa{0, nullptr, 0};
    e = launch_lag_reduce(p, partial, fa, d_out, st);
    if (e != cudaSuccess) return cuda_fail(e, "lag_reduce launch");
    return TCORR_OK;
}

}  // namespace

// The plain path's plan and size check, shared with the fixed-scratch entry
// point so that both produce bit-identical results for the same arguments.
BandPlan plain_band_plan(int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    return make_band_plan(T, N, tau_max, s, plain_tile_bo(), plain_tile_bf(), kPlainKseg, kMinItems);
}

bool corr_sizes_valid(int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    return valid_sizes(T, N, tau_max, s);
}

}  // namespace tcorr

using namespace tcorr;

extern "C" {

size_t tcorr_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t stride, int method) {
    if (!valid_sizes(T, N, tau_max, stride) || !known_method(method)) return 0;
    const int m = resolve_method(method, T, N, tau_max, stride);
    if (m == TCORR_PLAIN) return plain_workspace(T, N, tau_max, stride);
    return gram_workspace_size(T, N, tau_max, stride, m);
}

int tcorr_msd(const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride, int method,
              double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    return run_corr(0, d_x, T, N, tau_max, stride, method, d_out, d_ws, ws_bytes, stream);
}

int tcorr_acf(const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride, int method,
              double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    return run_corr(1, d_x, T, N, tau_max, stride, method, d_out, d_ws, ws_bytes, stream);
}

int gk_integrate(const double *d_c, int64_t n, double dt, double prefactor, double *d_running,
                 void *stream) {
    if (!d_c || !d_running || n < 1) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_c) & 7u) || (reinterpret_cast<uintptr_t>(d_running) & 7u))
        return TCORR_EALIGN;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(d_c), a1 = a0 + sizeof(double) * n;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(d_running), b1 = b0 + sizeof(double) * n;
    if (a0 < b1 && b0 < a1) return TCORR_EINVAL;   // overlapping buffers
    if (launch_gk_integrate(d_c, n, dt, prefactor, d_running, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess)
        return TCORR_ECUDA;
    return TCORR_OK;
}

int einstein_slope(const double *d_msd, int64_t n, double dt, int dim, int64_t lo, int64_t hi,
                   double *d_D, void *stream) {
    if (!d_msd || !d_D || dim < 1 || lo < 0 || hi <= lo || hi >= n || !(dt > 0.0))
        return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_msd) & 7u) || (reinterpret_cast<uintptr_t>(d_D) & 7u))
        return TCORR_EALIGN;
    if (launch_einstein(d_msd, n, dt, dim, lo, hi, d_D, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess)
        return TCORR_ECUDA;
    return TCORR_OK;
}

size_t tcorr_batch_workspace_size(const tcorr_instance *h_items, int count, int method) {
    if (!h_items || count < 1) return 0;
    size_t need = 0;
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &it = h_items[i];
        const size_t w = tcorr_workspace_size(it.T, it.N, it.tau_max, it.stride, method);
        if (w == 0) return 0;
        if (w > need) need = w;
    }
    return need;
}

int tcorr_batch(const tcorr_instance *h_items, int count, int method, void *d_ws, size_t ws_bytes,
                void *stream) {
    if (!h_items || count < 1 || !known_method(method)) return TCORR_EINVAL;
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &it = h_items[i];
        if ((it.kind != 0 && it.kind != 1) || !it.d_x || !it.d_out ||
            !valid_sizes(it.T, it.N, it.tau_max, it.stride))
            return TCORR_EINVAL;
    }
    const size_t need = tcorr_batch_workspace_size(h_items, count, method);
    if (ws_bytes < need) return TCORR_EWORKSPACE;
    // Instances run one after another on the stream and share the workspace.
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &it = h_items[i];
        const int rc = run_corr(it.kind, it.d_x, it.T, it.N, it.tau_max, it.stride, method, it.d_out,
                                d_ws, ws_bytes, stream);
        if (rc != TCORR_OK) return rc;
    }
    return TCORR_OK;
}

int tcorr_status_poll(void *stream) { return status_poll_and_clear(static_cast<cudaStream_t>(stream)); }

const char *tcorr_strerror(int code) {
    switch (code) {
        case TCORR_OK: return "TCORR_OK";
        case TCORR_EINVAL: return "TCORR_EINVAL: invalid argument";
        case TCORR_EALIGN: return "TCORR_EALIGN: misaligned pointer";
        case TCORR_ENOMEM: return "TCORR_ENOMEM: host allocation failed";
        case TCORR_EWORKSPACE: return "TCORR_EWORKSPACE: workspace too small";
        case TCORR_ECUDA: return "TCORR_ECUDA: CUDA call failed";
        case TCORR_ETIMEOUT: return "TCORR_ETIMEOUT: device-side wait gave up";
        case TCORR_EUNSUPPORTED: return "TCORR_EUNSUPPORTED: method cannot run this shape";
        default: return "unknown tcorr status";
    }
}

int tcorr_version(void) { return 100; }

}  // extern "C"
