// C ABI of libtcorr.so (declared in include/tcorr.h): argument validation,
// work planning, workspace carving and dispatch to the kernels.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

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
size_t gram_batch_workspace_size(const tcorr_instance *items, int count, int method);
int gram_batch_run(const tcorr_instance *items, int count, int method, void *d_ws, size_t ws_bytes,
                   cudaStream_t st);
int status_poll_and_clear(cudaStream_t st);
int selftest_timeout(cudaStream_t st);

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

void cap_origins(BandPlan *p, int64_t cap) {
    if (cap <= 0 || cap >= p->n_orig) return;
    p->n_orig = cap;
    p->n_rows = ceil_div(cap, p->BO);
    p->n_items = p->n_groups * p->n_res * p->n_rows * p->n_cols;
}

namespace {

bool valid_sizes(int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    if (T < 1 || N < 1 || s < 1 || tau_max < 0 || tau_max > T - 1) return false;
    // keep T * 3N and the padded forms far from int64 overflow
    if (N > (int64_t(1) << 40) || T > (int64_t(1) << 40)) return false;
    if (static_cast<double>(T) * static_cast<double>(N) * 3.0 > 9.0e15) return false;
    return true;
}

bool known_method(int m) { return (m >= TCORR_PLAIN && m <= TCORR_AUTO) || m == TCORR_FFT; }

size_t plain_workspace(int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    const BandPlan p = make_band_plan(T, N, tau_max, s, plain_tile_bo(), plain_tile_bf(), kPlainKseg,
                                      kMinItems);
    return align256(sizeof(double) * static_cast<size_t>(p.n_items) * p.WP);
}

// AUTO: the FFT route when its cost estimate is below the band form's, else
// the FP16 x3 tensor-core form (plain without a tensor-core device).  Costs
// per K column, calibrated on GB300: band about 6.5e-15 s per (origin, lag)
// pair (T (tau_max + 128) of them), FFT about 4e-12 s per L log2 L of the
// padded transform length (the library's double-float transforms, two
// columns per complex transform); e.g. T = 2e6 switches to the FFT above
// tau_max ~ 3e4, T = 1e5 above tau_max ~ 2.3e4.
int resolve_method(int method, int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    (void)N;
    (void)s;
    if (method != TCORR_AUTO) return method;
    if (!gram_method_available(TCORR_TC_FP16X3)) return TCORR_PLAIN;
    if (!fft_supported(T, tau_max)) return TCORR_TC_FP16X3;
    const double L = 2.0 * static_cast<double>(T + tau_max);      // padded length, within 2x
    const double band = 6.5e-15 * static_cast<double>(T) * static_cast<double>(tau_max + 128);
    const double fft = 4e-12 * L * std::log2(L);
    return fft < band ? TCORR_FFT : TCORR_TC_FP16X3;
}

}  // namespace

// Plain FP32 path for one trajectory, or one window of it (w != nullptr).
int plain_run(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s, double *d_out,
              void *d_ws, size_t ws_bytes, cudaStream_t st, const Window *w, const float *d_y) {
    BandPlan p = make_band_plan(T, N, tau_max, s, plain_tile_bo(), plain_tile_bf(), kPlainKseg, kMinItems);
    if (w) cap_origins(&p, w->orig_cap);
    const size_t need = align256(sizeof(double) * static_cast<size_t>(p.n_items) * p.WP);
    if (ws_bytes < need || (need > 0 && !d_ws)) return TCORR_EWORKSPACE;
    double *partial = static_cast<double *>(d_ws);
    cudaError_t e = launch_plain_tiles(kind, d_x, p, partial, st, d_y);
    if (e != cudaSuccess) return cuda_fail(e, "plain_tile_kernel launch");
    FinalizeArgs fa{0, nullptr, 0};
    e = launch_lag_reduce(p, partial, fa, d_out, st, w);
    if (e != cudaSuccess) return cuda_fail(e, "lag_reduce launch");
    return TCORR_OK;
}

size_t plain_window_workspace(int64_t T, int64_t N, int64_t tau_max, int64_t s, int64_t orig_cap) {
    BandPlan p = make_band_plan(T, N, tau_max, s, plain_tile_bo(), plain_tile_bf(), kPlainKseg, kMinItems);
    cap_origins(&p, orig_cap);
    return align256(sizeof(double) * static_cast<size_t>(p.n_items) * p.WP);
}

namespace {

int run_corr(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s,
             int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    if (!d_x || !d_out) return TCORR_EINVAL;
    if (!valid_sizes(T, N, tau_max, s) || !known_method(method)) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_x) & 3u) || (reinterpret_cast<uintptr_t>(d_out) & 7u) ||
        (reinterpret_cast<uintptr_t>(d_ws) & 255u))
        return TCORR_EALIGN;
    const int m = resolve_method(method, T, N, tau_max, s);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m == TCORR_FFT) return fft_run(kind, d_x, T, N, tau_max, s, d_out, d_ws, ws_bytes, st);
    if (m != TCORR_PLAIN)
        return gram_run(kind, d_x, T, N, tau_max, s, m, d_out, d_ws, ws_bytes, st);
    return plain_run(kind, d_x, T, N, tau_max, s, d_out, d_ws, ws_bytes, st, nullptr);
}

// ------------------------------------------------------------------ batch
// Plain method: one batched tile launch over every instance's work items
// (block -> instance by binary search) and one batched reduction.
struct PlainBatchLayout {
    std::vector<BandPlan> plans;
    std::vector<size_t> partial_off;
    size_t off_args = 0, off_red = 0, total = 0;
    int64_t total_items = 0, total_lags = 0;
};

void plain_batch_layout(const tcorr_instance *items, int count, PlainBatchLayout *B) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    B->off_args = take(plain_args_size() * count);
    B->off_red = take(sizeof(LagReduceDesc) * count);
    host_alloc_fault_point();
    B->plans.resize(count);
    B->partial_off.resize(count);
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &it = items[i];
        B->plans[i] = make_band_plan(it.T, it.N, it.tau_max, it.stride, plain_tile_bo(), plain_tile_bf(),
                                     kPlainKseg, kMinItems);
        B->partial_off[i] = take(sizeof(double) * static_cast<size_t>(B->plans[i].n_items) * B->plans[i].WP);
        B->total_items += B->plans[i].n_items;
        B->total_lags += it.tau_max + 1;
    }
    B->total = off;
}

int plain_batch_run(const tcorr_instance *items, int count, void *d_ws, size_t ws_bytes, cudaStream_t st) {
    PlainBatchLayout B;
    plain_batch_layout(items, count, &B);
    if (ws_bytes < B.total || !d_ws) return TCORR_EWORKSPACE;
    if (B.total_items > 0x7fffffffLL) return TCORR_EUNSUPPORTED;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    std::vector<uint8_t> args(plain_args_size() * count);
    std::vector<LagReduceDesc> red(count);
    int64_t item_begin = 0, lag_begin = 0;
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &it = items[i];
        double *partial = reinterpret_cast<double *>(ws + B.partial_off[i]);
        plain_args_write(args.data() + plain_args_size() * i, it.kind, it.d_x, B.plans[i], partial, item_begin);
        red[i] = lag_reduce_desc(B.plans[i], partial, FinalizeArgs{0, nullptr, 0}, it.d_out, lag_begin);
        item_begin += B.plans[i].n_items;
        lag_begin += it.tau_max + 1;
    }
    cudaError_t e;
    if ((e = upload_bytes(ws + B.off_args, args.data(), args.size(), st)) != cudaSuccess ||
        (e = upload_bytes(ws + B.off_red, red.data(), sizeof(LagReduceDesc) * count, st)) != cudaSuccess)
        return cuda_fail(e, "descriptor upload");
    if ((e = launch_plain_tiles_batch(ws + B.off_args, count, B.total_items, st)) != cudaSuccess)
        return cuda_fail(e, "plain_tile_batch_kernel launch");
    if ((e = launch_lag_reduce_batch(reinterpret_cast<const LagReduceDesc *>(ws + B.off_red), count,
                                     B.total_lags, st)) != cudaSuccess)
        return cuda_fail(e, "lag_reduce_batch launch");
    return TCORR_OK;
}

int batch_method(const tcorr_instance *items, int count, int method) {
    if (method != TCORR_AUTO) return method;
    (void)items;
    (void)count;
    return gram_method_available(TCORR_TC_FP16X3) ? TCORR_TC_FP16X3 : TCORR_PLAIN;
}

size_t batch_workspace(const tcorr_instance *items, int count, int m) {
    if (m == TCORR_PLAIN) {
        PlainBatchLayout B;
        plain_batch_layout(items, count, &B);
        return B.total;
    }
    return gram_batch_workspace_size(items, count, m);
}

int batch_run_direct(const tcorr_instance *items, int count, int m, void *d_ws, size_t ws_bytes,
                     cudaStream_t st) {
    if (m == TCORR_PLAIN) return plain_batch_run(items, count, d_ws, ws_bytes, st);
    return gram_batch_run(items, count, m, d_ws, ws_bytes, st);
}

// Graph cache: the first tcorr_batch call with a given argument set is
// captured into a CUDA graph and instantiated; later calls with the same
// instances, method, workspace, device and tuning knobs replay it with one
// cudaGraphLaunch.  Entries are dropped oldest first beyond kGraphCacheSize.
constexpr size_t kGraphCacheSize = 8;

struct GraphEntry {
    std::vector<tcorr_instance> items;
    int method;
    void *ws;
    size_t ws_bytes;
    int device;
    std::string knobs;
    cudaGraphExec_t exec;
};

std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;

std::string knob_string() {
    std::string k;
    for (const char *name : {"TCORR_KSEG", "TCORR_SUB_KB", "TCORR_SUPER"}) {
        const char *v = std::getenv(name);
        k += v ? v : "-";
        k += ';';
    }
    return k;
}

bool same_items(const std::vector<tcorr_instance> &a, const tcorr_instance *b, int count) {
    if (a.size() != static_cast<size_t>(count)) return false;
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &x = a[i], &y = b[i];
        if (x.kind != y.kind || x.d_x != y.d_x || x.T != y.T || x.N != y.N || x.tau_max != y.tau_max ||
            x.stride != y.stride || x.d_out != y.d_out)
            return false;
    }
    return true;
}

int batch_run_graph(const tcorr_instance *items, int count, int m, void *d_ws, size_t ws_bytes,
                    cudaStream_t st) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TCORR_ECUDA;
    const std::string knobs = knob_string();
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (const GraphEntry &g : g_graphs) {
        if (g.method == m && g.ws == d_ws && g.ws_bytes == ws_bytes && g.device == dev && g.knobs == knobs &&
            same_items(g.items, items, count)) {
            const cudaError_t e = cudaGraphLaunch(g.exec, st);
            return e == cudaSuccess ? TCORR_OK : cuda_fail(e, "cudaGraphLaunch");
        }
    }
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    int rc;
    try {
        rc = batch_run_direct(items, count, m, d_ws, ws_bytes, st);
    } catch (const std::bad_alloc &) {
        cudaGraph_t partial = nullptr;           // leave the stream out of capture mode
        if (cudaStreamEndCapture(st, &partial) == cudaSuccess && partial) cudaGraphDestroy(partial);
        throw;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (rc != TCORR_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    if (g_graphs.size() >= kGraphCacheSize) {
        cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(GraphEntry{std::vector<tcorr_instance>(items, items + count), m, d_ws, ws_bytes, dev,
                                  knobs, exec});
    e = cudaGraphLaunch(exec, st);
    return e == cudaSuccess ? TCORR_OK : cuda_fail(e, "cudaGraphLaunch");
}

}  // namespace

// Cross-correlation: products of d_a at the origin and d_b at the later frame,
// band form on either path (no polyphase: its operand copies hold one signal).
int run_xcf(const float *d_a, const float *d_b, int64_t T, int64_t N, int64_t tau_max, int64_t s, int method,
            double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    if (!d_a || !d_b || !d_out) return TCORR_EINVAL;
    if (!valid_sizes(T, N, tau_max, s) || !known_method(method)) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_a) & 3u) || (reinterpret_cast<uintptr_t>(d_b) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_out) & 7u) || (reinterpret_cast<uintptr_t>(d_ws) & 255u))
        return TCORR_EALIGN;
    const int m = resolve_method(method, T, N, tau_max, s);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m == TCORR_FFT) return fft_run(2, d_a, T, N, tau_max, s, d_out, d_ws, ws_bytes, st, d_b);
    if (m != TCORR_PLAIN) return gram_run(2, d_a, T, N, tau_max, s, m, d_out, d_ws, ws_bytes, st, nullptr, d_b);
    return plain_run(2, d_a, T, N, tau_max, s, d_out, d_ws, ws_bytes, st, nullptr, d_b);
}

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
    if (m == TCORR_FFT) return fft_workspace_size(T, N, tau_max, stride, 0);
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

size_t tcorr_weighted_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t stride, int method) {
    const size_t eng = tcorr_workspace_size(T, N, tau_max, stride, method);
    if (eng == 0) return 0;
    return weighted_copy_bytes(T, N) + eng;
}

static int run_weighted(int kind, const float *d_x, const float *d_w, int64_t T, int64_t N, int64_t tau_max,
                        int64_t s, int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    if (!d_x || !d_w || !d_out) return TCORR_EINVAL;
    if (!valid_sizes(T, N, tau_max, s) || !known_method(method)) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_x) & 3u) || (reinterpret_cast<uintptr_t>(d_w) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_out) & 7u) || (reinterpret_cast<uintptr_t>(d_ws) & 255u))
        return TCORR_EALIGN;
    const size_t need = tcorr_weighted_workspace_size(T, N, tau_max, s, method);
    if (need == 0) return TCORR_EUNSUPPORTED;
    if (!d_ws || ws_bytes < need) return TCORR_EWORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t copy = weighted_copy_bytes(T, N);
    cudaError_t e = launch_weight_copy(kind, d_x, d_w, T, N, d_ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "weighted copy launch");
    const int rc = run_corr(kind, static_cast<const float *>(d_ws), T, N, tau_max, s, method, d_out,
                            static_cast<uint8_t *>(d_ws) + copy, ws_bytes - copy, stream);
    if (rc != TCORR_OK) return rc;
    e = launch_weight_rescale(d_out, tau_max + 1, T, N, d_ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "weighted rescale launch");
    return TCORR_OK;
}

int tcorr_msd_weighted(const float *d_x, const float *d_w, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                       int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    return run_weighted(0, d_x, d_w, T, N, tau_max, stride, method, d_out, d_ws, ws_bytes, stream);
}

int tcorr_acf_weighted(const float *d_x, const float *d_w, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                       int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    return run_weighted(1, d_x, d_w, T, N, tau_max, stride, method, d_out, d_ws, ws_bytes, stream);
}

size_t tcorr_xcf_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t stride, int method) {
    if (!valid_sizes(T, N, tau_max, stride) || !known_method(method)) return 0;
    const int m = resolve_method(method, T, N, tau_max, stride);
    if (m == TCORR_PLAIN) return plain_workspace(T, N, tau_max, stride);
    if (m == TCORR_FFT) return fft_workspace_size(T, N, tau_max, stride, 2);
    return gram_workspace_size(T, N, tau_max, stride, m, nullptr, 2);
}

int tcorr_xcf(const float *d_a, const float *d_b, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
              int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    return run_xcf(d_a, d_b, T, N, tau_max, stride, method, d_out, d_ws, ws_bytes, stream);
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

int gk_integrate_batch(const double *d_c, int64_t n, int64_t count, int64_t ldc, double dt, double prefactor,
                       double *d_running, int64_t ldr, void *stream) {
    if (n < 1 || count < 0 || ldc < n || ldr < n) return TCORR_EINVAL;
    if (count == 0) return TCORR_OK;
    if (!d_c || !d_running) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_c) & 7u) || (reinterpret_cast<uintptr_t>(d_running) & 7u))
        return TCORR_EALIGN;
    if (count > (INT64_MAX / 8 - n) / ldc || count > (INT64_MAX / 8 - n) / ldr) return TCORR_EINVAL;
    // the spans [first series, end of the last) may not overlap
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(d_c), a1 = a0 + sizeof(double) * ((count - 1) * ldc + n);
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(d_running), b1 = b0 + sizeof(double) * ((count - 1) * ldr + n);
    if (a0 < b1 && b0 < a1) return TCORR_EINVAL;
    if (launch_gk_integrate_batch(d_c, n, count, ldc, dt, prefactor, d_running, ldr,
                                  static_cast<cudaStream_t>(stream)) != cudaSuccess)
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
    if (!h_items || count < 1 || !known_method(method)) return 0;
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &it = h_items[i];
        if (!valid_sizes(it.T, it.N, it.tau_max, it.stride)) return 0;
    }
    try {
        return batch_workspace(h_items, count, batch_method(h_items, count, method));
    } catch (const std::bad_alloc &) {
        return 0;
    }
}

int tcorr_batch(const tcorr_instance *h_items, int count, int method, void *d_ws, size_t ws_bytes,
                void *stream) {
    if (!h_items || count < 1 || !known_method(method)) return TCORR_EINVAL;
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &it = h_items[i];
        if ((it.kind != 0 && it.kind != 1) || !it.d_x || !it.d_out ||
            !valid_sizes(it.T, it.N, it.tau_max, it.stride))
            return TCORR_EINVAL;
        if ((reinterpret_cast<uintptr_t>(it.d_x) & 3u) || (reinterpret_cast<uintptr_t>(it.d_out) & 7u))
            return TCORR_EALIGN;
    }
    if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return TCORR_EALIGN;
    try {
        const int m = batch_method(h_items, count, method);
        const size_t need = batch_workspace(h_items, count, m);   // host plan: before any launch
        if (need == 0) return TCORR_EUNSUPPORTED;
        if (ws_bytes < need || !d_ws) return TCORR_EWORKSPACE;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (st != nullptr && cudaStreamIsCapturing(st, &cs) != cudaSuccess) return TCORR_ECUDA;
        if (st == nullptr || cs != cudaStreamCaptureStatusNone || std::getenv("TCORR_NO_GRAPH"))
            return batch_run_direct(h_items, count, m, d_ws, ws_bytes, st);
        return batch_run_graph(h_items, count, m, d_ws, ws_bytes, st);
    } catch (const std::bad_alloc &) {
        return TCORR_ENOMEM;      // a host allocation failed (the injected one, in the plan: nothing enqueued)
    }
}

int tcorr_status_poll(void *stream) { return status_poll_and_clear(static_cast<cudaStream_t>(stream)); }

int tcorr_selftest_timeout(void *stream) { return selftest_timeout(static_cast<cudaStream_t>(stream)); }

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
        case TCORR_EBOUNDS: return "TCORR_EBOUNDS: index check of a debug build failed";
        default: return "unknown tcorr status";
    }
}

int tcorr_version(void) { return 100; }

}  // extern "C"
