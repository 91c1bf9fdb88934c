// Streamed (out-of-core) correlation of a trajectory held in host memory.
//
// The whole-trajectory path needs X[T][N][3] resident on the device; the
// paper's Conclusion names that as the limit for dynamic quantities such as
// the MSD (all frames of a species on the device), and its two-particle
// section leaves splitting a trajectory to the user.  Here
// the origins are cut into windows of C frames: window c holds frames
// [cC, min(T, cC + C + tau_max)), i.e. its C origins plus a tau_max halo of
// partner frames.  Every pair (t0, t0 + tau) with t0 in the window's first C
// frames lies inside the window, so the windows together see each pair of
// Eq. 5 (MSD) and of the ACF numerator (Eq. 4) exactly once.  Each window
// runs the same engine as the whole-trajectory call, with its origins capped
// at C and its per-lag numerators added into d_out; one last kernel divides
// by N n_o(tau) of the whole trajectory.
//
// Copies: three window buffers rotate.  Window c's halo (its first tau_max
// frames) is the tail of window c-1 and is copied device to device; only the
// new frames cross from the host, so each frame crosses once.  Copies run
// on a second stream and overlap the earlier windows' kernels; events order
// buffer reuse.  With two buffers the copy of window c waited for window
// c-2's kernels, so whenever the window kernels queued behind other work on
// the device (an in-core call on another stream) the host link went idle;
// the third buffer lets the copies run one window further ahead.
#include <cstdint>
#include <vector>

#include "tcorr_internal.cuh"

namespace tcorr {

namespace {

constexpr int NBUF = 3;             // window buffers in rotation

// Origins per window when the caller passes 0: four halos' worth, at least
// 4096 frames, whole 128-origin row tiles.
int64_t default_chunk(int64_t tau_max, int64_t s) {
    int64_t c = 4 * (tau_max + 1);
    if (c < 4096) c = 4096;
    const int64_t q = 128 * s;
    return ceil_div(c, q) * q;
}

struct StreamPlan {
    int method;                 // resolved (never TCORR_AUTO)
    int64_t K, C, W, n_win;     // K = 3N; origins per window; largest window; windows
    std::vector<int64_t> start; // first frame of each window (multiples of s), then T
    int nbuf;                   // window buffers in use: min(NBUF, windows)
    size_t off_buf[NBUF], off_engine, engine_bytes, total;
};

// Windows of C origin frames, except that the last stretch is cut so that the
// final window holds at most a quarter of C: its kernels are the part of the
// call that no copy overlaps.
std::vector<int64_t> window_starts(int64_t T, int64_t C, int64_t s) {
    std::vector<int64_t> st;
    int64_t q = (C / 4 / s) * s;
    if (q < s) q = s;
    int64_t t = 0;
    while (t < T) {
        st.push_back(t);
        const int64_t rem = T - t;
        if (rem > C + q) t += C;
        else if (rem > q) t += ceil_div(rem - q, s) * s;
        else t = T;
    }
    st.push_back(T);
    return st;
}

// Frames held by window c: its origin frames plus the tau_max halo.
int64_t window_frames(const StreamPlan &P, int64_t T, int64_t tau_max, int64_t c) {
    const int64_t t0 = P.start[c], w = (P.start[c + 1] - t0) + tau_max;
    return T - t0 < w ? T - t0 : w;
}

Window window_of(const StreamPlan &P, int64_t c, int64_t s) {
    const int64_t len = P.start[c + 1] - P.start[c];     // frames whose origins start pairs here
    return Window{(len - 1) / s + 1, true};
}

bool make_stream_plan(int64_t T, int64_t N, int64_t tau_max, int64_t s, int method, int64_t chunk,
                      StreamPlan *P) {
    if (chunk < 0) return false;
    P->method = method;
    if (method == TCORR_AUTO) P->method = gram_method_available(TCORR_TC_FP16X3) ? TCORR_TC_FP16X3 : TCORR_PLAIN;
    P->K = 3 * N;
    int64_t C = chunk > 0 ? chunk : default_chunk(tau_max, s);
    C = ceil_div(C, s) * s;                              // windows start on origins
    const int64_t Tcap = ceil_div(T, s) * s;
    if (C > Tcap) C = Tcap;
    P->C = C;
    P->W = T < C + tau_max ? T : C + tau_max;
    P->start = window_starts(T, C, s);
    P->n_win = static_cast<int64_t>(P->start.size()) - 1;
    // Engine workspace: the largest over the windows.  A smaller window can
    // need more (its plan splits K into more groups to fill the GPU), so every
    // distinct window shape is sized; full windows all share one shape.
    P->engine_bytes = 0;
    bool full_seen = false;
    for (int64_t c = 0; c < P->n_win; ++c) {
        const int64_t len = P->start[c + 1] - P->start[c], Wc = window_frames(*P, T, tau_max, c);
        const bool full = len == C && Wc == C + tau_max;
        if (full && full_seen) continue;
        full_seen = full_seen || full;
        const int64_t tm = tau_max < Wc - 1 ? tau_max : Wc - 1;
        const Window w = window_of(*P, c, s);
        const size_t need = P->method == TCORR_PLAIN ? plain_window_workspace(Wc, N, tm, s, w.orig_cap)
                                                     : gram_workspace_size(Wc, N, tm, s, P->method, &w);
        if (need == 0 && P->method != TCORR_PLAIN) return false;
        if (need > P->engine_bytes) P->engine_bytes = need;
    }
    const size_t buf = align256(static_cast<size_t>(P->W) * static_cast<size_t>(P->K) * sizeof(float));
    P->nbuf = static_cast<int>(P->n_win < NBUF ? P->n_win : NBUF);
    for (int i = 0; i < NBUF; ++i) P->off_buf[i] = static_cast<size_t>(i < P->nbuf ? i : 0) * buf;
    P->off_engine = static_cast<size_t>(P->nbuf) * buf;
    P->total = static_cast<size_t>(P->nbuf) * buf + align256(P->engine_bytes);
    return true;
}

// Owns the side stream and events of one call; destroying them with work
// still queued is allowed (CUDA releases them when that work completes).
struct StreamRes {
    cudaStream_t side = nullptr;
    cudaEvent_t start = nullptr, copied[NBUF] = {}, freed[NBUF] = {};
    ~StreamRes() {
        if (start) cudaEventDestroy(start);
        for (int i = 0; i < NBUF; ++i) {
            if (copied[i]) cudaEventDestroy(copied[i]);
            if (freed[i]) cudaEventDestroy(freed[i]);
        }
        if (side) cudaStreamDestroy(side);
    }
    cudaError_t init() {
        cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) != cudaSuccess) return e;
        for (int i = 0; i < NBUF; ++i)
            if ((e = cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming)) != cudaSuccess)
                return e;
        return cudaSuccess;
    }
};

// The host frames: one array, or consecutive chunks (chunk i holds frames
// [first[i], first[i + 1]) as [frames][N][3] float32 rows).
struct HostFrames {
    const float *const *ptr;
    const int64_t *first;     // n + 1 entries, first[0] = 0, first[n] = T
    int n;
};

// Frames [f0, f0 + nf) into dst (rows of `row` bytes): one copy per chunk they touch.
cudaError_t copy_frames(const HostFrames &H, int64_t K, int64_t f0, int64_t nf, float *dst, size_t row,
                        cudaStream_t st) {
    int i = 0;
    while (i + 1 < H.n && H.first[i + 1] <= f0) ++i;
    while (nf > 0) {
        const int64_t in = f0 - H.first[i], take = H.first[i + 1] - f0 < nf ? H.first[i + 1] - f0 : nf;
        const cudaError_t e = cudaMemcpyAsync(dst, H.ptr[i] + static_cast<size_t>(in) * K, take * row,
                                              cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        dst += static_cast<size_t>(take) * K;
        f0 += take;
        nf -= take;
        ++i;
    }
    return cudaSuccess;
}

int run_stream(int kind, const HostFrames &H, int64_t T, int64_t N, int64_t tau_max, int64_t s, int method,
               int64_t chunk, double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    if (!d_out) return TCORR_EINVAL;
    if (!corr_sizes_valid(T, N, tau_max, s) || method < TCORR_PLAIN || method > TCORR_AUTO || chunk < 0)
        return TCORR_EINVAL;
    for (int i = 0; i < H.n; ++i) {
        if (!H.ptr[i]) return TCORR_EINVAL;
        if (reinterpret_cast<uintptr_t>(H.ptr[i]) & 3u) return TCORR_EALIGN;
    }
    if ((reinterpret_cast<uintptr_t>(d_out) & 7u) || (reinterpret_cast<uintptr_t>(d_ws) & 255u))
        return TCORR_EALIGN;
    StreamPlan P;
    if (!make_stream_plan(T, N, tau_max, s, method, chunk, &P)) return TCORR_EUNSUPPORTED;
    if (ws_bytes < P.total || !d_ws) return TCORR_EWORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StreamRes R;
    cudaError_t e = R.init();
    if (e != cudaSuccess) return cuda_fail(e, "stream resources");
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    float *buf[NBUF];
    for (int i = 0; i < NBUF; ++i) buf[i] = reinterpret_cast<float *>(ws + P.off_buf[i]);
    const size_t row = static_cast<size_t>(P.K) * sizeof(float);
    if ((e = cudaMemsetAsync(d_out, 0, sizeof(double) * static_cast<size_t>(tau_max + 1), st)) != cudaSuccess)
        return cuda_fail(e, "output reset");
    // the copy stream starts after everything already queued on the caller's stream
    if ((e = cudaEventRecord(R.start, st)) != cudaSuccess || (e = cudaStreamWaitEvent(R.side, R.start, 0)) != cudaSuccess)
        return cuda_fail(e, "stream fork");
    for (int64_t c = 0; c < P.n_win; ++c) {
        const int b = static_cast<int>(c % P.nbuf), pb = static_cast<int>((c + P.nbuf - 1) % P.nbuf);
        const int64_t t0 = P.start[c], Wc = window_frames(P, T, tau_max, c);
        if (c >= P.nbuf && (e = cudaStreamWaitEvent(R.side, R.freed[b], 0)) != cudaSuccess)
            return cuda_fail(e, "buffer reuse wait");
        int64_t have = 0;
        if (c > 0) {        // halo: frames [t0, t0 + h) follow the previous window's origin frames
            have = tau_max < Wc ? tau_max : Wc;
            const int64_t prev_len = t0 - P.start[c - 1];
            if (have > 0 &&
                (e = cudaMemcpyAsync(buf[b], buf[pb] + static_cast<size_t>(prev_len) * P.K, have * row,
                                     cudaMemcpyDeviceToDevice, R.side)) != cudaSuccess)
                return cuda_fail(e, "halo copy");
        }
        if (Wc > have &&
            (e = copy_frames(H, P.K, t0 + have, Wc - have, buf[b] + static_cast<size_t>(have) * P.K, row, R.side)) !=
                cudaSuccess)
            return cuda_fail(e, "window copy");
        if ((e = cudaEventRecord(R.copied[b], R.side)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, R.copied[b], 0)) != cudaSuccess)
            return cuda_fail(e, "window copy event");
        const int64_t tm = tau_max < Wc - 1 ? tau_max : Wc - 1;
        const Window w = window_of(P, c, s);
        const int rc = P.method == TCORR_PLAIN
                           ? plain_run(kind, buf[b], Wc, N, tm, s, d_out, ws + P.off_engine, P.engine_bytes, st, &w)
                           : gram_run(kind, buf[b], Wc, N, tm, s, P.method, d_out, ws + P.off_engine,
                                      P.engine_bytes, st, &w);
        if (rc != TCORR_OK) return rc;
        if ((e = cudaEventRecord(R.freed[b], st)) != cudaSuccess) return cuda_fail(e, "window done event");
    }
    if ((e = launch_normalize(d_out, T, N, tau_max, s, kind, st)) != cudaSuccess)
        return cuda_fail(e, "normalize launch");
    return TCORR_OK;
}

}  // namespace
}  // namespace tcorr

using namespace tcorr;

extern "C" size_t tcorr_stream_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                                              int method, int64_t chunk_frames) {
    if (!corr_sizes_valid(T, N, tau_max, stride) || method < TCORR_PLAIN || method > TCORR_AUTO) return 0;
    StreamPlan P;
    if (!make_stream_plan(T, N, tau_max, stride, method, chunk_frames, &P)) return 0;
    return P.total;
}

namespace {

int run_stream_one(int kind, const float *h_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride, int method,
                   int64_t chunk_frames, double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    if (!h_x) return TCORR_EINVAL;
    const float *ptrs[1] = {h_x};
    const int64_t first[2] = {0, T};
    return run_stream(kind, HostFrames{ptrs, first, 1}, T, N, tau_max, stride, method, chunk_frames, d_out, d_ws,
                      ws_bytes, stream);
}

int run_stream_chunks(int kind, const float *const *h_chunks, const int64_t *chunk_frames, int n_chunks,
                      int64_t N, int64_t tau_max, int64_t stride, int method, int64_t window_frames,
                      double *d_out, void *d_ws, size_t ws_bytes, void *stream) {
    if (!h_chunks || !chunk_frames || n_chunks < 1 || n_chunks > (1 << 24)) return TCORR_EINVAL;
    std::vector<int64_t> first(static_cast<size_t>(n_chunks) + 1, 0);
    for (int i = 0; i < n_chunks; ++i) {
        if (chunk_frames[i] < 1 || chunk_frames[i] > (int64_t(1) << 40)) return TCORR_EINVAL;
        first[i + 1] = first[i] + chunk_frames[i];
        if (first[i + 1] > (int64_t(1) << 40)) return TCORR_EINVAL;
    }
    return run_stream(kind, HostFrames{h_chunks, first.data(), n_chunks}, first[n_chunks], N, tau_max, stride,
                      method, window_frames, d_out, d_ws, ws_bytes, stream);
}

}  // namespace

extern "C" int tcorr_msd_stream(const float *h_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                                int method, int64_t chunk_frames, double *d_out, void *d_ws, size_t ws_bytes,
                                void *stream) {
    return run_stream_one(0, h_x, T, N, tau_max, stride, method, chunk_frames, d_out, d_ws, ws_bytes, stream);
}

extern "C" int tcorr_acf_stream(const float *h_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                                int method, int64_t chunk_frames, double *d_out, void *d_ws, size_t ws_bytes,
                                void *stream) {
    return run_stream_one(1, h_x, T, N, tau_max, stride, method, chunk_frames, d_out, d_ws, ws_bytes, stream);
}

extern "C" int tcorr_msd_stream_chunks(const float *const *h_chunks, const int64_t *chunk_frames, int n_chunks,
                                       int64_t N, int64_t tau_max, int64_t stride, int method,
                                       int64_t window_frames, double *d_out, void *d_ws, size_t ws_bytes,
                                       void *stream) {
    return run_stream_chunks(0, h_chunks, chunk_frames, n_chunks, N, tau_max, stride, method, window_frames, d_out,
                             d_ws, ws_bytes, stream);
}

extern "C" int tcorr_acf_stream_chunks(const float *const *h_chunks, const int64_t *chunk_frames, int n_chunks,
                                       int64_t N, int64_t tau_max, int64_t stride, int method,
                                       int64_t window_frames, double *d_out, void *d_ws, size_t ws_bytes,
                                       void *stream) {
    return run_stream_chunks(1, h_chunks, chunk_frames, n_chunks, N, tau_max, stride, method, window_frames, d_out,
                             d_ws, ws_bytes, stream);
}
