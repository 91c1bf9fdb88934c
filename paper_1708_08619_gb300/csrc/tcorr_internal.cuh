// Internal declarations shared by the translation units of libtcorr.so.
//
// Band tiling of the origin x frame plane (all methods)
// ----------------------------------------------------
// Origins are t0 = o*s (o = 0 .. n_orig-1).  A lag tau is split as
// tau = rho + m*s with residue rho = tau mod s, so the frame t0 + tau equals
// rho + (o+m)*s: for each residue rho the work is a stride-1 banded
// cross-correlation between the origin rows X[o*s] and the frame rows
// X[rho + k*s] (k = 0 .. n_rho-1), restricted to 0 <= k - o <= m_max(rho)
// with m_max(rho) = floor((tau_max - rho)/s).  For s = 1 there is one residue
// and this is the plain band |t - t'| <= tau_max of the Gram matrix X X^T.
//
// A tile (rho, r, c) covers origins o in [r*BO, r*BO+BO) and frame indices
// k in [r*BO + c*BF, r*BO + c*BF + BF).  Its entries fall on band offsets
// m = k - o in [c*BF - BO + 1, c*BF + BF - 1]; the tile stores its per-offset
// sums in a window of width BO+BF-1 indexed by w = m - c*BF + BO - 1.
// Work items are (K-group g, rho, r, c), c fastest, so that neighbouring
// blocks share origin rows and overlapping frame rows in L2.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tcorr.h"

namespace tcorr {

struct BandPlan {
    int64_t T, N, K;          // frames, atoms, K = 3N
    int64_t tau_max, s;       // max lag, origin stride
    int64_t n_orig;           // origins: floor((T-1)/s) + 1
    int64_t n_res;            // residues that carry lags: min(s, tau_max+1)
    int64_t m_max0;           // m_max(0) = floor(tau_max / s)
    int BO, BF;               // tile extent over origins / frame indices
    int WP;                   // padded window width (>= BO+BF-1)
    int64_t n_rows, n_cols;   // row tiles, column tiles per row tile
    int64_t kseg;             // K elements per FP32 accumulation segment
    int64_t segs_per_item;    // segments one work item walks
    int64_t n_groups;         // K groups: ceil(ceil(K/kseg)/segs_per_item)
    int64_t n_items;          // n_groups * n_res * n_rows * n_cols
    int pair = 0;             // CTA-pair tiling: odd row tiles r hold lags m = c BF - BO + j - i
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// n_o(tau) = floor((T-1-tau)/s) + 1 origins for lag tau.
__host__ __device__ inline int64_t n_origins(int64_t T, int64_t s, int64_t tau) {
    return (T - 1 - tau) / s + 1;
}

// Frame indices available for residue rho: frames rho, rho+s, ... <= T-1.
__host__ __device__ inline int64_t n_frames_res(int64_t T, int64_t s, int64_t rho) {
    return rho > T - 1 ? 0 : (T - 1 - rho) / s + 1;
}

// Build the plan.  `min_items` steers how many K segments one item walks so
// that the grid has enough blocks to fill the GPU.
BandPlan make_band_plan(int64_t T, int64_t N, int64_t tau_max, int64_t s, int BO, int BF,
                        int64_t kseg, int64_t min_items);

// One time window of a longer trajectory (the streamed path): only the
// window's first orig_cap origins (0: all) start pairs, and the lag
// reduction adds the per-lag numerators, sum over origins of |x(t+tau) -
// x(t)|^2 (MSD) or x(t).x(t+tau) (ACF), into the output instead of writing
// averages.  Summed over windows that tile the origins, these are the
// numerators of Eq. 5 and of the ACF (Eq. 4) over the whole trajectory.
struct Window {
    int64_t orig_cap;
    bool accumulate;
};
// Restricts a plan to its first `cap` origins (row tiles and items shrink).
void cap_origins(BandPlan *p, int64_t cap);

// Whole-path runs, kind 0 MSD, 1 ACF, 2 cross-correlation of d_x (at the
// origin) with d_y (at the later frame).  Tensor-core path (gram_tc.cu):
size_t gram_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t s, int method,
                           const Window *w = nullptr, int kind = 0);
int gram_run(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s, int method,
             double *d_out, void *d_ws, size_t ws_bytes, cudaStream_t st, const Window *w = nullptr,
             const float *d_y = nullptr);
bool gram_method_available(int method);
// Plain FP32 path (api.cu):
int plain_run(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s, double *d_out,
              void *d_ws, size_t ws_bytes, cudaStream_t st, const Window *w = nullptr,
              const float *d_y = nullptr);
size_t plain_window_workspace(int64_t T, int64_t N, int64_t tau_max, int64_t s, int64_t orig_cap);
bool corr_sizes_valid(int64_t T, int64_t N, int64_t tau_max, int64_t s);
// FFT route (fft.cu): the library's own double-float transforms; sizes are host arithmetic.
size_t fft_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t s, int kind);
// Whether the FFT route handles this padded length (T + tau_max up to about 8.4 million).
bool fft_supported(int64_t T, int64_t tau_max);
int fft_run(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s, double *d_out,
            void *d_ws, size_t ws_bytes, cudaStream_t st, const float *d_y = nullptr);
// prefix[rho][j] = sum_{j' < j} S(rho + j' s) for the residues rho < n_res (gram_tc.cu).
cudaError_t launch_s_prefix(const double *S, int64_t T, int64_t s, int64_t n_res, int64_t pstride,
                            double *prefix, cudaStream_t st);

// Maps a failed CUDA call to TCORR_ECUDA; with TCORR_VERBOSE set in the
// environment it also prints the call site and CUDA's error string.
inline int cuda_fail(cudaError_t e, const char *what) {
    if (std::getenv("TCORR_VERBOSE")) std::fprintf(stderr, "tcorr: %s: %s\n", what, cudaGetErrorString(e));
    return TCORR_ECUDA;
}

// Autotuner (tune.cu): per shape bucket, the tensor-core work-item length
// (kseg, K elements), the accumulation sub-chain length (sub_kb, K-blocks;
// 0 = the default for the kind and form) and the supertile of the band items'
// claim order (super_rows x super_cols tiles; 0 = the default).
struct TuneChoice {
    int64_t kseg;
    int sub_kb;
    int super_rows = 0;
    int super_cols = 0;
    int pair = -1;      // tile shape: 0 one CTA (M = 128), 1 a CTA pair (M = 256), -1 not chosen
};
// The default supertile (claim order) of the band kernel: 16 x 10 tiles.
constexpr int kDefaultSuperRows = 16;
constexpr int kDefaultSuperCols = 10;
int tune_mode();   // 0 off, 1 tune once per bucket, 2 re-tune every call
std::string tune_key(int method, int kind, int64_t K, int64_t tau_max, int64_t T, int64_t s);
bool tune_lookup(const std::string &key, TuneChoice *c);
void tune_store(const std::string &key, const TuneChoice &c);
const std::vector<TuneChoice> &tune_candidates();
int64_t tune_min_kseg();
void set_tune_override(const TuneChoice *c);
const TuneChoice *get_tune_override();
int64_t tune_default_kseg(int64_t K, int64_t tiles, int64_t n_cols);

// Diagnostics (profile.cu): events around one launch of the dominant kernel.
// kind: 0 MSD, 1 ACF, 2 a batched launch mixing both.
void prof_begin(int kind, cudaStream_t st);
void prof_end(cudaStream_t st);

// Test-only fault injection on the host.  With TCORR_FAULT_INJECT=host_alloc
// in the environment, the first host allocation of a batch plan (the per-
// instance layout, made before anything is enqueued) throws std::bad_alloc as
// if the host were out of memory; tcorr_batch returns it as TCORR_ENOMEM and
// tcorr_batch_workspace_size as 0.  Unset, this is one getenv per plan.
inline void host_alloc_fault_point() {
    const char *f = std::getenv("TCORR_FAULT_INJECT");
    if (f && std::string(f) == "host_alloc") throw std::bad_alloc();
}

// Debug builds (TCORR_DEBUG_BOUNDS, libtcorr_debug.so): kernels check the
// global-memory indices of the plain path (trajectory loads, partial-sum
// stores), of the lag reduction (partial-sum loads) and of the band kernel's
// window stores against the extents of their buffers before the access.  An
// index outside records TCORR_EBOUNDS in the device status word (read and
// cleared by tcorr_status_poll) and the access is skipped (a load reads 0), so
// a bad index shows as an error code instead of a fault.  In release builds
// the checks compile to nothing.  For a test of the mechanism,
// TCORR_DEBUG_SHRINK=1 in the environment makes the host declare every
// partial-sum buffer one window shorter than it is (the real buffer is intact,
// so the skipped accesses stay harmless) and the checks must fire.
unsigned int *status_word_device_ptr();     // the status word's device address (gram_tc.cu)
#ifdef TCORR_DEBUG_BOUNDS
__device__ __forceinline__ bool dbg_in_bounds(int64_t i, int64_t n, unsigned int *status) {
    if (i >= 0 && i < n) return true;
    atomicExch(status, static_cast<unsigned int>(TCORR_EBOUNDS));
    return false;
}
#define TCORR_IN_BOUNDS(i, n, status) ::tcorr::dbg_in_bounds((i), (n), (status))
inline int64_t dbg_shrink_elems(int64_t elems, int64_t window) {
    const char *v = std::getenv("TCORR_DEBUG_SHRINK");
    return (v && v[0] == '1' && elems >= window) ? elems - window : elems;
}
#else
#define TCORR_IN_BOUNDS(i, n, status) true
inline int64_t dbg_shrink_elems(int64_t elems, int64_t) { return elems; }
#endif

// Workspace layout helpers (byte offsets, 256-byte aligned).
inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Weighted averages (weighted.cu): the scaled copy y = sqrt(w) (x - x_ref) and
// W = sum w at the start of the workspace, then the result scaled by N / W.
size_t weighted_copy_bytes(int64_t T, int64_t N);
cudaError_t launch_weight_copy(int kind, const float *x, const float *w, int64_t T, int64_t N, void *d_copy,
                               cudaStream_t st);
cudaError_t launch_weight_rescale(double *out, int64_t n, int64_t T, int64_t N, const void *d_copy,
                                  cudaStream_t st);

// ------------------------------------------------------------------ kernels
// Plain FP32 path: per-item per-offset partial sums (double) into `partial`
// ([n_items][WP]).  kind 0 = MSD (differences), 1 = ACF (products), 2 =
// cross-correlation (products of d_x at the origin and d_xb at the later frame).
cudaError_t launch_plain_tiles(int kind, const float *d_x, const BandPlan &p, double *partial,
                               cudaStream_t st, const float *d_xb = nullptr);
// Batch of plain instances: d_descs holds one PlainArgs (plain.cu) per
// instance, plain_args_size() bytes each, written by plain_args_write.
size_t plain_args_size();
void plain_args_write(void *h_dst, int kind, const float *d_x, const BandPlan &p, double *partial,
                      int64_t item_begin);
cudaError_t launch_plain_tiles_batch(const void *d_descs, int n, int64_t total_items, cudaStream_t st);

// Fixed-order FP64 reduction of the per-item partials to per-lag sums D(tau),
// then the normalisation.  mode 0: out = D / (N n_o) (plain MSD and ACF);
// mode 1: out = (P + Q - 2 D) / (N n_o) using prefix sums of S (Gram MSD).
struct FinalizeArgs {
    int mode;
    const double *S_prefix;   // mode 1: [residue][prefix_stride] prefix sums of S
    int64_t prefix_stride;    // mode 1: entries per residue row of S_prefix
};
cudaError_t launch_lag_reduce(const BandPlan &p, const double *partial, const FinalizeArgs &fa,
                              double *d_out, cudaStream_t st, const Window *w = nullptr);
// out[tau] /= N n_o(tau) over the whole trajectory (MSD: out[0] = 0): turns
// the numerators accumulated over windows into averages.
cudaError_t launch_normalize(double *d_out, int64_t T, int64_t N, int64_t tau_max, int64_t s, int kind,
                             cudaStream_t st);

// One instance of the lag reduction (also one entry of a batch).
struct LagReduceDesc {
    const double *partial;
    int64_t partial_elems;    // doubles in partial (debug builds check the loads against it)
    unsigned int *dbg_status; // the status word (debug builds)
    int64_t T, N, s, tau_max;
    int64_t n_res, n_rows, n_cols, n_groups;
    int BO, BF, WP, mode;
    const double *S_prefix;
    int64_t prefix_stride;
    double *out;
    int64_t lag_begin;        // batch: first global lag of this instance
    int64_t n_orig;           // origins that start pairs (n_o(tau) is capped by it)
    int accumulate;           // 1: out[tau] += numerator (streamed windows)
    int pair;                 // CTA-pair tiling (see BandPlan::pair)
};
LagReduceDesc lag_reduce_desc(const BandPlan &p, const double *partial, const FinalizeArgs &fa,
                              double *d_out, int64_t lag_begin);
// Batch: one warp per (instance, lag); d_descs in device memory.
cudaError_t launch_lag_reduce_batch(const LagReduceDesc *d_descs, int n, int64_t total_lags,
                                    cudaStream_t st);

// Copies host bytes to device memory without a host-to-device memcpy: the
// bytes travel as kernel parameters (at most 28 KB per launch), so the copy
// needs no pinned buffer, allocates nothing and can be captured in a graph.
cudaError_t upload_bytes(void *d_dst, const void *h_src, size_t nbytes, cudaStream_t st);

cudaError_t launch_gk_integrate(const double *d_c, int64_t n, double dt, double prefactor,
                                double *d_running, cudaStream_t st);
// count series at once: series j reads d_c + j ldc, writes d_running + j ldr.
cudaError_t launch_gk_integrate_batch(const double *d_c, int64_t n, int64_t count, int64_t ldc, double dt,
                                      double prefactor, double *d_running, int64_t ldr, cudaStream_t st);
cudaError_t launch_einstein(const double *d_msd, int64_t n, double dt, int dim, int64_t lo,
                            int64_t hi, double *d_D, cudaStream_t st);

}  // namespace tcorr
