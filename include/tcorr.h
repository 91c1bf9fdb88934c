/*
 * tcorr.h -- C ABI of libtcorr.so: multiple-time-origin time correlation of
 * molecular-dynamics trajectories on one GB300 (sm_103a).
 *
 * The operations are those of arXiv 1708.08619, Sec. 3.5 ("Correlation
 * functions"):
 *   - the mean square displacement of Eq. 5, computed by the loop nest of
 *     Algorithms 10/11 (atoms, time intervals, time origins), averaged over
 *     atoms and over time origins;
 *   - the time autocorrelation <A(t0).A(t0+tau)> that Eq. 4 integrates,
 *     computed by the loop nest of Algorithms 8/9;
 *   - the running Green-Kubo integral of Eq. 4 (the quadrature loop that
 *     closes Algorithms 8 and 9);
 *   - the Einstein diffusion constant of Eq. 5.
 *
 * Common conventions
 * ------------------
 * Trajectory layout: x[T][N][3] float32, frame-major, contiguous (the linear
 * array of Sec. 2.3), i.e. a T x K row-major matrix with K = 3N.  For the MSD
 * it holds unwrapped positions (Algorithm 10 starts "from unwrapped
 * trajectory"); for the autocorrelation it holds the signal A (velocities,
 * or a per-frame flux such as (Pxy, Pxz, Pyz) with N = 1).
 *
 * Origins and lags: origins are t0 = 0, s, 2s, ... (stride s >= 1; s = 1 uses
 * every frame as the paper does); lags are tau = 0 .. tau_max with
 * 0 <= tau_max <= T-1.  For lag tau the origins used are those with
 * t0 + tau <= T-1; there are n_o(tau) = floor((T-1-tau)/s) + 1 of them.
 *
 * Normalisation: every per-lag output is divided by N * n_o(tau) (the average
 * over atoms and origins).  The paper leaves the normalisation unstated; this
 * is the textbook estimator it cites for Eq. 5.
 *
 * Memory: every pointer argument prefixed d_ is a device pointer on the
 * current CUDA device; h_ is a host pointer.  The caller owns every buffer.
 * The library allocates no device memory: scratch space is the caller's
 * workspace d_ws of at least tcorr_workspace_size(...) bytes, 256-byte
 * aligned.  Its contents on entry do not matter and are undefined on exit.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls enqueue work and return without synchronising, so a
 * returned TCORR_OK means "validated and enqueued".  Buffers must stay valid
 * until the stream reaches the work.  Two calls that share a workspace must be
 * ordered on the GPU (same stream, or events).
 *
 * Errors: argument errors are detected on the host before anything is
 * enqueued and returned as a tcorr_status; nothing is written in that case.
 * A CUDA launch failure returns TCORR_ECUDA.  Errors found by a kernel on the
 * device (a bounded wait that gave up) are recorded in a per-device status
 * word that tcorr_status_poll() reads and clears; no kernel traps.
 *
 * Determinism: for fixed arguments and method, results are bit-identical
 * from run to run (all cross-tile sums are fixed-order FP64 reductions).
 */
#ifndef TCORR_H
#define TCORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TCORR_OK = 0,
    TCORR_EINVAL = 1,        /* bad size, null pointer or unknown method        */
    TCORR_EALIGN = 2,        /* pointer not aligned as documented               */
    TCORR_ENOMEM = 3,        /* a host allocation failed                        */
    TCORR_EWORKSPACE = 4,    /* ws_bytes smaller than tcorr_workspace_size()    */
    TCORR_ECUDA = 5,         /* a CUDA runtime/driver call or launch failed     */
    TCORR_ETIMEOUT = 6,      /* a device-side bounded wait gave up (status word)*/
    TCORR_EUNSUPPORTED = 7,  /* method cannot run this shape or on this device  */
    TCORR_EBOUNDS = 8        /* debug build only: a kernel's index check found an
                                index outside its buffer and skipped the access
                                (status word)                                   */
} tcorr_status;

typedef enum {
    /* FP32 SIMT kernel: per-origin differences (MSD) or products (ACF),
       accumulated in FP32 over bounded segments of K, FP64 across segments
       and tiles.  Accuracy target: 1e-6 relative per lag. */
    TCORR_PLAIN = 0,
    /* tcgen05 tensor-core banded Gram X X^T over K = 3N with split operands:
       x = hi + lo, products hi.hi + hi.lo + lo.hi (x3) or also lo.lo (x4),
       FP32 accumulation in TMEM, FP64 per-lag sums.  The MSD is assembled as
       S(t0) + S(t0+tau) - 2 G(t0, t0+tau) with S(t) = |x_t|^2 in FP64, after
       referencing positions to the middle frame.  Accuracy target: 1e-5 relative to
       C(0) or MSD(tau_max). */
    TCORR_TC_TF32X3 = 1,
    TCORR_TC_BF16X3 = 2,
    TCORR_TC_BF16X4 = 3,
    TCORR_TC_FP16X3 = 4,     /* FP16 hi/lo with a power-of-two scale */
    TCORR_AUTO = 5,          /* the library picks (tensor-core when it can) */
    /* FFT route (not in the paper): per column, the lag sums up to tau_max are
       the inverse transform of the (cross) power spectrum of the column
       zero-padded to L >= T + tau_max (L = 2^a, 3 2^a or 5 2^a), two real
       columns per complex transform, computed by the library's own
       transforms in double-float arithmetic (about 48 significant bits),
       FP64 sums over columns; stride s uses the origin-masked signal on one
       side.  Cost O(K T log T) instead of O(K T tau_max): the choice when
       tau_max is a large fraction of T.  Padded lengths up to 2^23
       (T + tau_max up to 8,388,608); longer series return
       TCORR_EUNSUPPORTED (TCORR_AUTO then takes the tensor-core route).
       Accuracy target: 1e-5 relative to C(0) or MSD(tau_max).  Not
       available in tcorr_batch or the streamed calls. */
    TCORR_FFT = 6
} tcorr_method;

/*
 * Bytes of device workspace that tcorr_msd / tcorr_acf need for these
 * arguments and this method.  Returns 0 when the arguments are invalid or
 * the method cannot run this shape (the call itself then reports the error).
 * Host arithmetic only.
 */
size_t tcorr_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                            int method);

/*
 * Mean square displacement (Eq. 5; Algorithms 10 and 11):
 *   d_out[tau] = 1/(N n_o(tau)) sum_i sum_{t0} |x[t0+tau][i] - x[t0][i]|^2,
 *   tau = 0 .. tau_max.
 * d_x   : [T][N][3] float32 unwrapped positions, 4-byte aligned.
 * d_out : tau_max+1 doubles, 8-byte aligned.
 * d_ws  : workspace of ws_bytes >= tcorr_workspace_size(...) bytes,
 *         256-byte aligned (may be NULL when that size is 0).
 * Errors: TCORR_EINVAL (null pointer, T < 1, N < 1, tau_max outside
 * [0, T-1], stride < 1, unknown method), TCORR_EALIGN, TCORR_EWORKSPACE,
 * TCORR_EUNSUPPORTED, TCORR_ECUDA.
 */
int tcorr_msd(const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
              int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream);

/*
 * Time autocorrelation, the integrand of Eq. 4 (Algorithms 8 and 9):
 *   d_out[tau] = 1/(N n_o(tau)) sum_i sum_{t0} A[t0][i] . A[t0+tau][i].
 * Arguments, alignment and errors as tcorr_msd; d_x holds A.
 */
int tcorr_acf(const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
              int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream);

/*
 * Time cross-correlation of two signals of the same shape:
 *   d_out[tau] = 1/(N n_o(tau)) sum_i sum_{t0} A[t0][i] . B[t0+tau][i],
 *   tau = 0 .. tau_max (the product of Algorithm 8 with the later factor taken
 *   from B; for negative lags swap the arguments).  With A = B it is
 *   tcorr_acf.  Per-atom pairs give cross terms such as velocity-force or
 *   position-velocity correlations; with N = 1 and A, B summed over the atoms
 *   of two species (or weighted by charge) it gives the collective
 *   cross-correlations of Green-Kubo transport (interdiffusion, charge
 *   current).  The paper computes autocorrelations only; this is the same loop
 *   nest with two signals.  Small K (3N <= 24, stride 1, tau_max >= 383) uses
 *   the polyphase form as tcorr_acf does, with the unshifted operand copy of A
 *   on the origin side and the shifted copies of B on the other.
 * d_a, d_b: [T][N][3] float32, 4-byte aligned; d_out: tau_max+1 doubles,
 * 8-byte aligned; d_ws: tcorr_xcf_workspace_size(...) bytes (the tensor-core
 * methods keep split copies of both signals), 256-byte aligned.
 * Errors: as tcorr_msd.
 */
size_t tcorr_xcf_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t stride, int method);
int tcorr_xcf(const float *d_a, const float *d_b, int64_t T, int64_t N, int64_t tau_max,
              int64_t stride, int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream);

/*
 * Running Green-Kubo integral of Eq. 4, trapezoid rule on the frame grid
 * (the quadrature loop closing Algorithms 8/9, done on the GPU here):
 *   d_running[0] = 0,
 *   d_running[k] = prefactor * sum_{j=1..k} dt (c[j-1] + c[j]) / 2.
 * prefactor carries V/(k_B T) (and 1/3 to average three components).
 * d_c, d_running: n doubles (n >= 1), 8-byte aligned; they may not overlap.
 * The prefix sum is evaluated in a fixed order (deterministic).
 * Errors: TCORR_EINVAL, TCORR_EALIGN, TCORR_ECUDA.
 */
int gk_integrate(const double *d_c, int64_t n, double dt, double prefactor,
                 double *d_running, void *stream);

/*
 * gk_integrate for count correlation functions of n values each in one
 * launch: series j is read from d_c + j ldc and its running integral written
 * to d_running + j ldr (offsets in doubles; ldc, ldr >= n).  Each series gets
 * exactly the values a gk_integrate call on it would give.  The spans
 * [d_c, d_c + (count-1) ldc + n) and [d_running, d_running + (count-1) ldr + n)
 * may not overlap; both pointers 8-byte aligned.  count == 0 does nothing.
 * Errors: TCORR_EINVAL (n < 1, count < 0, ldc or ldr < n, null pointer,
 * overlapping spans), TCORR_EALIGN, TCORR_ECUDA.
 */
int gk_integrate_batch(const double *d_c, int64_t n, int64_t count, int64_t ldc, double dt,
                       double prefactor, double *d_running, int64_t ldr, void *stream);

/*
 * Weighted atom averages: tcorr_msd / tcorr_acf with atom i counted w_i
 * times in Eq. 5's average "over all the atoms (or a subclass)":
 *   MSD_w(tau) = sum_i w_i sum_{t0 in O(tau)} |x_i(t0+tau) - x_i(t0)|^2 / (W n_o(tau)),
 *   W = sum_i w_i (likewise the autocorrelation) -- a mass-weighted MSD, or a
 *   selection with 0/1 weights.
 * d_w: N float32 weights on the device, 4-byte aligned, each >= 0 (a negative
 * weight makes the result NaN), W > 0.  Method: the call writes
 * y_i = sqrt(w_i) x_i into its workspace (for the MSD relative to the middle
 * frame, which the MSD does not see), runs the unweighted engine of `method`
 * on y and scales by N / W; each y value is one FP32 rounding of the exact
 * product, so the accuracy is that of the method, plus rounding errors of the
 * products that average out over atoms and origins.  d_ws:
 * tcorr_weighted_workspace_size(...) bytes, 256-byte aligned (the copy of
 * the trajectory, W, then the method's own workspace).  Other arguments and
 * errors as tcorr_msd, plus TCORR_EINVAL for d_w == NULL.
 */
size_t tcorr_weighted_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t stride, int method);
int tcorr_msd_weighted(const float *d_x, const float *d_w, int64_t T, int64_t N, int64_t tau_max,
                       int64_t stride, int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream);
int tcorr_acf_weighted(const float *d_x, const float *d_w, int64_t T, int64_t N, int64_t tau_max,
                       int64_t stride, int method, double *d_out, void *d_ws, size_t ws_bytes, void *stream);

/*
 * Atom-sharded correlation (the Conclusion's division of a species' dynamic
 * data over several devices by atoms; Eq. 5 averages over atoms and n_o(tau)
 * is the same for every atom): each rank runs tcorr_msd / tcorr_acf (or the
 * weighted calls) on its own contiguous atom slice and writes one record of
 * n + 1 doubles, its per-lag averages a_r(0 .. n-1) followed by its weight
 * w_r (the slice's atom count N_r, or its weight sum W_r from
 * tcorr_weight_total for weighted averages).  The records of all ranks are
 * gathered in rank order (all-gather: the one exchange of the path) into
 * count rows of a row-major array with row stride ld >= n + 1 doubles, and
 *   d_out[i] = sum_r w_r d_rows[r ld + i] / sum_r w_r,   i = 0 .. n-1,
 * with both sums in FP64 in row order r = 0, 1, ... (fixed order: every rank
 * combining the same gathered rows gets the same bits).  Weights must be >= 0
 * with a positive total (else the result is Inf or NaN).
 * d_rows: device, 8-byte aligned; d_out: n doubles on the device, 8-byte
 * aligned, not overlapping the rows.  Errors: TCORR_EINVAL (null pointer,
 * n < 1, count < 1, ld < n + 1, overlap), TCORR_EALIGN, TCORR_ECUDA.
 */
int tcorr_combine_shards(const double *d_rows, int64_t n, int64_t count, int64_t ld, double *d_out,
                         void *stream);

/*
 * W = sum_i w_i of N float32 weights in FP64, summed in a fixed order (the
 * weight of one weighted shard, written where tcorr_combine_shards reads a
 * record's weight).  d_w: device, 4-byte aligned; d_W: one double on the
 * device, 8-byte aligned.  Errors: TCORR_EINVAL, TCORR_EALIGN, TCORR_ECUDA.
 */
int tcorr_weight_total(const float *d_w, int64_t N, double *d_W, void *stream);

/*
 * Collective signal of a trajectory, the input of collective transport
 * quantities (Eq. 4 with a collective flux, as the viscosity example
 * correlates the pressure tensor of the whole box):
 *   d_out[t][c] = sum_i w_i (x[t][i][c] - x[ref_frame][i][c])  (0 <= ref_frame < T)
 *   d_out[t][c] = sum_i w_i  x[t][i][c]                        (ref_frame = -1)
 * d_out is a [T][1][3] float32 trajectory of one "atom", ready for
 * tcorr_msd / tcorr_acf / tcorr_xcf with N = 1: with charges q_i as weights,
 * the MSD of the summed charged positions (Einstein-Helfand; take a reference
 * frame, which the MSD does not see, to keep the FP32 values small) or the
 * autocorrelation of the charge current (ref_frame = -1); with 0/1 weights,
 * the signal of an atom selection or species, e.g. for the velocity
 * cross-correlation of two species through tcorr_xcf.
 * d_x: [T][N][3] float32 (device, 4-byte aligned); d_w: N float32 weights
 * (device, 4-byte aligned) or NULL for unit weights; d_out: 3T floats, not
 * overlapping d_x or d_w.  Arithmetic: products and sums carried with their
 * rounding errors in FP32 (compensated dot product), combined per frame in
 * FP64 in a fixed order; with a reference frame its totals, formed the same
 * way, are subtracted in FP64; one rounding to FP32 (deterministic).
 * Errors: TCORR_EINVAL (null pointer, T < 1, N < 1, ref_frame outside
 * [-1, T-1], overlapping output), TCORR_EALIGN, TCORR_ECUDA.
 */
int tcorr_collective(const float *d_x, const float *d_w, int64_t T, int64_t N, int64_t ref_frame,
                     float *d_out, void *stream);

/*
 * Einstein relation (Eq. 5): with t = tau dt, d_D[0] = b / (2 dim) where b is
 * the ordinary least-squares slope of d_msd[tau] against t over
 * tau in [lo, hi]; d_D[1] = d_msd[hi] / (2 dim hi dt) (the literal ratio).
 * Needs 0 <= lo < hi < n, dim >= 1, dt > 0.  d_D: 2 doubles.
 * Errors: TCORR_EINVAL, TCORR_EALIGN, TCORR_ECUDA.
 */
int einstein_slope(const double *d_msd, int64_t n, double dt, int dim, int64_t lo,
                   int64_t hi, double *d_D, void *stream);

/* One entry of a batch: kind 0 = MSD, 1 = autocorrelation. */
typedef struct {
    int kind;
    const float *d_x;        /* [T][N][3] float32 on the device */
    int64_t T, N, tau_max, stride;
    double *d_out;           /* tau_max+1 doubles on the device */
} tcorr_instance;

/*
 * Many independent instances (trajectories, atom selections, signals of
 * uneven T, N, tau_max; Eq. 5 averages "over all the atoms in a given
 * subclass", so a subclass is an instance) in one call.  Each instance's
 * result equals what tcorr_msd / tcorr_acf would return for it.
 * h_items: host array of count entries; each is validated as tcorr_msd does.
 * Workspace: tcorr_batch_workspace_size(...) bytes.
 */
size_t tcorr_batch_workspace_size(const tcorr_instance *h_items, int count, int method);
int tcorr_batch(const tcorr_instance *h_items, int count, int method, void *d_ws,
                size_t ws_bytes, void *stream);

/*
 * Streamed (out-of-core) MSD / autocorrelation of a trajectory held in HOST
 * memory, for trajectories larger than device memory.  The paper's method
 * needs every frame on the device (its Conclusion names this as the limit for
 * dynamic quantities and leaves splitting a trajectory to the user); this
 * entry point removes that limit.  Result: Eq. 5 (tcorr_msd_stream) or the
 * autocorrelation of Eq. 4 (tcorr_acf_stream), exactly as tcorr_msd /
 * tcorr_acf define it over the whole trajectory, up to rounding order.
 * Method: the origins are cut into windows of chunk_frames frames (rounded up
 * to a multiple of stride; 0 picks max(4 (tau_max + 1), 4096) rounded up to
 * 128 stride).  Window c holds frames [c C, c C + C + tau_max); its first C
 * frames are the origins it owns, the rest is the tau_max halo of partner
 * frames.  Each window runs the tensor-core band kernel (or the plain
 * kernel) restricted to its own origins and adds the per-lag numerators into
 * d_out; one last kernel divides by N n_o(tau) of the whole trajectory.  Three
 * window buffers rotate: the halo is copied from the previous window on
 * the device and only the C new frames come from the host, on a second
 * stream that overlaps the earlier windows' kernels.  Polyphase (small K)
 * is not used in this mode; the band form handles every K.
 * h_x   : [T][N][3] float32 in host memory, 4-byte aligned.  Pinned memory
 *         (cudaHostAlloc / cudaHostRegister) lets the copies overlap the
 *         kernels; pageable memory works but each copy then blocks the host.
 *         h_x must stay valid and unchanged until `stream` has finished.
 * d_out : tau_max+1 doubles on the device, 8-byte aligned (overwritten).
 * d_ws  : device workspace of ws_bytes >= tcorr_stream_workspace_size(...),
 *         256-byte aligned: min(3, windows) window buffers of min(T, C + tau_max) frames
 *         plus the engine's workspace for one window.
 * The call enqueues work on `stream` and on a stream of its own, joined back
 * to `stream` through events; it cannot be captured in a CUDA graph.
 * Errors: as tcorr_msd, plus TCORR_EINVAL for chunk_frames < 0.
 */
size_t tcorr_stream_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                                   int method, int64_t chunk_frames);
int tcorr_msd_stream(const float *h_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                     int method, int64_t chunk_frames, double *d_out, void *d_ws,
                     size_t ws_bytes, void *stream);
int tcorr_acf_stream(const float *h_x, int64_t T, int64_t N, int64_t tau_max, int64_t stride,
                     int method, int64_t chunk_frames, double *d_out, void *d_ws,
                     size_t ws_bytes, void *stream);

/*
 * The same streamed MSD / autocorrelation (Eq. 5 / Eq. 4, as tcorr_msd_stream
 * and tcorr_acf_stream) for a trajectory held in host memory as consecutive
 * chunks of frames: chunk i holds chunk_frames[i] frames as [frames][N][3]
 * float32, and the trajectory is their concatenation (T = the sum).  The
 * windows, copies and kernels are those of the one-array call, so the result
 * is the same bit for bit; a window's new frames are copied from each chunk
 * they touch.  Pinning the trajectory as separately allocated chunks of about
 * 1 GiB keeps the host-to-device copies at the link's rate where one pinned
 * allocation of many GB was measured several times slower after load on the
 * host cores.
 * h_chunks     : n_chunks host pointers, each 4-byte aligned and non-null; the
 *                chunks must stay valid and unchanged until `stream` has finished.
 * chunk_frames : n_chunks frame counts, each >= 1 (host array).
 * n_chunks     : 1 .. 2^24.
 * window_frames: as chunk_frames of tcorr_msd_stream (origins per window; 0 =
 *                the default); the workspace is tcorr_stream_workspace_size(T,
 *                N, tau_max, stride, method, window_frames) with T the total.
 * Errors: as tcorr_msd_stream, plus TCORR_EINVAL for a null array, a null
 * chunk pointer, n_chunks out of range or a chunk of fewer than one frame, and
 * TCORR_EALIGN for a chunk pointer that is not 4-byte aligned.
 */
int tcorr_msd_stream_chunks(const float *const *h_chunks, const int64_t *chunk_frames, int n_chunks,
                            int64_t N, int64_t tau_max, int64_t stride, int method,
                            int64_t window_frames, double *d_out, void *d_ws, size_t ws_bytes,
                            void *stream);
int tcorr_acf_stream_chunks(const float *const *h_chunks, const int64_t *chunk_frames, int n_chunks,
                            int64_t N, int64_t tau_max, int64_t stride, int method,
                            int64_t window_frames, double *d_out, void *d_ws, size_t ws_bytes,
                            void *stream);

/*
 * Plain FP32 path without a caller workspace: the same result, bit for bit,
 * as tcorr_msd (kind 0) or tcorr_acf (kind 1) with method TCORR_PLAIN, but
 * the library allocates nothing and the caller passes no workspace.  The
 * paper has no counterpart; this entry point is for callers that cannot
 * allocate device memory, e.g. an analysis hook inside a simulation engine
 * whose device memory all belongs to the engine's own pool, or a host that
 * must not call cudaMalloc because it synchronises the device.
 * Scratch: one fixed 32 MiB array of device memory, held by every GPU that
 * loads this part of the library until the process exits.  Its device
 * address is looked up on the first call on each device (with that device
 * current), so make that first call before any stream capture.  All calls on
 * a device share the array: calls whose work overlaps on the GPU race.
 * Limit: the per-item partial sums must fit the array
 * (8 * 256 * n_items bytes, about 16k band tiles); larger shapes return
 * TCORR_EWORKSPACE without launching anything.
 * d_x: [T][N][3] float32, 4-byte aligned; d_out: tau_max+1 doubles, 8-byte
 * aligned.  Errors: TCORR_EINVAL, TCORR_EALIGN, TCORR_EWORKSPACE, TCORR_ECUDA.
 */
int tcorr_plain_static(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max,
                       int64_t stride, double *d_out, void *stream);

/*
 * Synchronises `stream`, then returns and clears the current device's status
 * word: TCORR_OK, or TCORR_ETIMEOUT if a kernel's bounded wait gave up since
 * the last poll, TCORR_EBOUNDS if an index check of a debug build
 * (libtcorr_debug.so, compiled with TCORR_DEBUG_BOUNDS) failed, or
 * TCORR_ECUDA if the synchronisation failed.
 */
int tcorr_status_poll(void *stream);

/*
 * Diagnostics, with no counterpart in the paper: when enabled, the library
 * records a pair of CUDA events on the launching stream around every launch
 * of its dominant kernel (the tensor-core band / polyphase kernel or the
 * plain tile kernel; not while the stream is being captured), so that a
 * caller can time that kernel alone.  tcorr_profile_read waits for the
 * recorded launches of one kind (0 = MSD, 1 = autocorrelation, 2 = batched
 * launches mixing both), returns their summed duration in milliseconds and
 * their count, and forgets them.  Errors: TCORR_EINVAL, TCORR_ECUDA.
 */
int tcorr_profile_enable(int on);
int tcorr_profile_read(int kind, double *total_ms, int *launches);

/*
 * Self-test of the device-side error path, with no counterpart in the paper:
 * enqueues one tiny kernel that waits on a barrier nothing completes; after
 * 10 ms the bounded wait gives up, the kernel records TCORR_ETIMEOUT in the
 * status word and returns (no trap, the context stays usable).  The next
 * tcorr_status_poll returns TCORR_ETIMEOUT.  Errors: TCORR_ECUDA.
 */
int tcorr_selftest_timeout(void *stream);

/* Human-readable name of a tcorr_status value (static string). */
const char *tcorr_strerror(int code);

/* Library version, major * 10000 + minor * 100 + patch. */
int tcorr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TCORR_H */
