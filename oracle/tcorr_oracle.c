/*
 * tcorr_oracle.c -- plain FP64 CPU oracle for multiple-time-origin time
 * correlation of MD trajectories (arXiv 1708.08619, Sec. 3.5).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * called only by the test suite, by the package's smoke check and by the
 * CPU-baseline leg of the benchmark.  The CUDA library never links, includes
 * or calls it, and it shares no code with the CUDA library.
 *
 * What it computes (the plain definition, evaluated in FP64 from FP32 inputs
 * promoted exactly):
 *
 *   Mean square displacement, Eq. 5 with the serial loop nest of Algorithm 10
 *   (atoms, then time intervals dt, then time origins t), averaged over all
 *   atoms and over all origins:
 *
 *     MSD(tau) = 1/(N n_o(tau)) * sum_i sum_{t0 in O(tau)} sum_c
 *                    (x[t0+tau][i][c] - x[t0][i][c])^2
 *
 *   Time autocorrelation, the integrand of Eq. 4 with the serial loop nest of
 *   Algorithm 8 (time intervals dt, then origins t, product of the signal at
 *   two times):
 *
 *     C(tau)   = 1/(N n_o(tau)) * sum_i sum_{t0 in O(tau)} sum_c
 *                    A[t0][i][c] * A[t0+tau][i][c]
 *
 *   Time cross-correlation of two signals A and B of the same shape (the
 *   product of Algorithm 8 with the second factor taken from B):
 *
 *     X(tau)   = 1/(N n_o(tau)) * sum_i sum_{t0 in O(tau)} sum_c
 *                    A[t0][i][c] * B[t0+tau][i][c]
 *
 *   where O(tau) = { t0 = 0, s, 2s, ... : t0 + tau <= T-1 } (origin stride
 *   s >= 1, s = 1 is the paper's "all time origins") and
 *   n_o(tau) = floor((T-1-tau)/s) + 1 is its size.
 *
 *   Running Green-Kubo integral, Eq. 4 with the quadrature loop that closes
 *   Algorithms 8 and 9, read as the trapezoid rule on the frame grid:
 *     I(0) = 0,  I(tau) = I(tau-1) + dt (C(tau-1) + C(tau)) / 2,
 *     eta(tau) = prefactor * I(tau).
 *
 *   Einstein diffusion constant, Eq. 5: the ordinary least-squares slope b of
 *   MSD(tau) against t = tau dt over [lo, hi], D = b / (2 d); and the literal
 *   ratio MSD(hi) / (2 d hi dt).
 *
 *   Collective signal (for collective transport coefficients): the weighted
 *   sum over atoms J[t] = sum_i w_i (x[t][i] - x[ref][i]).
 *
 * Layout of the trajectory: x[T][N][3] float32, row-major (frame-major),
 * the linear array of Sec. 2.3.
 *
 * Determinism: atoms are cut into fixed blocks of ORACLE_BLOCK atoms.  Each
 * block's per-lag sum is formed in atom order and stored on its own; block sums
 * are then added in block order.  The result therefore does not depend on the
 * number of threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_BLOCK 64

enum { ORACLE_KIND_MSD = 0, ORACLE_KIND_ACF = 1, ORACLE_KIND_XCF = 2 };

/* n_o(tau): number of origins t0 = 0, s, 2s, ... with t0 + tau <= T-1. */
static int64_t n_origins(int64_t T, int64_t tau, int64_t s) {
    if (tau > T - 1) return 0;
    return (T - 1 - tau) / s + 1;
}

typedef struct {
    const float *x;
    const float *y;           /* kind XCF: B, the signal at the later time t0 + tau */
    const float *w;           /* per-atom weights of the average, or NULL (equal weights) */
    int64_t T, N, s;
    const int64_t *lags;
    int64_t nlags;
    int kind;
    double *block_sums;       /* [nblocks][nlags] */
    int64_t nblocks;
    int64_t next_block;       /* shared work counter */
    pthread_mutex_t lock;
} job_t;

/* Per-lag sum over the atoms of one block, atoms in increasing order.
 * traj holds 3T values (6T for XCF: A's, then B's). */
static void do_block(job_t *J, int64_t b, double *traj) {
    const int64_t T = J->T, N = J->N, s = J->s;
    int64_t a0 = b * ORACLE_BLOCK, a1 = a0 + ORACLE_BLOCK;
    if (a1 > N) a1 = N;
    double *out = J->block_sums + b * J->nlags;
    double *later = J->kind == ORACLE_KIND_XCF ? traj + 3 * T : traj;   /* signal at t0 + tau */
    for (int64_t l = 0; l < J->nlags; ++l) out[l] = 0.0;
    for (int64_t i = a0; i < a1; ++i) {
        /* copy atom i's trajectory to a contiguous buffer traj[t][c] (FP64) */
        for (int64_t t = 0; t < T; ++t)
            for (int c = 0; c < 3; ++c)
                traj[3 * t + c] = (double)J->x[(t * N + i) * 3 + c];
        if (J->kind == ORACLE_KIND_XCF)
            for (int64_t t = 0; t < T; ++t)
                for (int c = 0; c < 3; ++c)
                    later[3 * t + c] = (double)J->y[(t * N + i) * 3 + c];
        for (int64_t l = 0; l < J->nlags; ++l) {
            const int64_t tau = J->lags[l];
            double acc = 0.0;
            for (int64_t t0 = 0; t0 + tau <= T - 1; t0 += s) {
                const double *p = traj + 3 * t0;
                const double *q = later + 3 * (t0 + tau);
                double term = 0.0;
                for (int c = 0; c < 3; ++c) {
                    if (J->kind == ORACLE_KIND_MSD) {
                        double d = q[c] - p[c];
                        term += d * d;
                    } else {
                        term += p[c] * q[c];
                    }
                }
                acc += term;
            }
            if (J->w) acc *= (double)J->w[i];
            out[l] += acc;
        }
    }
}

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    double *traj = (double *)malloc(sizeof(double) * (J->kind == ORACLE_KIND_XCF ? 6 : 3) * (size_t)J->T);
    if (!traj) return (void *)1;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t b = J->next_block++;
        pthread_mutex_unlock(&J->lock);
        if (b >= J->nblocks) break;
        do_block(J, b, traj);
    }
    free(traj);
    return NULL;
}

/*
 * oracle_corr: kind 0 = MSD, 1 = ACF, evaluated at the listed lags.
 * x: [T][N][3] float32.  lags: nlags values, each in [0, T-1].
 * out[l] = normalised result at lags[l].  Returns 0 on success, -1 on bad
 * arguments, -2 on allocation failure.
 */
static int corr_run(int kind, const float *x, const float *y, const float *w, int64_t T, int64_t N, int64_t s,
                    const int64_t *lags, int64_t nlags, double *out, int nthreads) {
    if (!x || !lags || !out || T < 1 || N < 1 || s < 1 || nlags < 0) return -1;
    if (kind != ORACLE_KIND_MSD && kind != ORACLE_KIND_ACF && kind != ORACLE_KIND_XCF) return -1;
    if (kind == ORACLE_KIND_XCF && !y) return -1;
    for (int64_t l = 0; l < nlags; ++l)
        if (lags[l] < 0 || lags[l] > T - 1) return -1;
    if (nthreads < 1) nthreads = 1;
    job_t J;
    J.x = x; J.y = y; J.w = w; J.T = T; J.N = N; J.s = s; J.lags = lags; J.nlags = nlags;
    J.kind = kind;
    J.nblocks = (N + ORACLE_BLOCK - 1) / ORACLE_BLOCK;
    J.next_block = 0;
    J.block_sums = (double *)malloc(sizeof(double) * (size_t)(J.nblocks * (nlags > 0 ? nlags : 1)));
    if (!J.block_sums) return -2;
    pthread_mutex_init(&J.lock, NULL);
    if (nthreads > J.nblocks) nthreads = (int)J.nblocks;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int rc = 0;
    if (!th) { rc = -2; goto done; }
    int started = 0;
    for (int k = 0; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, worker, &J) != 0) break;
        ++started;
    }
    if (started == 0) worker(&J);
    for (int k = 0; k < started; ++k) {
        void *ret = NULL;
        pthread_join(th[k], &ret);
        if (ret) rc = -2;
    }
    free(th);
    if (rc) goto done;
    double wsum = 0.0;
    if (w)
        for (int64_t i = 0; i < N; ++i) wsum += (double)w[i];
    for (int64_t l = 0; l < nlags; ++l) {
        double total = 0.0;
        for (int64_t b = 0; b < J.nblocks; ++b) total += J.block_sums[b * nlags + l];
        if (w) out[l] = total / (wsum * (double)n_origins(T, lags[l], s));
        else out[l] = total / ((double)N * (double)n_origins(T, lags[l], s));
    }
done:
    pthread_mutex_destroy(&J.lock);
    free(J.block_sums);
    return rc;
}

int oracle_corr(int kind, const float *x, int64_t T, int64_t N, int64_t s,
                const int64_t *lags, int64_t nlags, double *out, int nthreads) {
    if (kind == ORACLE_KIND_XCF) return -1;
    return corr_run(kind, x, NULL, NULL, T, N, s, lags, nlags, out, nthreads);
}

/*
 * oracle_corr_weighted: as oracle_corr, with the atom average weighted,
 *   MSD_w(tau) = 1/(W n_o(tau)) sum_i w_i sum_{t0} sum_c (x[t0+tau][i][c] - x[t0][i][c])^2,
 * W = sum_i w_i (likewise for the autocorrelation): the average "over all the
 * atoms (or a subclass)" of Eq. 5 with each atom counted w_i times, e.g. a
 * mass-weighted MSD or, with 0/1 weights, a selection.
 */
int oracle_corr_weighted(int kind, const float *x, const float *w, int64_t T, int64_t N, int64_t s,
                         const int64_t *lags, int64_t nlags, double *out, int nthreads) {
    if (kind == ORACLE_KIND_XCF || !w) return -1;
    return corr_run(kind, x, NULL, w, T, N, s, lags, nlags, out, nthreads);
}

/*
 * oracle_xcorr: cross-correlation X(tau) of a (at the origin t0) and b (at
 * t0 + tau), both [T][N][3] float32, at the listed lags.
 */
int oracle_xcorr(const float *a, const float *b, int64_t T, int64_t N, int64_t s,
                 const int64_t *lags, int64_t nlags, double *out, int nthreads) {
    return corr_run(ORACLE_KIND_XCF, a, b, NULL, T, N, s, lags, nlags, out, nthreads);
}

/* Running Green-Kubo integral (Eq. 4, trapezoid): running[0..n-1]. */
int oracle_gk_integrate(const double *c, int64_t n, double dt, double prefactor,
                        double *running) {
    if (!c || !running || n < 1) return -1;
    double I = 0.0;
    running[0] = 0.0;
    for (int64_t k = 1; k < n; ++k) {
        I += dt * (c[k - 1] + c[k]) / 2.0;
        running[k] = prefactor * I;
    }
    return 0;
}

/*
 * Collective signal: the system-wide sum whose time correlation gives a
 * collective transport coefficient (Eq. 4 with a collective flux, as the
 * viscosity example correlates the pressure tensor of the whole box; the
 * Einstein-Helfand form takes the MSD of the summed, weighted positions):
 *   J[t][c] = sum_i w[i] (x[t][i][c] - x[ref][i][c])   for 0 <= ref < T,
 *   J[t][c] = sum_i w[i] x[t][i][c]                     for ref = -1,
 * in FP64 from the FP32 inputs promoted exactly, atoms in increasing order;
 * w == NULL means unit weights.  J: T x 3 doubles.
 */
int oracle_collective(const float *x, const float *w, int64_t T, int64_t N, int64_t ref,
                      double *J) {
    if (!x || !J || T < 1 || N < 1 || ref < -1 || ref >= T) return -1;
    for (int64_t t = 0; t < T; ++t) {
        for (int c = 0; c < 3; ++c) {
            double sum = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double v = (double)x[(t * N + i) * 3 + c];
                if (ref >= 0) v -= (double)x[(ref * N + i) * 3 + c];
                sum += (w ? (double)w[i] : 1.0) * v;
            }
            J[t * 3 + c] = sum;
        }
    }
    return 0;
}

/*
 * Einstein relation (Eq. 5): least-squares slope of msd[tau] against
 * t = tau*dt over tau in [lo, hi]; D_slope = slope / (2 dim).  D_ratio is
 * msd[hi] / (2 dim hi dt).  Needs 0 <= lo < hi < n.
 */
int oracle_einstein(const double *msd, int64_t n, double dt, int dim,
                    int64_t lo, int64_t hi, double *D_slope, double *D_ratio) {
    if (!msd || !D_slope || !D_ratio || dim < 1 || lo < 0 || hi <= lo || hi >= n || !(dt > 0))
        return -1;
    const double m = (double)(hi - lo + 1);
    double sx = 0.0, sy = 0.0;
    for (int64_t k = lo; k <= hi; ++k) { sx += (double)k * dt; sy += msd[k]; }
    const double xbar = sx / m, ybar = sy / m;
    double sxy = 0.0, sxx = 0.0;
    for (int64_t k = lo; k <= hi; ++k) {
        const double dx = (double)k * dt - xbar;
        sxy += dx * (msd[k] - ybar);
        sxx += dx * dx;
    }
    *D_slope = (sxy / sxx) / (2.0 * dim);
    *D_ratio = msd[hi] / (2.0 * dim * (double)hi * dt);
    return 0;
}
