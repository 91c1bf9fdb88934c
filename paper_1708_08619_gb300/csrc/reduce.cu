// FP64 kernels that close the path:
//   lag_reduce   -- fixed-order sum of per-item band-offset partials into the
//                   per-lag sum D(tau), then the normalisation by N n_o(tau)
//                   (the "update global MSD array" step of Algorithm 11, done
//                   deterministically instead of by a race);
//   gk_integrate -- running trapezoid integral of Eq. 4 (the quadrature loop
//                   closing Algorithms 8 and 9, which the paper runs on the host);
//   einstein     -- least-squares slope of the MSD and D = slope / (2d), Eq. 5.
#include <algorithm>
#include <cstring>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// One warp per lag.  Lane l sums terms l, l+32, ... in order; the lanes are
// then combined by a fixed butterfly, so the result does not depend on timing.
// The lane's share of the window terms of lag m' = m + radd BO over row
// tiles rr rmul + radd (rr < nrow): term t = (gg, rr, cc) with cc fastest; the
// lane's first term is decoded once and each step of 32 terms is added as
// mixed-radix carries (no 64-bit division in the loop; a fixed order).
__device__ __forceinline__ double lag_terms(const LagReduceDesc &a, int64_t rho, int64_t mp, int64_t nrow,
                                            int64_t rmul, int64_t radd, int lane) {
    const int64_t c_lo = mp / a.BF;
    int64_t c_hi = (mp + a.BO - 1) / a.BF;
    if (c_hi > a.n_cols - 1) c_hi = a.n_cols - 1;
    const int64_t ncs = c_hi - c_lo + 1;
    double sum = 0.0;
    if (ncs <= 0 || nrow <= 0) return sum;
    const int64_t nterm = a.n_groups * nrow * ncs;
    int64_t cc = lane % ncs, q = lane / ncs;
    int64_t rr = q % nrow, gg = q / nrow;
    const int64_t dc = 32 % ncs, dq = 32 / ncs;
    for (int64_t t = lane; t < nterm; t += 32) {
        const int64_t c = c_lo + cc;
        const int64_t item = ((gg * a.n_res + rho) * a.n_rows + rr * rmul + radd) * a.n_cols + c;
        const int64_t w = mp - c * a.BF + a.BO - 1;
        const int64_t at = item * a.WP + w;
        if (TCORR_IN_BOUNDS(at, a.partial_elems, a.dbg_status)) sum += a.partial[at];
        cc += dc;
        int64_t carry = dq;
        if (cc >= ncs) {
            cc -= ncs;
            ++carry;
        }
        rr += carry;
        while (rr >= nrow) {
            rr -= nrow;
            ++gg;
        }
    }
    return sum;
}

__device__ __forceinline__ void lag_reduce_body(const LagReduceDesc &a, int64_t tau, int lane) {
    const int64_t rho = tau % a.s, m = tau / a.s;
    double sum;
    if (!a.pair) {
        sum = lag_terms(a, rho, m, a.n_rows, 1, 0, lane);
    } else {
        // CTA-pair tiling: even row tiles as in the plain tiling, odd ones hold lag m
        // at the window place of m + BO
        sum = lag_terms(a, rho, m, a.n_rows / 2, 2, 0, lane);
        sum += lag_terms(a, rho, m + a.BO, a.n_rows / 2, 2, 1, lane);
    }
    const double D = warp_sum(sum);
    if (lane == 0) {
        int64_t no = n_origins(a.T, a.s, tau);
        if (no > a.n_orig) no = a.n_orig;
        const double denom = a.accumulate ? 1.0 : static_cast<double>(a.N) * static_cast<double>(no);
        double v;
        if (a.mode == 0) {
            v = D / denom;
        } else if (tau == 0) {
            v = 0.0;   // |x - x|^2: exactly zero by definition
        } else {
            // P = sum_{o < n_o} S(o s);  Q = sum_{o < n_o} S(o s + tau).
            // S_prefix row rho' holds prefix sums over S(rho' + j s), j = 0, 1, ...
            const double *p0 = a.S_prefix;
            const double P = p0[no];
            const int64_t qq = tau / a.s;
            const double *pr = a.S_prefix + (tau % a.s) * a.prefix_stride;
            const double Q = pr[qq + no] - pr[qq];
            v = (P + Q - 2.0 * D) / denom;
        }
        if (a.accumulate) a.out[tau] += v;
        else a.out[tau] = v;
    }
}

__global__ void lag_reduce_kernel(const __grid_constant__ LagReduceDesc a) {
    const int64_t tau = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (tau > a.tau_max) return;
    lag_reduce_body(a, tau, threadIdx.x & 31);
}

__global__ void lag_reduce_batch_kernel(const LagReduceDesc *__restrict__ d, int n, int64_t total) {
    const int64_t g = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (g >= total) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].lag_begin <= g) lo = mid;
        else hi = mid - 1;
    }
    lag_reduce_body(d[lo], g - d[lo].lag_begin, threadIdx.x & 31);
}

constexpr int kChunkBytes = 28672;
struct ByteChunk {
    alignas(16) uint8_t bytes[kChunkBytes];
    uint32_t n;
};

// Parameter memory serves one address per lane at a time, so the chunk is
// read in 16-byte words where the destination allows it.
__global__ void write_bytes_kernel(uint8_t *dst, const __grid_constant__ ByteChunk c) {
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        const uint32_t n16 = c.n / 16;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(c.bytes);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (uint32_t i = threadIdx.x; i < n16; i += blockDim.x) d4[i] = s4[i];
        done = n16 * 16;
    }
    for (uint32_t i = done + threadIdx.x; i < c.n; i += blockDim.x) dst[i] = c.bytes[i];
}

// Running trapezoid, I(k) = I(k-1) + dt (c[k-1] + c[k]) / 2, spread over
// blocks of GK_SPAN increments (FP64 throughput per SM is low on this part,
// so one block would be slow).  Each block integrates its span (GK_PER
// increments per thread combined by a warp-shuffle scan) on top of the
// integral up to the span, which comes, in a fixed order, from:
//   up to GK_RESUM_BLOCKS blocks: one launch; block b sums the values before
//     its span strided over its threads, S = sum_{k<k0} c[k], and the
//     integral there is dt (2 S - c[0] - c[k0-1]) / 2;
//   more blocks (the re-summing would grow as n^2 / GK_SPAN): three
//     launches; each block sums its span's increments into the first output
//     slot of its span, one block scans those totals in place (exclusive),
//     and each block reads its own slot before it writes its span (only
//     block b writes that slot, so nothing is read after being overwritten).
// Deterministic for a given n.
constexpr int GK_THREADS = 256;
constexpr int GK_PER = 8;
constexpr int64_t GK_SPAN = int64_t(GK_THREADS) * GK_PER;
constexpr int GK_SCAN_THREADS = 1024;
constexpr int64_t GK_RESUM_BLOCKS = 32;

__device__ __forceinline__ double gk_inc(const double *c, int64_t k, int64_t n, double dt) {
    return k < n ? dt * (c[k - 1] + c[k]) / 2.0 : 0.0;
}

// Exclusive block scan of one value per thread (fixed shuffle tree); also
// returns the block total in *total.
template <int NT>
__device__ __forceinline__ double block_excl_scan(double v, double *sh, double *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += u;
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    double base = 0.0, tot = 0.0;
    for (int i = 0; i < NT / 32; ++i) {
        if (i < w) base += sh[i];
        tot += sh[i];
    }
    __syncthreads();
    *total = tot;
    return base + (inc - v);
}

// Batched launches: grid.y indexes the series; series y reads c + y ldc and
// writes running + y ldr.
__global__ void __launch_bounds__(GK_THREADS) gk_block_total_kernel(const double *c, int64_t n, double dt,
                                                                     double *running, int64_t ldc,
                                                                     int64_t ldr) {
    __shared__ double sh[GK_THREADS / 32];
    c += static_cast<int64_t>(blockIdx.y) * ldc;
    running += static_cast<int64_t>(blockIdx.y) * ldr;
    const int64_t k0 = 1 + static_cast<int64_t>(blockIdx.x) * GK_SPAN;
    const int64_t kb = k0 + static_cast<int64_t>(threadIdx.x) * GK_PER;
    double mine = 0.0;
#pragma unroll
    for (int i = 0; i < GK_PER; ++i) mine += gk_inc(c, kb + i, n, dt);
    double tot;
    block_excl_scan<GK_THREADS>(mine, sh, &tot);
    if (threadIdx.x == 0) running[k0] = tot;
}

// In place: running[1 + b SPAN] <- sum of the totals of blocks before b.
__global__ void __launch_bounds__(GK_SCAN_THREADS) gk_scan_totals_kernel(double *running, int64_t nb,
                                                                          int64_t ldr) {
    __shared__ double sh[GK_SCAN_THREADS / 32];
    running += static_cast<int64_t>(blockIdx.y) * ldr;
    const int64_t per = ceil_div(nb, GK_SCAN_THREADS);
    const int64_t b0 = static_cast<int64_t>(threadIdx.x) * per, b1 = min(nb, b0 + per);
    double mine = 0.0;
    for (int64_t b = b0; b < b1; ++b) mine += running[1 + b * GK_SPAN];
    double tot;
    double run = block_excl_scan<GK_SCAN_THREADS>(mine, sh, &tot);
    for (int64_t b = b0; b < b1; ++b) {
        const double t = running[1 + b * GK_SPAN];
        running[1 + b * GK_SPAN] = run;
        run += t;
    }
}

// from_slot: the integral up to this span is the scanned slot; otherwise the
// block re-sums the values before its span (0 for the first block).
__global__ void __launch_bounds__(GK_THREADS) gk_integrate_kernel(const double *c, int64_t n, double dt,
                                                                   double prefactor, double *running,
                                                                   int from_slot, int64_t ldc, int64_t ldr) {
    __shared__ double sh[GK_THREADS / 32];
    __shared__ double before_sh;
    c += static_cast<int64_t>(blockIdx.y) * ldc;
    running += static_cast<int64_t>(blockIdx.y) * ldr;
    const int64_t k0 = 1 + static_cast<int64_t>(blockIdx.x) * GK_SPAN;
    double before = 0.0;
    if (from_slot) {
        if (threadIdx.x == 0) before_sh = running[k0];
        __syncthreads();                    // the slot is read before this block writes its span
        before = before_sh;
    } else if (k0 > 1) {
        // eight interleaved partial sums keep eight loads in flight per thread
        // (one running sum waits out a load latency per element); fixed order
        double p[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int64_t k = threadIdx.x;
        for (; k + 7 * GK_THREADS < k0; k += 8 * GK_THREADS) {
#pragma unroll
            for (int j = 0; j < 8; ++j) p[j] += c[k + j * GK_THREADS];
        }
#pragma unroll
        for (int j = 0; j < 7; ++j) {              // fewer than 8 strides remain
            const int64_t kk = k + j * GK_THREADS;
            if (kk < k0) p[j] += c[kk];
        }
        const double S = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
        double tot;
        block_excl_scan<GK_THREADS>(S, sh, &tot);
        before = dt * (2.0 * tot - c[0] - c[k0 - 1]) / 2.0;
    }
    const int64_t kb = k0 + static_cast<int64_t>(threadIdx.x) * GK_PER;
    double loc[GK_PER];
    double mine = 0.0;
#pragma unroll
    for (int i = 0; i < GK_PER; ++i) {
        loc[i] = gk_inc(c, kb + i, n, dt);
        mine += loc[i];
    }
    double tot;
    double I = before + block_excl_scan<GK_THREADS>(mine, sh, &tot);
    if (blockIdx.x == 0 && threadIdx.x == 0) running[0] = 0.0;
#pragma unroll
    for (int i = 0; i < GK_PER; ++i) {
        const int64_t k = kb + i;
        if (k < n) {
            I += loc[i];
            running[k] = prefactor * I;
        }
    }
}

constexpr int EIN_THREADS = 256;

__device__ double block_sum(double v, double *sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = EIN_THREADS / 2; off > 0; off >>= 1) {
        if (t < off) sh[t] += sh[t + off];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void einstein_kernel(const double *msd, double dt, int dim, int64_t lo, int64_t hi,
                                double *D) {
    __shared__ double sh[EIN_THREADS];
    const int t = threadIdx.x;
    const double m = static_cast<double>(hi - lo + 1);
    double sx = 0.0, sy = 0.0;
    for (int64_t k = lo + t; k <= hi; k += EIN_THREADS) {
        sx += static_cast<double>(k) * dt;
        sy += msd[k];
    }
    const double xbar = block_sum(sx, sh) / m;
    const double ybar = block_sum(sy, sh) / m;
    double sxy = 0.0, sxx = 0.0;
    for (int64_t k = lo + t; k <= hi; k += EIN_THREADS) {
        const double dx = static_cast<double>(k) * dt - xbar;
        sxy += dx * (msd[k] - ybar);
        sxx += dx * dx;
    }
    const double Sxy = block_sum(sxy, sh);
    const double Sxx = block_sum(sxx, sh);
    if (t == 0) {
        D[0] = (Sxy / Sxx) / (2.0 * dim);
        D[1] = msd[hi] / (2.0 * dim * static_cast<double>(hi) * dt);
    }
}

}  // namespace

LagReduceDesc lag_reduce_desc(const BandPlan &p, const double *partial, const FinalizeArgs &fa,
                              double *d_out, int64_t lag_begin) {
    LagReduceDesc a;
    a.partial = partial;
    a.partial_elems = dbg_shrink_elems(p.n_items * p.WP, p.WP);
#ifdef TCORR_DEBUG_BOUNDS
    a.dbg_status = status_word_device_ptr();
#else
    a.dbg_status = nullptr;
#endif
    a.T = p.T;
    a.N = p.N;
    a.s = p.s;
    a.tau_max = p.tau_max;
    a.n_res = p.n_res;
    a.n_rows = p.n_rows;
    a.n_cols = p.n_cols;
    a.n_groups = p.n_groups;
    a.BO = p.BO;
    a.BF = p.BF;
    a.WP = p.WP;
    a.mode = fa.mode;
    a.S_prefix = fa.S_prefix;
    a.prefix_stride = fa.prefix_stride;
    a.out = d_out;
    a.lag_begin = lag_begin;
    a.n_orig = p.n_orig;
    a.accumulate = 0;
    a.pair = p.pair;
    return a;
}

cudaError_t launch_lag_reduce(const BandPlan &p, const double *partial, const FinalizeArgs &fa,
                              double *d_out, cudaStream_t st, const Window *w) {
    LagReduceDesc a = lag_reduce_desc(p, partial, fa, d_out, 0);
    if (w && w->accumulate) a.accumulate = 1;
    const int64_t warps = p.tau_max + 1;
    const int threads = 256;
    const int64_t blocks = ceil_div(warps * 32, threads);
    lag_reduce_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(a);
    return cudaGetLastError();
}

__global__ void normalize_kernel(double *out, int64_t T, int64_t N, int64_t tau_max, int64_t s, int kind) {
    const int64_t tau = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tau > tau_max) return;
    if (kind == 0 && tau == 0) {
        out[0] = 0.0;
        return;
    }
    out[tau] /= static_cast<double>(N) * static_cast<double>(n_origins(T, s, tau));
}

cudaError_t launch_normalize(double *d_out, int64_t T, int64_t N, int64_t tau_max, int64_t s, int kind,
                             cudaStream_t st) {
    normalize_kernel<<<static_cast<unsigned>(ceil_div(tau_max + 1, 256)), 256, 0, st>>>(d_out, T, N, tau_max, s,
                                                                                         kind);
    return cudaGetLastError();
}

cudaError_t launch_lag_reduce_batch(const LagReduceDesc *d_descs, int n, int64_t total_lags,
                                    cudaStream_t st) {
    if (total_lags <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = ceil_div(total_lags * 32, threads);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    lag_reduce_batch_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(d_descs, n, total_lags);
    return cudaGetLastError();
}

cudaError_t upload_bytes(void *d_dst, const void *h_src, size_t nbytes, cudaStream_t st) {
    const uint8_t *src = static_cast<const uint8_t *>(h_src);
    uint8_t *dst = static_cast<uint8_t *>(d_dst);
    ByteChunk c;
    for (size_t off = 0; off < nbytes; off += kChunkBytes) {
        const size_t n = nbytes - off < size_t(kChunkBytes) ? nbytes - off : size_t(kChunkBytes);
        c.n = static_cast<uint32_t>(n);
        std::memcpy(c.bytes, src + off, n);
        write_bytes_kernel<<<1, 256, 0, st>>>(dst + off, c);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gk_integrate_batch(const double *d_c, int64_t n, int64_t count, int64_t ldc, double dt,
                                      double prefactor, double *d_running, int64_t ldr, cudaStream_t st) {
    const int64_t blocks = n > 1 ? ceil_div(n - 1, GK_SPAN) : 1;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool three_pass = blocks > GK_RESUM_BLOCKS;
    constexpr int64_t kMaxY = 65535;           // grid.y limit: series in chunks
    for (int64_t s0 = 0; s0 < count; s0 += kMaxY) {
        const dim3 g(static_cast<unsigned>(blocks), static_cast<unsigned>(std::min(kMaxY, count - s0)));
        const double *c = d_c + s0 * ldc;
        double *r = d_running + s0 * ldr;
        if (three_pass) {
            gk_block_total_kernel<<<g, GK_THREADS, 0, st>>>(c, n, dt, r, ldc, ldr);
            gk_scan_totals_kernel<<<dim3(1, g.y), GK_SCAN_THREADS, 0, st>>>(r, blocks, ldr);
        }
        gk_integrate_kernel<<<g, GK_THREADS, 0, st>>>(c, n, dt, prefactor, r, three_pass ? 1 : 0, ldc, ldr);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gk_integrate(const double *d_c, int64_t n, double dt, double prefactor,
                                double *d_running, cudaStream_t st) {
    return launch_gk_integrate_batch(d_c, n, 1, n, dt, prefactor, d_running, n, st);
}

cudaError_t launch_einstein(const double *d_msd, int64_t n, double dt, int dim, int64_t lo,
                            int64_t hi, double *d_D, cudaStream_t st) {
    (void)n;
    einstein_kernel<<<1, EIN_THREADS, 0, st>>>(d_msd, dt, dim, lo, hi, d_D);
    return cudaGetLastError();
}

}  // namespace tcorr
