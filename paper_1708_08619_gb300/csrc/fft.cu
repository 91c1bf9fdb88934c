// FFT (Wiener-Khinchin) route for the MSD and the autocorrelation.
//
// The band kernels cost O(T tau_max K); when tau_max approaches T the lag sums
// are cheaper through the correlation theorem: per column k of the T x K
// matrix, r_k(tau) = sum_t a_k(t) a_k(t + tau) is the inverse transform of
// |F a_k|^2 once a_k is zero-padded to a length L >= T + tau_max (then the
// circular wrap adds nothing to lags <= tau_max).  Origins thinned to a
// stride s use the cross form: with m_k(t) = a_k(t) for t in sZ and 0
// otherwise, sum_{t0 in sZ} a_k(t0) a_k(t0 + tau) = IFFT(conj(F m_k) F a_k).
// The MSD uses the same lag sums D(tau) of the frame-0-referenced positions
// and MSD = (P + Q - 2 D) / (N n_o) with P, Q from FP64 prefix sums of
// S(t) = |x_t|^2, as the band path does (expanding |a - b|^2, Eq. 5).
//
// The cross-correlation of A (origin side) with B (later side) is the same
// with IFFT(conj(F m_A) F b).
//
// Work per chunk of Kc columns: a tiled transpose gathers the columns into
// zero-padded FP64 rows, cuFFT transforms them (real to complex, the work
// area in the caller's workspace), one kernel forms the (cross) power
// spectrum, cuFFT transforms back, and one thread per lag adds the chunk's
// columns to an FP64 accumulator in column order (deterministic).
//
// Precision: a transform's rounding error is spread evenly over the lags at
// about eps times the signal energy, and the lag sums are then divided by
// n_o(tau), which is 1 at tau = T - 1; so the error relative to C(0) or
// MSD(tau_max) grows with T / n_o.  FP32 transforms missed 1e-5 at
// tau_max = T - 1 (measured 5.9e-5 on T = 1000), hence FP64 throughout; the
// inputs are FP32 and are promoted exactly.
#include <cufft.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int64_t kFftChunkElems = int64_t(1) << 26;   // real elements of one chunk buffer (512 MB)

// Smallest L >= n of the form 2^a, 3 2^a or 5 2^a (sizes cuFFT handles fast).
int64_t fft_length(int64_t n) {
    int64_t best = 0;
    for (int64_t m : {int64_t(1), int64_t(3), int64_t(5)}) {
        int64_t L = m;
        while (L < n) L *= 2;
        if (best == 0 || L < best) best = L;
    }
    return best;
}

struct FftLayout {
    int64_t T, N, K, tau_max, s, L, Lc, Kc, n_chunks, pstride;
    size_t off_r, off_rm, off_c, off_cm, off_d, off_S, off_prefix, off_work, total;
    size_t work_bytes;
};

// Cached cuFFT plans per (device, L, batch, direction); cuFFT's own plan data
// is created once, its work area is always the caller's workspace.
struct PlanKey {
    int dev;
    int64_t L, batch;
    int dir;
    bool operator<(const PlanKey &o) const {
        return std::tie(dev, L, batch, dir) < std::tie(o.dev, o.L, o.batch, o.dir);
    }
};
struct PlanVal {
    cufftHandle h;
    size_t work;
};
std::mutex g_plan_mu, g_exec_mu;
std::map<PlanKey, PlanVal> g_plans;

// dir 0: real -> complex, 1: complex -> real; batch transforms of length L,
// rows L (real) or L/2+1 (complex) apart.
bool get_plan(int64_t L, int64_t batch, int dir, PlanVal *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(g_plan_mu);
    const PlanKey key{dev, L, batch, dir};
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        *out = it->second;
        return true;
    }
    cufftHandle h;
    if (cufftCreate(&h) != CUFFT_SUCCESS) return false;
    if (cufftSetAutoAllocation(h, 0) != CUFFT_SUCCESS) {
        cufftDestroy(h);
        return false;
    }
    long long n[1] = {L};
    long long inembed[1] = {dir == 0 ? L : L / 2 + 1};
    long long onembed[1] = {dir == 0 ? L / 2 + 1 : L};
    size_t work = 0;
    if (cufftMakePlanMany64(h, 1, n, inembed, 1, inembed[0], onembed, 1, onembed[0],
                            dir == 0 ? CUFFT_D2Z : CUFFT_Z2D, batch, &work) != CUFFT_SUCCESS) {
        cufftDestroy(h);
        return false;
    }
    const PlanVal v{h, work};
    g_plans[key] = v;
    *out = v;
    return true;
}

bool make_fft_layout(int64_t T, int64_t N, int64_t tau_max, int64_t s, int kind, FftLayout *F) {
    F->T = T;
    F->N = N;
    F->K = 3 * N;
    F->tau_max = tau_max;
    F->s = s;
    F->L = fft_length(T + tau_max);
    F->Lc = F->L / 2 + 1;
    int64_t kc = kFftChunkElems / F->L;
    if (kc < 1) kc = 1;
    if (kc > 65535 * 32) kc = 65535 * 32;           // the gather grid's y extent
    F->Kc = kc < F->K ? kc : F->K;
    F->n_chunks = ceil_div(F->K, F->Kc);
    F->pstride = (T - 1) / s + 2;
    const int64_t n_res = s < tau_max + 1 ? s : tau_max + 1;
    PlanVal fwd, inv;
    if (!get_plan(F->L, F->Kc, 0, &fwd) || !get_plan(F->L, F->Kc, 1, &inv)) return false;
    F->work_bytes = fwd.work > inv.work ? fwd.work : inv.work;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t rbytes = sizeof(double) * static_cast<size_t>(F->Kc) * F->L;
    const size_t cbytes = sizeof(cufftDoubleComplex) * static_cast<size_t>(F->Kc) * F->Lc;
    const bool two = s > 1 || kind == 2;           // a separate origin-side transform
    F->off_r = take(rbytes);
    F->off_rm = take(two ? rbytes : 0);
    F->off_c = take(cbytes);
    F->off_cm = take(two ? cbytes : 0);
    F->off_d = take(sizeof(double) * static_cast<size_t>(tau_max + 1));
    F->off_S = take(kind == 0 ? sizeof(double) * static_cast<size_t>(T) : 0);
    F->off_prefix = take(kind == 0 ? sizeof(double) * static_cast<size_t>(n_res * F->pstride) : 0);
    F->off_work = take(F->work_bytes);
    F->total = off;
    return true;
}

// Columns k0 .. k0+Kc-1 of x (minus frame 0 when ref) into zero-padded rows
// R[c][0..L), keeping only frames t in sZ when mask_s > 1 (origins).  32 x 32
// tiles through shared memory: reads along k, writes along t.
__global__ void fft_gather_kernel(const float *__restrict__ x, int64_t T, int64_t K, int64_t k0, int64_t Kc,
                                  int64_t L, int ref, int64_t mask_s, double *R) {
    __shared__ double tile[32][33];
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * 32, c0 = static_cast<int64_t>(blockIdx.y) * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += blockDim.y) {
        const int64_t t = t0 + i, c = c0 + tx, k = k0 + c;
        float v = 0.f;
        if (t < T && c < Kc && k < K && t % mask_s == 0) {
            v = x[t * K + k];
            if (ref) v -= x[k];          // exact in FP32 (nearby values)
        }
        tile[i][tx] = static_cast<double>(v);
    }
    __syncthreads();
    for (int i = ty; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, t = t0 + tx;
        if (c < Kc && t < L) R[c * L + t] = tile[tx][i];
    }
}

// The same for a handful of columns (Kc <= 8, e.g. a flux series with K = 3):
// one thread per frame reads its Kc values and writes one to each row, so no
// tile lanes sit idle.
constexpr int64_t kNarrowGather = 8;
__global__ void fft_gather_narrow_kernel(const float *__restrict__ x, int64_t T, int64_t K, int64_t k0,
                                         int64_t Kc, int64_t L, int ref, int64_t mask_s, double *R) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= L) return;
    const bool live = t < T && t % mask_s == 0;
    for (int64_t c = 0; c < Kc; ++c) {
        const int64_t k = k0 + c;
        float v = 0.f;
        if (live && k < K) {
            v = x[t * K + k];
            if (ref) v -= x[k];
        }
        R[c * L + t] = static_cast<double>(v);
    }
}

// C <- |C|^2 (s = 1) or conj(Cm) C (s > 1): the transform of the lag sums.
__global__ void fft_power_kernel(cufftDoubleComplex *C, const cufftDoubleComplex *Cm, int64_t n) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cufftDoubleComplex a = C[i];
    if (Cm == nullptr) {
        C[i] = make_cuDoubleComplex(a.x * a.x + a.y * a.y, 0.0);
    } else {
        const cufftDoubleComplex m = Cm[i];
        C[i] = make_cuDoubleComplex(m.x * a.x + m.y * a.y, m.x * a.y - m.y * a.x);
    }
}

// D[tau] += (sum over the chunk's columns, in column order) / L.
__global__ void fft_lag_sum_kernel(const double *R, int64_t Kc, int64_t L, int64_t tau_max, double *D) {
    const int64_t tau = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tau > tau_max) return;
    double acc = 0.0;
    for (int64_t c = 0; c < Kc; ++c) acc += R[c * L + tau];
    D[tau] += acc / static_cast<double>(L);
}

// S(t) = |x_t - x_0|^2 in FP64 from the exact FP32 differences, one block per frame.
constexpr int FS_THREADS = 256;
__global__ void __launch_bounds__(FS_THREADS) fft_s_kernel(const float *__restrict__ x, int64_t K, double *S) {
    __shared__ double red[FS_THREADS / 32];
    const int64_t t = blockIdx.x;
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < K; k += FS_THREADS) {
        const double d = static_cast<double>(x[t * K + k] - x[k]);
        acc += d * d;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < FS_THREADS / 32; ++i) tot += red[i];
        S[t] = tot;
    }
}

// out[tau] = D / (N n_o) (ACF) or (P + Q - 2D) / (N n_o) (MSD, out[0] = 0).
__global__ void fft_finalize_kernel(const double *D, int64_t T, int64_t N, int64_t s, int64_t tau_max, int kind,
                                    const double *prefix, int64_t pstride, double *out) {
    const int64_t tau = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tau > tau_max) return;
    const int64_t no = n_origins(T, s, tau);
    const double denom = static_cast<double>(N) * static_cast<double>(no);
    if (kind != 0) {
        out[tau] = D[tau] / denom;
    } else if (tau == 0) {
        out[tau] = 0.0;
    } else {
        const double P = prefix[no];
        const int64_t qq = tau / s;
        const double *pr = prefix + (tau % s) * pstride;
        const double Q = pr[qq + no] - pr[qq];
        out[tau] = (P + Q - 2.0 * D[tau]) / denom;
    }
}

}  // namespace

// kind 0 (MSD) needs the most of 0 and 1; kind 2 adds the origin-side buffers.
size_t fft_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t s, int kind) {
    FftLayout F;
    if (!make_fft_layout(T, N, tau_max, s, kind, &F)) return 0;
    return F.total;
}

// kind 0 MSD, 1 ACF of d_x; 2 cross-correlation of d_x (origins) with d_y.
int fft_run(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s, double *d_out,
            void *d_ws, size_t ws_bytes, cudaStream_t st, const float *d_y) {
    FftLayout F;
    if (!make_fft_layout(T, N, tau_max, s, kind, &F)) return TCORR_EUNSUPPORTED;
    if (ws_bytes < F.total || !d_ws) return TCORR_EWORKSPACE;
    const bool two = s > 1 || kind == 2;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    double *R = reinterpret_cast<double *>(ws + F.off_r);
    double *Rm = two ? reinterpret_cast<double *>(ws + F.off_rm) : nullptr;
    cufftDoubleComplex *C = reinterpret_cast<cufftDoubleComplex *>(ws + F.off_c);
    cufftDoubleComplex *Cm = two ? reinterpret_cast<cufftDoubleComplex *>(ws + F.off_cm) : nullptr;
    double *D = reinterpret_cast<double *>(ws + F.off_d);
    PlanVal fwd, inv;
    if (!get_plan(F.L, F.Kc, 0, &fwd) || !get_plan(F.L, F.Kc, 1, &inv)) return TCORR_EUNSUPPORTED;
    // plans are shared: their stream and work area are set and used under one lock
    std::lock_guard<std::mutex> lock(g_exec_mu);
    for (cufftHandle h : {fwd.h, inv.h})
        if (cufftSetStream(h, st) != CUFFT_SUCCESS || cufftSetWorkArea(h, ws + F.off_work) != CUFFT_SUCCESS)
            return TCORR_ECUDA;
    cudaError_t e = cudaMemsetAsync(D, 0, sizeof(double) * static_cast<size_t>(tau_max + 1), st);
    if (e != cudaSuccess) return cuda_fail(e, "lag-sum reset");
    const int64_t nspec = F.Kc * F.Lc;
    for (int64_t ch = 0; ch < F.n_chunks; ++ch) {
        const int64_t k0 = ch * F.Kc;
        const dim3 g(static_cast<unsigned>(ceil_div(F.L, 32)), static_cast<unsigned>(ceil_div(F.Kc, 32)));
        const unsigned gn = static_cast<unsigned>(ceil_div(F.L, 256));
        auto gather = [&](const float *src, int64_t mask_s, double *dst) {
            if (F.Kc <= kNarrowGather)
                fft_gather_narrow_kernel<<<gn, 256, 0, st>>>(src, T, F.K, k0, F.Kc, F.L, kind == 0, mask_s, dst);
            else
                fft_gather_kernel<<<g, dim3(32, 8), 0, st>>>(src, T, F.K, k0, F.Kc, F.L, kind == 0, mask_s, dst);
        };
        // later side: B (cross) or the signal itself; origin side: the signal, masked to sZ
        gather(kind == 2 ? d_y : d_x, 1, R);
        if (two) gather(d_x, s, Rm);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_gather launch");
        if (cufftExecD2Z(fwd.h, R, C) != CUFFT_SUCCESS) return TCORR_ECUDA;
        if (two && cufftExecD2Z(fwd.h, Rm, Cm) != CUFFT_SUCCESS) return TCORR_ECUDA;
        fft_power_kernel<<<static_cast<unsigned>(ceil_div(nspec, 256)), 256, 0, st>>>(C, Cm, nspec);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_power launch");
        if (cufftExecZ2D(inv.h, C, R) != CUFFT_SUCCESS) return TCORR_ECUDA;
        // the last chunk's columns past K were gathered as zeros and add nothing
        fft_lag_sum_kernel<<<static_cast<unsigned>(ceil_div(tau_max + 1, 256)), 256, 0, st>>>(R, F.Kc, F.L,
                                                                                           tau_max, D);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_lag_sum launch");
    }
    const double *prefix = nullptr;
    if (kind == 0) {
        double *S = reinterpret_cast<double *>(ws + F.off_S);
        double *pre = reinterpret_cast<double *>(ws + F.off_prefix);
        fft_s_kernel<<<static_cast<unsigned>(T), FS_THREADS, 0, st>>>(d_x, F.K, S);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_s launch");
        const int64_t n_res = s < tau_max + 1 ? s : tau_max + 1;
        if ((e = launch_s_prefix(S, T, s, n_res, F.pstride, pre, st)) != cudaSuccess)
            return cuda_fail(e, "s_prefix launch");
        prefix = pre;
    }
    fft_finalize_kernel<<<static_cast<unsigned>(ceil_div(tau_max + 1, 256)), 256, 0, st>>>(
        D, T, N, s, tau_max, kind, prefix, F.pstride, d_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_finalize launch");
    return TCORR_OK;
}

}  // namespace tcorr
