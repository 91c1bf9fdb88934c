// FFT (Wiener-Khinchin) route for the MSD and the autocorrelation, with the
// library's own transforms.
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
// S(t) = |x_t|^2, as the band path does (expanding |a - b|^2, Eq. 5).  The
// cross-correlation of A (origin side) with B (later side) is
// IFFT(conj(F m_A) F b).
//
// Two real columns per complex transform.  The route needs only the SUM of
// the columns' lag sums, so columns 2c and 2c+1 travel as one complex signal
// z = a + i b: with w = m_a + i m_b the origin-side signal (w = z without a
// mask), Re IFFT(conj(F w) F z)(tau) = sum_t m_a(t) a(t+tau) + m_b(t) b(t+tau),
// exactly the two columns' lag sums; the imaginary part (their cross terms)
// is dropped.  No real-to-complex packing step is needed.
//
// Transforms: complex, length L = L1 L2 (L of the form 2^a, 3 2^a, 5 2^a;
// L1 a power of two <= 2048, L2 <= 4096), as the four-step factorisation
// with n = L2 n1 + n2 and k = k1 + L1 k2:
//   column pass: Y[k1][n2] = W_L^(n2 k1) sum_n1 x[L2 n1 + n2] W_L1^(n1 k1)
//   row pass:    X[k1 + L1 k2] = sum_n2 Y[k1][n2] W_L2^(n2 k2)
// Both passes work in place on a row-major L1 x L2 array, so the spectrum
// comes out in the transposed order [k1][k2].  The power spectrum is formed
// point by point, which does not care about the order, and the inverse
// transform takes the same order back to natural time order (row pass, then
// column pass, with conjugate twiddles).  The row pass does the forward row
// transform, the power spectrum and the inverse row transform of one row in
// shared memory, so a chunk costs three passes over the data: column pass,
// fused row pass, inverse column pass.  L <= 4096 is the row pass alone
// (L1 = 1).  Each pass is a Stockham FFT in shared memory (radix 2/4 stages
// and one radix-3 or radix-5 stage), every thread holding its butterflies'
// outputs in registers across the barrier that separates a stage's reads
// from its writes.
//
// Arithmetic: double-float.  Each real part is an unevaluated sum hi + lo of
// two FP32 values (about 48 significant bits), computed on the FP32 pipe with
// error-free transformations: Knuth's two-sum, Dekker's fast two-sum and the
// FMA form of the exact product (the double-float arithmetic of Dekker 1971;
// the addition keeps the hi error term exactly and folds the lo terms in, so
// its absolute error is about 2^-47 (|a| + |b|)).  FP64 would be the other
// choice, but this part's FP64 rate is a small fraction of its FP32 rate.
// Precision matters: a transform's rounding error spreads evenly over the
// lags at about eps times the signal energy, and the lag sums are then
// divided by n_o(tau), which is 1 at tau = T - 1, so the error relative to
// C(0) or MSD(tau_max) grows with T / n_o; FP32 transforms missed 1e-5 at
// tau_max = T - 1 (measured 5.9e-5 on T = 1000).  The inputs are FP32 and
// enter exactly (lo = 0); twiddles come from FP64 sincospi split into hi + lo.
// The lag sums leave the transform as FP64 (hi + lo) and are summed over the
// chunk's rows in row order in FP64 (deterministic).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

// ------------------------------------------------------ double-float numbers
struct DF {
    float h, l;
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.h, -a.l}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
// a * c (c a double-float constant): exact product of the hi parts by FMA,
// cross terms folded into the error word.
__device__ __forceinline__ DF df_mul(DF a, DF c) {
    const float p = __fmul_rn(a.h, c.h);
    float e = fmaf(a.h, c.h, -p);
    e = fmaf(a.h, c.l, e);
    e = fmaf(a.l, c.h, e);
    return fast_two_sum(p, e);
}
// a b + c d in one rounding chain: the two hi products are exact (FMA), their
// sum is a two-sum, the small terms go into the error word.
__device__ __forceinline__ DF df_dot2(DF a, DF b, DF c, DF d) {
    const float p = __fmul_rn(a.h, b.h);
    const float ep = fmaf(a.h, b.h, -p);
    const float q = __fmul_rn(c.h, d.h);
    const float eq = fmaf(c.h, d.h, -q);
    DF s = two_sum(p, q);
    float e = __fadd_rn(s.l, __fadd_rn(ep, eq));
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    e = fmaf(c.h, d.l, e);
    e = fmaf(c.l, d.h, e);
    return fast_two_sum(s.h, e);
}
__device__ __forceinline__ DF df_from(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - static_cast<double>(h))};
}
__device__ __forceinline__ double df_to(DF a) { return static_cast<double>(a.h) + static_cast<double>(a.l); }

// A complex number in double-float (16 bytes, the element of every buffer).
struct __align__(16) Z {
    DF x, y;
};
__device__ __forceinline__ Z zadd(Z a, Z b) { return {df_add(a.x, b.x), df_add(a.y, b.y)}; }
__device__ __forceinline__ Z zsub(Z a, Z b) { return {df_sub(a.x, b.x), df_sub(a.y, b.y)}; }
// a * w
__device__ __forceinline__ Z zmul(Z a, Z w) {
    return {df_dot2(a.x, w.x, df_neg(a.y), w.y), df_dot2(a.x, w.y, a.y, w.x)};
}
// a * conj(w)
__device__ __forceinline__ Z zmulc(Z a, Z w) {
    return {df_dot2(a.x, w.x, a.y, w.y), df_dot2(a.y, w.x, df_neg(a.x), w.y)};
}
// a * (s i), s = +-1
__device__ __forceinline__ Z zrot(Z a, int s) { return s > 0 ? Z{df_neg(a.y), a.x} : Z{a.y, df_neg(a.x)}; }
__device__ __forceinline__ Z zscale(Z a, DF c) { return {df_mul(a.x, c), df_mul(a.y, c)}; }
__device__ __forceinline__ Z zload(const Z *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void zstore(Z *p, Z a) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.x.h, a.x.l, a.y.h, a.y.l);
}

// Real constants of the radix-3 and radix-5 butterflies, as double-float
// (from the host's libm in FP64, split into hi + lo).
struct Consts {
    DF s3;             // sin(2 pi / 3)
    DF c51, c52;       // cos(2 pi / 5), cos(4 pi / 5)
    DF s51, s52;       // sin(2 pi / 5), sin(4 pi / 5)
};

// ------------------------------------------------------------ butterflies
// In-register DFT of length R.  dir = -1 forward (W = e^(-2 pi i / R)),
// +1 inverse (conjugate W).
template <int R>
__device__ __forceinline__ void dft(Z (&a)[R], int dir, const Consts &K);

template <>
__device__ __forceinline__ void dft<2>(Z (&a)[2], int, const Consts &) {
    const Z t = a[0];
    a[0] = zadd(t, a[1]);
    a[1] = zsub(t, a[1]);
}

template <>
__device__ __forceinline__ void dft<4>(Z (&a)[4], int dir, const Consts &) {
    const Z t0 = zadd(a[0], a[2]), t1 = zsub(a[0], a[2]);
    const Z t2 = zadd(a[1], a[3]), t3 = zrot(zsub(a[1], a[3]), dir);   // (a1 - a3) W_4^(+-1)
    a[0] = zadd(t0, t2);
    a[2] = zsub(t0, t2);
    a[1] = zadd(t1, t3);
    a[3] = zsub(t1, t3);
}

// b0 = a0 + s;  b1,2 = a0 - s/2 -+ i dir' (sqrt3/2)(a1 - a2),  s = a1 + a2
template <>
__device__ __forceinline__ void dft<3>(Z (&a)[3], int dir, const Consts &K) {
    const Z s = zadd(a[1], a[2]);
    const Z d = zscale(zsub(a[1], a[2]), K.s3);
    const DF half = {0.5f, 0.f};
    const Z m = zsub(a[0], zscale(s, half));
    a[0] = zadd(a[0], s);
    const Z r = zrot(d, dir);          // (sqrt3/2)(a1 - a2) * (dir i)
    a[1] = zadd(m, r);
    a[2] = zsub(m, r);
}

// with s1 = a1 + a4, d1 = a1 - a4, s2 = a2 + a3, d2 = a2 - a3:
//   b1,4 = a0 + c1 s1 + c2 s2 + (dir i)(+-)(sn1 d1 + sn2 d2)
//   b2,3 = a0 + c2 s1 + c1 s2 + (dir i)(+-)(sn2 d1 - sn1 d2)
template <>
__device__ __forceinline__ void dft<5>(Z (&a)[5], int dir, const Consts &K) {
    const Z s1 = zadd(a[1], a[4]), d1 = zsub(a[1], a[4]);
    const Z s2 = zadd(a[2], a[3]), d2 = zsub(a[2], a[3]);
    const Z e1 = zadd(a[0], zadd(zscale(s1, K.c51), zscale(s2, K.c52)));
    const Z e2 = zadd(a[0], zadd(zscale(s1, K.c52), zscale(s2, K.c51)));
    const Z o1 = zrot(zadd(zscale(d1, K.s51), zscale(d2, K.s52)), dir);
    const Z o2 = zrot(zsub(zscale(d1, K.s52), zscale(d2, K.s51)), dir);
    a[0] = zadd(a[0], zadd(s1, s2));
    a[1] = zadd(e1, o1);
    a[4] = zsub(e1, o1);
    a[2] = zadd(e2, o2);
    a[3] = zsub(e2, o2);
}

constexpr int kThreads = 512;         // threads per FFT block
constexpr int kMaxElems = 4096;       // complex elements per block's shared buffer (64 KB)
constexpr int kMaxL1 = 2048;
constexpr int kMaxL2 = 4096;
constexpr int64_t kTwSplit = 2048;    // W_L^j = W_L^(j mod 2048) W_L^(2048 floor(j / 2048))

// One Stockham stage of radix R over nfft transforms of length P stored in
// shared memory at buf[e * es + f * fs] (element e of transform f).  Before
// the stage the transforms of length Ns are done; butterfly idx (0 <= idx <
// P/R) reads elements idx + r P/R, applies W_(Ns R)^(dir r k), k = idx mod
// Ns, and writes element (idx / Ns) Ns R + k + r Ns.  tw holds W_P^j, j < P
// (forward direction).
template <int R>
__device__ __forceinline__ void stockham_stage(Z *buf, int P, int Ns, int es, int fs, int nfft, int dir,
                                               const Z *__restrict__ tw, const Consts &K) {
    constexpr int MAXB = (kMaxElems / R + kThreads - 1) / kThreads;
    const int nb = P / R;
    const int total = nb * nfft;
    const int tstep = P / (Ns * R);
    Z out[MAXB][R];
    int dst[MAXB];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int u = threadIdx.x + b * kThreads;
        dst[b] = -1;
        if (u < total) {
            const int f = u % nfft, idx = u / nfft;
            const int k = idx % Ns;
            Z a[R];
#pragma unroll
            for (int r = 0; r < R; ++r) a[r] = buf[(idx + r * nb) * es + f * fs];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const Z w = zload(tw + r * k * tstep);
                    a[r] = dir < 0 ? zmul(a[r], w) : zmulc(a[r], w);
                }
            }
            dft<R>(a, dir, K);
#pragma unroll
            for (int r = 0; r < R; ++r) out[b][r] = a[r];
            dst[b] = ((idx / Ns) * Ns * R + k) * es + f * fs;
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        if (dst[b] >= 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[dst[b] + r * Ns * es] = out[b][r];
        }
    }
    __syncthreads();
}

// Length-P DFT (P = m 2^a, m in {1, 3, 5}) of nfft transforms in shared memory,
// natural order in and out; the caller has synchronised after filling buf.
__device__ void fft_smem(Z *buf, int P, int es, int fs, int nfft, int dir, const Z *__restrict__ tw,
                         const Consts &K) {
    const int m = (P % 3 == 0) ? 3 : (P % 5 == 0) ? 5 : 1;
    int rem = P / m;                     // power of two
    int Ns = 1;
    if (rem > 1 && (__ffs(rem) - 1) % 2 == 1) {
        stockham_stage<2>(buf, P, Ns, es, fs, nfft, dir, tw, K);
        Ns *= 2;
        rem /= 2;
    }
    while (rem >= 4) {
        stockham_stage<4>(buf, P, Ns, es, fs, nfft, dir, tw, K);
        Ns *= 4;
        rem /= 4;
    }
    if (m == 3) stockham_stage<3>(buf, P, Ns, es, fs, nfft, dir, tw, K);
    if (m == 5) stockham_stage<5>(buf, P, Ns, es, fs, nfft, dir, tw, K);
}

// W_L^j from the two-level table (j < L).
__device__ __forceinline__ Z twiddle_L(const Z *__restrict__ ta, const Z *__restrict__ tb, int64_t j) {
    return zmul(zload(ta + (j % kTwSplit)), zload(tb + j / kTwSplit));
}

// ------------------------------------------------------------------ kernels

// Twiddle tables, W_N^j = exp(-2 pi i j / N) from FP64 sincospi, as
// double-float: tw1[j] = W_L1^j (j < L1), tw2[j] = W_L2^j (j < L2),
// ta[j] = W_L^j (j < 2048), tb[j] = W_L^(2048 j) (j < ceil(L / 2048)).
__global__ void fft_twiddle_kernel(Z *tw1, int L1, Z *tw2, int L2, Z *ta, Z *tb, int64_t L, int64_t ntb) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    auto put = [](Z *dst, int64_t j, int64_t n) {
        double sn, cs;
        sincospi(2.0 * static_cast<double>(j) / static_cast<double>(n), &sn, &cs);
        zstore(dst, Z{df_from(cs), df_from(-sn)});
    };
    if (i < L1) put(tw1 + i, i, L1);
    if (i < L2) put(tw2 + i, i, L2);
    if (i < kTwSplit) put(ta + i, i, L);
    if (i < ntb) put(tb + i, (i * kTwSplit) % L, L);
}

// Columns k0 .. k0+Kc-1 of x (minus frame 0 when ref) into complex rows
// Zr[c][t] = (x_(k0+2c)(t), x_(k0+2c+1)(t)), zero-padded to L, keeping only
// frames t in sZ when mask_s > 1.  Tiles of 32 frames x 32 column pairs
// through shared memory: reads along k, writes along t.
__global__ void fft_gather_kernel(const float *__restrict__ x, int64_t T, int64_t K, int64_t k0, int64_t Kc,
                                  int64_t L, int ref, int64_t mask_s, Z *Zr) {
    __shared__ float tile[32][65];
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * 32, p0 = static_cast<int64_t>(blockIdx.y) * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;     // 32 x 8
    for (int i = ty; i < 32; i += 8) {
        const int64_t t = t0 + i;
        const bool live = t < T && t % mask_s == 0;
        for (int h = 0; h < 2; ++h) {
            const int64_t c = 2 * p0 + 32 * h + tx;      // column within the chunk
            const int64_t k = k0 + c;
            float v = 0.f;
            if (live && c < Kc && k < K) {
                v = x[t * K + k];
                if (ref) v -= x[k];                       // exact in FP32 (nearby values)
            }
            tile[i][32 * h + tx] = v;
        }
    }
    __syncthreads();
    const int64_t npairs = (Kc + 1) / 2;
    for (int i = ty; i < 32; i += 8) {
        const int64_t p = p0 + i, t = t0 + tx;
        if (p < npairs && t < L)
            zstore(Zr + p * L + t, Z{{tile[tx][2 * i], 0.f}, {tile[tx][2 * i + 1], 0.f}});
    }
}

// The same for a handful of columns (Kc <= 8, e.g. a flux series with K = 3):
// one thread per frame.
constexpr int64_t kNarrowGather = 8;
__global__ void fft_gather_narrow_kernel(const float *__restrict__ x, int64_t T, int64_t K, int64_t k0,
                                         int64_t Kc, int64_t L, int ref, int64_t mask_s, Z *Zr) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= L) return;
    const bool live = t < T && t % mask_s == 0;
    for (int64_t p = 0; 2 * p < Kc; ++p) {
        float v[2];
        for (int h = 0; h < 2; ++h) {
            const int64_t c = 2 * p + h, k = k0 + c;
            v[h] = 0.f;
            if (live && c < Kc && k < K) {
                v[h] = x[t * K + k];
                if (ref) v[h] -= x[k];
            }
        }
        zstore(Zr + p * L + t, Z{{v[0], 0.f}, {v[1], 0.f}});
    }
}

// Column pass over the rows of data ([rows][L], each a row-major L1 x L2
// array): block (row, column group) transforms CB adjacent columns n2 of
// length L1.  Forward: then multiplies by W_L^(n2 k1).  Inverse: the plain
// conjugate transform (the row pass applied the conjugate twiddle).
template <bool FWD>
__global__ void __launch_bounds__(kThreads) fft_col_kernel(Z *data, int64_t L, int L1, int L2, int CB,
                                                           const Z *__restrict__ tw1, const Z *__restrict__ ta,
                                                           const Z *__restrict__ tb, Consts K) {
    extern __shared__ __align__(16) Z cbuf[];            // [L1][CB]
    Z *g = data + static_cast<int64_t>(blockIdx.x) * L;
    const int n20 = blockIdx.y * CB;
    const int n = L1 * CB;
    for (int e = threadIdx.x; e < n; e += kThreads) cbuf[e] = zload(g + static_cast<int64_t>(e / CB) * L2 + n20 + e % CB);
    __syncthreads();
    fft_smem(cbuf, L1, CB, 1, CB, FWD ? -1 : 1, tw1, K);
    for (int e = threadIdx.x; e < n; e += kThreads) {
        const int k1 = e / CB, n2 = n20 + e % CB;
        Z v = cbuf[e];
        if (FWD) v = zmul(v, twiddle_L(ta, tb, static_cast<int64_t>(n2) * k1));
        zstore(g + static_cast<int64_t>(k1) * L2 + n2, v);
    }
}

// Row pass, fused: block (row, k1) loads row k1 of data (and of mdata, the
// origin-side signal, when MASK), transforms it forward, forms the power
// spectrum |Z|^2 (or conj(Zm) Z), transforms back and multiplies by
// W_L^(-n2 k1) (skipped when L1 = 1).
template <bool MASK>
__global__ void __launch_bounds__(kThreads) fft_row_kernel(Z *data, const Z *mdata, int64_t L, int L1, int L2,
                                                           const Z *__restrict__ tw2, const Z *__restrict__ ta,
                                                           const Z *__restrict__ tb, Consts K) {
    extern __shared__ __align__(16) Z rbuf[];            // [L2] (+ [L2] origin side)
    const int k1 = blockIdx.y;
    const int64_t off = static_cast<int64_t>(blockIdx.x) * L + static_cast<int64_t>(k1) * L2;
    Z *g = data + off;
    Z *mb = rbuf + L2;
    for (int e = threadIdx.x; e < L2; e += kThreads) {
        rbuf[e] = zload(g + e);
        if (MASK) mb[e] = zload(mdata + off + e);
    }
    __syncthreads();
    fft_smem(rbuf, L2, 1, 0, 1, -1, tw2, K);
    if (MASK) fft_smem(mb, L2, 1, 0, 1, -1, tw2, K);
    for (int e = threadIdx.x; e < L2; e += kThreads) {
        const Z z = rbuf[e];
        rbuf[e] = MASK ? zmulc(z, mb[e]) : Z{df_dot2(z.x, z.x, z.y, z.y), {0.f, 0.f}};
    }
    __syncthreads();
    fft_smem(rbuf, L2, 1, 0, 1, 1, tw2, K);
    for (int e = threadIdx.x; e < L2; e += kThreads) {
        Z v = rbuf[e];
        if (L1 > 1) v = zmulc(v, twiddle_L(ta, tb, static_cast<int64_t>(e) * k1));
        zstore(g + e, v);
    }
}

// D[tau] += (sum over the chunk's rows, in row order, of Re Zr[c][tau]) / L, in FP64.
__global__ void fft_lag_sum_kernel(const Z *Zr, int64_t rows, int64_t L, int64_t tau_max, double *D) {
    const int64_t tau = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tau > tau_max) return;
    double acc = 0.0;
    for (int64_t c = 0; c < rows; ++c) acc += df_to(zload(Zr + c * L + tau).x);
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

// ------------------------------------------------------------------- plan
constexpr int64_t kChunkElems = int64_t(1) << 23;   // complex elements of one chunk buffer (128 MB)

// Smallest L >= n of the form 2^a, 3 2^a or 5 2^a.
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
    int64_t T, N, K, tau_max, s, L, Kc, rows, n_chunks, pstride, ntb;
    int L1, L2, CB;
    size_t off_z, off_zm, off_tw1, off_tw2, off_ta, off_tb, off_d, off_S, off_prefix, total;
};

bool make_fft_layout(int64_t T, int64_t N, int64_t tau_max, int64_t s, int kind, FftLayout *F) {
    F->T = T;
    F->N = N;
    F->K = 3 * N;
    F->tau_max = tau_max;
    F->s = s;
    F->L = fft_length(T + tau_max);
    const int64_t L = F->L;
    if (L <= kMaxL2) {
        F->L1 = 1;
        F->L2 = static_cast<int>(L);
    } else {
        int64_t l1 = 2;
        while (L / l1 > kMaxL2) l1 *= 2;
        if (l1 > kMaxL1 || L % l1 != 0) return false;           // beyond this route's sizes
        F->L1 = static_cast<int>(l1);
        F->L2 = static_cast<int>(L / l1);
    }
    // column group: a power of two dividing L2 with L1 * CB <= kMaxElems
    int cb = kMaxElems / F->L1;
    while (cb > 1 && F->L2 % cb != 0) cb /= 2;
    F->CB = F->L1 > 1 ? cb : 1;
    int64_t rows = kChunkElems / L;
    if (rows < 1) rows = 1;
    F->Kc = 2 * rows < F->K ? 2 * rows : F->K;
    F->rows = (F->Kc + 1) / 2;
    F->n_chunks = ceil_div(F->K, F->Kc);
    F->pstride = (T - 1) / s + 2;
    F->ntb = ceil_div(L, kTwSplit);
    const int64_t n_res = s < tau_max + 1 ? s : tau_max + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t zbytes = sizeof(Z) * static_cast<size_t>(F->rows) * L;
    const bool two = s > 1 || kind == 2;           // a separate origin-side signal
    F->off_z = take(zbytes);
    F->off_zm = take(two ? zbytes : 0);
    F->off_tw1 = take(sizeof(Z) * static_cast<size_t>(F->L1));
    F->off_tw2 = take(sizeof(Z) * static_cast<size_t>(F->L2));
    F->off_ta = take(sizeof(Z) * static_cast<size_t>(kTwSplit));
    F->off_tb = take(sizeof(Z) * static_cast<size_t>(F->ntb));
    F->off_d = take(sizeof(double) * static_cast<size_t>(tau_max + 1));
    F->off_S = take(kind == 0 ? sizeof(double) * static_cast<size_t>(T) : 0);
    F->off_prefix = take(kind == 0 ? sizeof(double) * static_cast<size_t>(n_res * F->pstride) : 0);
    F->total = off;
    return true;
}

Consts host_consts() {
    const double pi = std::acos(-1.0);
    auto split = [](double v) {
        DF d;
        d.h = static_cast<float>(v);
        d.l = static_cast<float>(v - static_cast<double>(d.h));
        return d;
    };
    Consts K;
    K.s3 = split(std::sin(2.0 * pi / 3.0));
    K.c51 = split(std::cos(2.0 * pi / 5.0));
    K.c52 = split(std::cos(4.0 * pi / 5.0));
    K.s51 = split(std::sin(2.0 * pi / 5.0));
    K.s52 = split(std::sin(4.0 * pi / 5.0));
    return K;
}

cudaError_t set_smem_attrs() {
    static cudaError_t done = [] {
        cudaError_t e = cudaFuncSetAttribute(fft_col_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(sizeof(Z) * kMaxElems));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fft_col_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(sizeof(Z) * kMaxElems));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fft_row_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(sizeof(Z) * kMaxL2));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fft_row_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(2 * sizeof(Z) * kMaxL2));
        return e;
    }();
    return done;
}

}  // namespace

// kind 0 (MSD) needs the most of 0 and 1; kind 2 adds the origin-side buffer.
// Host arithmetic only; 0 when the padded length is beyond the route's sizes.
size_t fft_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t s, int kind) {
    FftLayout F;
    if (!make_fft_layout(T, N, tau_max, s, kind, &F)) return 0;
    return F.total;
}

bool fft_supported(int64_t T, int64_t tau_max) {
    FftLayout F;
    return make_fft_layout(T, 1, tau_max, 1, 1, &F);
}

// kind 0 MSD, 1 ACF of d_x; 2 cross-correlation of d_x (origins) with d_y.
int fft_run(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s, double *d_out,
            void *d_ws, size_t ws_bytes, cudaStream_t st, const float *d_y) {
    FftLayout F;
    if (!make_fft_layout(T, N, tau_max, s, kind, &F)) return TCORR_EUNSUPPORTED;
    if (ws_bytes < F.total || !d_ws) return TCORR_EWORKSPACE;
    cudaError_t e = set_smem_attrs();
    if (e != cudaSuccess) return cuda_fail(e, "fft shared-memory attributes");
    const bool two = s > 1 || kind == 2;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    Z *Zr = reinterpret_cast<Z *>(ws + F.off_z);
    Z *Zm = two ? reinterpret_cast<Z *>(ws + F.off_zm) : nullptr;
    Z *tw1 = reinterpret_cast<Z *>(ws + F.off_tw1);
    Z *tw2 = reinterpret_cast<Z *>(ws + F.off_tw2);
    Z *ta = reinterpret_cast<Z *>(ws + F.off_ta);
    Z *tb = reinterpret_cast<Z *>(ws + F.off_tb);
    double *D = reinterpret_cast<double *>(ws + F.off_d);
    const Consts K = host_consts();
    const int64_t L = F.L;
    {
        const int64_t n = std::max<int64_t>(std::max<int64_t>(F.L1, F.L2), std::max<int64_t>(kTwSplit, F.ntb));
        fft_twiddle_kernel<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(tw1, F.L1, tw2, F.L2, ta, tb, L,
                                                                                    F.ntb);
    }
    e = cudaMemsetAsync(D, 0, sizeof(double) * static_cast<size_t>(tau_max + 1), st);
    if (e != cudaSuccess) return cuda_fail(e, "lag-sum reset");
    const size_t col_smem = sizeof(Z) * static_cast<size_t>(F.L1) * F.CB;
    const size_t row_smem = sizeof(Z) * static_cast<size_t>(F.L2) * (two ? 2 : 1);
    for (int64_t ch = 0; ch < F.n_chunks; ++ch) {
        const int64_t k0 = ch * F.Kc;
        const int64_t kc = std::min(F.Kc, F.K - k0);
        const int64_t rows = (kc + 1) / 2;
        auto gather = [&](const float *src, int64_t mask_s, Z *dst) {
            if (kc <= kNarrowGather) {
                fft_gather_narrow_kernel<<<static_cast<unsigned>(ceil_div(L, 256)), 256, 0, st>>>(
                    src, T, F.K, k0, kc, L, kind == 0, mask_s, dst);
            } else {
                const dim3 g(static_cast<unsigned>(ceil_div(L, 32)), static_cast<unsigned>(ceil_div(rows, 32)));
                fft_gather_kernel<<<g, dim3(32, 8), 0, st>>>(src, T, F.K, k0, kc, L, kind == 0, mask_s, dst);
            }
        };
        // later side: B (cross) or the signal itself; origin side: the signal, masked to sZ
        gather(kind == 2 ? d_y : d_x, 1, Zr);
        if (two) gather(d_x, s, Zm);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_gather launch");
        if (F.L1 > 1) {
            const dim3 gc(static_cast<unsigned>(rows), static_cast<unsigned>(F.L2 / F.CB));
            fft_col_kernel<true><<<gc, kThreads, col_smem, st>>>(Zr, L, F.L1, F.L2, F.CB, tw1, ta, tb, K);
            if (two) fft_col_kernel<true><<<gc, kThreads, col_smem, st>>>(Zm, L, F.L1, F.L2, F.CB, tw1, ta, tb, K);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_col launch");
        }
        const dim3 gr(static_cast<unsigned>(rows), static_cast<unsigned>(F.L1));
        if (two) fft_row_kernel<true><<<gr, kThreads, row_smem, st>>>(Zr, Zm, L, F.L1, F.L2, tw2, ta, tb, K);
        else fft_row_kernel<false><<<gr, kThreads, row_smem, st>>>(Zr, nullptr, L, F.L1, F.L2, tw2, ta, tb, K);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_row launch");
        if (F.L1 > 1) {
            const dim3 gc(static_cast<unsigned>(rows), static_cast<unsigned>(F.L2 / F.CB));
            fft_col_kernel<false><<<gc, kThreads, col_smem, st>>>(Zr, L, F.L1, F.L2, F.CB, tw1, ta, tb, K);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fft_col launch");
        }
        // the last chunk's missing column of an odd pair was gathered as zeros and adds nothing
        fft_lag_sum_kernel<<<static_cast<unsigned>(ceil_div(tau_max + 1, 256)), 256, 0, st>>>(Zr, rows, L, tau_max,
                                                                                           D);
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
