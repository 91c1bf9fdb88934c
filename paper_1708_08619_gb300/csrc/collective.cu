// Collective (weighted atom-sum) signal of a trajectory:
//
//   J[t][c] = sum_i w_i (x[t][i][c] - x[ref][i][c])   (0 <= ref < T)
//   J[t][c] = sum_i w_i  x[t][i][c]                   (ref = -1)
//
// the input of collective transport quantities: the autocorrelation of a
// current sum_i q_i v_i (Eq. 4 with a collective flux, as the viscosity
// example correlates the pressure tensor of the whole box), the
// Einstein-Helfand MSD of sum_i q_i r_i, or, with 0/1 weights, one species'
// signal for a cross-correlation between species.  The result is written as
// a [T][1][3] float32 trajectory of one "atom", ready for tcorr_msd,
// tcorr_acf and tcorr_xcf with N = 1.
//
// One block per frame, threads strided over the atoms.  Each product w_i v and
// each addition carries its rounding error along (the compensated dot product
// of Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26 (2005): the FMA gives a product's exact error, Knuth's two-sum an
// addition's), so the FP32 pipe delivers about twice the FP32 precision and
// the kernel stays bound by its one read of x from HBM; the per-thread
// (sum, error) pairs are combined in FP64 in a fixed order (deterministic).
// With a reference frame, each block forms that frame's totals once the same
// way and subtracts them in FP64 from every frame's totals: both carry an
// error of about 2^-44 of sum_i |w_i x_i|, far below the final rounding to
// FP32 for unwrapped positions, and J(ref) comes out exactly zero.  Rows of a
// multiple of four atoms, 16-byte aligned, are read as float4 (four atoms =
// three float4 per thread and step).
#include <cstdint>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int COL_THREADS = 256;

// s + e = a + b exactly (Knuth's two-sum); the _rn intrinsics keep the compiler
// from fusing these steps into FMAs, which would break the identity.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// One term w x into (s, e).
__device__ __forceinline__ void add_term(float &s, float &e, float w, float x) {
    const float p = __fmul_rn(w, x);
    const float pe = fmaf(w, x, -p);                      // w x - p, exact
    float q;
    two_sum(s, p, s, q);
    e = __fadd_rn(e, __fadd_rn(pe, q));
}

// This thread's (sum, error) pairs of sum_i w_i row[i][c] over its atoms.
template <bool VEC>
__device__ __forceinline__ void row_partials(const float *__restrict__ row, const float *__restrict__ w, int64_t N,
                                             float (&s)[3], float (&e)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] = e[c] = 0.f;
    if (VEC) {
        // four atoms per step: three float4 of the row
        const float4 *row4 = reinterpret_cast<const float4 *>(row);
        for (int64_t a = threadIdx.x; a < N / 4; a += COL_THREADS) {
            float xv[12], wv[4] = {1.f, 1.f, 1.f, 1.f};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 f = __ldg(row4 + 3 * a + k);
                xv[4 * k] = f.x; xv[4 * k + 1] = f.y; xv[4 * k + 2] = f.z; xv[4 * k + 3] = f.w;
            }
            if (w) {
                const float4 g = __ldg(reinterpret_cast<const float4 *>(w) + a);
                wv[0] = g.x; wv[1] = g.y; wv[2] = g.z; wv[3] = g.w;
            }
#pragma unroll
            for (int j = 0; j < 12; ++j) add_term(s[j % 3], e[j % 3], wv[j / 3], xv[j]);
        }
    } else {
#pragma unroll 4
        for (int64_t i = threadIdx.x; i < N; i += COL_THREADS) {
            const float wi = w ? __ldg(w + i) : 1.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) add_term(s[c], e[c], wi, __ldg(row + 3 * i + c));
        }
    }
}

// Block totals in FP64, fixed order: lane tree within each warp, warps in
// order; the three totals land in tot[] (shared) for every thread.
__device__ __forceinline__ void block_totals(const float (&s)[3], const float (&e)[3],
                                             double (*part)[COL_THREADS / 32], double *tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d = static_cast<double>(s[c]) + static_cast<double>(e[c]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
        if (lane == 0) part[c][warp] = d;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < COL_THREADS / 32; ++k) sum += part[threadIdx.x][k];
        tot[threadIdx.x] = sum;
    }
    __syncthreads();
}

template <bool VEC>
__global__ void __launch_bounds__(COL_THREADS) collective_kernel(const float *__restrict__ x,
                                                                  const float *__restrict__ w, int64_t T,
                                                                  int64_t N, int64_t ref,
                                                                  float *__restrict__ out) {
    __shared__ double part[3][COL_THREADS / 32];
    __shared__ double base[3], tot[3];
    float s[3], e[3];
    if (ref >= 0) {
        row_partials<VEC>(x + ref * 3 * N, w, N, s, e);
        block_totals(s, e, part, base);
    } else if (threadIdx.x < 3) {
        base[threadIdx.x] = 0.0;
    }
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
        row_partials<VEC>(x + t * 3 * N, w, N, s, e);
        block_totals(s, e, part, tot);   // its barriers also order base[] before the reads below
        if (threadIdx.x < 3) out[t * 3 + threadIdx.x] = static_cast<float>(tot[threadIdx.x] - base[threadIdx.x]);
    }
}

}  // namespace

cudaError_t launch_collective(const float *x, const float *w, int64_t T, int64_t N, int64_t ref, float *out,
                              cudaStream_t st) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return cudaErrorInvalidDevice;
    const int64_t cap = static_cast<int64_t>(sms) * 16;
    const unsigned grid = static_cast<unsigned>(T < cap ? T : cap);
    const bool vec = N % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0 &&
                     (w == nullptr || (reinterpret_cast<uintptr_t>(w) & 15u) == 0);
    if (vec) collective_kernel<true><<<grid, COL_THREADS, 0, st>>>(x, w, T, N, ref, out);
    else collective_kernel<false><<<grid, COL_THREADS, 0, st>>>(x, w, T, N, ref, out);
    return cudaGetLastError();
}

}  // namespace tcorr

using namespace tcorr;

extern "C" int tcorr_collective(const float *d_x, const float *d_w, int64_t T, int64_t N, int64_t ref_frame,
                                float *d_out, void *stream) {
    if (!d_x || !d_out || T < 1 || N < 1 || ref_frame < -1 || ref_frame >= T) return TCORR_EINVAL;
    if (N > (INT64_MAX / 12) / T) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_x) & 3u) || (reinterpret_cast<uintptr_t>(d_out) & 3u) ||
        (d_w && (reinterpret_cast<uintptr_t>(d_w) & 3u)))
        return TCORR_EALIGN;
    const uintptr_t o0 = reinterpret_cast<uintptr_t>(d_out), o1 = o0 + sizeof(float) * 3 * T;
    const uintptr_t x0 = reinterpret_cast<uintptr_t>(d_x), x1 = x0 + sizeof(float) * 3 * T * N;
    if (o0 < x1 && x0 < o1) return TCORR_EINVAL;                  // output overlaps the trajectory
    if (d_w) {
        const uintptr_t w0 = reinterpret_cast<uintptr_t>(d_w), w1 = w0 + sizeof(float) * N;
        if (o0 < w1 && w0 < o1) return TCORR_EINVAL;              // output overlaps the weights
    }
    if (launch_collective(d_x, d_w, T, N, ref_frame, d_out, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return TCORR_ECUDA;
    return TCORR_OK;
}
