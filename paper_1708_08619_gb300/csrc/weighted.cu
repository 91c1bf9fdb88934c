// Weighted atom averages: Eq. 5's average "over all the atoms (or a
// subclass)" with atom i counted w_i times (a mass-weighted MSD, or 0/1
// weights for a selection):
//
//   MSD_w(tau) = sum_i w_i sum_{t0} |x_i(t0+tau) - x_i(t0)|^2 / (W n_o(tau)),   W = sum_i w_i,
//
// and likewise for the autocorrelation.  The weighted numerator is the plain
// numerator of y_i = sqrt(w_i) x_i, so the call writes y into its workspace
// (square roots of the weights once, then one pass over x, four atoms per
// thread and step when the rows allow),
// runs the unweighted engine of the chosen method on it and scales the result
// by N / W.  For the MSD, y is taken relative to the middle frame first
// (y_i(t) = sqrt(w_i) (x_i(t) - x_i(m)); the MSD does not see the shift), so
// that the one rounding of each product is relative to the displacement
// scale rather than to the absolute positions.  The weights must be >= 0.
#include <algorithm>
#include <cstdint>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int WCOPY_THREADS = 256;

// sw[i] = sqrt(w[i]).
__global__ void __launch_bounds__(WCOPY_THREADS) weight_sqrt_kernel(const float *__restrict__ w, int64_t N,
                                                                     float *__restrict__ sw) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * WCOPY_THREADS + threadIdx.x; i < N;
         i += static_cast<int64_t>(gridDim.x) * WCOPY_THREADS)
        sw[i] = sqrtf(w[i]);
}

// y[t][i][c] = sw[i] (x[t][i][c] - ref[i][c]) (ref = nullptr: no reference).
// VEC: four atoms per thread and step, three float4 of the row (and of the
// reference row) and one float4 of sw (N % 4 == 0, x 16-byte aligned).
template <bool VEC, bool REF>
__global__ void __launch_bounds__(WCOPY_THREADS) weight_copy_kernel(const float *__restrict__ x,
                                                                     const float *__restrict__ sw, int64_t T,
                                                                     int64_t N, const float *__restrict__ ref,
                                                                     float *__restrict__ y) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * WCOPY_THREADS;
    const int64_t K = 3 * N;
    for (int64_t t = blockIdx.y; t < T; t += gridDim.y) {
        if (VEC) {
            const float4 *x4 = reinterpret_cast<const float4 *>(x + t * K);
            const float4 *r4 = reinterpret_cast<const float4 *>(ref);
            float4 *y4 = reinterpret_cast<float4 *>(y + t * K);
            for (int64_t a = static_cast<int64_t>(blockIdx.x) * WCOPY_THREADS + threadIdx.x; a < N / 4; a += stride) {
                const float4 s4 = __ldg(reinterpret_cast<const float4 *>(sw) + a);
                const float sa[4] = {s4.x, s4.y, s4.z, s4.w};
                float v[12];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float4 f = __ldg(x4 + 3 * a + k);
                    if (REF) {
                        const float4 r = __ldg(r4 + 3 * a + k);
                        f.x -= r.x; f.y -= r.y; f.z -= r.z; f.w -= r.w;
                    }
                    v[4 * k] = f.x; v[4 * k + 1] = f.y; v[4 * k + 2] = f.z; v[4 * k + 3] = f.w;
                }
#pragma unroll
                for (int j = 0; j < 12; ++j) v[j] *= sa[j / 3];
#pragma unroll
                for (int k = 0; k < 3; ++k) y4[3 * a + k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            }
        } else {
            for (int64_t k = static_cast<int64_t>(blockIdx.x) * WCOPY_THREADS + threadIdx.x; k < K; k += stride) {
                float v = __ldg(x + t * K + k);
                if (REF) v -= __ldg(ref + k);
                y[t * K + k] = v * __ldg(sw + k / 3);
            }
        }
    }
}

// W = sum_i w_i in FP64, fixed order (one block).
__global__ void __launch_bounds__(WCOPY_THREADS) weight_sum_kernel(const float *__restrict__ w, int64_t N,
                                                                    double *__restrict__ W) {
    __shared__ double part[WCOPY_THREADS / 32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += WCOPY_THREADS) s += static_cast<double>(w[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
#pragma unroll
        for (int k = 0; k < WCOPY_THREADS / 32; ++k) tot += part[k];
        *W = tot;
    }
}

// out[l] *= N / W: the engine divided by N n_o(tau), the weighted average wants W n_o(tau).
__global__ void weight_rescale_kernel(double *__restrict__ out, int64_t n, int64_t N, const double *__restrict__ W) {
    const int64_t l = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (l < n) out[l] = out[l] * (static_cast<double>(N) / *W);
}

}  // namespace

// Copy region: y (T x 3N floats), W (one double), sqrt(w) (N floats).
size_t weighted_copy_bytes(int64_t T, int64_t N) {
    return align256(static_cast<size_t>(T) * static_cast<size_t>(3 * N) * sizeof(float)) + 256 +
           align256(static_cast<size_t>(N) * sizeof(float));
}

cudaError_t launch_weight_copy(int kind, const float *x, const float *w, int64_t T, int64_t N, void *d_copy,
                               cudaStream_t st) {
    const int64_t K = 3 * N;
    float *y = static_cast<float *>(d_copy);
    double *W = reinterpret_cast<double *>(static_cast<uint8_t *>(d_copy) +
                                           align256(static_cast<size_t>(T) * static_cast<size_t>(K) * sizeof(float)));
    float *sw = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(W) + 256);
    weight_sqrt_kernel<<<static_cast<unsigned>(std::min<int64_t>(ceil_div(N, WCOPY_THREADS), 1024)), WCOPY_THREADS,
                         0, st>>>(w, N, sw);
    weight_sum_kernel<<<1, WCOPY_THREADS, 0, st>>>(w, N, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float *ref = kind == 0 ? x + ((T - 1) / 2) * K : nullptr;
    const bool vec = N % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    const int64_t per_row = vec ? N / 4 : K;
    const dim3 grid(static_cast<unsigned>(std::min<int64_t>(ceil_div(per_row, WCOPY_THREADS), 64)),
                    static_cast<unsigned>(std::min<int64_t>(T, 65535)));
    if (vec) {
        if (ref) weight_copy_kernel<true, true><<<grid, WCOPY_THREADS, 0, st>>>(x, sw, T, N, ref, y);
        else weight_copy_kernel<true, false><<<grid, WCOPY_THREADS, 0, st>>>(x, sw, T, N, ref, y);
    } else {
        if (ref) weight_copy_kernel<false, true><<<grid, WCOPY_THREADS, 0, st>>>(x, sw, T, N, ref, y);
        else weight_copy_kernel<false, false><<<grid, WCOPY_THREADS, 0, st>>>(x, sw, T, N, ref, y);
    }
    return cudaGetLastError();
}

cudaError_t launch_weight_sum(const float *w, int64_t N, double *W, cudaStream_t st) {
    weight_sum_kernel<<<1, WCOPY_THREADS, 0, st>>>(w, N, W);
    return cudaGetLastError();
}

cudaError_t launch_weight_rescale(double *out, int64_t n, int64_t T, int64_t N, const void *d_copy,
                                  cudaStream_t st) {
    const double *W = reinterpret_cast<const double *>(
        static_cast<const uint8_t *>(d_copy) + align256(static_cast<size_t>(T) * static_cast<size_t>(3 * N) * sizeof(float)));
    weight_rescale_kernel<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(out, n, N, W);
    return cudaGetLastError();
}

}  // namespace tcorr
