// Atom-sharded correlation: the per-lag averages of disjoint atom slices of
// one trajectory combined into the average over all atoms.
//
// The Conclusion of the paper notes that the dynamic data of a species can be
// divided over several devices by atoms, and the parallelisation paragraph
// before Algorithm 11 already gives each thread its own atoms: Eq. 5 averages
// over atoms, and the origin count n_o(tau) is the same for every atom (same T
// and stride).  So if shard r holds N_r atoms and its per-lag average a_r(tau)
// (what tcorr_msd / tcorr_acf return for its slice), the average over all
// atoms is  sum_r N_r a_r(tau) / sum_r N_r.  For weighted averages N_r is the
// shard's weight sum W_r (tcorr_weight_total).
//
// Each rank writes one record [a_r(0) .. a_r(n-1), N_r]; the records of all
// ranks are gathered (all-gather, the one exchange of the path) into rows of
// a [count][ld] array, and tcorr_combine_shards forms the weighted mean with
// FP64 sums in shard order, so every rank gets the same bits whatever the
// collective's own summation order would have been.
#include "tcorr_internal.cuh"

namespace tcorr {

cudaError_t launch_weight_sum(const float *w, int64_t N, double *W, cudaStream_t st);

namespace {

constexpr int kCombineThreads = 256;

// out[i] = sum_r w_r rows[r][i] / sum_r w_r with w_r = rows[r][n], r = 0, 1, ... in order.
__global__ void __launch_bounds__(kCombineThreads) combine_shards_kernel(const double *__restrict__ rows, int64_t n,
                                                                          int64_t count, int64_t ld,
                                                                          double *__restrict__ out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kCombineThreads + threadIdx.x;
    if (i >= n) return;
    double num = 0.0, den = 0.0;
    for (int64_t r = 0; r < count; ++r) {
        const double w = rows[r * ld + n];
        num += w * rows[r * ld + i];
        den += w;
    }
    out[i] = num / den;
}

}  // namespace
}  // namespace tcorr

using namespace tcorr;

extern "C" int tcorr_combine_shards(const double *d_rows, int64_t n, int64_t count, int64_t ld, double *d_out,
                                    void *stream) {
    if (!d_rows || !d_out || n < 1 || count < 1 || ld < n + 1) return TCORR_EINVAL;
    if (count > (int64_t(1) << 40) / ld) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_rows) & 7u) || (reinterpret_cast<uintptr_t>(d_out) & 7u)) return TCORR_EALIGN;
    // the output may not overlap the records it is formed from
    const uintptr_t r0 = reinterpret_cast<uintptr_t>(d_rows);
    const uintptr_t r1 = r0 + static_cast<uintptr_t>((count - 1) * ld + n + 1) * sizeof(double);
    const uintptr_t o0 = reinterpret_cast<uintptr_t>(d_out);
    const uintptr_t o1 = o0 + static_cast<uintptr_t>(n) * sizeof(double);
    if (o0 < r1 && r0 < o1) return TCORR_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    combine_shards_kernel<<<static_cast<unsigned>(ceil_div(n, kCombineThreads)), kCombineThreads, 0, st>>>(
        d_rows, n, count, ld, d_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TCORR_OK : cuda_fail(e, "combine_shards_kernel launch");
}

extern "C" int tcorr_weight_total(const float *d_w, int64_t N, double *d_W, void *stream) {
    if (!d_w || !d_W || N < 1) return TCORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_w) & 3u) || (reinterpret_cast<uintptr_t>(d_W) & 7u)) return TCORR_EALIGN;
    const cudaError_t e = launch_weight_sum(d_w, N, d_W, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? TCORR_OK : cuda_fail(e, "weight_sum_kernel launch");
}
