// Plain FP32 SIMT path: per-origin differences (MSD, Algorithm 11) or
// products (autocorrelation, Algorithm 9), summed over atoms and components.
//
// The paper gives one thread one (lag, atom) pair and lets it walk the
// origins.  Here one block owns a 128 x 128 tile of the origin x frame plane
// (see the band tiling in tcorr_internal.cuh) and walks K = 3N in chunks of
// 16 staged in shared memory; each thread keeps an 8 x 8 register tile of
// pair sums, so every staged value is reused 64 times from registers.
//
//   MSD:  acc(o, f) += (x[f][k] - x[o][k])^2      2 FP32 instructions / k
//   ACF:  acc(o, f) += x[o][k] * x[f][k]          1 FP32 instruction  / k
//
// Accumulation, in three levels so that no FP32 run is long:
//   1. each pair sum over one staged chunk of BK = 16 K elements starts from
//      zero (a run of 16 terms);
//   2. the chunk totals are added into a running FP32 pair sum for a segment
//      of `kseg` K elements (256: a run of 16 chunk totals);
//   3. at the end of a segment the tile goes to shared memory and each thread
//      sums one diagonal (one band offset m = f - o) as eight interleaved
//      chains of eight entries combined in a fixed tree, and adds it to an
//      FP64 accumulator that spans the item's segments.
// A sequential FP32 sum of n positive terms errs by at most (n - 1) 2^-24 of
// the sum; with these levels the longest run is 16 terms, so when every
// origin gives the same pair sum (ballistic motion, where rounding cannot
// average out over origins) the result stays near a few 2^-24 instead of the
// (K - 1) 2^-24 of one run over all of K.  The result of an item is a window
// of per-offset FP64 sums, reduced across items by lag_reduce (reduce.cu).
#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int BO = 128;       // origins per tile
constexpr int BF = 128;       // frame indices per tile
constexpr int BK = 16;        // K elements per pipeline stage
constexpr int NT = 256;       // threads: 16 x 16, 8 x 8 pairs each
constexpr int STAGES = 4;
constexpr int LDS = 132;      // floats per staged k-row (128 + 4, float4 aligned)
constexpr int PLD = 129;      // floats per row of the flush tile
constexpr int WP = 256;       // window width stored per item (>= BO+BF-1)
constexpr size_t SMEM_BYTES = sizeof(float) * (2 * STAGES * BK * LDS + 64 * PLD);

}  // namespace

// One instance of the plain path (also one entry of a batch).
struct PlainArgs {
    const float *x;         // origin rows (A of a cross-correlation)
    const float *xb;        // partner-frame rows: B of a cross-correlation, else x
    int64_t T, K, s, tau_max, n_orig;
    int64_t n_res, n_rows, n_cols, kseg, segs_per_item;
    double *partial;        // [n_items][WP] of this instance
    int64_t item_begin;     // batch: first global block of this instance
    int kind;               // batch: 0 = MSD, 1 = ACF
    int64_t x_elems;        // floats in x and in xb (debug builds check the loads against it)
    int64_t partial_elems;  // doubles in partial (debug builds check the stores against it)
    unsigned int *dbg_status;
};

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const float *src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Row r of a staged k-row lives at column r ^ ((kk >> 3) << 4): the two
// half-warps that store k-rows kk and kk+8 then hit disjoint banks, and every
// aligned group of four rows stays contiguous for float4 reads.
__device__ __forceinline__ int swz(int row, int kk) { return row ^ ((kk >> 3) << 4); }

template <int KIND>
__device__ __forceinline__ void plain_tile_body(const PlainArgs &a, int64_t item_in) {
    extern __shared__ __align__(16) float smem[];
    float *sA = smem;                              // [STAGES][BK][LDS] origin rows
    float *sB = smem + STAGES * BK * LDS;          // [STAGES][BK][LDS] frame rows
    float *sP = smem + 2 * STAGES * BK * LDS;      // [64][PLD] flush tile (half)

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    int64_t item = item_in;
    const int64_t c = item % a.n_cols;
    item /= a.n_cols;
    const int64_t r = item % a.n_rows;
    item /= a.n_rows;
    const int64_t rho = item % a.n_res;
    const int64_t g = item / a.n_res;

    double *outp = a.partial + item_in * WP;
    const int64_t n_rho = n_frames_res(a.T, a.s, rho);
    const int64_t m_max = (a.tau_max - rho) / a.s;
    const int64_t o0 = r * BO;
    const int64_t k0 = o0 + c * BF;
    if (c * BF - BO + 1 > m_max || k0 >= n_rho) {   // no pair of this tile is in the band
        if (TCORR_IN_BOUNDS(item_in * WP + tid, a.partial_elems, a.dbg_status)) outp[tid] = 0.0;
        return;
    }

    // Loader role: thread loads 8 consecutive k of one origin row and one frame row.
    const int lrow = tid >> 1;
    const int lk = (tid & 1) * 8;
    const int lcol = swz(lrow, lk);
    const int64_t oA = o0 + lrow, kB = k0 + lrow;
    const bool vA = oA < a.n_orig, vB = kB < n_rho;
    const float *gA = a.x + (vA ? oA * a.s * a.K : 0);
    const float *gB = a.xb + (vB ? (rho + kB * a.s) * a.K : 0);
    const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);

    const int64_t kbeg = g * a.segs_per_item * a.kseg;
    const int64_t kend = min(a.K, kbeg + a.segs_per_item * a.kseg);

    double dacc = 0.0;   // this thread's diagonal (w = tid), summed over segments

    for (int64_t sb = kbeg; sb < kend; sb += a.kseg) {
        const int64_t se = min(kend, sb + a.kseg);
        const int nch = static_cast<int>(ceil_div(se - sb, BK));

        auto load_chunk = [&](int buf, int64_t kc) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int kk = lk + q;
                const int64_t kg = kc + kk;
                const bool ok = kg < se;
                const uint32_t off = static_cast<uint32_t>(((buf * BK + kk) * LDS + lcol) * 4);
                const bool la = ok && vA && TCORR_IN_BOUNDS(oA * a.s * a.K + kg, a.x_elems, a.dbg_status);
                const bool lb = ok && vB && TCORR_IN_BOUNDS((rho + kB * a.s) * a.K + kg, a.x_elems, a.dbg_status);
                cp_async4(sA0 + off, la ? gA + kg : a.x, la ? 4 : 0);
                cp_async4(sB0 + off, lb ? gB + kg : a.x, lb ? 4 : 0);
            }
        };

        float racc[8][8];   // running pair sums of this segment: chunk totals added in FP32
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) racc[i][j] = 0.f;

#pragma unroll
        for (int st = 0; st < STAGES - 1; ++st) {
            if (st < nch) load_chunk(st, sb + st * BK);
            cp_async_commit();
        }
        for (int ch = 0; ch < nch; ++ch) {
            cp_async_wait<STAGES - 2>();
            __syncthreads();
            const int nxt = ch + STAGES - 1;
            if (nxt < nch) load_chunk(nxt % STAGES, sb + static_cast<int64_t>(nxt) * BK);
            cp_async_commit();

            const float *cA = sA + (ch % STAGES) * BK * LDS;
            const float *cB = sB + (ch % STAGES) * BK * LDS;
            float acc[8][8];    // this chunk's pair sums, a fresh run of BK terms
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(cA + kk * LDS + swz(4 * ty, kk));
                const float4 a1 = *reinterpret_cast<const float4 *>(cA + kk * LDS + swz(64 + 4 * ty, kk));
                const float4 b0 = *reinterpret_cast<const float4 *>(cB + kk * LDS + swz(4 * tx, kk));
                const float4 b1 = *reinterpret_cast<const float4 *>(cB + kk * LDS + swz(64 + 4 * tx, kk));
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (KIND == 0) {
                            const float d = bv[j] - av[i];
                            acc[i][j] = kk == 0 ? d * d : fmaf(d, d, acc[i][j]);
                        } else {
                            acc[i][j] = kk == 0 ? av[i] * bv[j] : fmaf(av[i], bv[j], acc[i][j]);
                        }
                    }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) racc[i][j] += acc[i][j];
        }
        cp_async_wait<0>();

        // Flush: mask pairs outside the band or past the ends, then sum
        // diagonals in a fixed order, one half of the origins at a time.
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int il = 4 * ty + q;          // local origin row within half h
                const int i = 64 * h + il;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = (jj < 4) ? 4 * tx + jj : 64 + 4 * tx + (jj - 4);
                    const int64_t m = c * BF + j - i;
                    const bool ok = (o0 + i < a.n_orig) && (k0 + j < n_rho) && m >= 0 && m <= m_max;
                    sP[il * PLD + j] = ok ? racc[4 * h + q][jj] : 0.f;
                }
            }
            __syncthreads();
            // diagonal w = tid: entries (il, j) with j - (64h + il) + BO - 1 = w,
            // as eight chains (entry il goes to chain il % 8) and a fixed tree
            float sd[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) sd[e] = 0.f;
            const int jb = tid + 64 * h - (BO - 1);
#pragma unroll 2
            for (int il = 0; il < 64; il += 8) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = jb + il + e;
                    if (j >= 0 && j < BF) sd[e] += sP[(il + e) * PLD + j];
                }
            }
            dacc += static_cast<double>(((sd[0] + sd[1]) + (sd[2] + sd[3])) + ((sd[4] + sd[5]) + (sd[6] + sd[7])));
        }
    }
    if (TCORR_IN_BOUNDS(item_in * WP + tid, a.partial_elems, a.dbg_status)) outp[tid] = dacc;
}

template <int KIND>
// One block per SM is enough (the compiler keeps the 8 x 8 tile, the next
// k-slice and the addresses in registers without spilling): measured on the
// mid-size case, MSD unchanged and ACF 8% faster than with two blocks per SM.
__global__ void __launch_bounds__(NT, 1) plain_tile_kernel(const __grid_constant__ PlainArgs a) {
    plain_tile_body<KIND>(a, blockIdx.x);
}

// Batch: block b belongs to the instance whose [item_begin, next item_begin)
// holds b (binary search over the descriptors); the kind is per instance.
__global__ void __launch_bounds__(NT, 1) plain_tile_batch_kernel(const PlainArgs *__restrict__ d, int n) {
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].item_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    __shared__ PlainArgs sa;    // the instance's descriptor, read on demand from shared memory
    if (threadIdx.x == 0) sa = d[lo];
    __syncthreads();
    if (sa.kind == 0) plain_tile_body<0>(sa, b - sa.item_begin);
    else plain_tile_body<1>(sa, b - sa.item_begin);
}

}  // namespace

PlainArgs plain_args(int kind, const float *d_x, const BandPlan &p, double *partial, int64_t item_begin);

cudaError_t launch_plain_tiles(int kind, const float *d_x, const BandPlan &p, double *partial,
                               cudaStream_t st, const float *d_xb) {
    if (p.BO != BO || p.BF != BF || p.WP != WP) return cudaErrorInvalidValue;
    PlainArgs a = plain_args(kind == 2 ? 1 : kind, d_x, p, partial, 0);
    if (kind == 2) a.xb = d_xb;          // cross-correlation: products, B at the later frame
    if (p.n_items <= 0) return cudaSuccess;
    if (p.n_items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (kind == 0) {
        e = cudaFuncSetAttribute(plain_tile_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(SMEM_BYTES));
        if (e != cudaSuccess) return e;
        prof_begin(0, st);
        plain_tile_kernel<0><<<static_cast<unsigned>(p.n_items), NT, SMEM_BYTES, st>>>(a);
        prof_end(st);
    } else {
        e = cudaFuncSetAttribute(plain_tile_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(SMEM_BYTES));
        if (e != cudaSuccess) return e;
        prof_begin(1, st);
        plain_tile_kernel<1><<<static_cast<unsigned>(p.n_items), NT, SMEM_BYTES, st>>>(a);
        prof_end(st);
    }
    return cudaGetLastError();
}

PlainArgs plain_args(int kind, const float *d_x, const BandPlan &p, double *partial, int64_t item_begin) {
    PlainArgs a;
    a.x = d_x;
    a.xb = d_x;
    a.T = p.T;
    a.K = p.K;
    a.s = p.s;
    a.tau_max = p.tau_max;
    a.n_orig = p.n_orig;
    a.n_res = p.n_res;
    a.n_rows = p.n_rows;
    a.n_cols = p.n_cols;
    a.kseg = p.kseg;
    a.segs_per_item = p.segs_per_item;
    a.partial = partial;
    a.item_begin = item_begin;
    a.kind = kind;
    a.x_elems = p.T * p.K;
    a.partial_elems = dbg_shrink_elems(p.n_items * WP, WP);
#ifdef TCORR_DEBUG_BOUNDS
    a.dbg_status = status_word_device_ptr();
#else
    a.dbg_status = nullptr;
#endif
    return a;
}

size_t plain_args_size() { return sizeof(PlainArgs); }

void plain_args_write(void *h_dst, int kind, const float *d_x, const BandPlan &p, double *partial,
                      int64_t item_begin) {
    *static_cast<PlainArgs *>(h_dst) = plain_args(kind, d_x, p, partial, item_begin);
}

cudaError_t launch_plain_tiles_batch(const void *d_descs, int n, int64_t total_items, cudaStream_t st) {
    if (total_items <= 0) return cudaSuccess;
    if (total_items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(plain_tile_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SMEM_BYTES));
    if (e != cudaSuccess) return e;
    plain_tile_batch_kernel<<<static_cast<unsigned>(total_items), NT, SMEM_BYTES, st>>>(
        static_cast<const PlainArgs *>(d_descs), n);
    return cudaGetLastError();
}

int plain_tile_bo() { return BO; }
int plain_tile_bf() { return BF; }
int plain_tile_wp() { return WP; }

}  // namespace tcorr
