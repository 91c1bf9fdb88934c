// Tensor-core banded Gram path (tcgen05, TMA, TMEM) for sm_103a.
//
// The origin x lag sum of Algorithms 9 and 11 is recast as a banded Gram
// product.  With x_t the row of frame t (K = 3N values):
//   ACF:  sum_{t0} x_{t0} . x_{t0+tau}                            = D(tau)
//   MSD:  sum_{t0} |x_{t0+tau} - x_{t0}|^2 = P(tau) + Q(tau) - 2 D(tau)
// where D(tau) sums the Gram entries G(t0, t0+tau) = x_{t0} . x_{t0+tau}
// along one band offset, P(tau) = sum_{t0} S(t0), Q(tau) = sum_{t0} S(t0+tau)
// and S(t) = |x_t|^2 (expanding |a - b|^2 = |a|^2 + |b|^2 - 2 a.b).  For the
// MSD the positions are first referenced to the middle frame m (x_t = r_t - r_m;
// the MSD only sees differences) so that S and G stay small.
//
// Split precision: each FP32 value is written as x = hi + lo with hi and lo in
// a 16-bit (or TF32) format and G is accumulated from hi.hi + hi.lo + lo.hi
// (x3; x4 adds lo.lo) in FP32 in tensor memory.  FP16 operands carry a
// power-of-two scale per (frame, K-group) (so |x| <= 2^14 and hi, lo stay
// normal; a K-group is the K range one work item contracts); BF16 and TF32
// need none.  S(t) is formed from the FP32 values in FP64.
//
// Kernels, in launch order:
//   split_kernel      one block per (frame, K-group): reference, scale,
//                     split, the group's part of S(t)
//   s_combine_kernel  S(t) = sum of the group parts (MSD only)
//   s_prefix_kernel   per-residue FP64 prefix sums of S (MSD only)
//   gram_band_kernel  persistent, warp-specialised band tiles (below)
//   lag_reduce        (reduce.cu) fixed-order FP64 reduction + MSD assembly
// A cross-correlation splits its two signals separately (B into its own
// copies) and skips S; small K uses the polyphase form further down.
//
// gram_band_kernel: one CTA per SM, 10 warps.
//   warp 0     TMA producer: claims work items from a global counter and,
//              per K-block, loads A_hi, A_lo (128 origin rows) and B_hi,
//              B_lo (192 frame rows; the narrow last column tile of a band
//              row only the 32-row boxes it needs) into a 5-stage smem ring
//              (64-byte rows, 64B swizzle).
//   warp 1     allocates TMEM (two 128 x 192 FP32 accumulators)
//              and, from one lane, issues the tcgen05.mma chain.  The chain
//              of a work item is cut into sub-chains (sub_kb K-blocks of 6
//              MMAs each for x3) that alternate between the two
//              accumulators: the tensor core's FP32 accumulation loses low
//              bits on every accumulate step, so a long chain drifts low;
//              short chains keep that loss small.
//   warps 2-9  epilogue: two warps per TMEM lane quadrant, 96 columns each.
//              Each sub-chain's accumulator is read with tcgen05.ld and added
//              (FP32, round to nearest) into a per-thread register copy of
//              its 96 entries; at the end of the item the band mask, the
//              per-(frame, group) unscale and the diagonal sums (band offset
//              w = j - i + 127) go to per-warp shared buffers, and a
//              fixed-order combine writes one FP64 window per work item.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tcorr_internal.cuh"

namespace tcorr {

__device__ unsigned int g_status;   // device status word (TCORR_OK or an error code)

namespace {

constexpr int BO = 128;             // origins per tile (MMA M)
constexpr int BF = 192;             // frames per tile (MMA N)
constexpr int POLY_L = 3 * BO;      // polyphase phases: 384 = 3 row tiles = 2 column tiles
constexpr int STAGES = 5;
constexpr int ROWB = 64;            // bytes of K per staged row = one 64B swizzle span
constexpr int A_BYTES = BO * ROWB;  // 8 KB
constexpr int B_BYTES = BF * ROWB;  // 12 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NBOX = 32;            // B rows per box of the narrow-tile maps (full tiles: one BF box)
constexpr int NBOX_BYTES = NBOX * ROWB;
static_assert(BF % NBOX == 0, "a narrow B tile is a whole number of boxes");
constexpr int NMAPS = 6;            // A hi, A lo, B hi, B lo, then B hi / lo with NBOX-row boxes
constexpr int WPG = 320;            // window width per item (>= BO + BF - 1 = 319)
constexpr int NTHREADS = 320;   // 10 warps
constexpr int NEPI = 8;          // epilogue warps
constexpr uint32_t TMEM_COLS = 512;
// K-blocks per TMEM accumulation sub-chain (defaults).  The tensor core's FP32
// accumulation drifts low by about the same amount per accumulate step, so the
// error grows linearly with the chain while longer chains hand fewer partial
// sums to the epilogue.  The MSD is assembled as P + Q - 2D with D several
// times MSD(tau_max), which multiplies the drift: referenced to frame 0 the
// water-scale MSD erred 3.8 / 8.2 e-6 of MSD(tau_max) at 4 / 8 K-blocks;
// referenced to the middle frame 1.8 / 2.9 / 4.0 e-6 at 4 / 6 / 8 K-blocks
// (launch 7.67 / 7.21 / 7.08 ms).  A correlation is compared with C(0)
// directly (water-scale VACF 0.76 / 1.47 / 2.42 / 3.10 e-6 of C(0) at
// 4 / 8 / 12 / 16 K-blocks, launch 7.70 / 7.41 / 7.27 / 7.18 ms; flux ACF
// 1.3 / 1.7 / 2.7 / 3.6 e-6 at 6 / 8 / 12 / 16, step 8.84 / 8.29 / 7.66 /
// 7.38 ms).
// Chain lengths are set by accuracy per kind, not tuned for speed.
constexpr int kSubKb = 8;          // band form, MSD
constexpr int kSubKbCorr = 12;     // band form, auto- and cross-correlation
constexpr int kSubKbPoly = 12;     // polyphase form (correlations only)

int default_sub_kb(int kind, bool poly) {
    if (poly) return kSubKbPoly;
    return kind == 0 ? kSubKb : kSubKbCorr;
}

// Manual overrides: TCORR_KSEG (K elements per work item, a multiple of 64)
// and TCORR_SUB_KB (K-blocks per accumulation sub-chain, 1..16).  Longer
// sub-chains trade accuracy for fewer accumulator hand-offs.
int64_t env_kseg() {
    const char *e = std::getenv("TCORR_KSEG");
    const long long v = e ? std::atoll(e) : 0;
    return (v >= 64 && v % 64 == 0 && v <= (1 << 20)) ? v : 0;
}
int env_sub_kb() {
    const char *e = std::getenv("TCORR_SUB_KB");
    const int v = e ? std::atoi(e) : 0;
    return (v >= 1 && v <= 16) ? v : 0;
}

// TCORR_SUPER=RxC overrides the supertile of the band items' claim order
// (R row tiles x C column tiles, each 1..4096).
void supertile_env(int64_t *rows, int64_t *cols) {
    if (const char *e = std::getenv("TCORR_SUPER")) {
        long long r = 0, c = 0;
        if (std::sscanf(e, "%lldx%lld", &r, &c) == 2 && r >= 1 && c >= 1 && r <= 4096 && c <= 4096) {
            *rows = r;
            *cols = c;
        }
    }
}

// Band contraction on CTA pairs (gram_pair_kernel) for single instances:
// TCORR_PAIR=0 / 1 first, then the tuned tile shape (tuned >= 0), then the
// default (one-CTA tiles).
constexpr bool kPairDefault = false;
bool pair_enabled(int tuned) {
    if (const char *e = std::getenv("TCORR_PAIR")) return std::strcmp(e, "0") != 0;
    if (tuned >= 0) return tuned != 0;
    return kPairDefault;
}


constexpr unsigned long long kWaitNs = 2000000000ull;

constexpr size_t SMEM_STAGES = size_t(STAGES) * STAGE_BYTES;
constexpr size_t SMEM_LAG = NEPI * WPG * sizeof(float);
constexpr size_t SMEM_CS = BF * sizeof(float);
constexpr size_t SMEM_BAR = 32 * 8;
constexpr int IQ = 4;               // depth of the work-item queue (producer -> MMA, epilogue)
constexpr size_t SMEM_TOTAL = 1024 + SMEM_STAGES + SMEM_LAG + SMEM_CS + SMEM_BAR + 16 + IQ * 8;

enum Prec { P_FP16 = 0, P_BF16 = 1, P_TF32 = 2 };

struct GramArgs {
    int64_t T, s, tau_max, n_orig, n_res, n_rows, n_cols, n_items;
    int64_t kb_total;       // K-blocks that hold data: ceil(K / BKe)
    int64_t kb_per_item;    // K-blocks per work item
    const float *inv_scale; // 2^-e per frame (FP16): [group][scale_stride] (band) or [phase] (polyphase)
    int64_t scale_stride;   // band: T_pad (one row of scales per K-group); polyphase: 0
    const float *inv_scale_b;   // scales of the frame (column) operand: B's for a cross-correlation
    double *partial;        // [n_items][WPG]
    int b3d;                // 0 band, stride 1; 1 band, stride > 1; 2 polyphase (tensor maps)
    int sub_kb;             // K-blocks per accumulation sub-chain
    unsigned long long *counter;   // work-item counter (zeroed before the launch)
    int mode;               // 0 = band tiles, 1 = polyphase blocks
    int64_t nq;             // polyphase: block shifts q = 0 .. nq-1
    int64_t partial_elems;  // doubles in partial (debug builds check the window stores)
    unsigned int *dbg_status;
    int64_t super_rows, super_cols;   // band: supertile of the claim order (row tiles x column tiles)
    const uint8_t *xa_h, *xa_l;       // band: tile images of the origin (A) operand, hi / lo
    const uint8_t *xb_h, *xb_l;       // band: tile images of the frame (B) operand, hi / lo
    int64_t nkp, rows;                // band: tile-image rows per residue / per K-block plane
};

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if it gave up (status word set) or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            const unsigned long long now = globaltimer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kWaitNs) {
                atomicExch(&g_status, static_cast<unsigned int>(TCORR_ETIMEOUT));
                *abort_flag = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int32_t c0,
                                            int32_t c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
// Plain bulk copy global -> shared (contiguous bytes, 16-byte aligned).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
template <int PREC>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (PREC == P_TF32) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}
// 32 lanes x 32 columns of FP32 from TMEM, waited on before returning.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}
// Two 32-column loads in flight, one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, "
        "%43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, "
        "%62, %63}, [%65];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
          "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]),
          "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]),
          "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]),
          "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]), "=r"(v[56]), "=r"(v[57]),
          "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
        : "r"(taddr), "r"(taddr + 32u)
        : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// ---- CTA-pair (cta_group::2) helpers: a cluster of two CTAs on one TPC
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// The address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void st_cluster_u64(uint32_t cluster_addr, int64_t v) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(cluster_addr), "l"(v) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait with cluster-scope acquire (arrivals may come from the peer CTA).
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            const unsigned long long now = globaltimer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kWaitNs) {
                atomicExch(&g_status, static_cast<unsigned int>(TCORR_ETIMEOUT));
                *abort_flag = 1;
                return false;
            }
        }
    }
}
// Tensor copy into this CTA's shared memory that completes on a barrier of
// either CTA of the pair (cluster address `bar`).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map, int32_t c0, int32_t c1,
                                                 uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
// Arrive on barrier `bar` (same offset) in every CTA of `mask` when the MMAs
// this thread issued so far have completed.
__device__ __forceinline__ void tc_commit_pair(uint32_t bar, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 ::"r"(bar), "h"(mask)
                 : "memory");
}
template <int PREC>
__device__ __forceinline__ void tc_mma_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (PREC == P_TF32) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

// Shared-memory matrix descriptor for a K-major tile with 64-byte rows and the
// 64B swizzle: 8-row groups are 512 bytes apart (stride byte offset), the
// leading byte offset is unused for this layout, version field = 1.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(1u) << 16;                  // leading byte offset (unused)
    d |= static_cast<uint64_t>((512u >> 4) & 0x3FFFu) << 32; // stride byte offset
    d |= static_cast<uint64_t>(1u) << 46;                  // descriptor version
    d |= static_cast<uint64_t>(4u) << 61;                  // 64B swizzle
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B K-major, M = 128, N = BF = 192
// (the narrow last tile of a band row overrides N per item).
template <int PREC>
__host__ __device__ constexpr uint32_t make_idesc() {
    return (1u << 4)                                                       // D format F32
           | ((PREC == P_FP16 ? 0u : PREC == P_BF16 ? 1u : 2u) << 7)       // A format
           | ((PREC == P_FP16 ? 0u : PREC == P_BF16 ? 1u : 2u) << 10)      // B format
           | (static_cast<uint32_t>(BF >> 3) << 17)                        // N >> 3
           | (static_cast<uint32_t>(BO >> 4) << 24);                       // M >> 4
}

// One work item, decoded.  A rows start at a_y, B rows at (b_x, b_y, b_z)
// (b_x: extra K offset; b_z: shifted operand copy, polyphase only).  Entry
// (row i, column j) of the tile holds band offset / lag m = moff + j - i,
// kept if 0 <= m <= m_max.  Within the item's K-group g, the FP16 scale of
// row i is inv_scale[g][sa0 + i*sstr] and of column j
// inv_scale_b[g][sb0 + j*sstr] (one row per group; polyphase: per phase).  Only
// columns j < ncol can hold a kept lag (m_max - moff + BO of them, rounded
// up to the MMA's N granularity of 16): the last column tile of a band row
// is issued that narrow.
struct Item {
    int64_t canon;                    // index of the item's partial window (see decode_item)
    int64_t rho, a_y, b_x, b_y, b_z, moff, m_max, kb0, kb1;
    int64_t sa0, sb0, sstr, a_rows;   // a_rows: A rows that hold data (scale lookups)
    int ncol;
    bool empty;
};

__device__ __forceinline__ int item_ncol(int64_t moff, int64_t m_max) {
    const int64_t need = m_max - moff + BO;
    if (need >= BF) return BF;
    return need <= 16 ? 16 : static_cast<int>((need + 15) & ~int64_t(15));
}

// Band items are claimed in supertile order: within one (K-group, residue),
// row tiles are taken super_rows at a time and, inside such a row block,
// column tiles super_cols at a time (column fastest); 16 x 10 by default, the
// autotuner may pick another shape.  The ~152 items in flight then form a
// compact block of the origin x frame plane whose CTAs read the same A rows
// (one row tile, several columns) and overlapping B rows (neighbouring row
// tiles are 128 frames apart) at about the same K-block, so the operands are
// shared in L2.  With column-fastest order over whole rows a band of 53
// column tiles (tau_max = 10000) left only about 3 row tiles in flight and
// each B tile was read from DRAM once per row tile.  The item's partial
// window is stored at its canonical index ((g n_res + rho) n_rows + r) n_cols
// + c, which the lag reduction reads.
__device__ __forceinline__ Item decode_item(const GramArgs &a, int64_t item) {
    Item I;
    int64_t t = item;
    if (a.mode == 0) {
        const int64_t per = a.n_rows * a.n_cols;
        const int64_t gr = t / per;                          // (K-group, residue) block
        int64_t u = t - gr * per;
        const int64_t srows = a.super_rows;
        const int64_t cs = a.n_cols < a.super_cols ? a.n_cols : a.super_cols;
        const int64_t rb = u / (srows * a.n_cols);           // row block (all but the last are full)
        u -= rb * srows * a.n_cols;
        const int64_t rcount = min(srows, a.n_rows - rb * srows);
        const int64_t cb = u / (rcount * cs);                // column block within the row block
        u -= cb * rcount * cs;
        const int64_t ccount = min(cs, a.n_cols - cb * cs);
        const int64_t r = rb * srows + u / ccount;
        const int64_t c = cb * cs + u % ccount;
        I.canon = (gr * a.n_rows + r) * a.n_cols + c;
        I.rho = gr % a.n_res;
        const int64_t g = gr / a.n_res;
        const int64_t o0 = r * BO, k0 = o0 + c * BF;
        I.a_y = o0;
        I.b_x = 0;
        I.b_y = k0;
        I.b_z = I.rho;
        I.moff = c * BF;
        I.m_max = (a.tau_max - I.rho) / a.s;
        I.sa0 = o0 * a.s;
        I.sb0 = I.rho + k0 * a.s;
        I.sstr = a.s;
        I.a_rows = a.n_orig - o0;
        const int64_t n_rho = n_frames_res(a.T, a.s, I.rho);
        I.kb0 = g * a.kb_per_item;
        I.kb1 = min(a.kb_total, I.kb0 + a.kb_per_item);
        I.empty = (c * BF - BO + 1 > I.m_max) || (k0 >= n_rho) || (I.kb0 >= I.kb1);
        I.ncol = item_ncol(I.moff, I.m_max);
    } else {
        // polyphase block (q, h, c) of M_q = sum_p Y[.][p] Y[.][p+q]^T, rows = phases
        I.canon = item;
        const int64_t c = t % 2;
        t /= 2;
        const int64_t h = t % 3;
        t /= 3;
        const int64_t q = t % a.nq;
        const int64_t g = t / a.nq;
        I.rho = 0;
        I.a_y = BO * h;
        I.b_x = q - (q & 7);
        I.b_y = BF * c;
        I.b_z = q & 7;
        I.moff = q * (3 * BO) + BF * c - BO * h;
        I.m_max = a.tau_max;
        I.sa0 = BO * h;
        I.sb0 = BF * c;
        I.sstr = 1;
        I.a_rows = BO;
        I.kb0 = g * a.kb_per_item;
        I.kb1 = min(a.kb_total, I.kb0 + a.kb_per_item);
        I.empty = (I.moff + BF - 1 < 0) || (I.moff - (BO - 1) > a.tau_max) || (I.kb0 >= I.kb1);
        I.ncol = item_ncol(I.moff, I.m_max);
    }
    return I;
}

// Band item of a CTA pair (cta_group::2): row tiles 2 rp (rank 0) and
// 2 rp + 1 (rank 1) against one column tile of frames k0 = 2 rp BO + c BF,
// one M = 256 product whose B rows (frames) are split between the two CTAs:
// rank 0 loads rows k0 .. k0 + ncol/2 - 1, rank 1 the next ncol/2.  Each CTA
// keeps its own 128 x ncol accumulator, whose entry (i, j) holds lag
// m = moff + j - i with moff = c BF - rank BO.  Pair items are claimed in
// supertile order over (pair row, column); emptiness and ncol are decided for
// the pair, so both CTAs agree on them.  The number of row tiles is even in a
// pair layout (a last odd row tile gets a partner whose origins are all past
// the last origin and are masked), and n_cols covers the lags of both ranks.
__device__ __forceinline__ Item decode_pair(const GramArgs &a, int64_t item, int cr) {
    Item I;
    const int64_t n_prow = a.n_rows >> 1;
    const int64_t per = n_prow * a.n_cols;
    const int64_t gr = item / per;
    int64_t u = item - gr * per;
    const int64_t srows = a.super_rows >= 2 ? a.super_rows / 2 : 1;
    const int64_t cs = a.n_cols < a.super_cols ? a.n_cols : a.super_cols;
    const int64_t rb = u / (srows * a.n_cols);
    u -= rb * srows * a.n_cols;
    const int64_t rcount = min(srows, n_prow - rb * srows);
    const int64_t cb = u / (rcount * cs);
    u -= cb * rcount * cs;
    const int64_t ccount = min(cs, a.n_cols - cb * cs);
    const int64_t rp = rb * srows + u / ccount;
    const int64_t c = cb * cs + u % ccount;
    const int64_t r = 2 * rp + cr;
    I.canon = (gr * a.n_rows + r) * a.n_cols + c;
    I.rho = gr % a.n_res;
    const int64_t g = gr / a.n_res;
    const int64_t o0 = r * BO, k0 = 2 * rp * BO + c * BF;
    I.a_y = o0;
    I.b_x = 0;
    I.b_z = I.rho;
    I.moff = k0 - o0;
    I.m_max = (a.tau_max - I.rho) / a.s;
    I.sa0 = o0 * a.s;
    I.sb0 = I.rho + k0 * a.s;
    I.sstr = a.s;
    I.a_rows = a.n_orig - o0;
    const int64_t n_rho = n_frames_res(a.T, a.s, I.rho);
    I.kb0 = g * a.kb_per_item;
    I.kb1 = min(a.kb_total, I.kb0 + a.kb_per_item);
    I.empty = (c * BF - 2 * BO + 1 > I.m_max) || (k0 >= n_rho) || (I.kb0 >= I.kb1);
    const int64_t need = I.m_max - c * BF + 2 * BO;      // columns that can hold a kept lag, either rank
    I.ncol = need >= BF ? BF : (need <= 32 ? 32 : static_cast<int>((need + 31) & ~int64_t(31)));
    I.b_y = k0 + cr * (I.ncol / 2);
    return I;
}

// Where a work item's instance lives: one instance whose tensor maps and
// arguments are kernel parameters, or a batch of instances described in
// device memory (item -> instance by binary search over item offsets).
struct InstDesc {                // CUtensorMap members keep it 64-byte aligned
    CUtensorMap maps[NMAPS];  // A hi, A lo, B hi, B lo, narrow B hi, narrow B lo
    GramArgs ga;
    int64_t item_begin;       // first global work item of this instance
};

struct SrcSingle {
    const CUtensorMap *m[NMAPS];
    const GramArgs *a;
    __device__ __forceinline__ int64_t n_items() const { return a->n_items; }
    __device__ __forceinline__ unsigned long long *counter() const { return a->counter; }
};

struct SrcBatch {
    const InstDesc *d;
    int n;
    int64_t total;
    unsigned long long *ctr;
    __device__ __forceinline__ int64_t n_items() const { return total; }
    __device__ __forceinline__ unsigned long long *counter() const { return ctr; }
    __device__ __forceinline__ const GramArgs *get(int64_t item, int64_t &local, const CUtensorMap *&m0) const {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d[mid].item_begin <= item) lo = mid;
            else hi = mid - 1;
        }
        local = item - d[lo].item_begin;
        m0 = d[lo].maps;
        return &d[lo].ga;
    }
};

// Resolve an item to (its instance's arguments, its four tensor maps, local index).
__device__ __forceinline__ const GramArgs *resolve(const SrcSingle &src, int64_t item, int64_t &local,
                                                   const CUtensorMap *(&maps)[NMAPS]) {
    local = item;
    for (int i = 0; i < NMAPS; ++i) maps[i] = src.m[i];
    return src.a;
}
__device__ __forceinline__ const GramArgs *resolve(const SrcBatch &src, int64_t item, int64_t &local,
                                                   const CUtensorMap *(&maps)[NMAPS]) {
    const CUtensorMap *m0;
    const GramArgs *a = src.get(item, local, m0);
    for (int i = 0; i < NMAPS; ++i) maps[i] = m0 + i;
    return a;
}

// 10 warps: three share one SM sub-partition's 16K registers, so at most
// 168 registers per thread (the epilogue keeps 96 FP32 accumulators).
template <int PREC, bool X4, class Src>
__device__ __forceinline__ void gram_body(const Src &src) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *stages = smem;
    float *lagbuf = reinterpret_cast<float *>(smem + SMEM_STAGES);            // [NEPI][WPG]
    float *cs = reinterpret_cast<float *>(smem + SMEM_STAGES + SMEM_LAG);     // [BF]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SMEM_STAGES + SMEM_LAG + SMEM_CS);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 32);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int64_t *item_q = reinterpret_cast<volatile int64_t *>(tmem_slot + 4);   // [IQ]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int st) { return bar0 + 8u * st; };
    auto empty_bar = [&](int st) { return bar0 + 8u * (STAGES + st); };
    auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
    const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
    auto iq_full_bar = [&](int q) { return bar0 + 8u * (2 * STAGES + 5 + q); };
    auto iq_empty_bar = [&](int q) { return bar0 + 8u * (2 * STAGES + 5 + IQ + q); };

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(full_bar(st), 1);
            mbar_init(empty_bar(st), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), NEPI);
        }
        mbar_init(drain_bar, 1);
        for (int q = 0; q < IQ; ++q) {
            mbar_init(iq_full_bar(q), 1);
            mbar_init(iq_empty_bar(q), 1 + NEPI);   // the MMA thread and one lane per epilogue warp
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp >= 2) {
        for (int i = threadIdx.x - 64; i < NEPI * WPG; i += 32 * NEPI) lagbuf[i] = 0.f;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int64_t n_items = src.n_items();

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        int st = 0;
        uint32_t ph = 0;
        const CUtensorMap *last_map = nullptr;
        unsigned long long *ctr = src.counter();
        for (uint32_t it = 0;; ++it) {
            // claim the next work item and publish it to the MMA and epilogue warps
            const int qs = it % IQ;
            if (!mbar_wait(iq_empty_bar(qs), ((it / IQ) & 1u) ^ 1u, abort_flag)) goto producer_done;
            const int64_t claimed = static_cast<int64_t>(atomicAdd(ctr, 1ull));
            const int64_t item = claimed < n_items ? claimed : -1;
            item_q[qs] = item;
            mbar_arrive(iq_full_bar(qs));
            if (item < 0) break;
            int64_t local;
            const CUtensorMap *mp[NMAPS];
            const GramArgs &a = *resolve(src, item, local, mp);
            const Item I = decode_item(a, local);
            if (I.empty) continue;
            const int b3d = a.b3d;
            // a full tile loads BF rows of B; a narrow one only the NBOX-row groups it uses
            const bool narrow = I.ncol < BF;
            const int nbox = narrow ? (I.ncol + NBOX - 1) / NBOX : 1;
            const int32_t brows = narrow ? NBOX : BF;
            const uint32_t b_bytes = static_cast<uint32_t>(nbox * brows * ROWB);
            const uint32_t stage_tx = 2 * A_BYTES + 2 * b_bytes;
            if (b3d == 2) {
                // polyphase: tensor maps over row-major (K, copy * POLY_L + phase) operands
                if (mp[0] != last_map) {      // new instance: bring its descriptors close to the TMA unit
                    for (int i = 0; i < NMAPS; ++i) prefetch_tensormap(mp[i]);
                    last_map = mp[0];
                }
                const int32_t ay = static_cast<int32_t>(I.a_y), by = static_cast<int32_t>(I.b_y);
                const int32_t bz = static_cast<int32_t>(I.b_z), bx = static_cast<int32_t>(I.b_x);
                const CUtensorMap *mbh = narrow ? mp[4] : mp[2], *mbl = narrow ? mp[5] : mp[3];
                for (int64_t kb = I.kb0; kb < I.kb1; ++kb) {
                    if (!mbar_wait(empty_bar(st), ph ^ 1u, abort_flag)) goto producer_done;
                    mbar_arrive_expect_tx(full_bar(st), stage_tx);
                    const uint32_t sbase = smem_u32(stages + size_t(st) * STAGE_BYTES);
                    const int32_t kx = static_cast<int32_t>(kb * (PREC == P_TF32 ? 16 : 32));
                    tma_load_2d(sbase, mp[0], kx, ay, full_bar(st));
                    tma_load_2d(sbase + A_BYTES, mp[1], kx, ay, full_bar(st));
                    for (int j = 0; j < nbox; ++j) {
                        const uint32_t sh = sbase + 2 * A_BYTES + j * NBOX_BYTES, sl = sh + B_BYTES;
                        tma_load_2d(sh, mbh, kx + bx, bz * POLY_L + by + j * NBOX, full_bar(st));
                        tma_load_2d(sl, mbl, kx + bx, bz * POLY_L + by + j * NBOX, full_bar(st));
                    }
                    if (++st == STAGES) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
            } else {
                // band: each operand tile is one contiguous, pre-swizzled piece of its
                // K-block plane (A: residue 0, rows o0 ..; B: residue rho, rows k0 ..)
                const int64_t ra = I.a_y, rb = I.b_z * a.nkp + I.b_y;
                for (int64_t kb = I.kb0; kb < I.kb1; ++kb) {
                    if (!mbar_wait(empty_bar(st), ph ^ 1u, abort_flag)) goto producer_done;
                    mbar_arrive_expect_tx(full_bar(st), stage_tx);
                    const uint32_t sbase = smem_u32(stages + size_t(st) * STAGE_BYTES);
                    const int64_t plane = kb * a.rows;
                    const int64_t oa = (plane + ra) * ROWB, ob = (plane + rb) * ROWB;
                    bulk_load(sbase, a.xa_h + oa, A_BYTES, full_bar(st));
                    bulk_load(sbase + A_BYTES, a.xa_l + oa, A_BYTES, full_bar(st));
                    bulk_load(sbase + 2 * A_BYTES, a.xb_h + ob, b_bytes, full_bar(st));
                    bulk_load(sbase + 2 * A_BYTES + B_BYTES, a.xb_l + ob, b_bytes, full_bar(st));
                    if (++st == STAGES) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
    producer_done:;
    } else if (warp == 1 && lane == 0) {
        // --------------------------------------------------------------- MMA
        constexpr uint32_t idesc = make_idesc<PREC>();
        int st = 0;
        uint32_t ph = 0, chain = 0;
        bool issued = false, aborted = false;
        for (uint32_t it = 0; !aborted; ++it) {
            const int qs = it % IQ;
            if (!mbar_wait(iq_full_bar(qs), (it / IQ) & 1u, abort_flag)) break;
            const int64_t item = item_q[qs];
            mbar_arrive(iq_empty_bar(qs));
            if (item < 0) break;
            int64_t local;
            const CUtensorMap *mp[NMAPS];
            const GramArgs &a = *resolve(src, item, local, mp);
            const Item I = decode_item(a, local);
            if (I.empty) continue;
            const uint32_t idesc_i = (idesc & ~(0x3Fu << 17)) | (static_cast<uint32_t>(I.ncol >> 3) << 17);
            const int64_t sub_kb = a.sub_kb;
            for (int64_t kc = I.kb0; kc < I.kb1 && !aborted; kc += sub_kb) {
                const int64_t kc1 = min(I.kb1, kc + sub_kb);
                const int b = chain & 1;
                if (!mbar_wait(tempty_bar(b), ((chain >> 1) & 1u) ^ 1u, abort_flag)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + static_cast<uint32_t>(b * BF);
                for (int64_t kb = kc; kb < kc1; ++kb) {
                    if (!mbar_wait(full_bar(st), ph, abort_flag)) {
                        aborted = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sA = smem_u32(stages + size_t(st) * STAGE_BYTES);
                    const uint64_t dAh = smem_desc_sw64(sA);
                    const uint64_t dAl = smem_desc_sw64(sA + A_BYTES);
                    const uint64_t dBh = smem_desc_sw64(sA + 2 * A_BYTES);
                    const uint64_t dBl = smem_desc_sw64(sA + 2 * A_BYTES + B_BYTES);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t adv = static_cast<uint64_t>(ks * 2);   // 32 bytes of K in 16-byte units
                        const uint32_t acc = (kb != kc || ks != 0) ? 1u : 0u;
                        tc_mma<PREC>(d, dAh + adv, dBh + adv, idesc_i, acc);
                        tc_mma<PREC>(d, dAh + adv, dBl + adv, idesc_i, 1u);
                        tc_mma<PREC>(d, dAl + adv, dBh + adv, idesc_i, 1u);
                        if (X4) tc_mma<PREC>(d, dAl + adv, dBl + adv, idesc_i, 1u);
                    }
                    issued = true;
                    tc_commit(empty_bar(st));
                    if (++st == STAGES) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
                if (aborted) break;
                tc_commit(tfull_bar(b));
                ++chain;
            }
        }
        if (issued) {   // wait (bounded) until every MMA this thread issued has completed
            tc_commit(drain_bar);
            int dummy = 0;
            volatile int *never = &dummy;
            mbar_wait(drain_bar, 0u, never);
        }
    } else if (warp >= 2) {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        const int half = (warp - 2) >> 2;     // which 96 accumulator columns
        const int row = 32 * q + lane;        // accumulator row = origin o0 + row
        const int et = threadIdx.x - 64;      // 0 .. 32*NEPI-1
        float *lb = lagbuf + (warp - 2) * WPG;
        uint32_t chain = 0;
        bool aborted = false;
        for (uint32_t it = 0;; ++it) {
            const int qs = it % IQ;
            if (!mbar_wait(iq_full_bar(qs), (it / IQ) & 1u, abort_flag)) break;
            const int64_t item = item_q[qs];
            __syncwarp();
            if (lane == 0) mbar_arrive(iq_empty_bar(qs));
            if (item < 0) break;
            int64_t local;
            const CUtensorMap *mp[NMAPS];
            const GramArgs &a = *resolve(src, item, local, mp);
            int64_t kb0, kb1;
            int ncol;
            float cs_pre = 1.f, rs_pre = 1.f;   // FP16 scales, requested before the sub-chains
            {
                const Item I0 = decode_item(a, local);
                if (I0.empty) {
                    double *outp0 = a.partial + I0.canon * WPG;
                    for (int w = et; w < WPG; w += 32 * NEPI)
                        if (TCORR_IN_BOUNDS(I0.canon * WPG + w, a.partial_elems, a.dbg_status)) outp0[w] = 0.0;
                    continue;
                }
                kb0 = I0.kb0;
                kb1 = I0.kb1;
                ncol = I0.ncol;
                if (PREC == P_FP16) {
                    const int64_t nscale = a.mode == 0 ? a.T : 3 * BO;
                    const int64_t gofs = (I0.kb0 / a.kb_per_item) * a.scale_stride;
                    if (et < BF) {
                        const int64_t f = I0.sb0 + et * I0.sstr;
                        cs_pre = f < nscale ? a.inv_scale_b[gofs + f] : 1.f;
                    }
                    if (row < I0.a_rows) rs_pre = a.inv_scale[gofs + I0.sa0 + row * I0.sstr];
                }
            }
            // columns of this warp's half that the MMA wrote (the rest is stale and masked)
            const int hcols = ncol - (BF / 2) * half;
            const int64_t sub_kb = a.sub_kb;
            float acc2[BF / 2];
#pragma unroll
            for (int j = 0; j < BF / 2; ++j) acc2[j] = 0.f;
            for (int64_t kc = kb0; kc < kb1; kc += sub_kb) {
                const int b = chain & 1;
                if (!mbar_wait(tfull_bar(b), (chain >> 1) & 1u, abort_flag)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem_base + (static_cast<uint32_t>(32 * q) << 16) +
                                       static_cast<uint32_t>(b * BF + (BF / 2) * half);
                if (hcols > 0) {
                    uint32_t v[64];
                    tmem_ld64(tbase, v);
#pragma unroll
                    for (int jj = 0; jj < 64; ++jj) acc2[jj] += __uint_as_float(v[jj]);
                }
                if (hcols > 64) {
                    uint32_t v[32];
                    tmem_ld32(tbase + 64, v);
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) acc2[64 + jj] += __uint_as_float(v[jj]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty_bar(b));
                ++chain;
            }
            if (aborted) break;
            const Item I = decode_item(a, local);     // decoded again: keeps registers free above
            double *outp = a.partial + I.canon * WPG;
            float rs = 1.f;
            if (PREC == P_FP16) {
                if (et < BF) cs[et] = cs_pre;
                rs = rs_pre;
                named_bar_sync(1, 32 * NEPI);
            }
            // Diagonal sums of this warp's 32 x 96 block: entry (lane l, column jj)
            // lies on diagonal d = jj - l in [-31, 95].  Lane L keeps the diagonals
            // d = L - 32 + 32 k (k = 0..3); for each jj it takes the entry of lane
            // (jj - L) mod 32 by a shuffle, whose diagonal is L - 32 + 32 k with
            // k = floor((jj - L) / 32) + 1.  Each diagonal adds its entries in
            // increasing jj, and the sums go to this warp's own slice of lagbuf.
            const int64_t mrow = I.moff - row;        // band offset / lag m = mrow + j
            float dg0 = 0.f, dg1 = 0.f, dg2 = 0.f, dg3 = 0.f;
#pragma unroll
            for (int jj = 0; jj < BF / 2; ++jj) {
                const int j = (BF / 2) * half + jj;
                const int64_t m = mrow + j;
                float val = 0.f;
                if (m >= 0 && m <= I.m_max && row < I.a_rows) {
                    val = acc2[jj];
                    if (PREC == P_FP16) val = (val * rs) * cs[j];
                }
                const float got = __shfl_sync(0xffffffffu, val, (jj - lane) & 31);
                const int k = (jj - lane + 32) >> 5;
                dg0 += k == 0 ? got : 0.f;
                dg1 += k == 1 ? got : 0.f;
                dg2 += k == 2 ? got : 0.f;
                dg3 += k == 3 ? got : 0.f;
            }
            {
                // diagonal d of this block is window slot d + 96 half - 32 q + BO - 1 (0 .. 318)
                float *lw = lb + (BF / 2) * half - 32 * q + (BO - 1) + lane;
                if (lane > 0) lw[-32] = dg0;      // lane 0: d = -32 holds no entry
                lw[0] = dg1;
                lw[32] = dg2;
                lw[64] = dg3;
            }
            named_bar_sync(1, 32 * NEPI);
            for (int w = et; w < WPG; w += 32 * NEPI) {
                float sum = 0.f;
#pragma unroll
                for (int e = 0; e < NEPI; ++e) {
                    sum += lagbuf[e * WPG + w];
                    lagbuf[e * WPG + w] = 0.f;
                }
                if (TCORR_IN_BOUNDS(I.canon * WPG + w, a.partial_elems, a.dbg_status)) outp[w] = static_cast<double>(sum);
            }
            named_bar_sync(1, 32 * NEPI);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

template <int PREC, bool X4>
__global__ void __launch_bounds__(NTHREADS, 1)
    gram_band_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                     const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                     const __grid_constant__ CUtensorMap tmBhn, const __grid_constant__ CUtensorMap tmBln,
                     const __grid_constant__ GramArgs a) {
    SrcSingle src;
    src.m[0] = &tmAh;
    src.m[1] = &tmAl;
    src.m[2] = &tmBh;
    src.m[3] = &tmBl;
    src.m[4] = &tmBhn;
    src.m[5] = &tmBln;
    src.a = &a;
    gram_body<PREC, X4>(src);
}

template <int PREC, bool X4>
__global__ void __launch_bounds__(NTHREADS, 1) gram_band_batch_kernel(const __grid_constant__ SrcBatch src) {
    gram_body<PREC, X4>(src);
}

// ------------------------------------------------------------------ prep
// One block per padded frame row t.  x = X[t] - X[m] (MSD, m the middle frame) or X[t] (ACF);
// FP16 rows are scaled by 2^e_t with e_t chosen so max |x| * 2^e_t < 2^14.
// ---------------------------------------------------- CTA-pair band kernel
// The band contraction on CTA pairs (cta_group::2, clusters of two CTAs on one
// TPC): each pair item is one M = 256 product (the two CTAs' row tiles) over
// one column tile whose B rows are split between the CTAs, so each CTA loads
// its A tile and half of B per K-block: 28 KB instead of 40 KB.  Roles per
// CTA: warp 0 lane 0 loads the CTA's operands (the leader, rank 0, also claims
// the items and publishes them to both CTAs); warp 1 lane 0 of the leader
// issues the MMAs; warps 2..9 are the epilogue of the CTA's own accumulator.
// The operand tiles are read as 2-D views of their tile images (rows of 512
// bytes) by tensor copies that complete on the leader's full barrier, so one
// barrier sees both CTAs' bytes.  Leader barriers count the peer's arrivals
// (tempty: 2 x 8 warps, item slots: 2 + 2 x 8); commits go to both CTAs by
// multicast.  Every wait is bounded as in gram_body.
constexpr int STAGES_P = 7;
constexpr int BH_BYTES = (BF / 2) * ROWB;                    // half of a B tile, 6 KB
constexpr int STAGE_BYTES_P = 2 * A_BYTES + 2 * BH_BYTES;     // 28 KB
constexpr size_t SMEM_STAGES_P = size_t(STAGES_P) * STAGE_BYTES_P;
constexpr size_t SMEM_TOTAL_P = 1024 + SMEM_STAGES_P + SMEM_LAG + SMEM_CS + SMEM_BAR + 16 + IQ * 8;
static_assert(SMEM_TOTAL_P <= 227 * 1024, "pair kernel shared memory");
static_assert(2 * STAGES_P + 5 + 2 * IQ <= 32, "pair kernel barriers");

template <int PREC, bool X4>
__device__ __forceinline__ void gram_pair_body(const GramArgs &a, const CUtensorMap *const *mp) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *stages = smem;
    float *lagbuf = reinterpret_cast<float *>(smem + SMEM_STAGES_P);            // [NEPI][WPG]
    float *cs = reinterpret_cast<float *>(smem + SMEM_STAGES_P + SMEM_LAG);     // [BF]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SMEM_STAGES_P + SMEM_LAG + SMEM_CS);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 32);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int64_t *item_q = reinterpret_cast<volatile int64_t *>(tmem_slot + 4);   // [IQ]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t cr = cluster_rank();
    const bool leader = cr == 0;
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int st) { return bar0 + 8u * st; };
    auto empty_bar = [&](int st) { return bar0 + 8u * (STAGES_P + st); };
    auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES_P + b); };
    auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES_P + 2 + b); };
    const uint32_t drain_bar = bar0 + 8u * (2 * STAGES_P + 4);
    auto iq_full_bar = [&](int q) { return bar0 + 8u * (2 * STAGES_P + 5 + q); };
    auto iq_empty_bar = [&](int q) { return bar0 + 8u * (2 * STAGES_P + 5 + IQ + q); };
    // arrive on a barrier of the leader: locally in the leader, remotely from the peer
    auto arrive_leader = [&](uint32_t bar) {
        if (leader) mbar_arrive(bar);
        else mbar_arrive_cluster(map_to_rank(bar, 0));
    };

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES_P; ++st) {
            mbar_init(full_bar(st), 1);
            mbar_init(empty_bar(st), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), 2 * NEPI);
        }
        mbar_init(drain_bar, 1);
        for (int q = 0; q < IQ; ++q) {
            mbar_init(iq_full_bar(q), 1);
            mbar_init(iq_empty_bar(q), 2 + 2 * NEPI);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp >= 2) {
        for (int i = threadIdx.x - 64; i < NEPI * WPG; i += 32 * NEPI) lagbuf[i] = 0.f;
    }
    if (warp == 1) {   // one allocation for the pair, made by one warp of each CTA together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // both CTAs' barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int64_t n_items = a.n_items;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        int st = 0;
        uint32_t ph = 0;
        unsigned long long *ctr = a.counter;
        for (uint32_t it = 0;; ++it) {
            const int qs = it % IQ;
            int64_t item;
            if (leader) {   // claim the next pair item and publish it to both CTAs
                if (!mbar_wait_cluster(iq_empty_bar(qs), ((it / IQ) & 1u) ^ 1u, abort_flag)) break;
                const int64_t claimed = static_cast<int64_t>(atomicAdd(ctr, 1ull));
                item = claimed < n_items ? claimed : -1;
                item_q[qs] = item;
                st_cluster_u64(map_to_rank(smem_u32(const_cast<int64_t *>(&item_q[qs])), 1), item);
                mbar_arrive(iq_full_bar(qs));
                mbar_arrive_cluster(map_to_rank(iq_full_bar(qs), 1));
            } else {
                if (!mbar_wait_cluster(iq_full_bar(qs), (it / IQ) & 1u, abort_flag)) break;
                item = item_q[qs];
                mbar_arrive_cluster(map_to_rank(iq_empty_bar(qs), 0));
            }
            if (item < 0) break;
            const Item I = decode_pair(a, item, static_cast<int>(cr));
            if (I.empty) continue;
            // each operand tile is a contiguous tile image, read through a 2-D view of
            // 512-byte rows (8 tile rows each); every copy of both CTAs completes on
            // the leader's full barrier, whose expected bytes count both CTAs
            const uint32_t b_bytes = static_cast<uint32_t>(I.ncol / 2) * ROWB;
            const uint32_t pair_tx = 2 * (2 * A_BYTES + 2 * b_bytes);
            const bool narrow = I.ncol < BF;
            const int nbox = narrow ? I.ncol / 32 : 1;          // narrow B half: 1 KB boxes
            const CUtensorMap *mbh = narrow ? mp[4] : mp[2], *mbl = narrow ? mp[5] : mp[3];
            const int64_t ra = I.a_y, rb = I.b_z * a.nkp + I.b_y;
            for (int64_t kb = I.kb0; kb < I.kb1; ++kb) {
                if (!mbar_wait(empty_bar(st), ph ^ 1u, abort_flag)) goto pair_producer_done;
                const uint32_t fb = leader ? full_bar(st) : map_to_rank(full_bar(st), 0);
                if (leader) mbar_arrive_expect_tx(full_bar(st), pair_tx);
                const uint32_t sbase = smem_u32(stages + size_t(st) * STAGE_BYTES_P);
                const int64_t plane = kb * a.rows;
                const int32_t ya = static_cast<int32_t>((plane + ra) >> 3), yb = static_cast<int32_t>((plane + rb) >> 3);
                tma_load_2d_pair(sbase, mp[0], 0, ya, fb);
                tma_load_2d_pair(sbase + A_BYTES, mp[1], 0, ya, fb);
                for (int j = 0; j < nbox; ++j) {
                    tma_load_2d_pair(sbase + 2 * A_BYTES + j * 1024, mbh, 0, yb + 2 * j, fb);
                    tma_load_2d_pair(sbase + 2 * A_BYTES + BH_BYTES + j * 1024, mbl, 0, yb + 2 * j, fb);
                }
                if (++st == STAGES_P) {
                    st = 0;
                    ph ^= 1u;
                }
            }
        }
    pair_producer_done:;
    } else if (warp == 1 && lane == 0 && leader) {
        // --------------------------------------------------------- MMA (leader)
        constexpr uint32_t idesc = (make_idesc<PREC>() & ~(0x1Fu << 24)) | (static_cast<uint32_t>((2 * BO) >> 4) << 24);
        int st = 0;
        uint32_t ph = 0, chain = 0;
        bool issued = false, aborted = false;
        for (uint32_t it = 0; !aborted; ++it) {
            const int qs = it % IQ;
            if (!mbar_wait_cluster(iq_full_bar(qs), (it / IQ) & 1u, abort_flag)) break;
            const int64_t item = item_q[qs];
            arrive_leader(iq_empty_bar(qs));
            if (item < 0) break;
            const Item I = decode_pair(a, item, static_cast<int>(cr));
            if (I.empty) continue;
            const uint32_t idesc_i = (idesc & ~(0x3Fu << 17)) | (static_cast<uint32_t>(I.ncol >> 3) << 17);
            const int64_t sub_kb = a.sub_kb;
            for (int64_t kc = I.kb0; kc < I.kb1 && !aborted; kc += sub_kb) {
                const int64_t kc1 = min(I.kb1, kc + sub_kb);
                const int b = chain & 1;
                if (!mbar_wait_cluster(tempty_bar(b), ((chain >> 1) & 1u) ^ 1u, abort_flag)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + static_cast<uint32_t>(b * BF);
                for (int64_t kb = kc; kb < kc1; ++kb) {
                    if (!mbar_wait(full_bar(st), ph, abort_flag)) {
                        aborted = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sA = smem_u32(stages + size_t(st) * STAGE_BYTES_P);
                    const uint64_t dAh = smem_desc_sw64(sA);
                    const uint64_t dAl = smem_desc_sw64(sA + A_BYTES);
                    const uint64_t dBh = smem_desc_sw64(sA + 2 * A_BYTES);
                    const uint64_t dBl = smem_desc_sw64(sA + 2 * A_BYTES + BH_BYTES);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t adv = static_cast<uint64_t>(ks * 2);
                        const uint32_t acc = (kb != kc || ks != 0) ? 1u : 0u;
                        tc_mma_pair<PREC>(d, dAh + adv, dBh + adv, idesc_i, acc);
                        tc_mma_pair<PREC>(d, dAh + adv, dBl + adv, idesc_i, 1u);
                        tc_mma_pair<PREC>(d, dAl + adv, dBh + adv, idesc_i, 1u);
                        if (X4) tc_mma_pair<PREC>(d, dAl + adv, dBl + adv, idesc_i, 1u);
                    }
                    issued = true;
                    tc_commit_pair(empty_bar(st), 3);
                    if (++st == STAGES_P) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
                if (aborted) break;
                tc_commit_pair(tfull_bar(b), 3);
                ++chain;
            }
        }
        if (issued) {   // wait (bounded) until every MMA issued has completed
            tc_commit_pair(drain_bar, 1);
            int dummy = 0;
            volatile int *never = &dummy;
            mbar_wait_cluster(drain_bar, 0u, never);
        }
    }
    else if (warp >= 2) {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        const int half = (warp - 2) >> 2;     // which 96 accumulator columns
        const int row = 32 * q + lane;        // accumulator row = origin o0 + row
        const int et = threadIdx.x - 64;
        float *lb = lagbuf + (warp - 2) * WPG;
        uint32_t chain = 0;
        bool aborted = false;
        for (uint32_t it = 0;; ++it) {
            const int qs = it % IQ;
            if (!mbar_wait_cluster(iq_full_bar(qs), (it / IQ) & 1u, abort_flag)) break;
            const int64_t item = item_q[qs];
            __syncwarp();
            if (lane == 0) arrive_leader(iq_empty_bar(qs));
            if (item < 0) break;
            int64_t kb0, kb1;
            int ncol;
            float cs_pre = 1.f, rs_pre = 1.f;   // FP16 scales, requested before the sub-chains
            {
                const Item I0 = decode_pair(a, item, static_cast<int>(cr));
                if (I0.empty) {
                    double *outp0 = a.partial + I0.canon * WPG;
                    for (int w = et; w < WPG; w += 32 * NEPI)
                        if (TCORR_IN_BOUNDS(I0.canon * WPG + w, a.partial_elems, a.dbg_status)) outp0[w] = 0.0;
                    continue;
                }
                kb0 = I0.kb0;
                kb1 = I0.kb1;
                ncol = I0.ncol;
                if (PREC == P_FP16) {
                    const int64_t gofs = (I0.kb0 / a.kb_per_item) * a.scale_stride;
                    if (et < BF) {
                        const int64_t f = I0.sb0 + et * I0.sstr;
                        cs_pre = f < a.T ? a.inv_scale_b[gofs + f] : 1.f;
                    }
                    if (row < I0.a_rows) rs_pre = a.inv_scale[gofs + I0.sa0 + row * I0.sstr];
                }
            }
            const int hcols = ncol - (BF / 2) * half;
            const int64_t sub_kb = a.sub_kb;
            float acc2[BF / 2];
#pragma unroll
            for (int j = 0; j < BF / 2; ++j) acc2[j] = 0.f;
            for (int64_t kc = kb0; kc < kb1; kc += sub_kb) {
                const int b = chain & 1;
                if (!mbar_wait(tfull_bar(b), (chain >> 1) & 1u, abort_flag)) {
                    aborted = true;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem_base + (static_cast<uint32_t>(32 * q) << 16) +
                                       static_cast<uint32_t>(b * BF + (BF / 2) * half);
                if (hcols > 0) {
                    uint32_t v[64];
                    tmem_ld64(tbase, v);
#pragma unroll
                    for (int jj = 0; jj < 64; ++jj) acc2[jj] += __uint_as_float(v[jj]);
                }
                if (hcols > 64) {
                    uint32_t v[32];
                    tmem_ld32(tbase + 64, v);
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) acc2[64 + jj] += __uint_as_float(v[jj]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) arrive_leader(tempty_bar(b));
                ++chain;
            }
            if (aborted) break;
            const Item I = decode_pair(a, item, static_cast<int>(cr));
            double *outp = a.partial + I.canon * WPG;
            float rs = 1.f;
            if (PREC == P_FP16) {
                if (et < BF) cs[et] = cs_pre;
                rs = rs_pre;
                named_bar_sync(1, 32 * NEPI);
            }
            // diagonal sums by warp shuffles, as in gram_body
            const int64_t mrow = I.moff - row;
            float dg0 = 0.f, dg1 = 0.f, dg2 = 0.f, dg3 = 0.f;
#pragma unroll
            for (int jj = 0; jj < BF / 2; ++jj) {
                const int j = (BF / 2) * half + jj;
                const int64_t m = mrow + j;
                float val = 0.f;
                if (m >= 0 && m <= I.m_max && row < I.a_rows) {
                    val = acc2[jj];
                    if (PREC == P_FP16) val = (val * rs) * cs[j];
                }
                const float got = __shfl_sync(0xffffffffu, val, (jj - lane) & 31);
                const int k = (jj - lane + 32) >> 5;
                dg0 += k == 0 ? got : 0.f;
                dg1 += k == 1 ? got : 0.f;
                dg2 += k == 2 ? got : 0.f;
                dg3 += k == 3 ? got : 0.f;
            }
            {
                float *lw = lb + (BF / 2) * half - 32 * q + (BO - 1) + lane;
                if (lane > 0) lw[-32] = dg0;
                lw[0] = dg1;
                lw[32] = dg2;
                lw[64] = dg3;
            }
            named_bar_sync(1, 32 * NEPI);
            for (int w = et; w < WPG; w += 32 * NEPI) {
                float sum = 0.f;
#pragma unroll
                for (int e = 0; e < NEPI; ++e) {
                    sum += lagbuf[e * WPG + w];
                    lagbuf[e * WPG + w] = 0.f;
                }
                if (TCORR_IN_BOUNDS(I.canon * WPG + w, a.partial_elems, a.dbg_status)) outp[w] = static_cast<double>(sum);
            }
            named_bar_sync(1, 32 * NEPI);
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // no remote arrival or MMA into this CTA's memory after this point
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

// Maps: A hi / lo (16-row boxes: one 8 KB tile), B hi / lo (12-row boxes: a
// full half tile of 6 KB), B hi / lo (2-row boxes of 1 KB, narrow tiles);
// rows of 512 bytes.
template <int PREC, bool X4>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    gram_pair_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                     const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                     const __grid_constant__ CUtensorMap tmBhn, const __grid_constant__ CUtensorMap tmBln,
                     const __grid_constant__ GramArgs a) {
    const CUtensorMap *mp[NMAPS] = {&tmAh, &tmAl, &tmBh, &tmBl, &tmBhn, &tmBln};
    gram_pair_body<PREC, X4>(a, mp);
}

constexpr int PREP_THREADS = 256;

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Band operand layout (tile images).  K-block kb (64 bytes of K) of frame
// t = rho + kk s sits in row R = rho nkp + kk of plane kb; a plane holds
// rows = s nkp rows, nkp >= n_k + BF per residue, and the rows past n_k are
// zero.  The rows of one tile (consecutive kk of one residue) are then one
// contiguous piece of memory, stored as the 64B-swizzled shared-memory image
// the MMA reads: in row R the 16-byte chunk c sits at position
// c ^ ((R >> 1) & 3).  Tiles start at rows that are multiples of 8, so one
// bulk copy of the piece reproduces the image in shared memory.
__device__ __forceinline__ int64_t tile_chunk_byte(int64_t kb, int64_t R, int64_t rows, int c) {
    return (kb * rows + R) * 64 + (static_cast<int64_t>(c ^ static_cast<int>((R >> 1) & 3)) << 4);
}

// Eight values x scaled (FP16) and split into hi / lo, packed as they are
// stored: two 16-byte vectors each for TF32, one each for FP16 / BF16.
template <int PREC>
__device__ __forceinline__ void split_pack8(const float (&x)[8], float scale, uint4 (&vh)[2], uint4 (&vl)[2]) {
    if (PREC == P_TF32) {
        uint32_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            h[i] = tf32_rna(x[i]);
            l[i] = tf32_rna(x[i] - __uint_as_float(h[i]));
        }
        vh[0] = make_uint4(h[0], h[1], h[2], h[3]);
        vh[1] = make_uint4(h[4], h[5], h[6], h[7]);
        vl[0] = make_uint4(l[0], l[1], l[2], l[3]);
        vl[1] = make_uint4(l[4], l[5], l[6], l[7]);
    } else {
        uint16_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (PREC == P_FP16) {
                const float xs = x[i] * scale;
                const __half hh = __float2half_rn(xs);
                const __half ll = __float2half_rn(xs - __half2float(hh));
                h[i] = __half_as_ushort(hh);
                l[i] = __half_as_ushort(ll);
            } else {
                const __nv_bfloat16 hh = __float2bfloat16_rn(x[i]);
                const __nv_bfloat16 ll = __float2bfloat16_rn(x[i] - __bfloat162float(hh));
                h[i] = __bfloat16_as_ushort(hh);
                l[i] = __bfloat16_as_ushort(ll);
            }
        }
        vh[0] = make_uint4(h[0] | (uint32_t(h[1]) << 16), h[2] | (uint32_t(h[3]) << 16),
                           h[4] | (uint32_t(h[5]) << 16), h[6] | (uint32_t(h[7]) << 16));
        vl[0] = make_uint4(l[0] | (uint32_t(l[1]) << 16), l[2] | (uint32_t(l[3]) << 16),
                           l[4] | (uint32_t(l[5]) << 16), l[6] | (uint32_t(l[7]) << 16));
        vh[1] = vl[1] = make_uint4(0, 0, 0, 0);
    }
}

// Band: the eight values of row R at K positions k0 .. k0+7 (k0 a multiple
// of 8), stored at their tile-image places.
template <int PREC>
__device__ __forceinline__ void split_store8(const float (&x)[8], float scale, void *Xh, void *Xl, int64_t R,
                                             int64_t k0, int64_t rows) {
    uint8_t *bh = static_cast<uint8_t *>(Xh), *bl = static_cast<uint8_t *>(Xl);
    uint4 vh[2], vl[2];
    split_pack8<PREC>(x, scale, vh, vl);
    if (PREC == P_TF32) {
        const int64_t kb = k0 / 16;
        const int c0 = static_cast<int>((k0 % 16) / 4);
        const int64_t o0 = tile_chunk_byte(kb, R, rows, c0), o1 = tile_chunk_byte(kb, R, rows, c0 + 1);
        *reinterpret_cast<uint4 *>(bh + o0) = vh[0];
        *reinterpret_cast<uint4 *>(bh + o1) = vh[1];
        *reinterpret_cast<uint4 *>(bl + o0) = vl[0];
        *reinterpret_cast<uint4 *>(bl + o1) = vl[1];
    } else {
        const int64_t o = tile_chunk_byte(k0 / 32, R, rows, static_cast<int>((k0 % 32) / 8));
        *reinterpret_cast<uint4 *>(bh + o) = vh[0];
        *reinterpret_cast<uint4 *>(bl + o) = vl[0];
    }
}

// Polyphase: the eight values at element offset off of a row-major array.
template <int PREC>
__device__ __forceinline__ void split_store8_rm(const float (&x)[8], float scale, void *Xh, void *Xl, int64_t off) {
    uint4 vh[2], vl[2];
    split_pack8<PREC>(x, scale, vh, vl);
    constexpr int ES = PREC == P_TF32 ? 4 : 2;
    uint4 *ph = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(Xh) + off * ES);
    uint4 *pl = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(Xl) + off * ES);
    ph[0] = vh[0];
    pl[0] = vl[0];
    if (PREC == P_TF32) {
        ph[1] = vh[1];
        pl[1] = vl[1];
    }
}

// Eight consecutive values x = X[t][k..k+7] (- ref[k..k+7] for the MSD),
// zero past K.  VEC: rows are 16-byte aligned and K % 4 == 0 (float4 loads).
template <int KIND, bool VEC>
__device__ __forceinline__ void load8(const float *__restrict__ row, const float *__restrict__ ref, int64_t k,
                                      int64_t K, float (&x)[8]) {
    if (VEC && k + 8 <= K) {
        const float4 a0 = __ldg(reinterpret_cast<const float4 *>(row + k));
        const float4 a1 = __ldg(reinterpret_cast<const float4 *>(row + k + 4));
        x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
        x[4] = a1.x; x[5] = a1.y; x[6] = a1.z; x[7] = a1.w;
        if (KIND == 0) {
            const float4 r0 = __ldg(reinterpret_cast<const float4 *>(ref + k));
            const float4 r1 = __ldg(reinterpret_cast<const float4 *>(ref + k + 4));
            x[0] -= r0.x; x[1] -= r0.y; x[2] -= r0.z; x[3] -= r0.w;
            x[4] -= r1.x; x[5] -= r1.y; x[6] -= r1.z; x[7] -= r1.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t kk = k + i;
            x[i] = kk < K ? (KIND == 0 ? __ldg(row + kk) - __ldg(ref + kk) : __ldg(row + kk)) : 0.f;
        }
    }
}

// One prep entry: an instance's frames cut into K-groups of kseg elements,
// the K range one Gram work item contracts.  The FP16 scale and the FP64
// partial of S(t) are kept per (group, frame): inv_scale[g][T_pad], S[g][T].
struct SplitDesc {
    const float *X;
    const float *ref;         // MSD: the reference frame's row (the middle frame)
    int64_t T, K, Kp, T_pad, kseg, n_groups;
    int64_t s, n_k, nkp, rows;   // tile-image rows: R = (t % s) nkp + t / s, rows = s nkp per plane
    void *Xh, *Xl;
    float *inv_scale;
    double *S;
    int kind, vec;
    int warp_mode;            // groups of at most kWarpSeg columns: one warp per (frame, group)
    int64_t blk_begin;        // batch: first global block of this instance
};

// Groups of up to kWarpSeg columns (small K) are split by one warp each,
// eight frames per block: a 256-thread block per (frame, group) would leave
// most lanes idle and spend more on its reductions than on the data.
constexpr int64_t kWarpSeg = 1024;
constexpr int kWarpFrames = PREP_THREADS / 32;


// Block-wide max of |x| -> power-of-two scale 2^e with max |x| 2^e < 2^14,
// so that FP16 hi and lo stay normal; stores 2^-e for the epilogue.
__device__ __forceinline__ float fp16_scale(float mx, float *red_f, float *inv_out) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((tid & 31) == 0) red_f[tid >> 5] = mx;
    __syncthreads();
    mx = red_f[0];
#pragma unroll
    for (int i = 1; i < PREP_THREADS / 32; ++i) mx = fmaxf(mx, red_f[i]);
    int e = 0;
    if (mx > 0.f) {
        int ex;
        frexpf(mx, &ex);          // mx < 2^ex
        e = 14 - ex;
        e = e < -60 ? -60 : (e > 60 ? 60 : e);
    }
    if (tid == 0) *inv_out = ldexpf(1.f, -e);
    return ldexpf(1.f, e);
}

// One block per (padded frame t, K-group g): x = r_t - r_m (MSD) or A_t
// (ACF) over the group's columns, scaled (FP16) and split into hi/lo, and the
// group's part of S(t) = |x_t|^2 in FP64.  A group of up to 8 x 2048 columns
// is held in registers: one read from DRAM, then the max, then the stores.
template <int PREC, int KIND, bool VEC>
__device__ __forceinline__ void split_body(const SplitDesc &q, int64_t R, int64_t g) {
    __shared__ float red_f[PREP_THREADS / 32];
    __shared__ double red_d[PREP_THREADS / 32];
    __shared__ float inv_dummy;
    const int tid = threadIdx.x;
    const float *X = q.X;
    const int64_t rho = R / q.nkp, kk = R - rho * q.nkp;
    const int64_t t = rho + kk * q.s;
    const bool real = kk < q.n_k;              // a frame < T_pad (else a zero pad row)
    const bool live = real && t < q.T;
    const float *row = X + (live ? t : 0) * q.K;
    const int64_t Klive = live ? q.K : 0;      // padding rows are all zero
    const int64_t kb = g * q.kseg;
    const int64_t ke = g == q.n_groups - 1 ? q.Kp : min(q.Kp, kb + q.kseg);
    constexpr int64_t STEP = PREP_THREADS * 8;
    constexpr int NCH = 8;
    float *inv_out = real ? q.inv_scale + g * q.T_pad + t : &inv_dummy;
    float scale = 1.f;
    double sacc = 0.0;
    if (ke - kb <= NCH * STEP) {
        float x[NCH][8];
        float mx = 0.f;
        // every chunk of the row is requested first (the loads from DRAM all in flight at
        // once); the MSD's reference-frame values (L2-resident) follow half the chunks at a
        // time, so that the registers hold the row plus half a row of references
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int64_t k0 = kb + c * STEP + static_cast<int64_t>(tid) * 8;
            if (k0 < ke) {
                load8<1, VEC>(row, X, k0, Klive, x[c]);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) x[c][i] = 0.f;
            }
        }
        constexpr int NH = KIND == 0 ? NCH / 2 : NCH;
#pragma unroll
        for (int h = 0; h < NCH / NH; ++h) {
            float r[KIND == 0 ? NH : 1][8];
            if (KIND == 0) {
#pragma unroll
                for (int cc = 0; cc < NH; ++cc) {
                    const int64_t k0 = kb + (h * NH + cc) * STEP + static_cast<int64_t>(tid) * 8;
                    if (k0 < ke) {
                        load8<1, VEC>(q.ref, q.ref, k0, Klive, r[cc]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) r[cc][i] = 0.f;
                    }
                }
            }
#pragma unroll
            for (int cc = 0; cc < NH; ++cc) {
                const int c = h * NH + cc;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (KIND == 0) x[c][i] -= r[cc][i];
                    mx = fmaxf(mx, fabsf(x[c][i]));
                }
            }
        }
        if (PREC == P_FP16) scale = fp16_scale(mx, red_f, inv_out);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int64_t k0 = kb + c * STEP + static_cast<int64_t>(tid) * 8;
            if (k0 < ke) {
                if (KIND == 0) {
                    float sq = 0.f;
#pragma unroll
                    for (int i = 0; i < 8; ++i) sq = fmaf(x[c][i], x[c][i], sq);
                    sacc += static_cast<double>(sq);
                }
                split_store8<PREC>(x[c], scale, q.Xh, q.Xl, R, k0, q.rows);
            }
        }
    } else {
        // a longer group: a max pass, then the conversion pass (second read from L2)
        if (PREC == P_FP16) {
            float mx = 0.f;
            for (int64_t k0 = kb + static_cast<int64_t>(tid) * 8; k0 < ke; k0 += STEP) {
                float x[8];
                load8<KIND, VEC>(row, q.ref, k0, Klive, x);
#pragma unroll
                for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(x[i]));
            }
            scale = fp16_scale(mx, red_f, inv_out);
        }
        for (int64_t k0 = kb + static_cast<int64_t>(tid) * 8; k0 < ke; k0 += STEP) {
            float x[8];
            load8<KIND, VEC>(row, q.ref, k0, Klive, x);
            if (KIND == 0) {
                float sq = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) sq = fmaf(x[i], x[i], sq);
                sacc += static_cast<double>(sq);
            }
            split_store8<PREC>(x, scale, q.Xh, q.Xl, R, k0, q.rows);
        }
    }
    if (KIND == 0 && q.S != nullptr) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
        if ((tid & 31) == 0) red_d[tid >> 5] = sacc;
        __syncthreads();
        if (tid == 0 && live) {
            double tot = 0.0;
#pragma unroll
            for (int i = 0; i < PREP_THREADS / 32; ++i) tot += red_d[i];
            q.S[g * q.T + t] = tot;
        }
    }
}

// One warp per (frame t, K-group g) of at most kWarpSeg columns: the same
// values as split_body, with warp shuffles in place of block reductions.
template <int PREC, int KIND, bool VEC>
__device__ __forceinline__ void split_warp_body(const SplitDesc &q, int64_t R, int64_t g) {
    if (R >= q.rows) return;                   // past the last row of the plane (whole warp)
    const int lane = threadIdx.x & 31;
    const float *X = q.X;
    const int64_t rho = R / q.nkp, kk = R - rho * q.nkp;
    const int64_t t = rho + kk * q.s;
    const bool real = kk < q.n_k;
    const bool live = real && t < q.T;
    const float *row = X + (live ? t : 0) * q.K;
    const int64_t Klive = live ? q.K : 0;
    const int64_t kb = g * q.kseg;
    const int64_t ke = g == q.n_groups - 1 ? q.Kp : min(q.Kp, kb + q.kseg);
    constexpr int NCW = static_cast<int>(kWarpSeg / 256);    // 8 columns per lane per chunk
    float x[NCW][8];
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < NCW; ++c) {
        const int64_t k0 = kb + c * 256 + lane * 8;
        if (k0 < ke) {
            load8<KIND, VEC>(row, q.ref, k0, Klive, x[c]);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[c][i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(x[c][i]));
    }
    float scale = 1.f;
    if (PREC == P_FP16) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        int e = 0;
        if (mx > 0.f) {
            int ex;
            frexpf(mx, &ex);
            e = 14 - ex;
            e = e < -60 ? -60 : (e > 60 ? 60 : e);
        }
        scale = ldexpf(1.f, e);
        if (lane == 0 && real) q.inv_scale[g * q.T_pad + t] = ldexpf(1.f, -e);
    }
    double sacc = 0.0;
#pragma unroll
    for (int c = 0; c < NCW; ++c) {
        const int64_t k0 = kb + c * 256 + lane * 8;
        if (k0 < ke) {
            if (KIND == 0) {
                float sq = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) sq = fmaf(x[c][i], x[c][i], sq);
                sacc += static_cast<double>(sq);
            }
            split_store8<PREC>(x[c], scale, q.Xh, q.Xl, R, k0, q.rows);
        }
    }
    if (KIND == 0 && q.S != nullptr) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
        if (lane == 0 && live) q.S[g * q.T + t] = sacc;
    }
}

template <int PREC, int KIND, bool VEC>
__global__ void __launch_bounds__(PREP_THREADS, 2) split_kernel(const __grid_constant__ SplitDesc q) {
    split_body<PREC, KIND, VEC>(q, blockIdx.x, blockIdx.y);
}

template <int PREC, int KIND, bool VEC>
__global__ void __launch_bounds__(PREP_THREADS, 2) split_warp_kernel(const __grid_constant__ SplitDesc q) {
    split_warp_body<PREC, KIND, VEC>(q, static_cast<int64_t>(blockIdx.x) * kWarpFrames + (threadIdx.x >> 5),
                                     blockIdx.y);
}

// Batch: the instances of one prep class (kind, float4 loads, warp mode) in
// one grid, block -> instance by binary search; each class is its own
// specialisation, so the kernel carries only the registers its class needs.
template <int PREC, int KIND, bool VEC, bool WARP>
__global__ void __launch_bounds__(PREP_THREADS, 2) split_batch_kernel(const SplitDesc *__restrict__ d, int n) {
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].blk_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const SplitDesc &q = d[lo];
    const int64_t local = b - q.blk_begin;
    const int64_t tb = local / q.n_groups, g = local - tb * q.n_groups;
    if (WARP) split_warp_body<PREC, KIND, VEC>(q, tb * kWarpFrames + (threadIdx.x >> 5), g);
    else split_body<PREC, KIND, VEC>(q, tb, g);
}

// prefix[rho][j] = sum_{j' < j} S(rho + j' s), j = 0 .. n_rho.  One block per
// residue; each thread owns a contiguous chunk; chunk totals are scanned with
// a fixed warp-shuffle tree, so the result does not depend on timing.
constexpr int PFX_THREADS = 1024;

__device__ __forceinline__ double block_exclusive_scan(double v, double *warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += u;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        double x = lane < (blockDim.x >> 5) ? warp_tot[lane] : 0.0;
        double xi = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, xi, off);
            if (lane >= off) xi += u;
        }
        warp_tot[lane] = xi - x;     // exclusive prefix of warp totals
    }
    __syncthreads();
    return warp_tot[w] + (inc - v);
}

// S(f) = sum over K-groups g of S[g][f], added in group order.
__device__ __forceinline__ double s_total(const double *S, int64_t T, int64_t n_groups, int64_t f) {
    double v = 0.0;
    for (int64_t g = 0; g < n_groups; ++g) v += S[g * T + f];
    return v;
}

__device__ __forceinline__ void s_prefix_body(const double *S, int64_t T, int64_t n_groups, int64_t s,
                                              int64_t pstride, double *prefix, int64_t rho) {
    __shared__ double warp_tot[32];
    const int tid = threadIdx.x;
    const int64_t n = n_frames_res(T, s, rho);
    double *pr = prefix + rho * pstride;
    const int64_t per = ceil_div(n > 0 ? n : 1, PFX_THREADS);
    const int64_t b = tid * per, e = min(n, b + per);
    double acc = 0.0;
    for (int64_t j = b; j < e; ++j) acc += s_total(S, T, n_groups, rho + j * s);
    double run = block_exclusive_scan(acc, warp_tot);
    if (tid == 0) pr[0] = 0.0;
    for (int64_t j = b; j < e; ++j) {
        run += s_total(S, T, n_groups, rho + j * s);
        pr[j + 1] = run;
    }
}

__global__ void __launch_bounds__(PFX_THREADS) s_prefix_kernel(const double *S, int64_t T, int64_t n_groups,
                                                                int64_t s, int64_t pstride, double *prefix) {
    s_prefix_body(S, T, n_groups, s, pstride, prefix, blockIdx.x);
}

// S[0][f] = sum over K-groups g of S[g][f] (group order), in place: then
// the prefix pass reads one value per frame.
__global__ void s_combine_kernel(double *S, int64_t T, int64_t n_groups) {
    const int64_t f = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (f >= T) return;
    S[f] = s_total(S, T, n_groups, f);
}

struct PfxDesc {
    const double *S;
    int64_t T, n_groups, s, pstride;
    double *prefix;
    int64_t blk_begin;        // first global block (residue) of this instance
    int64_t frame_begin;      // first global frame of this instance (S combine pass)
};

// Batch: S[0][f] = sum over groups of S[g][f] for every frame of every MSD
// instance, one thread per (instance, frame).
__global__ void s_combine_batch_kernel(const PfxDesc *__restrict__ d, int n, int64_t total) {
    const int64_t f = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (f >= total) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].frame_begin <= f) lo = mid;
        else hi = mid - 1;
    }
    const PfxDesc &q = d[lo];
    double *S = const_cast<double *>(q.S);
    const int64_t t = f - q.frame_begin;
    S[t] = s_total(S, q.T, q.n_groups, t);
}

__global__ void __launch_bounds__(PFX_THREADS) s_prefix_batch_kernel(const PfxDesc *__restrict__ d, int n) {
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].blk_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const PfxDesc &q = d[lo];
    s_prefix_body(q.S, q.T, q.n_groups, q.s, q.pstride, q.prefix, b - q.blk_begin);
}

// ------------------------------------------------------------- polyphase
// Small K (a few series, e.g. the three off-diagonal pressure components):
// with L = 384 phases, Y[j][(series, p)] = a_series(p L + j) and
// M_q = sum_p Y[.][p] Y[.][p+q]^T; entry (j, j') of M_q is the sum of
// a(t) a(t + tau) over origins t = p L + j with tau = q L + j' - j.  The
// shift q of the contraction index is split into an aligned part (a TMA
// coordinate) and q mod 8, served by one of 8 copies of Y pre-shifted by
// 0..7 elements.  Each series occupies Pp >= P + nq slots of the contraction
// so that shifted reads never reach the next series.

struct PolyPrepArgs {
    const float *X;
    int64_t T, K, P, Pp, Kprime, Kalloc;
    void *Yh, *Yl;                   // [8][L][Kalloc]
    float *inv_scale;                // [L]
    unsigned *rowmax;                // [L] FP16: bits of the largest |value| per phase row (zeroed first)
    int kind;
    int ncopies;                     // shifted copies written: 8, or 1 for the origin side of a cross-correlation
    int64_t rm_begin, tile_begin;    // batch: first row-max block / prep tile of this instance
};

constexpr int RM_P = 16;                          // frame blocks p per row-max block
constexpr int PT_K = 32;                          // contraction columns per prep tile
constexpr int PT_ROWS = PT_K + 7;                 // + the largest copy shift
constexpr int PT_LD = POLY_L + 1;                 // shared row stride (floats), conflict-free reads
constexpr size_t PT_SMEM = size_t(PT_ROWS) * PT_LD * sizeof(float) + POLY_L * sizeof(float) +
                           2 * PT_ROWS * sizeof(int);
static_assert(POLY_L > PREP_THREADS && POLY_L <= 2 * PREP_THREADS, "two phases per prep thread");

__host__ __device__ __forceinline__ int64_t poly_rm_blocks(int64_t P) { return (P + RM_P - 1) / RM_P; }
__host__ __device__ __forceinline__ int64_t poly_tiles(int64_t Kalloc) { return Kalloc / PT_K; }

// FP16 only: largest |value| of each phase row j over all series and frame
// blocks, one block per RM_P frame blocks (384 threads, one per phase, reads
// consecutive frames), folded into rowmax[] with an unsigned max on the bit
// pattern (order-preserving for non-negative floats).
__device__ __forceinline__ void poly_rowmax_body(const PolyPrepArgs &a, int64_t blk) {
    const int j = threadIdx.x;
    const int64_t p0 = blk * RM_P;
    float mx = 0.f;
#pragma unroll 4
    for (int dp = 0; dp < RM_P; ++dp) {
        const int64_t t = (p0 + dp) * POLY_L + j;
        if (p0 + dp >= a.P || t >= a.T) break;
        for (int64_t ser = 0; ser < a.K; ++ser) {
            const float v = a.X[t * a.K + ser];
            mx = fmaxf(mx, fabsf(a.kind == 0 ? v - a.X[ser] : v));
        }
    }
    if (mx > 0.f) atomicMax(a.rowmax + j, __float_as_uint(mx));
}

__global__ void __launch_bounds__(POLY_L) poly_rowmax_kernel(const __grid_constant__ PolyPrepArgs a) {
    poly_rowmax_body(a, blockIdx.x);
}

__global__ void __launch_bounds__(POLY_L) poly_rowmax_batch_kernel(const PolyPrepArgs *__restrict__ d, int n) {
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].rm_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    poly_rowmax_body(d[lo], b - d[lo].rm_begin);
}

// One block per tile of PT_K contraction columns [k0, k0 + PT_K): stages the
// values of columns k0 .. k0 + PT_K + 6 for all 384 phases in shared memory
// (reads along phases, i.e. consecutive frames), then writes the 8 copies
// Y_r[j][k] = value(j, k + r) as hi/lo pairs, 8 consecutive k per thread.
template <int PREC>
__device__ __forceinline__ void poly_split_body(const PolyPrepArgs &a, int64_t tile, float *sm) {
    float *V = sm;                                   // [PT_ROWS][PT_LD]
    float *sc = sm + PT_ROWS * PT_LD;                // [L] per-row scale
    int *rser = reinterpret_cast<int *>(sc + POLY_L);    // [PT_ROWS] series of column k0 + row
    int *rp = rser + PT_ROWS;                        // [PT_ROWS] its frame block, -1: zero column
    const int tid = threadIdx.x;
    const int k0 = static_cast<int>(tile) * PT_K;
    if (tid < PT_ROWS) {
        const int kk = k0 + tid;
        const int Pp = static_cast<int>(a.Pp);
        const int ser = kk / Pp, p = kk - ser * Pp;
        rser[tid] = ser;
        rp[tid] = (kk < a.Kprime && p < a.P) ? p : -1;
    }
    for (int j = tid; j < POLY_L; j += PREP_THREADS) {
        float s = 1.f;
        if (PREC == P_FP16) {
            const float mx = __uint_as_float(a.rowmax[j]);
            int e = 0;
            if (mx > 0.f) {
                int ex;
                frexpf(mx, &ex);
                e = 14 - ex;
                e = e < -60 ? -60 : (e > 60 ? 60 : e);
            }
            s = ldexpf(1.f, e);
            if (tile == 0) a.inv_scale[j] = ldexpf(1.f, -e);
        }
        sc[j] = s;
    }
    __syncthreads();
    // phases j = tid and tid + 256 of every staged column: consecutive frames,
    // independent loads (unrolled) so that many are in flight per thread
    const bool two = tid < POLY_L - PREP_THREADS;
#pragma unroll 13
    for (int row = 0; row < PT_ROWS; ++row) {
        const int p = rp[row], ser = rser[row];
        float v0 = 0.f, v1 = 0.f;
        if (p >= 0) {
            const int64_t t0 = static_cast<int64_t>(p) * POLY_L + tid;
            const float ref = a.kind == 0 ? a.X[ser] : 0.f;
            if (t0 < a.T) v0 = a.X[t0 * a.K + ser] - ref;
            if (two && t0 + PREP_THREADS < a.T) v1 = a.X[(t0 + PREP_THREADS) * a.K + ser] - ref;
        }
        V[row * PT_LD + tid] = v0;
        if (two) V[row * PT_LD + tid + PREP_THREADS] = v1;
    }
    __syncthreads();
    const int units = a.ncopies * POLY_L * (PT_K / 8);   // (copy r, phase j, octet) -> 8 elements
    for (int u = tid; u < units; u += PREP_THREADS) {
        const int oct = u & (PT_K / 8 - 1);
        const int rj = u / (PT_K / 8);
        const int r = rj / POLY_L, j = rj - r * POLY_L;
        float x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = V[(oct * 8 + r + i) * PT_LD + j];
        const int64_t off = (static_cast<int64_t>(r) * POLY_L + j) * a.Kalloc + k0 + oct * 8;
        split_store8_rm<PREC>(x, sc[j], a.Yh, a.Yl, off);
    }
}

template <int PREC>
__global__ void __launch_bounds__(PREP_THREADS) poly_split_kernel(const __grid_constant__ PolyPrepArgs a) {
    extern __shared__ __align__(16) float poly_sm[];
    poly_split_body<PREC>(a, blockIdx.x, poly_sm);
}

// Batch: tiles of all instances in one grid; tile -> instance by binary search.
template <int PREC>
__global__ void __launch_bounds__(PREP_THREADS) poly_split_batch_kernel(const PolyPrepArgs *__restrict__ d, int n) {
    extern __shared__ __align__(16) float poly_sm[];
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].tile_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    poly_split_body<PREC>(d[lo], b - d[lo].tile_begin, poly_sm);
}

// S(t) = |x_t|^2 (FP64) for the polyphase MSD: one thread per frame.
__global__ void poly_s_kernel(const float *X, int64_t T, int64_t K, double *S) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double acc = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        const double d = static_cast<double>(X[t * K + k] - X[k]);
        acc += d * d;
    }
    S[t] = acc;
}

struct PolyReduceArgs {
    const double *partial;
    int64_t T, N, tau_max, nq, n_groups;
    int kind;
    const double *S_prefix;          // kind 0: prefix sums of S, T+1 entries
    double *out;
    int64_t lag_begin;               // batch: first global lag of this instance
};

// One thread per lag.  Block (g, q, h, c) holds lag tau at window slot
// w = tau + 128 h - 192 c + 127 - q L; the window (319 slots) is shorter
// than L, so for each (g, h, c) only q = floor(base / L) can hold it.  The
// terms are added in the fixed order g, h, c; neighbouring lags read
// neighbouring slots.
__device__ __forceinline__ void poly_reduce_body(const PolyReduceArgs &a, int64_t tau) {
    double sum = 0.0;
    const int nq = static_cast<int>(a.nq);
    for (int64_t g = 0; g < a.n_groups; ++g) {
#pragma unroll
        for (int hc = 0; hc < 6; ++hc) {
            const int h = hc >> 1, c = hc & 1;
            const int base = static_cast<int>(tau) + BO * h - BF * c + (BO - 1);
            if (base < 0) continue;
            const int q = base / POLY_L;
            const int w = base - q * POLY_L;
            if (q >= nq || w > BO + BF - 2) continue;
            const int64_t item = ((g * nq + q) * 3 + h) * 2 + c;
            sum += a.partial[item * WPG + w];
        }
    }
    const int64_t no = a.T - tau;
    const double denom = static_cast<double>(a.N) * static_cast<double>(no);
    double v;
    if (a.kind != 0) {             // autocorrelation or cross-correlation
        v = sum / denom;
    } else if (tau == 0) {
        v = 0.0;
    } else {
        const double P = a.S_prefix[no];
        const double Q = a.S_prefix[a.T] - a.S_prefix[tau];
        v = (P + Q - 2.0 * sum) / denom;
    }
    a.out[tau] = v;
}

__global__ void poly_reduce_kernel(const __grid_constant__ PolyReduceArgs a) {
    const int64_t tau = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tau > a.tau_max) return;
    poly_reduce_body(a, tau);
}

__global__ void poly_reduce_batch_kernel(const PolyReduceArgs *__restrict__ d, int n, int64_t total) {
    const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].lag_begin <= g) lo = mid;
        else hi = mid - 1;
    }
    poly_reduce_body(d[lo], g - d[lo].lag_begin);
}

// ------------------------------------------------------------------ host
struct GramLayout {
    BandPlan p;
    int prec;
    bool x4;
    int64_t Kp, T_pad, n_k, esize, bke, pstride, kseg;
    int sub_kb;
    int super_rows = kDefaultSuperRows, super_cols = kDefaultSuperCols;   // band claim order
    int64_t nkp = 0, rows = 0;      // band tile images: rows per residue (>= n_k + 2 BO) and per plane (s nkp)
    bool pair = false;              // band on CTA pairs (gram_pair_kernel)
    bool poly;                      // polyphase layout (small K, stride 1)
    int64_t P, Pp, nq, Kprime, Kalloc;
    size_t off_xh, off_xl, off_scale, off_S, off_prefix, off_partial, off_counter, total;
    bool cross = false;             // cross-correlation: B operand from a second signal
    size_t off_bh = 0, off_bl = 0, off_scale_b = 0;
};

bool method_prec(int method, int *prec, bool *x4) {
    switch (method) {
        case TCORR_TC_FP16X3: *prec = P_FP16; *x4 = false; return true;
        case TCORR_TC_BF16X3: *prec = P_BF16; *x4 = false; return true;
        case TCORR_TC_BF16X4: *prec = P_BF16; *x4 = true; return true;
        case TCORR_TC_TF32X3: *prec = P_TF32; *x4 = false; return true;
        default: return false;
    }
}

// Polyphase pays off when K is too small to fill an MMA's K dimension and
// the lag range spans at least one phase block.
bool use_polyphase(int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    if (std::getenv("TCORR_NO_POLYPHASE")) return false;
    return s == 1 && 3 * N <= 24 && tau_max + 1 >= POLY_L && T >= POLY_L;
}

bool make_poly_layout(int64_t T, int64_t N, int64_t tau_max, int method, int kind, GramLayout *L) {
    (void)method;
    const int64_t K = 3 * N;
    L->P = ceil_div(T, POLY_L);
    L->nq = (tau_max + POLY_L - 1) / POLY_L + 1;
    L->Pp = ceil_div(L->P + L->nq + 1, 64) * 64;
    L->Kprime = K * L->Pp;
    L->Kalloc = ceil_div(L->Kprime + L->nq + 8, 64) * 64;
    L->Kp = L->Kalloc;
    if (L->Kalloc >= (int64_t(1) << 31)) return false;
    const int64_t kb_total = ceil_div(L->Kprime, L->bke);
    {
        TuneChoice c{tune_default_kseg(L->Kprime, 6 * L->nq, 2), 0};
        if (const TuneChoice *o = get_tune_override()) c = *o;
        if (const int64_t ek = env_kseg()) c.kseg = ek;
        if (c.sub_kb <= 0) c.sub_kb = default_sub_kb(kind, true);
        if (const int es = env_sub_kb()) c.sub_kb = es;
        L->kseg = c.kseg;
        L->sub_kb = c.sub_kb;
    }
    const int64_t kb_per_item = L->kseg / L->bke;
    L->p = BandPlan{};
    L->p.T = T;
    L->p.N = N;
    L->p.K = K;
    L->p.tau_max = tau_max;
    L->p.s = 1;
    L->p.n_orig = T;
    L->p.n_res = 1;
    L->p.BO = BO;
    L->p.BF = BF;
    L->p.WP = WPG;
    L->p.n_groups = ceil_div(kb_total, kb_per_item);
    L->p.n_items = L->p.n_groups * L->nq * 6;
    L->T_pad = T;
    L->n_k = T;
    L->pstride = T + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t copies = size_t(8) * POLY_L * L->Kalloc * L->esize;
    L->cross = kind == 2;
    // a cross-correlation reads only the unshifted copy of its origin-side signal A
    L->off_xh = take(L->cross ? copies / 8 : copies);
    L->off_xl = take(L->cross ? copies / 8 : copies);
    L->off_scale = take(size_t(2 * POLY_L) * sizeof(float));      // inv_scale, then row maxima
    if (L->cross) {
        L->off_bh = take(copies);
        L->off_bl = take(copies);
        L->off_scale_b = take(size_t(2 * POLY_L) * sizeof(float));
    }
    L->off_S = take(kind == 0 ? size_t(T) * sizeof(double) : 0);
    L->off_prefix = take(kind == 0 ? size_t(T + 1) * sizeof(double) : 0);
    L->off_partial = take(size_t(L->p.n_items) * WPG * sizeof(double));
    L->off_counter = take(sizeof(unsigned long long));
    L->total = off;
    return true;
}

// w != nullptr: one window of a streamed trajectory (band form only: the
// polyphase contraction cannot stop origins at a cap).
bool make_layout(int64_t T, int64_t N, int64_t tau_max, int64_t s, int method, int kind, GramLayout *L,
                 const Window *w = nullptr, bool allow_pair = false) {
    if (!method_prec(method, &L->prec, &L->x4)) return false;
    L->esize = L->prec == P_TF32 ? 4 : 2;
    L->bke = L->prec == P_TF32 ? 16 : 32;
    const int64_t K = 3 * N;
    L->cross = kind == 2;
    L->poly = !w && use_polyphase(T, N, tau_max, s);
    if (L->poly) return make_poly_layout(T, N, tau_max, method, kind, L);
    L->Kp = ceil_div(K, 64) * 64;
    L->n_k = ceil_div(T, s);
    L->nkp = ceil_div(L->n_k + 2 * BO, 8) * 8;   // a tile starting at a real row never leaves its residue
    L->rows = s * L->nkp;
    L->T_pad = L->n_k * s;           // rows rho + k s for every rho < s, k < n_k exist
    // kseg / sub_kb / supertile / tile shape: tuning override, then environment, then tuned
    // cache, then defaults
    int tuned_pair = -1;
    {
        const BandPlan p0 = make_band_plan(T, N, tau_max, s, BO, BF, 64, 1);
        const int64_t tiles = p0.n_res * p0.n_rows * p0.n_cols;
        TuneChoice c{tune_default_kseg(K, tiles, p0.n_cols), 0};
        TuneChoice cached;
        if (const TuneChoice *o = get_tune_override()) c = *o;
        else if (tune_mode() != 0 && tune_lookup(tune_key(method, kind, K, tau_max, T, s), &cached)) c = cached;
        if (const int64_t ek = env_kseg()) c.kseg = ek;
        if (c.sub_kb <= 0) c.sub_kb = default_sub_kb(kind, false);
        if (const int es = env_sub_kb()) c.sub_kb = es;
        L->kseg = c.kseg;
        L->sub_kb = c.sub_kb;
        tuned_pair = c.pair;
        if (c.super_rows > 0 && c.super_cols > 0) {
            L->super_rows = c.super_rows;
            L->super_cols = c.super_cols;
        }
    }
    L->p = make_band_plan(T, N, tau_max, s, BO, BF, L->kseg, 1);
    if (w) cap_origins(&L->p, w->orig_cap);
    L->p.WP = WPG;
    L->pair = allow_pair && pair_enabled(tuned_pair);
    if (L->pair) {   // an even number of row tiles; columns for the lags of both ranks of a pair
        L->p.pair = 1;
        L->p.n_rows = ceil_div(L->p.n_rows, 2) * 2;
        L->p.n_cols = ceil_div(2 * BO + L->p.m_max0, BF);
    }
    // one K group per segment of kseg elements
    const int64_t kb_total = ceil_div(K, L->bke);
    const int64_t kb_per_item = L->kseg / L->bke;
    L->p.n_groups = ceil_div(kb_total, kb_per_item);
    L->p.segs_per_item = 1;
    L->p.n_items = L->p.n_groups * L->p.n_res * L->p.n_rows * L->p.n_cols;
    L->pstride = (T - 1) / s + 2;
    // TMA coordinates are 32-bit
    if (L->Kp >= (int64_t(1) << 31) || L->rows >= (int64_t(1) << 31)) return false;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L->off_xh = take(size_t(L->rows) * L->Kp * L->esize);
    L->off_xl = take(size_t(L->rows) * L->Kp * L->esize);
    L->off_scale = take(size_t(L->p.n_groups) * L->T_pad * sizeof(float));
    if (L->cross) {
        L->off_bh = take(size_t(L->rows) * L->Kp * L->esize);
        L->off_bl = take(size_t(L->rows) * L->Kp * L->esize);
        L->off_scale_b = take(size_t(L->p.n_groups) * L->T_pad * sizeof(float));
    }
    L->off_S = take(kind == 0 ? size_t(L->p.n_groups) * T * sizeof(double) : 0);
    L->off_prefix = take(kind == 0 ? size_t(L->p.n_res) * L->pstride * sizeof(double) : 0);
    L->off_partial = take(size_t(L->p.n_items) * WPG * sizeof(double));
    L->off_counter = take(sizeof(unsigned long long));
    L->total = off;
    return true;
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

bool device_is_sm103(int *num_sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    return major == 10 && minor == 3;
}

template <int PREC, bool X4>
cudaError_t launch_gram(const CUtensorMap *maps, const GramArgs &ga, int grid, cudaStream_t st, int kind) {
    cudaError_t e = cudaFuncSetAttribute(gram_band_kernel<PREC, X4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SMEM_TOTAL));
    if (e != cudaSuccess) return e;
    prof_begin(kind, st);
    gram_band_kernel<PREC, X4><<<grid, NTHREADS, SMEM_TOTAL, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4],
                                                                      maps[5], ga);
    prof_end(st);
    return cudaGetLastError();
}

template <int PREC, bool X4>
cudaError_t launch_gram_pair(const CUtensorMap *maps, const GramArgs &ga, int grid, cudaStream_t st, int kind) {
    cudaError_t e = cudaFuncSetAttribute(gram_pair_kernel<PREC, X4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SMEM_TOTAL_P));
    if (e != cudaSuccess) return e;
    prof_begin(kind, st);
    gram_pair_kernel<PREC, X4><<<grid, NTHREADS, SMEM_TOTAL_P, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4],
                                                                      maps[5], ga);
    prof_end(st);
    return cudaGetLastError();
}

template <int PREC, bool X4>
cudaError_t launch_gram_batch(const SrcBatch &src, int grid, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(gram_band_batch_kernel<PREC, X4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SMEM_TOTAL));
    if (e != cudaSuccess) return e;
    prof_begin(2, st);
    gram_band_batch_kernel<PREC, X4><<<grid, NTHREADS, SMEM_TOTAL, st>>>(src);
    prof_end(st);
    return cudaGetLastError();
}

// Prep mode of a layout: one warp per (frame, group) when no group is longer
// than kWarpSeg columns (the last group runs to Kp), else one block.
bool split_warp_mode(const GramLayout &L) {
    const int64_t kseg = (L.kseg / L.bke) * L.bke;
    const int64_t last = L.Kp - (L.p.n_groups - 1) * kseg;
    return (kseg > last ? kseg : last) <= kWarpSeg;
}

int64_t split_block_count(const GramLayout &L) {
    return split_warp_mode(L) ? ceil_div(L.rows, kWarpFrames) * L.p.n_groups : L.rows * L.p.n_groups;
}

// The MSD is unchanged by a constant shift of an atom's positions, so any
// frame may serve as the reference x_t = r_t - r_ref.  The middle frame keeps
// |x_t|^2, and with it the Gram sum D that P + Q - 2D cancels, about half as
// large as frame 0 does for a diffusive walk (a quarter for ballistic motion),
// which halves the effect of the tensor core's accumulation drift on the MSD.
int64_t msd_ref_frame(int64_t T) { return (T - 1) / 2; }

SplitDesc split_desc(int kind, const float *X, const GramLayout &L, uint8_t *base, int64_t blk_begin) {
    SplitDesc q;
    q.X = X;
    q.ref = X + msd_ref_frame(L.p.T) * L.p.K;
    q.T = L.p.T;
    q.K = L.p.K;
    q.Kp = L.Kp;
    q.s = L.p.s;
    q.n_k = L.n_k;
    q.nkp = L.nkp;
    q.rows = L.rows;
    q.T_pad = L.T_pad;
    q.kseg = (L.kseg / L.bke) * L.bke;     // the K range of one Gram work item
    q.n_groups = L.p.n_groups;
    q.Xh = base + L.off_xh;
    q.Xl = base + L.off_xl;
    q.inv_scale = reinterpret_cast<float *>(base + L.off_scale);
    q.S = kind == 0 ? reinterpret_cast<double *>(base + L.off_S) : nullptr;
    q.kind = kind;
    q.vec = (q.K % 4 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
    q.warp_mode = split_warp_mode(L) ? 1 : 0;
    q.blk_begin = blk_begin;
    return q;
}

template <int PREC>
cudaError_t launch_split(const SplitDesc &q, cudaStream_t st) {
    if (q.n_groups > 65535 || q.rows > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (q.warp_mode) {
        const dim3 gw(static_cast<unsigned>(ceil_div(q.rows, kWarpFrames)), static_cast<unsigned>(q.n_groups));
        if (q.kind == 0) {
            if (q.vec) split_warp_kernel<PREC, 0, true><<<gw, PREP_THREADS, 0, st>>>(q);
            else split_warp_kernel<PREC, 0, false><<<gw, PREP_THREADS, 0, st>>>(q);
        } else {
            if (q.vec) split_warp_kernel<PREC, 1, true><<<gw, PREP_THREADS, 0, st>>>(q);
            else split_warp_kernel<PREC, 1, false><<<gw, PREP_THREADS, 0, st>>>(q);
        }
        return cudaGetLastError();
    }
    const dim3 g(static_cast<unsigned>(q.rows), static_cast<unsigned>(q.n_groups));
    if (q.kind == 0) {
        if (q.vec) split_kernel<PREC, 0, true><<<g, PREP_THREADS, 0, st>>>(q);
        else split_kernel<PREC, 0, false><<<g, PREP_THREADS, 0, st>>>(q);
    } else {
        if (q.vec) split_kernel<PREC, 1, true><<<g, PREP_THREADS, 0, st>>>(q);
        else split_kernel<PREC, 1, false><<<g, PREP_THREADS, 0, st>>>(q);
    }
    return cudaGetLastError();
}

// Prep class of a batch entry: kind (0 MSD, 1 ACF), float4 loads, warp mode.
int split_class(const SplitDesc &q) { return q.kind * 4 + q.vec * 2 + q.warp_mode; }

template <int PREC>
cudaError_t launch_split_batch_class(int cls, const SplitDesc *d, int n, int64_t blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned g = static_cast<unsigned>(blocks);
    switch (cls) {
        case 0: split_batch_kernel<PREC, 0, false, false><<<g, PREP_THREADS, 0, st>>>(d, n); break;
        case 1: split_batch_kernel<PREC, 0, false, true><<<g, PREP_THREADS, 0, st>>>(d, n); break;
        case 2: split_batch_kernel<PREC, 0, true, false><<<g, PREP_THREADS, 0, st>>>(d, n); break;
        case 3: split_batch_kernel<PREC, 0, true, true><<<g, PREP_THREADS, 0, st>>>(d, n); break;
        case 4: split_batch_kernel<PREC, 1, false, false><<<g, PREP_THREADS, 0, st>>>(d, n); break;
        case 5: split_batch_kernel<PREC, 1, false, true><<<g, PREP_THREADS, 0, st>>>(d, n); break;
        case 6: split_batch_kernel<PREC, 1, true, false><<<g, PREP_THREADS, 0, st>>>(d, n); break;
        default: split_batch_kernel<PREC, 1, true, true><<<g, PREP_THREADS, 0, st>>>(d, n); break;
    }
    return cudaGetLastError();
}

// Tensor maps of one instance: A rows are origins o (frame o s); B rows are
// frames rho + k s (2-D map for s = 1, (K, residue, frame index) for s > 1).
// The band operands are read as tile images by plain bulk copies, so a band
// instance carries no tensor maps: its map slots are zeroed (only polyphase
// instances, whose maps poly_setup encodes, touch them).
int encode_maps(const GramLayout &, uint8_t *, int64_t, CUtensorMap *maps) {
    std::memset(maps, 0, sizeof(CUtensorMap) * NMAPS);
    return TCORR_OK;
}

// CTA-pair kernel maps: each operand's tile images as a 2-D array of 512-byte
// rows (8 tile rows each; 512 / esize elements per row), no swizzle (the
// images are stored swizzled), boxes of 16 rows (A), 12 rows (full B half) and
// 2 rows (narrow B halves in 1 KB steps).
int encode_pair_maps(const GramLayout &L, uint8_t *base, CUtensorMap *maps) {
    EncodeFn encode = get_encode();
    if (!encode) return TCORR_EUNSUPPORTED;
    const CUtensorMapDataType dt = L.prec == P_FP16   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : L.prec == P_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t per_row = static_cast<cuuint64_t>(512 / L.esize);
    const cuuint64_t n512 = static_cast<cuuint64_t>(L.Kp / L.bke) * static_cast<cuuint64_t>(L.rows) / 8;
    const cuuint64_t dim[2] = {per_row, n512};
    const cuuint64_t str[1] = {512};
    const cuuint32_t es[2] = {1, 1};
    uint8_t *bufs[4] = {base + L.off_xh, base + L.off_xl, base + (L.cross ? L.off_bh : L.off_xh),
                        base + (L.cross ? L.off_bl : L.off_xl)};
    const int buf_of[NMAPS] = {0, 1, 2, 3, 2, 3};
    const cuuint32_t rows_of[NMAPS] = {16, 16, 12, 12, 2, 2};
    for (int i = 0; i < NMAPS; ++i) {
        const cuuint32_t box[2] = {static_cast<cuuint32_t>(per_row), rows_of[i]};
        if (encode(&maps[i], dt, 2, bufs[buf_of[i]], dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cuda_fail(cudaErrorInvalidValue, "cuTensorMapEncodeTiled (pair)");
    }
    return TCORR_OK;
}

GramArgs gram_args(const GramLayout &L, uint8_t *base, int64_t T, int64_t N, int64_t tau_max, int64_t s) {
    GramArgs ga{};
    ga.mode = 0;
    ga.nq = 0;
    ga.T = T;
    ga.s = s;
    ga.tau_max = tau_max;
    ga.n_orig = L.p.n_orig;
    ga.n_res = L.p.n_res;
    ga.n_rows = L.p.n_rows;
    ga.n_cols = L.p.n_cols;
    ga.n_items = L.pair ? L.p.n_items / 2 : L.p.n_items;   // pair items cover two row tiles
    ga.kb_total = ceil_div(3 * N, L.bke);
    ga.kb_per_item = L.kseg / L.bke;
    ga.inv_scale = reinterpret_cast<const float *>(base + L.off_scale);
    ga.scale_stride = L.T_pad;
    ga.inv_scale_b = reinterpret_cast<const float *>(base + (L.cross ? L.off_scale_b : L.off_scale));
    ga.partial = reinterpret_cast<double *>(base + L.off_partial);
    ga.b3d = s > 1 ? 1 : 0;
    ga.sub_kb = L.sub_kb;
    ga.counter = reinterpret_cast<unsigned long long *>(base + L.off_counter);
    ga.partial_elems = dbg_shrink_elems(L.p.n_items * WPG, WPG);
#ifdef TCORR_DEBUG_BOUNDS
    ga.dbg_status = status_word_device_ptr();
#else
    ga.dbg_status = nullptr;
#endif
    ga.super_rows = L.super_rows;
    ga.super_cols = L.super_cols;
    supertile_env(&ga.super_rows, &ga.super_cols);
    ga.xa_h = base + L.off_xh;
    ga.xa_l = base + L.off_xl;
    ga.xb_h = base + (L.cross ? L.off_bh : L.off_xh);
    ga.xb_l = base + (L.cross ? L.off_bl : L.off_xl);
    ga.nkp = L.nkp;
    ga.rows = L.rows;
    return ga;
}

FinalizeArgs finalize_args(int kind, const GramLayout &L, uint8_t *base) {
    FinalizeArgs fa{kind == 0 ? 1 : 0, kind == 0 ? reinterpret_cast<const double *>(base + L.off_prefix) : nullptr,
                    L.pstride};
    return fa;
}

// Batch plan: instances in decreasing order of tensor work (longest first),
// each with its own workspace region after the descriptor arrays.
struct BatchLayout {
    int n = 0, n_msd = 0, prec = 0;
    bool x4 = false;
    std::vector<int> order;
    std::vector<GramLayout> L;
    std::vector<size_t> base;
    size_t off_inst = 0, off_split = 0, off_pfx = 0, off_red = 0, off_counter = 0, total = 0;
    size_t off_pprep = 0, off_pred = 0, off_rowmax = 0;
    int64_t total_items = 0, total_frames = 0, total_pfx = 0, total_lags = 0;
};

bool make_batch_layout(const tcorr_instance *items, int count, int method, BatchLayout *B) {
    if (!method_prec(method, &B->prec, &B->x4)) return false;
    B->n = count;
    B->L.resize(count);
    host_alloc_fault_point();
    std::vector<double> work(count);
    for (int i = 0; i < count; ++i) {
        const tcorr_instance &it = items[i];
        if (!make_layout(it.T, it.N, it.tau_max, it.stride, method, it.kind, &B->L[i])) return false;
        const BandPlan &p = B->L[i].p;
        work[i] = static_cast<double>(p.n_res * p.n_rows * p.n_cols) * static_cast<double>(B->L[i].Kp);
        if (it.kind == 0) ++B->n_msd;
    }
    B->order.resize(count);
    for (int i = 0; i < count; ++i) B->order[i] = i;
    std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b) { return work[a] > work[b]; });
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    B->off_inst = take(sizeof(InstDesc) * count);
    B->off_split = take(sizeof(SplitDesc) * count);
    B->off_pfx = take(2 * sizeof(PfxDesc) * (B->n_msd > 0 ? B->n_msd : 1));   // combine, then prefix
    B->off_red = take(sizeof(LagReduceDesc) * count);
    B->off_counter = take(sizeof(unsigned long long));
    B->off_pprep = take(sizeof(PolyPrepArgs) * count);
    B->off_pred = take(sizeof(PolyReduceArgs) * count);
    B->off_rowmax = take(sizeof(unsigned) * POLY_L * count);    // polyphase row maxima, one reset
    B->base.resize(count);
    for (int k = 0; k < count; ++k) {
        const int i = B->order[k];
        B->base[i] = take(B->L[i].total);
        if (B->L[i].poly) continue;      // polyphase instances have prep and reduction of their own
        B->total_items += B->L[i].p.n_items;
        B->total_frames += split_block_count(B->L[i]);             // prep blocks
        if (items[i].kind == 0) B->total_pfx += B->L[i].p.n_res;
        B->total_lags += items[i].tau_max + 1;
    }
    B->total = off;
    return B->total_frames < (int64_t(1) << 31) && B->total_items < (int64_t(1) << 40);
}

// Host-side description of one polyphase instance: prep arguments, the Gram
// kernel's tensor maps and arguments, and the reduction arguments.
struct PolySetup {
    PolyPrepArgs prep;
    PolyPrepArgs prep_b;            // cross-correlation: the later-side signal B
    InstDesc gram;
    PolyReduceArgs red;
};

int poly_setup(int kind, const float *d_x, const GramLayout &L, uint8_t *base, double *d_out, PolySetup *P,
               const float *d_y = nullptr) {
    const int64_t T = L.p.T, N = L.p.N;
    PolyPrepArgs &pa = P->prep;
    pa.X = d_x;
    pa.T = T;
    pa.K = 3 * N;
    pa.P = L.P;
    pa.Pp = L.Pp;
    pa.Kprime = L.Kprime;
    pa.Kalloc = L.Kalloc;
    pa.Yh = base + L.off_xh;
    pa.Yl = base + L.off_xl;
    pa.inv_scale = reinterpret_cast<float *>(base + L.off_scale);
    pa.rowmax = reinterpret_cast<unsigned *>(base + L.off_scale) + POLY_L;
    pa.kind = L.cross ? 1 : kind;
    pa.ncopies = L.cross ? 1 : 8;
    pa.rm_begin = 0;
    pa.tile_begin = 0;
    if (L.cross) {
        PolyPrepArgs &pb = P->prep_b;
        pb = pa;
        pb.X = d_y;
        pb.Yh = base + L.off_bh;
        pb.Yl = base + L.off_bl;
        pb.inv_scale = reinterpret_cast<float *>(base + L.off_scale_b);
        pb.rowmax = reinterpret_cast<unsigned *>(base + L.off_scale_b) + POLY_L;
        pb.ncopies = 8;
    }
    EncodeFn encode = get_encode();
    if (!encode) return TCORR_EUNSUPPORTED;
    const CUtensorMapDataType dt = L.prec == P_FP16   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : L.prec == P_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMap *maps = P->gram.maps;
    void *bases[2] = {base + L.off_xh, base + L.off_xl};
    void *bbases[2] = {base + (L.cross ? L.off_bh : L.off_xh), base + (L.cross ? L.off_bl : L.off_xl)};
    const cuuint64_t rowb = static_cast<cuuint64_t>(L.Kalloc * L.esize);
    for (int h = 0; h < 2; ++h) {
        const cuuint64_t dimA[2] = {static_cast<cuuint64_t>(L.Kalloc), POLY_L};
        const cuuint64_t strA[1] = {rowb};
        const cuuint32_t boxA[2] = {static_cast<cuuint32_t>(L.bke), static_cast<cuuint32_t>(BO)};
        const cuuint32_t es2[2] = {1, 1};
        if (encode(&maps[h], dt, 2, bases[h], dimA, strA, boxA, es2, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cuda_fail(cudaErrorInvalidValue, "cuTensorMapEncodeTiled (polyphase A)");
        // the 8 shifted copies are consecutive blocks of POLY_L rows: one 2-D map,
        // row = copy * POLY_L + phase (a 2-D box moves faster than a 3-D one)
        const cuuint64_t dimB[2] = {static_cast<cuuint64_t>(L.Kalloc), 8 * POLY_L};
        const cuuint64_t strB[1] = {rowb};
        for (int v = 0; v < 2; ++v) {          // B with BF-row boxes, then with NBOX-row boxes
            const cuuint32_t boxB[2] = {static_cast<cuuint32_t>(L.bke), static_cast<cuuint32_t>(v == 0 ? BF : NBOX)};
            if (encode(&maps[2 + 2 * v + h], dt, 2, bbases[h], dimB, strB, boxB, es2, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cuda_fail(cudaErrorInvalidValue, "cuTensorMapEncodeTiled (polyphase B)");
        }
    }
    GramArgs &ga = P->gram.ga;
    ga = GramArgs{};
    ga.T = T;
    ga.s = 1;
    ga.tau_max = L.p.tau_max;
    ga.n_orig = T;
    ga.n_res = 1;
    ga.n_rows = 3;
    ga.n_cols = 2;
    ga.n_items = L.p.n_items;
    ga.kb_total = ceil_div(L.Kprime, L.bke);
    ga.kb_per_item = L.kseg / L.bke;
    ga.inv_scale = reinterpret_cast<const float *>(base + L.off_scale);
    ga.inv_scale_b = L.cross ? reinterpret_cast<const float *>(base + L.off_scale_b) : ga.inv_scale;
    ga.partial = reinterpret_cast<double *>(base + L.off_partial);
    ga.b3d = 2;
    ga.xa_h = ga.xa_l = ga.xb_h = ga.xb_l = nullptr;
    ga.nkp = ga.rows = 0;
    ga.sub_kb = L.sub_kb;
    ga.counter = reinterpret_cast<unsigned long long *>(base + L.off_counter);
    ga.mode = 1;
    ga.nq = L.nq;
    ga.super_rows = kDefaultSuperRows;
    ga.super_cols = kDefaultSuperCols;
    ga.partial_elems = dbg_shrink_elems(L.p.n_items * WPG, WPG);
#ifdef TCORR_DEBUG_BOUNDS
    ga.dbg_status = status_word_device_ptr();
#else
    ga.dbg_status = nullptr;
#endif
    P->gram.item_begin = 0;
    PolyReduceArgs &ra = P->red;
    ra.partial = ga.partial;
    ra.T = T;
    ra.N = N;
    ra.tau_max = L.p.tau_max;
    ra.nq = L.nq;
    ra.n_groups = L.p.n_groups;
    ra.kind = kind;
    ra.S_prefix = kind == 0 ? reinterpret_cast<const double *>(base + L.off_prefix) : nullptr;
    ra.out = d_out;
    ra.lag_begin = 0;
    return TCORR_OK;
}

// Operand copies of one instance (single: *args by value) or of a batch
// (batch: args points at n device descriptors), `grid` prep tiles.
cudaError_t poly_split_launch(int prec, bool batch, const PolyPrepArgs *args, int n, unsigned grid,
                              cudaStream_t st) {
    auto go = [&](auto single_k, auto batch_k) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(batch ? reinterpret_cast<const void *>(batch_k)
                                                   : reinterpret_cast<const void *>(single_k),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(PT_SMEM));
        if (e != cudaSuccess) return e;
        if (batch) batch_k<<<grid, PREP_THREADS, PT_SMEM, st>>>(args, n);
        else single_k<<<grid, PREP_THREADS, PT_SMEM, st>>>(*args);
        return cudaGetLastError();
    };
    switch (prec) {
        case P_FP16: return go(poly_split_kernel<P_FP16>, poly_split_batch_kernel<P_FP16>);
        case P_BF16: return go(poly_split_kernel<P_BF16>, poly_split_batch_kernel<P_BF16>);
        default: return go(poly_split_kernel<P_TF32>, poly_split_batch_kernel<P_TF32>);
    }
}

// S(t) and its prefix sums for a polyphase MSD instance.
cudaError_t poly_msd_s(const float *d_x, const GramLayout &L, uint8_t *base, cudaStream_t st) {
    const int64_t T = L.p.T;
    double *S = reinterpret_cast<double *>(base + L.off_S);
    double *prefix = reinterpret_cast<double *>(base + L.off_prefix);
    poly_s_kernel<<<static_cast<unsigned>(ceil_div(T, 256)), 256, 0, st>>>(d_x, T, 3 * L.p.N, S);
    s_prefix_kernel<<<1, PFX_THREADS, 0, st>>>(S, T, 1, 1, T + 1, prefix);
    return cudaGetLastError();
}

// Enqueues one polyphase instance: operand copies, S(t) and its prefix sums
// (MSD), the Gram kernel over (q, h, c) blocks, and the lag reduction.
int poly_run(int kind, const float *d_x, const GramLayout &L, uint8_t *base, double *d_out, int num_sms,
             cudaStream_t st, const float *d_y = nullptr) {
    PolySetup P;
    int rc = poly_setup(kind, d_x, L, base, d_out, &P, d_y);
    if (rc != TCORR_OK) return rc;
    cudaError_t e = cudaSuccess;
    for (int side = 0; side < (L.cross ? 2 : 1); ++side) {      // the signal, then B of a cross-correlation
        const PolyPrepArgs &pp = side == 0 ? P.prep : P.prep_b;
        if (L.prec == P_FP16) {
            if ((e = cudaMemsetAsync(pp.rowmax, 0, POLY_L * sizeof(unsigned), st)) != cudaSuccess)
                return cuda_fail(e, "row-max reset");
            poly_rowmax_kernel<<<static_cast<unsigned>(poly_rm_blocks(L.P)), POLY_L, 0, st>>>(pp);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "poly_rowmax_kernel launch");
        }
        if ((e = poly_split_launch(L.prec, false, &pp, 1, static_cast<unsigned>(poly_tiles(L.Kalloc)), st)) !=
            cudaSuccess)
            return cuda_fail(e, "poly_split_kernel launch");
    }
    if (kind == 0 && (e = poly_msd_s(d_x, L, base, st)) != cudaSuccess) return cuda_fail(e, "poly S launch");
    const GramArgs &ga = P.gram.ga;
    if ((e = cudaMemsetAsync(ga.counter, 0, sizeof(unsigned long long), st)) != cudaSuccess)
        return cuda_fail(e, "work-item counter reset");
    const int grid = static_cast<int>(ga.n_items < num_sms ? ga.n_items : num_sms);
    switch (L.prec * 2 + (L.x4 ? 1 : 0)) {
        case P_FP16 * 2: e = launch_gram<P_FP16, false>(P.gram.maps, ga, grid, st, kind & 1); break;
        case P_BF16 * 2: e = launch_gram<P_BF16, false>(P.gram.maps, ga, grid, st, kind & 1); break;
        case P_BF16 * 2 + 1: e = launch_gram<P_BF16, true>(P.gram.maps, ga, grid, st, kind & 1); break;
        default: e = launch_gram<P_TF32, false>(P.gram.maps, ga, grid, st, kind & 1); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "gram_band_kernel (polyphase) launch");
    poly_reduce_kernel<<<static_cast<unsigned>(ceil_div(L.p.tau_max + 1, 256)), 256, 0, st>>>(P.red);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "poly_reduce launch");
    return TCORR_OK;
}

}  // namespace

// Workspace bound: the MSD layout (a superset of the ACF one) with the chosen
// parameters, and with the shortest candidate work item when tuning may run.
size_t gram_workspace_size(int64_t T, int64_t N, int64_t tau_max, int64_t s, int method, const Window *w,
                           int kind) {
    GramLayout L;
    if (!make_layout(T, N, tau_max, s, method, kind, &L, w, true)) return 0;
    size_t need = L.total;
    if (!w && tune_mode() != 0) {   // every candidate: the shortest item length, either tile shape
        const TuneChoice *prev = get_tune_override();
        for (int pair : {0, 1}) {
            TuneChoice shortest{tune_min_kseg(), 0};
            shortest.pair = pair;
            set_tune_override(&shortest);
            GramLayout Ls;
            if (make_layout(T, N, tau_max, s, method, kind, &Ls, nullptr, true) && Ls.total > need) need = Ls.total;
        }
        set_tune_override(prev);
    }
    return need;
}

cudaError_t launch_s_prefix(const double *S, int64_t T, int64_t s, int64_t n_res, int64_t pstride,
                            double *prefix, cudaStream_t st) {
    s_prefix_kernel<<<static_cast<unsigned>(n_res), PFX_THREADS, 0, st>>>(S, T, 1, s, pstride, prefix);
    return cudaGetLastError();
}

size_t gram_batch_workspace_size(const tcorr_instance *items, int count, int method) {
    BatchLayout B;
    if (!make_batch_layout(items, count, method, &B)) return 0;
    return B.total;
}

bool gram_method_available(int method) {
    int prec;
    bool x4;
    int sms = 0;
    return method_prec(method, &prec, &x4) && device_is_sm103(&sms) && get_encode() != nullptr;
}

namespace {

// kind 0 MSD, 1 ACF, 2 cross-correlation of d_x (origins) with d_y (later frames).
int gram_run_once(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s, int method,
                  double *d_out, void *d_ws, size_t ws_bytes, cudaStream_t st, const Window *w = nullptr,
                  const float *d_y = nullptr) {
    GramLayout L;
    if (!make_layout(T, N, tau_max, s, method, kind, &L, w, true)) return TCORR_EUNSUPPORTED;
    if (ws_bytes < L.total || !d_ws) return TCORR_EWORKSPACE;
    int num_sms = 0;
    if (!device_is_sm103(&num_sms)) return TCORR_EUNSUPPORTED;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    if (L.poly) return poly_run(kind, d_x, L, ws, d_out, num_sms, st, d_y);

    auto split = [&](const SplitDesc &q) {
        switch (L.prec) {
            case P_FP16: return launch_split<P_FP16>(q, st);
            case P_BF16: return launch_split<P_BF16>(q, st);
            default: return launch_split<P_TF32>(q, st);
        }
    };
    cudaError_t e = split(split_desc(kind == 2 ? 1 : kind, d_x, L, ws, 0));
    if (e != cudaSuccess) return cuda_fail(e, "split_kernel launch");
    if (kind == 2) {                  // B: its own hi/lo copies and scales
        SplitDesc qb = split_desc(1, d_y, L, ws, 0);
        qb.Xh = ws + L.off_bh;
        qb.Xl = ws + L.off_bl;
        qb.inv_scale = reinterpret_cast<float *>(ws + L.off_scale_b);
        if ((e = split(qb)) != cudaSuccess) return cuda_fail(e, "split_kernel launch (B)");
    }
    if (kind == 0) {
        double *S = reinterpret_cast<double *>(ws + L.off_S);
        if (L.p.n_groups > 1)
            s_combine_kernel<<<static_cast<unsigned>(ceil_div(T, 256)), 256, 0, st>>>(S, T, L.p.n_groups);
        s_prefix_kernel<<<static_cast<unsigned>(L.p.n_res), PFX_THREADS, 0, st>>>(
            S, T, 1, s, L.pstride, reinterpret_cast<double *>(ws + L.off_prefix));
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "s_prefix_kernel launch");
    }
    CUtensorMap maps[NMAPS];
    const int rc = encode_maps(L, ws, s, maps);
    if (rc != TCORR_OK) return rc;
    const GramArgs ga = gram_args(L, ws, T, N, tau_max, s);
    e = cudaMemsetAsync(ga.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "work-item counter reset");
    if (L.pair) {   // one cluster of two CTAs per TPC
        CUtensorMap pmaps[NMAPS];
        const int prc = encode_pair_maps(L, ws, pmaps);
        if (prc != TCORR_OK) return prc;
        const int64_t pairs = num_sms / 2;
        const int grid = 2 * static_cast<int>(ga.n_items < pairs ? ga.n_items : pairs);
        switch (L.prec * 2 + (L.x4 ? 1 : 0)) {
            case P_FP16 * 2: e = launch_gram_pair<P_FP16, false>(pmaps, ga, grid, st, kind & 1); break;
            case P_BF16 * 2: e = launch_gram_pair<P_BF16, false>(pmaps, ga, grid, st, kind & 1); break;
            case P_BF16 * 2 + 1: e = launch_gram_pair<P_BF16, true>(pmaps, ga, grid, st, kind & 1); break;
            default: e = launch_gram_pair<P_TF32, false>(pmaps, ga, grid, st, kind & 1); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "gram_pair_kernel launch");
        e = launch_lag_reduce(L.p, ga.partial, finalize_args(kind, L, ws), d_out, st, w);
        if (e != cudaSuccess) return cuda_fail(e, "lag_reduce launch");
        return TCORR_OK;
    }
    const int grid = static_cast<int>(L.p.n_items < num_sms ? L.p.n_items : num_sms);
    switch (L.prec * 2 + (L.x4 ? 1 : 0)) {
        case P_FP16 * 2: e = launch_gram<P_FP16, false>(maps, ga, grid, st, kind & 1); break;
        case P_BF16 * 2: e = launch_gram<P_BF16, false>(maps, ga, grid, st, kind & 1); break;
        case P_BF16 * 2 + 1: e = launch_gram<P_BF16, true>(maps, ga, grid, st, kind & 1); break;
        default: e = launch_gram<P_TF32, false>(maps, ga, grid, st, kind & 1); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "gram_band_kernel launch");
    e = launch_lag_reduce(L.p, ga.partial, finalize_args(kind, L, ws), d_out, st, w);
    if (e != cudaSuccess) return cuda_fail(e, "lag_reduce launch");
    return TCORR_OK;
}

// Times every tuning candidate (work-item length; the sub-chain length stays
// the kind's default) on the stream, synchronising, and keeps the fastest.
int gram_tune(const std::string &key, int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s,
              int method, double *d_out, void *d_ws, size_t ws_bytes, cudaStream_t st, TuneChoice *best,
              const float *d_y) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TCORR_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TCORR_ECUDA;
    }
    // A candidate that fails to launch (a launch-configuration error, which does not stick to the
    // context) is skipped; the call fails only when no candidate runs, or on an error that
    // stays with the context (every later candidate then fails too).
    float best_ms = -1.f;
    int rc = TCORR_OK, last_err = TCORR_OK;
    bool sync_failed = false;
    for (const TuneChoice &c : tune_candidates()) {
        set_tune_override(&c);
        rc = gram_run_once(kind, d_x, T, N, tau_max, s, method, d_out, d_ws, ws_bytes, st, nullptr, d_y);   // warm-up
        if (rc == TCORR_OK) {
            cudaEventRecord(e0, st);
            rc = gram_run_once(kind, d_x, T, N, tau_max, s, method, d_out, d_ws, ws_bytes, st, nullptr, d_y);
            cudaEventRecord(e1, st);
        }
        set_tune_override(nullptr);
        if (rc != TCORR_OK) {
            last_err = rc;
            cudaGetLastError();
            continue;
        }
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            sync_failed = true;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (sync_failed) return TCORR_ECUDA;
    if (best_ms < 0.f) return last_err != TCORR_OK ? last_err : TCORR_ECUDA;
    tune_store(key, *best);
    return TCORR_OK;
}

}  // namespace

int gram_run(int kind, const float *d_x, int64_t T, int64_t N, int64_t tau_max, int64_t s, int method,
             double *d_out, void *d_ws, size_t ws_bytes, cudaStream_t st, const Window *w, const float *d_y) {
    if (w) return gram_run_once(kind, d_x, T, N, tau_max, s, method, d_out, d_ws, ws_bytes, st, w, d_y);
    const int mode = tune_mode();
    if (mode != 0 && !env_kseg() && !env_sub_kb()) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            const std::string key = tune_key(method, kind, 3 * N, tau_max, T, s);
            TuneChoice c;
            if (mode == 2 || !tune_lookup(key, &c)) {
                const int rc = gram_tune(key, kind, d_x, T, N, tau_max, s, method, d_out, d_ws, ws_bytes, st, &c,
                                         d_y);
                if (rc != TCORR_OK) return rc;
            }
            set_tune_override(&c);
            const int rc = gram_run_once(kind, d_x, T, N, tau_max, s, method, d_out, d_ws, ws_bytes, st, nullptr,
                                         d_y);
            set_tune_override(nullptr);
            return rc;
        }
    }
    return gram_run_once(kind, d_x, T, N, tau_max, s, method, d_out, d_ws, ws_bytes, st, nullptr, d_y);
}

// Whole batch: one batched prep launch, one batched S-prefix launch, Gram
// tiles (one launch per instance with many work items, one shared
// persistent launch for the rest), one batched reduction, plus the
// descriptor uploads.  Callers check arguments; d_ws holds
// gram_batch_workspace_size().
int gram_batch_run(const tcorr_instance *items, int count, int method, void *d_ws, size_t ws_bytes,
                   cudaStream_t st) {
    BatchLayout B;
    if (!make_batch_layout(items, count, method, &B)) return TCORR_EUNSUPPORTED;
    if (ws_bytes < B.total || !d_ws) return TCORR_EWORKSPACE;
    int num_sms = 0;
    if (!device_is_sm103(&num_sms)) return TCORR_EUNSUPPORTED;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);

    // Instances with many work items get a launch of their own (tensor maps as
    // kernel parameters, which the TMA unit reaches faster than maps in
    // global memory); the rest share one persistent launch.  An own-launch
    // band instance has its prep (split, S combine and prefix) enqueued just
    // before its Gram launch, and these instances go in the caller's order:
    // with every instance's prep first and the Gram launches by decreasing
    // work, the 256-instance uneven workload took 464 ms on GB300 against
    // 441 ms this way (per-instance calls: 441 ms); the results are identical.
    const int64_t big_items = 8 * static_cast<int64_t>(num_sms);
    std::vector<InstDesc> inst;
    std::vector<SplitDesc> spl(count);
    std::vector<PfxDesc> pfx;
    std::vector<LagReduceDesc> red(count);
    struct OwnLaunch {
        InstDesc d;
        int index;             // position in the caller's array
        bool band_prep;        // band form: split (and S prefix) enqueued with the Gram launch
        SplitDesc q;
        const GramLayout *L;
        int kind;
        int64_t T, s;
        double *S, *prefix;
    };
    std::vector<OwnLaunch> own;
    int ns = 0;                          // band instances whose prep is batched
    int64_t item_begin = 0, frame_begin = 0, pfx_begin = 0, lag_begin = 0, s_frames = 0;
    std::vector<PolyPrepArgs> pprep;
    std::vector<PolyReduceArgs> pred;
    std::vector<int> poly_msd;
    int64_t plag_begin = 0, prm_begin = 0, ptile_begin = 0;
    int nb = 0;                          // band instances, in descriptor order
    for (int k = 0; k < count; ++k) {
        const int i = B.order[k];
        const tcorr_instance &it = items[i];
        const GramLayout &L = B.L[i];
        uint8_t *base = ws + B.base[i];
        if (L.poly) {
            PolySetup P;
            const int rc = poly_setup(it.kind, it.d_x, L, base, it.d_out, &P);
            if (rc != TCORR_OK) return rc;
            if (L.p.n_items >= big_items) {
                own.push_back(OwnLaunch{P.gram, i, false, SplitDesc{}, &L, it.kind, it.T, it.stride, nullptr,
                                        nullptr});
            } else {
                P.gram.item_begin = item_begin;
                item_begin += L.p.n_items;
                inst.push_back(P.gram);
            }
            P.prep.rowmax = reinterpret_cast<unsigned *>(ws + B.off_rowmax) + pprep.size() * POLY_L;
            P.prep.rm_begin = prm_begin;
            P.prep.tile_begin = ptile_begin;
            prm_begin += poly_rm_blocks(L.P);
            ptile_begin += poly_tiles(L.Kalloc);
            pprep.push_back(P.prep);
            P.red.lag_begin = plag_begin;
            plag_begin += it.tau_max + 1;
            pred.push_back(P.red);
            if (it.kind == 0) poly_msd.push_back(i);
            continue;
        }
        InstDesc d;
        const int rc = encode_maps(L, base, it.stride, d.maps);
        if (rc != TCORR_OK) return rc;
        d.ga = gram_args(L, base, it.T, it.N, it.tau_max, it.stride);
        if (L.p.n_items >= big_items) {
            d.item_begin = 0;
            own.push_back(OwnLaunch{d, i, true, split_desc(it.kind, it.d_x, L, base, 0), &L, it.kind, it.T,
                                    it.stride, reinterpret_cast<double *>(base + L.off_S),
                                    reinterpret_cast<double *>(base + L.off_prefix)});
        } else {
            d.item_begin = item_begin;
            item_begin += L.p.n_items;
            inst.push_back(d);
            spl[ns++] = split_desc(it.kind, it.d_x, L, base, frame_begin);
            frame_begin += split_block_count(L);
        }
        if (it.kind == 0 && L.p.n_items < big_items) {
            PfxDesc q;
            q.S = reinterpret_cast<const double *>(base + L.off_S);
            q.T = it.T;
            q.n_groups = L.p.n_groups;
            q.s = it.stride;
            q.pstride = L.pstride;
            q.prefix = reinterpret_cast<double *>(base + L.off_prefix);
            q.blk_begin = pfx_begin;
            q.frame_begin = s_frames;
            s_frames += it.T;
            pfx_begin += L.p.n_res;
            pfx.push_back(q);
        }
        red[nb] = lag_reduce_desc(L.p, d.ga.partial, finalize_args(it.kind, L, base), it.d_out, lag_begin);
        lag_begin += it.tau_max + 1;
        ++nb;
    }
    // the prefix pass reads S after the group parts were combined into group 0
    std::vector<PfxDesc> pfx1(pfx);
    for (PfxDesc &q : pfx1) q.n_groups = 1;
    // prep descriptors grouped by class, block offsets counted within each class
    std::vector<SplitDesc> spl_by_class;
    int cls_start[9] = {0};
    int64_t cls_blocks[8] = {0};
    for (int c = 0; c < 8; ++c) {
        cls_start[c] = static_cast<int>(spl_by_class.size());
        for (int k = 0; k < ns; ++k) {
            if (split_class(spl[k]) != c) continue;
            SplitDesc q = spl[k];
            q.blk_begin = cls_blocks[c];
            cls_blocks[c] += q.warp_mode ? ceil_div(q.rows, kWarpFrames) * q.n_groups : q.rows * q.n_groups;
            spl_by_class.push_back(q);
        }
    }
    cls_start[8] = static_cast<int>(spl_by_class.size());
    const int np = static_cast<int>(pprep.size());
    cudaError_t e = cudaSuccess;
    if ((!inst.empty() &&
         (e = upload_bytes(ws + B.off_inst, inst.data(), sizeof(InstDesc) * inst.size(), st)) != cudaSuccess) ||
        (ns > 0 &&
         (e = upload_bytes(ws + B.off_split, spl_by_class.data(), sizeof(SplitDesc) * ns, st)) != cudaSuccess) ||
        (nb > 0 && (e = upload_bytes(ws + B.off_red, red.data(), sizeof(LagReduceDesc) * nb, st)) != cudaSuccess) ||
        (!pfx.empty() && (e = upload_bytes(ws + B.off_pfx, pfx.data(), sizeof(PfxDesc) * pfx.size(), st)) != cudaSuccess) ||
        (!pfx.empty() && (e = upload_bytes(ws + B.off_pfx + sizeof(PfxDesc) * pfx.size(), pfx1.data(),
                                           sizeof(PfxDesc) * pfx1.size(), st)) != cudaSuccess) ||
        (np > 0 && (e = upload_bytes(ws + B.off_pprep, pprep.data(), sizeof(PolyPrepArgs) * np, st)) != cudaSuccess) ||
        (np > 0 && (e = upload_bytes(ws + B.off_pred, pred.data(), sizeof(PolyReduceArgs) * np, st)) != cudaSuccess))
        return cuda_fail(e, "descriptor upload");
    if (np > 0) {
        const PolyPrepArgs *d_pp = reinterpret_cast<const PolyPrepArgs *>(ws + B.off_pprep);
        if (B.prec == P_FP16) {
            if ((e = cudaMemsetAsync(ws + B.off_rowmax, 0, sizeof(unsigned) * POLY_L * np, st)) != cudaSuccess)
                return cuda_fail(e, "row-max reset");
            poly_rowmax_batch_kernel<<<static_cast<unsigned>(prm_begin), POLY_L, 0, st>>>(d_pp, np);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "poly_rowmax_batch_kernel launch");
        }
        if ((e = poly_split_launch(B.prec, true, d_pp, np, static_cast<unsigned>(ptile_begin), st)) != cudaSuccess)
            return cuda_fail(e, "poly_split_batch_kernel launch");
        for (int i : poly_msd)
            if ((e = poly_msd_s(items[i].d_x, B.L[i], ws + B.base[i], st)) != cudaSuccess)
                return cuda_fail(e, "poly S launch");
    }

    const SplitDesc *d_spl = reinterpret_cast<const SplitDesc *>(ws + B.off_split);
    for (int c = 0; c < 8; ++c) {
        const int n = cls_start[c + 1] - cls_start[c];
        if (n == 0) continue;
        const SplitDesc *dc = d_spl + cls_start[c];
        switch (B.prec) {
            case P_FP16: e = launch_split_batch_class<P_FP16>(c, dc, n, cls_blocks[c], st); break;
            case P_BF16: e = launch_split_batch_class<P_BF16>(c, dc, n, cls_blocks[c], st); break;
            default: e = launch_split_batch_class<P_TF32>(c, dc, n, cls_blocks[c], st); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "split_batch_kernel launch");
    }
    if (!pfx.empty()) {
        // the group parts of S(t) are combined in parallel (in place, into group 0),
        // then the prefix pass reads one value per frame (its descriptors say 1 group)
        const PfxDesc *d_pfx = reinterpret_cast<const PfxDesc *>(ws + B.off_pfx);
        s_combine_batch_kernel<<<static_cast<unsigned>(ceil_div(s_frames, 256)), 256, 0, st>>>(
            d_pfx, static_cast<int>(pfx.size()), s_frames);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "s_combine_batch_kernel launch");
        s_prefix_batch_kernel<<<static_cast<unsigned>(B.total_pfx), PFX_THREADS, 0, st>>>(
            reinterpret_cast<const PfxDesc *>(ws + B.off_pfx + sizeof(PfxDesc) * pfx.size()),
            static_cast<int>(pfx.size()));
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "s_prefix_batch_kernel launch");
    }
    std::stable_sort(own.begin(), own.end(), [](const OwnLaunch &a, const OwnLaunch &b) { return a.index < b.index; });
    for (const OwnLaunch &o : own) {
        const InstDesc &d = o.d;
        if (o.band_prep) {
            switch (B.prec) {
                case P_FP16: e = launch_split<P_FP16>(o.q, st); break;
                case P_BF16: e = launch_split<P_BF16>(o.q, st); break;
                default: e = launch_split<P_TF32>(o.q, st); break;
            }
            if (e != cudaSuccess) return cuda_fail(e, "split_kernel launch");
            if (o.kind == 0) {
                if (o.L->p.n_groups > 1)
                    s_combine_kernel<<<static_cast<unsigned>(ceil_div(o.T, 256)), 256, 0, st>>>(o.S, o.T,
                                                                                             o.L->p.n_groups);
                s_prefix_kernel<<<static_cast<unsigned>(o.L->p.n_res), PFX_THREADS, 0, st>>>(o.S, o.T, 1, o.s,
                                                                                              o.L->pstride, o.prefix);
                if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "s_prefix_kernel launch");
            }
        }
        if ((e = cudaMemsetAsync(d.ga.counter, 0, sizeof(unsigned long long), st)) != cudaSuccess)
            return cuda_fail(e, "work-item counter reset");
        const int grid = static_cast<int>(d.ga.n_items < num_sms ? d.ga.n_items : num_sms);
        switch (B.prec * 2 + (B.x4 ? 1 : 0)) {
            case P_FP16 * 2: e = launch_gram<P_FP16, false>(d.maps, d.ga, grid, st, 2); break;
            case P_BF16 * 2: e = launch_gram<P_BF16, false>(d.maps, d.ga, grid, st, 2); break;
            case P_BF16 * 2 + 1: e = launch_gram<P_BF16, true>(d.maps, d.ga, grid, st, 2); break;
            default: e = launch_gram<P_TF32, false>(d.maps, d.ga, grid, st, 2); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "gram_band_kernel launch");
    }
    if (!inst.empty() && item_begin > 0) {
        SrcBatch src;
        src.d = reinterpret_cast<const InstDesc *>(ws + B.off_inst);
        src.n = static_cast<int>(inst.size());
        src.total = item_begin;
        src.ctr = reinterpret_cast<unsigned long long *>(ws + B.off_counter);
        if ((e = cudaMemsetAsync(src.ctr, 0, sizeof(unsigned long long), st)) != cudaSuccess)
            return cuda_fail(e, "work-item counter reset");
        const int grid = static_cast<int>(src.total < num_sms ? src.total : num_sms);
        switch (B.prec * 2 + (B.x4 ? 1 : 0)) {
            case P_FP16 * 2: e = launch_gram_batch<P_FP16, false>(src, grid, st); break;
            case P_BF16 * 2: e = launch_gram_batch<P_BF16, false>(src, grid, st); break;
            case P_BF16 * 2 + 1: e = launch_gram_batch<P_BF16, true>(src, grid, st); break;
            default: e = launch_gram_batch<P_TF32, false>(src, grid, st); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "gram_band_batch_kernel launch");
    }
    if (nb > 0) {
        e = launch_lag_reduce_batch(reinterpret_cast<const LagReduceDesc *>(ws + B.off_red), nb, B.total_lags, st);
        if (e != cudaSuccess) return cuda_fail(e, "lag_reduce_batch launch");
    }
    if (np > 0) {
        poly_reduce_batch_kernel<<<static_cast<unsigned>(ceil_div(plag_begin, 256)), 256, 0, st>>>(
            reinterpret_cast<const PolyReduceArgs *>(ws + B.off_pred), np, plag_begin);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "poly_reduce_batch launch");
    }
    return TCORR_OK;
}

namespace {

// Waits on an mbarrier that nothing completes, with a short limit, through the
// same bounded-wait path as the band kernel: the wait gives up, the status
// word records TCORR_ETIMEOUT, and the kernel returns normally.
__global__ void timeout_probe_kernel(unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    fence_barrier_init();
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(b, 0u)) return;              // never: nobody arrives
        if ((it & 255u) == 255u && globaltimer() - t0 > limit_ns) {
            atomicExch(&g_status, static_cast<unsigned int>(TCORR_ETIMEOUT));
            return;
        }
    }
}

}  // namespace

int selftest_timeout(cudaStream_t st) {
    timeout_probe_kernel<<<1, 32, 0, st>>>(10000000ull);   // 10 ms
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TCORR_OK : cuda_fail(e, "timeout_probe_kernel launch");
}

unsigned int *status_word_device_ptr() {
    static unsigned int *ptr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
        ptr[dev] = static_cast<unsigned int *>(p);
    }
    return ptr[dev];
}

int status_poll_and_clear(cudaStream_t st) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return TCORR_ECUDA;
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof(v)) != cudaSuccess) return TCORR_ECUDA;
    const unsigned int zero = 0;
    if (cudaMemcpyToSymbol(g_status, &zero, sizeof(zero)) != cudaSuccess) return TCORR_ECUDA;
    return static_cast<int>(v);
}

}  // namespace tcorr
