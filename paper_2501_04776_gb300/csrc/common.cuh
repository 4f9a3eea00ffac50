// Shared internals of the IQP library: workspace plan, status word, launch
// accounting and the PTX wrappers (mbarrier, TMA, tcgen05) used by the
// kernels. Internal header; the public ABI is include/iqp.h.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "iqp.h"

namespace iqp {

// ---------------------------------------------------------------- sizes

constexpr int kPartColsSimt = 128;  // samples per (S, M2) partial, FP32 form
constexpr int kPartColsTc = 64;     // samples per (S, M2) partial, tensor-core form
constexpr int kATile = 128;      // observables per gradient partial row (single-CTA gradient kernel)
constexpr int kGradObs = 256;    // observables per tile of the CTA-pair gradient kernel (two partial rows each)
// Split phase tiles: one 128 x 256 FP32 partial accumulator per (part, CTA),
// for at most kMaxSplitCtas CTAs, then one int counter per (tile, CTA).
constexpr int64_t kSplitSlotFloats = 128 * 256;
constexpr int kMaxSplitCtas = 160;
// Balanced split of the two-sample-tile phase's last round: kSplitSlots slots
// (one per piece, CTA and accumulator), then kMaxSplitCtas counters.
constexpr int kSplitSlots = 640;
// Two-sample-tile phase kernels: the running sums of both accumulators, per
// CTA (at most kMaxSplitCtas CTAs).
constexpr int64_t kDtSumFloats = 2 * 128 * 256;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// Workspace layout. Every region is 256-byte aligned. Regions a given op does
// not use have size 0.
struct Plan {
    int64_t n, m, l, s, N;
    int op, prec;
    int64_t ldp;    // words per row of P_A / P_Z (bits over m), multiple of 4
    int64_t ldzt;   // words per row of P_Z^T (bits over s), multiple of 4
    int64_t ldlt;   // words per row of P_A^T (bits over l), multiple of 4
    int64_t mpad;   // ldp * 64 (length of the split-theta arrays)
    int64_t ldw;    // elements per row of W (multiple of 64)
    int64_t pw;     // samples per (S, M2) partial
    int64_t nparts; // (S, M2) partials per observable: ceil(s / pw)
    int64_t natile; // room for gradient partial rows: 2 ceil(l / 128)
    size_t off_status, off_pa, off_pz, off_pzt, off_pat, off_rt, off_c, off_part, off_w, off_gpart;
    size_t off_ab, off_s12, off_T, off_terms, off_zt, off_sup, total;
    // low-order form: C (+ d), M = C S, V, H, single-gate partials; ldc floats per row of C and H
    size_t off_lo_c, off_lo_m, off_lo_v, off_lo_h, off_lo_gs, off_lo_a;
    size_t off_skp;  // split BF16: partial accumulators and counters of split phase tiles (0 if none)
    size_t off_gsum; // split BF16: per-CTA running sums of the two-sample-tile phase kernels (0 if none)
    size_t off_skx;  // split BF16: pieces and counters of the two-tile phase's balanced last round (0 if none)
    size_t off_phi;  // MMD gradient (split BF16, row-sparse): room for Phi, l x ldw fp32 (0 if none)
    // Kept Phi (l x ldphi fp32, ldphi a multiple of 64 >= s; the layout is the
    // precision's own): phi_out = the statistics pass writes it, phi_in = the
    // gradient pass forms W from it instead of recomputing Phi.
    float *phi;
    int64_t ldphi;
    bool phi_out, phi_in;
    int64_t ldc;
    bool indep;     // one sample batch per observable (Z has l * s rows)
    const uint64_t *G;  // generators (read by the independent-batch kernels)
    int64_t ldg;
    const uint64_t *A;  // observables (read by the low-order kernels)
    int64_t lda;
};

// Independent-batch arguments of the row-sparse kernels.
struct SparseIndep {
    const int4 *sup;    // per gate: first three support qubits and |supp|
    const uint64_t *G;  // generators, for |supp| > 3
    int64_t ldg;
    int64_t n;
};

Plan make_plan(int op, int64_t n, int64_t m, int64_t l, int64_t s, int64_t N, int prec);
// The smallest workspace an op runs with (without the optional split-tile
// scratch at the end of its plan); 0 for invalid arguments.
size_t workspace_min_bytes(int op, int64_t n, int64_t m, int64_t l, int64_t s, int64_t N, int prec);

// Host-side argument checks of iqp_expval (sizes, pointers, alignment,
// precision), without the workspace.
iqp_status expval_arg_check(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                            int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                            iqp_precision prec, const double *expval, const double *std_err);

// Dense contraction on the tensor cores (split BF16, FP32 accumulation):
//   out[r][c] = sum_{k < K} (a_hi[r][k] + a_lo[r][k]) (1 - 2 bit k of b row c)
// for r < rows, c < nb. a_hi / a_lo: rows x kpad BF16 (row-major, kpad a
// multiple of 64, zero for k >= K); b_bits: nb rows of ldb words (even,
// >= 4, bits >= K zero or multiplied by zero); out: row-major, ldo elements
// per row (a multiple of 4), FP32 or FP64. cudaErrorNotSupported when a
// shape or layout rule does not hold (nothing is launched then).
cudaError_t launch_tc_dense(const __nv_bfloat16 *a_hi, const __nv_bfloat16 *a_lo, int64_t rows, int64_t kpad,
                            int64_t k, const uint64_t *b_bits, int64_t nb, int64_t ldb, void *out, int64_t ldo,
                            bool out_f64, uint32_t *status, cudaStream_t st);

// ---------------------------------------------------------------- status

// Device status word at the start of the workspace (uint32): 0 = OK, else an
// iqp_status recorded by the first kernel that failed.
__device__ inline void record_status(uint32_t *status, uint32_t code) {
    if (status) atomicCAS(status, 0u, code);
}

// Optional self-checks (build with -DIQP_CHECKS): every global index a
// kernel derives from the caller's shapes is compared with the extent of its
// buffer before the access; an index outside records 200 + site in this
// translation unit's check word (the first failure wins) and the access is
// skipped. iqp_check_status() reads and clears the words of all units. In
// the default build the checks compile to nothing. Nothing traps.
#ifdef IQP_CHECKS
static __device__ uint32_t g_check_word;
__device__ __forceinline__ bool check_in(int64_t idx, int64_t extent, uint32_t site) {
    if (idx >= 0 && idx < extent) return true;
    atomicCAS(&g_check_word, 0u, 200u + site);
    return false;
}
#define IQP_IN(idx, extent, site) ::iqp::check_in((int64_t)(idx), (int64_t)(extent), (uint32_t)(site))
// This unit's check word, cleared (host; synchronises the device).
static inline uint32_t take_check_word() {
    uint32_t v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_word, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
    if (cudaMemcpyToSymbol(g_check_word, &z, sizeof(z)) != cudaSuccess) return 0xFFFFFFFFu;
    return v;
}
#else
#define IQP_IN(idx, extent, site) true
static inline uint32_t take_check_word() { return 0u; }
#endif

// Host-side launch accounting (iqp_launch_count) and optional per-kernel
// event timing (iqp_profile_*). Construct one right before each launch.
struct LaunchScope {
    LaunchScope(int kernel, cudaStream_t st);
    ~LaunchScope();
    int kernel;
    cudaStream_t st;
    cudaEvent_t ev0, ev1;
};
iqp_status cuda_status(cudaError_t e);
int num_sms();
int device_cc();  // major*10+minor of the current device

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` of `bar`. Gives up when the
// CTA-wide abort flag is raised or after `limit_ns`; on its own timeout it
// raises the abort flag and records IQP_ERR_TIMEOUT. Returns false on give-up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint32_t *status, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u) {
            if (*abort_flag) return false;
            if (globaltimer_ns() - t0 > limit_ns) {
                *abort_flag = 1;
                record_status(status, IQP_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

// Bounded wait that ignores the abort flag, for draining work that always
// completes by itself (issued copies, issued MMAs) before a CTA exits.
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity, uint32_t *status, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && globaltimer_ns() - t0 > limit_ns) {
            record_status(status, IQP_ERR_TIMEOUT);
            return false;
        }
    }
}

// 2D tiled TMA load into shared memory, completing on `bar` (tx bytes).
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 2D tiled TMA load into this CTA's shared memory whose completion (tx
// bytes) is signalled to an mbarrier of the CTA pair given by its
// shared::cluster address `bar_cluster` (the leader's barrier, so that one
// barrier tracks both CTAs' halves of a pair operand).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const void *tmap, uint32_t bar_cluster, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}

// Prefetch the 2D tile of `tmap` at {x, y} into L2 (no shared memory, no barrier).
__device__ __forceinline__ void tma_prefetch_2d(const void *tmap, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(tmap), "r"(x), "r"(y)
                 : "memory");
}

// 1D bulk copy global -> shared (16-byte aligned, size multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const void *tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// ---- tcgen05 (5th-generation tensor cores, accumulators in tensor memory)

__device__ __forceinline__ void tmem_alloc(uint32_t *slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, kind::f16 (BF16 in, FP32 acc).
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// ---- clusters and the CTA-pair (cta_group::2) forms

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared::cluster address of the object at shared::cta address `addr` in CTA `rank`.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Arrive (release, cluster scope) on an mbarrier named by a shared::cluster address.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait with cluster-scope acquire (arrivals come from the peer CTA too).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                                  uint32_t *status, uint64_t limit_ns) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 63u) == 0u) {
            if (*abort_flag) return false;
            if (globaltimer_ns() - t0 > limit_ns) {
                *abort_flag = 1;
                record_status(status, IQP_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

// Every thread of both CTAs of the cluster (not warp-aligned).
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Pair MMA (issued by the even CTA): M = 256 split over the two CTAs' shared
// memory (A rows 0..127 here, 128..255 in the peer, same offsets), B's N
// columns split in halves likewise; each CTA's TMEM receives its 128 rows.
__device__ __forceinline__ void umma_f16_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Pair MMA with the A operand in tensor memory: rows 0..127 of A are TMEM
// lanes 0..127 of this CTA at column address `a_tmem`, rows 128..255 the same
// lanes and columns of the peer's TMEM; a 16-bit A element (row r, k) is half
// k & 1 (0 = low) of the 32-bit cell (lane r, column a_tmem + k / 2).
__device__ __forceinline__ void umma_f16_pair_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                                 uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Two MMAs of one K step, issued back to back: D (+)= A1 B1 (accumulating
// iff `acc` != 0), then D += A2 B2. The split-BF16 hi and lo products share one
// operand; each operand is a shared-memory descriptor or, where named
// `*_tmem`, a TMEM address. Pair forms: cta_group::2, issued by the even CTA.
__device__ __forceinline__ void umma2_pair_ss(uint32_t d, uint64_t a1, uint64_t a2, uint64_t b, uint32_t idesc,
                                              uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %5, 0;\n\t"
        "setp.eq.b32 q, %5, %5;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %3, %4, p;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %2, %3, %4, q;\n\t}\n"
        ::"r"(d), "l"(a1), "l"(a2), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma2_pair_ts(uint32_t d, uint32_t a1_tmem, uint32_t a2_tmem, uint64_t b,
                                              uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %5, 0;\n\t"
        "setp.eq.b32 q, %5, %5;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %3, %4, p;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%2], %3, %4, q;\n\t}\n"
        ::"r"(d), "r"(a1_tmem), "r"(a2_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma2_pair_ts_b(uint32_t d, uint32_t a_tmem, uint64_t b1, uint64_t b2,
                                                uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %5, 0;\n\t"
        "setp.eq.b32 q, %5, %5;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %4, p;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %3, %4, q;\n\t}\n"
        ::"r"(d), "r"(a_tmem), "l"(b1), "l"(b2), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma2_ss(uint32_t d, uint64_t a1, uint64_t a2, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %5, 0;\n\t"
        "setp.eq.b32 q, %5, %5;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %4, p;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %3, %4, q;\n\t}\n"
        ::"r"(d), "l"(a1), "l"(a2), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// One operand stage of MMAs from a single asm statement (descriptors and
// TMEM addresses of the later K steps formed inside it), so that the issuing
// thread spends as few instructions as possible per MMA. Every stage issues
// the hi and lo products of each 16-wide K step back to back into D; the
// first MMA accumulates iff `acc` != 0, every later one accumulates.
// Shared-memory operand descriptors advance 32 bytes (2 in the start-address
// field) per K step within a 128-byte swizzle atom.
// Four K steps, all operands in shared memory (A hi, A lo, B).
__device__ __forceinline__ void umma_stage4_pair_ss(uint32_t d, uint64_t ahi, uint64_t alo, uint64_t b, uint32_t idesc,
                                             uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t.reg .b64 h, l, bb;\n\t"
        "setp.ne.b32 p, %5, 0;\n\tsetp.eq.b32 q, %5, %5;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %3, %4, p;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %2, %3, %4, q;\n\t"
        "add.s64 h, %1, 2;\n\tadd.s64 l, %2, 2;\n\tadd.s64 bb, %3, 2;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], h, bb, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], l, bb, %4, q;\n\t"
        "add.s64 h, %1, 4;\n\tadd.s64 l, %2, 4;\n\tadd.s64 bb, %3, 4;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], h, bb, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], l, bb, %4, q;\n\t"
        "add.s64 h, %1, 6;\n\tadd.s64 l, %2, 6;\n\tadd.s64 bb, %3, 6;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], h, bb, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], l, bb, %4, q;\n}\n"
        ::"r"(d), "l"(ahi), "l"(alo), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_stage4_ss(uint32_t d, uint64_t ahi, uint64_t alo, uint64_t b, uint32_t idesc,
                                             uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t.reg .b64 h, l, bb;\n\t"
        "setp.ne.b32 p, %5, 0;\n\tsetp.eq.b32 q, %5, %5;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %4, p;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %3, %4, q;\n\t"
        "add.s64 h, %1, 2;\n\tadd.s64 l, %2, 2;\n\tadd.s64 bb, %3, 2;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], h, bb, %4, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], l, bb, %4, q;\n\t"
        "add.s64 h, %1, 4;\n\tadd.s64 l, %2, 4;\n\tadd.s64 bb, %3, 4;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], h, bb, %4, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], l, bb, %4, q;\n\t"
        "add.s64 h, %1, 6;\n\tadd.s64 l, %2, 6;\n\tadd.s64 bb, %3, 6;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], h, bb, %4, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], l, bb, %4, q;\n}\n"
        ::"r"(d), "l"(ahi), "l"(alo), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// Four K steps, A hi / A lo in TMEM (64 columns; K step k: hi at ta + 16 k,
// lo at ta + 16 k + 8), B in shared memory.
__device__ __forceinline__ void umma_stage4_pair_ts(uint32_t d, uint32_t ta, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t.reg .b32 th, tl;\n\t.reg .b64 bb;\n\t"
        "setp.ne.b32 p, %4, 0;\n\tsetp.eq.b32 q, %4, %4;\n\t"
        "add.u32 tl, %1, 8;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [tl], %2, %3, q;\n\t"
        "add.u32 th, %1, 16;\n\tadd.u32 tl, %1, 24;\n\tadd.s64 bb, %2, 2;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [th], bb, %3, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [tl], bb, %3, q;\n\t"
        "add.u32 th, %1, 32;\n\tadd.u32 tl, %1, 40;\n\tadd.s64 bb, %2, 4;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [th], bb, %3, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [tl], bb, %3, q;\n\t"
        "add.u32 th, %1, 48;\n\tadd.u32 tl, %1, 56;\n\tadd.s64 bb, %2, 6;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [th], bb, %3, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [tl], bb, %3, q;\n}\n"
        ::"r"(d), "r"(ta), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// Eight K steps (two 128-byte K atoms of B, `atom` bytes apart), A in TMEM at
// ta + 8 k, B hi / B lo in shared memory.
__device__ __forceinline__ void umma_stage8_pair_ts_b(uint32_t d, uint32_t ta, uint64_t bhi, uint64_t blo, uint32_t idesc,
                                             uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t.reg .b32 t;\n\t.reg .b64 h, l;\n\t"
        "setp.ne.b32 p, %5, 0;\n\tsetp.eq.b32 q, %5, %5;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %4, p;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %3, %4, q;\n\t"
        "add.u32 t, %1, 8;\n\tadd.s64 h, %2, 2;\n\tadd.s64 l, %3, 2;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], h, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], l, %4, q;\n\t"
        "add.u32 t, %1, 16;\n\tadd.s64 h, %2, 4;\n\tadd.s64 l, %3, 4;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], h, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], l, %4, q;\n\t"
        "add.u32 t, %1, 24;\n\tadd.s64 h, %2, 6;\n\tadd.s64 l, %3, 6;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], h, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], l, %4, q;\n\t"
        "add.u32 t, %1, 32;\n\tadd.s64 h, %2, 1024;\n\tadd.s64 l, %3, 1024;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], h, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], l, %4, q;\n\t"
        "add.u32 t, %1, 40;\n\tadd.s64 h, %2, 1026;\n\tadd.s64 l, %3, 1026;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], h, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], l, %4, q;\n\t"
        "add.u32 t, %1, 48;\n\tadd.s64 h, %2, 1028;\n\tadd.s64 l, %3, 1028;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], h, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], l, %4, q;\n\t"
        "add.u32 t, %1, 56;\n\tadd.s64 h, %2, 1030;\n\tadd.s64 l, %3, 1030;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], h, %4, q;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [t], l, %4, q;\n}\n"
        ::"r"(d), "r"(ta), "l"(bhi), "l"(blo), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive once on the barrier at `bar`'s offset in both CTAs of the pair when
// all previously issued pair MMAs of this thread complete.
__device__ __forceinline__ void umma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// Arrive once on `bar` when all previously issued tcgen05.mma of this thread complete.
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 columns of 32-bit words: thread t of the warp gets columns
// [col, col+32) of TMEM lane (lane_base + t). The load and its wait are one
// asm statement, so no use of r[] can be scheduled before the data lands.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// Store 8 columns of 32-bit words to TMEM lane (lane_base + t), no wait
// (tmem_wait_st completes every store of the thread).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
        : "memory");
}
// Store 16 columns of 32-bit words to TMEM lane (lane_base + t), no wait.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Store 32 columns of 32-bit words to TMEM lane (lane_base + t), then wait.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n\t"
        "tcgen05.wait::st.sync.aligned;"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
          "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
          "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile stored in the
// 128-byte-swizzle canonical layout: rows of 128 B (64 BF16 along K), the
// 16-byte chunks of row r permuted by chunk ^ (r & 7), 8-row groups 1024 B
// apart (stride byte offset). Tile base must be 1024-byte aligned.
__device__ __forceinline__ uint64_t sdesc_k128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);         // start address
    d |= (uint64_t)1u << 16;                          // leading byte offset (unused here)
    d |= (uint64_t)(1024u >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1u << 46;                          // descriptor version (tcgen05)
    d |= (uint64_t)2u << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of 16-byte chunk `chunk` (0..7) of row `row` in a 128B-swizzled tile.
__device__ __forceinline__ uint32_t swz128(uint32_t row, uint32_t chunk) {
    return row * 128u + ((chunk ^ (row & 7u)) << 4);
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Eight +-1 BF16 values from 8 parity bits: bit k set -> -1 (odd parity),
// clear -> +1. S = 1 - 2P exactly. Word p holds elements 2p (low half) and
// 2p+1 (high half).
__device__ __forceinline__ uint4 expand_pm1(uint32_t b) {
    // t * (2^15 + 2^30) puts bit 0 of t at 15 and bit 1 at 31 with no carries.
    uint4 o;
    o.x = ((b * 0x40008000u) & 0x80008000u) | 0x3F803F80u;
    o.y = (((b >> 2) * 0x40008000u) & 0x80008000u) | 0x3F803F80u;
    o.z = (((b >> 4) * 0x40008000u) & 0x80008000u) | 0x3F803F80u;
    o.w = (((b >> 6) * 0x40008000u) & 0x80008000u) | 0x3F803F80u;
    return o;
}

// Half-word masks (0x0000 / 0xFFFF) of 8 bits: word p masks elements 2p, 2p+1.
__device__ __forceinline__ uint4 expand_mask(uint32_t b) {
    // h * 0x10204080 places bit k of a nibble at the top of byte k (no carries);
    // prmt with sign-replicating selectors broadcasts those bits over halves.
    const uint32_t v0 = (b & 0xFu) * 0x10204080u;
    const uint32_t v1 = ((b >> 4) & 0xFu) * 0x10204080u;
    uint4 o;
    o.x = prmt(v0, 0u, 0x9988u);
    o.y = prmt(v0, 0u, 0xBBAAu);
    o.z = prmt(v1, 0u, 0x9988u);
    o.w = prmt(v1, 0u, 0xBBAAu);
    return o;
}

}  // namespace iqp
