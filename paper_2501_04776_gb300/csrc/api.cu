// The C ABI of include/iqp.h: argument checks, workspace plan and the launch
// sequence of each call. Every step of the computation runs in the kernels of
// parity.cu, simt.cu and tc.cu; this file only validates and orders them.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "parity.cuh"

namespace iqp {

// ---- kernels (parity.cu, simt.cu, tc.cu)
cudaError_t launch_parity(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr, const uint64_t *G, int64_t m,
                          int64_t ldg, uint64_t *P, int64_t ldp, uint64_t *PT, int64_t ldpt, cudaStream_t st);
cudaError_t launch_parity_gather(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr, const uint64_t *G,
                                 int64_t m, int64_t ldg, uint64_t *P, int64_t ldp, uint64_t *PT, int64_t ldpt,
                                 uint64_t *RT, cudaStream_t st, const int4 *sup = nullptr);
cudaError_t launch_parity_sum(int64_t n, const uint64_t *A, int64_t l, int64_t lda, const uint64_t *X, int64_t N,
                              int64_t ldx, int64_t *T, cudaStream_t st);
cudaError_t launch_theta_prep(const float *theta, int64_t m, int64_t mpad, float *c32, __nv_bfloat16 *hi,
                              __nv_bfloat16 *lo, cudaStream_t st);
cudaError_t launch_phase_simt(int mode, const uint64_t *PA, const uint64_t *PZ, int64_t ldp, const float *c,
                              int64_t l, int64_t s, int64_t m, double2 *part, int64_t nparts, const double *alpha,
                              const double *beta, float *W, int64_t ldw, cudaStream_t st);
cudaError_t launch_grad_simt(const float *W, int64_t ldw, const uint64_t *PZ, const uint64_t *PA, int64_t ldp,
                             int64_t l, int64_t s, int64_t m, double *gpart, cudaStream_t st);
cudaError_t launch_finalize(const double2 *part, int64_t nparts, int64_t pw, int64_t l, int64_t s, double *expval,
                            double *std_err, double *S1, double *S2, cudaStream_t st);
cudaError_t launch_grad_reduce(const double *gpart, int64_t ntiles, int64_t m, double *grad, cudaStream_t st);
cudaError_t launch_mmd_combine(const int64_t *T, const double *S1, const double *S2, int64_t l, int64_t s, int64_t N,
                               int unbiased, bool sqrt_loss, double *terms, double *alpha, double *beta, double *loss,
                               cudaStream_t st);
cudaError_t launch_phase_tc(int mode, const Plan &p, void *ws, const double *alpha, const double *beta,
                            cudaStream_t st, iqp_status *why);
cudaError_t launch_w_from_phi(const Plan &p, void *ws, const double *alpha, const double *beta, cudaStream_t st);
cudaError_t launch_grad_tc(const Plan &p, void *ws, cudaStream_t st, iqp_status *why);
int64_t grad_tc_rows(const Plan &p);
// per-translation-unit self-check words (builds with -DIQP_CHECKS; 0 otherwise)
uint32_t check_word_parity();
uint32_t check_word_simt();
uint32_t check_word_tc();
uint32_t check_word_sparse();
uint32_t check_word_bitflip();
uint32_t check_word_variants();
cudaError_t launch_timeout_selftest(uint32_t *status, uint64_t limit_ns, cudaStream_t st);
int64_t sparse_part_samples();
cudaError_t launch_sparse_stats(const uint64_t *PA, int64_t ldp, const uint64_t *PZT, int64_t ldzt, const float *c,
                                int64_t l, int64_t s, int64_t m, double2 *part, int64_t nparts,
                                const SparseIndep *indep, float *phi, int64_t ldphi, cudaStream_t st);
cudaError_t launch_sparse_grad(const uint64_t *PA, int64_t ldp, const uint64_t *PZT, int64_t ldzt, const float *c,
                               int64_t l, int64_t s, int64_t m, int64_t nparts, const double *alpha,
                               const double *beta, double *scale, unsigned long long *gfx, double *grad,
                               const SparseIndep *indep, const float *phi, int64_t ldphi, cudaStream_t st);
cudaError_t launch_sparse_value_grad(const uint64_t *PA, int64_t ldp, const uint64_t *PZT, int64_t ldzt,
                                     const float *c, int64_t l, int64_t s, int64_t m, int64_t nparts, double2 *part,
                                     const double *alpha, const double *beta, double *scale, unsigned long long *gfx,
                                     double *grad, cudaStream_t st);
cudaError_t launch_bit_transpose_batched(const uint64_t *in, int64_t batch, int64_t in_rows, int64_t in_cols,
                                         int64_t ld_in, uint64_t *out, int64_t ld_out, cudaStream_t st);
cudaError_t launch_support_list(const uint64_t *G, int64_t m, int64_t ldg, int64_t n, int4 *sup, cudaStream_t st);
cudaError_t launch_expand_params(const float *theta_p, int64_t np, const int64_t *start, int64_t m, float *theta_gen,
                                 cudaStream_t st);
cudaError_t launch_reduce_params(const double *grad_gen, int64_t m, const int64_t *start, int64_t np,
                                 double *grad_p, cudaStream_t st);
cudaError_t launch_embed_bits(const uint64_t *src, int64_t rows, int64_t ld_src, const int32_t *wires, int64_t nw,
                              uint64_t *dst, int64_t ld_dst, int64_t n, cudaStream_t st);
cudaError_t launch_uniform_bits(uint64_t seed, uint64_t stream, int64_t rows, int64_t n, int64_t ld, uint64_t *out,
                                cudaStream_t st);
cudaError_t launch_bernoulli_bits(uint64_t seed, uint64_t stream, int64_t rows, int64_t n, double p, int64_t ld,
                                  uint64_t *out, cudaStream_t st);
int64_t lo_part_samples();
int64_t lo_split_elems(int64_t n, int64_t lds);
cudaError_t launch_lo_prepare(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *Z, int64_t s,
                              int64_t ldz, const float *c, int4 *sup, uint64_t *ZT, int64_t ldzt, float *C,
                              int64_t ldc, float *M, int64_t lds, __nv_bfloat16 *split, unsigned long long *fx,
                              uint32_t *status, cudaStream_t st);
cudaError_t launch_lo_stats(const uint64_t *A, int64_t lda, int64_t n, int64_t l, const uint64_t *ZT, int64_t ldzt,
                            const float *M, int64_t lds, const float *C, int64_t ldc, int64_t s, double2 *part,
                            int64_t nparts, float *phi, int64_t ldphi, uint32_t *status, cudaStream_t st);
cudaError_t launch_lo_grad(const uint64_t *A, int64_t lda, int64_t n, int64_t l, const uint64_t *ZT, int64_t ldzt,
                           const float *M, int64_t lds, const float *C, int64_t ldc, int64_t s, int64_t m,
                           const int4 *sup, const double *alpha, const double *beta, uint64_t *AT, int64_t ldlt,
                           float *W, float *V, double *H, double *gsp, unsigned long long *Kfx, double *grad,
                           __nv_bfloat16 *split, const float *phi, int64_t ldphi, uint32_t *status,
                           cudaStream_t st);
cudaError_t launch_bitflip_gates(const float *theta, int64_t m, int64_t mpad, double *c, double *t, cudaStream_t st);
cudaError_t launch_bitflip_rows(const uint64_t *PA, int64_t ldp, int64_t l, const double *c, double *expval,
                                cudaStream_t st);
cudaError_t launch_bitflip_grad(const uint64_t *PAT, int64_t ldlt, int64_t m, int64_t l, const double *w,
                                const double *ev, double *v, const double *t, double *grad, cudaStream_t st);

// ---------------------------------------------------------------- plan

Plan make_plan(int op, int64_t n, int64_t m, int64_t l, int64_t s, int64_t N, int prec) {
    Plan p;
    std::memset(&p, 0, sizeof(p));
    p.indep = op >= IQP_OP_EXPVAL_INDEP && op <= IQP_OP_MMD_LOSS_GRAD_INDEP;
    if (p.indep) prec = IQP_SPARSE_FP32;  // the independent-batch estimator is row-sparse FP32
    p.op = op;
    p.prec = prec;
    p.n = n;
    p.m = m;
    p.l = l;
    p.s = s;
    p.N = N;
    p.ldp = round_up(cdiv(m, 64), 4);
    p.ldzt = round_up(cdiv(s, 64), 4);
    p.ldlt = round_up(cdiv(l, 64), 4);
    p.mpad = p.ldp * 64;
    p.ldw = round_up(s, 64);
    p.pw = prec == IQP_SPLIT_BF16    ? kPartColsTc
           : prec == IQP_SPARSE_FP32 ? sparse_part_samples()
           : prec == IQP_LOWORDER_FP32 ? lo_part_samples()
                                       : kPartColsSimt;
    p.ldc = round_up(n, 4);
    p.nparts = cdiv(s, p.pw);
    p.natile = 2 * cdiv(l, kATile);  // enough for every gradient kernel form (at least 128 observables per tile)
    const bool grad = op == IQP_OP_EXPVAL_GRAD || op == IQP_OP_MMD_LOSS_GRAD || op == IQP_OP_EXPVAL_INDEP_GRAD ||
                      op == IQP_OP_MMD_LOSS_GRAD_INDEP;
    const bool mmd = op == IQP_OP_MMD_LOSS || op == IQP_OP_MMD_LOSS_GRAD || op == IQP_OP_MMD_LOSS_INDEP ||
                     op == IQP_OP_MMD_LOSS_GRAD_INDEP;
    const bool indep = p.indep;
    const bool bitflip = op == IQP_OP_BITFLIP;
    const bool sparse = prec == IQP_SPARSE_FP32 && !bitflip;
    const bool lo = prec == IQP_LOWORDER_FP32 && !bitflip && !indep;
    size_t off = 0;
    auto take = [&](int64_t bytes) {
        const size_t o = off;
        off += (size_t)round_up(bytes > 0 ? bytes : 0, 256);
        return o;
    };
    p.off_status = take(256);
    p.off_pa = take(lo ? 0 : l * p.ldp * 8);
    p.off_pz = take(bitflip || sparse || lo ? 0 : s * p.ldp * 8);
    p.off_pzt = take(bitflip || indep ? 0 : (lo ? n : m) * p.ldzt * 8);  // low-order: the samples transposed
    p.off_pat = take(lo ? 0 : m * p.ldlt * 8);
    p.off_rt = take(n * (p.ldzt + p.ldlt) * 8);  // R^T of A, then of Z (one fused parity launch for both)
    p.off_c = take(bitflip ? p.mpad * 16 : p.mpad * 4);  // bitflip: cos(2 theta), -2 tan(2 theta) in FP64
    p.off_part = take(bitflip ? l * 16 : l * p.nparts * 16);  // bitflip: expval, w * expval
    p.off_w = take(grad && !sparse ? l * p.ldw * 4 : 0);
    p.off_lo_c = take(lo ? (n + 1) * p.ldc * 4 + n * cdiv(n, 64) * 8 : 0);  // C, d, pair-existence bits E
    p.off_lo_m = take(lo ? n * p.ldw * 4 : 0);
    p.off_lo_v = take(lo && grad ? n * p.ldw * 4 : 0);
    p.off_lo_h = take(lo && grad ? n * p.ldc * 8 : 0);
    p.off_lo_gs = take(lo && grad ? n * cdiv(s, lo_part_samples()) * 8 : 0);
    p.off_lo_a = take(lo ? lo_split_elems(n, p.ldw) * 2 : 0);  // split-BF16 operand of the pair contractions
    // sparse: 64-bit fixed-point gradient accumulators and their scale
    // low-order: also the fixed-point sums that build C and d (n x n + n, and
    // the largest |c_j|), before the gradient's pair corrections reuse it
    p.off_gpart = take(lo ? n * n * 8 + n * 8 + 64 : (grad ? (sparse ? m * 8 + 8 : p.natile * m * 8) : 0));
    p.off_ab = take(mmd ? l * 16 : 0);
    p.off_s12 = take(mmd ? l * 16 : 0);
    p.off_T = take(mmd ? l * 8 : 0);
    p.off_terms = take(mmd ? l * 8 : 0);
    p.off_zt = take(indep ? l * n * p.ldzt * 8 : 0);  // every batch transposed: n rows of bits over samples
    p.off_sup = take(m * 16);  // int4 support list per gate (parity gathers, independent batches, low-order)
    // MMD gradient (split BF16, row-sparse; shared batches): Phi kept from
    // the statistics pass, so W needs no second phase pass (the loss's alpha,
    // beta come between). The low-order form keeps it in its W buffer.
    p.off_phi = (op == IQP_OP_MMD_LOSS_GRAD && (prec == IQP_SPLIT_BF16 || prec == IQP_SPARSE_FP32)) ? take(l * p.ldw * 4)
                                                                                                : 0;
    p.phi = nullptr;
    p.ldphi = 0;
    p.phi_out = p.phi_in = false;
    // Last, and optional: the split-tile scratch of the tensor-core phase (a
    // workspace that ends before it runs every phase tile whole), the running
    // sums of the two-sample-tile phase kernels (a workspace that ends before
    // them runs one sample tile per tile), and the scratch of their balanced
    // last round (a workspace that ends before it runs that round as single
    // tiles).
    p.off_skp = p.off_gsum = p.off_skx = 0;
    if (prec == IQP_SPLIT_BF16 && !bitflip && !indep) {
        p.off_skp = take((int64_t)kMaxSplitCtas * kSplitSlotFloats * 4 + (int64_t)kMaxSplitCtas * 4);
        p.off_gsum = take((int64_t)kMaxSplitCtas * kDtSumFloats * 4);
        p.off_skx = take((int64_t)kSplitSlots * kSplitSlotFloats * 4 + (int64_t)kMaxSplitCtas * 4);
    }
    p.total = off;
    return p;
}

// Bytes of the workspace below which `p` cannot run (the optional regions at
// its end left out).
size_t plan_min_bytes(const Plan &p) { return p.off_skp != 0 ? p.off_skp : p.total; }

// The smallest workspace `op` runs with (iqp_workspace_bytes less the
// optional split-tile scratch at its end); 0 for invalid arguments (the
// checks of iqp_workspace_bytes).
size_t workspace_min_bytes(int op, int64_t n, int64_t m, int64_t l, int64_t s, int64_t N, int prec) {
    if (n < 1 || m < 1 || l < 1 || s < 1) return 0;
    if (op < IQP_OP_EXPVAL || op > IQP_OP_MMD_LOSS_GRAD_INDEP) return 0;
    if (prec != IQP_FP32 && prec != IQP_SPLIT_BF16 && prec != IQP_SPARSE_FP32 && prec != IQP_LOWORDER_FP32) return 0;
    return plan_min_bytes(make_plan(op, n, m, l, s, N, prec));
}

// ---------------------------------------------------------------- misc

static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_profiling{0};
static std::mutex g_prof_mu;
struct PendingEvent {
    int kernel;
    cudaEvent_t a, b;
};
static std::vector<PendingEvent> g_pending;
static double g_prof_ms[IQP_KERNEL_COUNT];
static uint64_t g_prof_n[IQP_KERNEL_COUNT];

// A stream being captured into a CUDA graph gets no timing events: events
// recorded into a capture exist only inside the graph, and waiting on them
// from the host would fail or block.
static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

LaunchScope::LaunchScope(int k, cudaStream_t s) : kernel(k), st(s), ev0(nullptr), ev1(nullptr) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_profiling.load(std::memory_order_relaxed) && !capturing(s)) {
        if (cudaEventCreate(&ev0) == cudaSuccess && cudaEventCreate(&ev1) == cudaSuccess) {
            cudaEventRecord(ev0, st);
        } else {
            ev0 = ev1 = nullptr;
        }
    }
}

LaunchScope::~LaunchScope() {
    if (ev0 != nullptr) {
        cudaEventRecord(ev1, st);
        std::lock_guard<std::mutex> g(g_prof_mu);
        g_pending.push_back({kernel, ev0, ev1});
    }
}

static void drain_pending() {
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_prof_ms[p.kernel] += ms;
            g_prof_n[p.kernel] += 1;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
}

iqp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? IQP_OK : IQP_ERR_CUDA; }

int num_sms() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return v;
}

int device_cc() {
    int dev = 0, ma = 0, mi = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev);
    return ma * 10 + mi;
}

namespace {

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

iqp_status check_bits(const uint64_t *M, int64_t rows, int64_t ld, int64_t n) {
    if (rows < 1) return IQP_ERR_ARG;
    if (M == nullptr) return IQP_ERR_ARG;
    if (ld < cdiv(n, 64) || (ld & 1)) return IQP_ERR_ARG;
    if (!aligned(M, 16)) return IQP_ERR_ALIGN;
    return IQP_OK;
}

iqp_status check_common(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                        int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                        iqp_precision prec) {
    if (n < 1 || m < 1 || l < 1 || s < 1) return IQP_ERR_ARG;
    if (m > (int64_t)1 << 36 || l > (int64_t)1 << 31 || s > (int64_t)1 << 31) return IQP_ERR_ARG;
    iqp_status st;
    if ((st = check_bits(G, m, ldg, n)) != IQP_OK) return st;
    if ((st = check_bits(A, l, lda, n)) != IQP_OK) return st;
    if ((st = check_bits(Z, s, ldz, n)) != IQP_OK) return st;
    if (theta == nullptr) return IQP_ERR_ARG;
    if (!aligned(theta, 4)) return IQP_ERR_ALIGN;
    if (prec != IQP_FP32 && prec != IQP_SPLIT_BF16 && prec != IQP_SPARSE_FP32 && prec != IQP_LOWORDER_FP32)
        return IQP_ERR_ARG;
    if (prec == IQP_SPLIT_BF16 && !iqp_tensor_path_available()) return IQP_ERR_UNSUPPORTED;
    // low-order form: observables on grid x, 256-sample blocks on y; its n x n
    // pair matrices (C, H, K: 20 n^2 bytes) bound n
    if (prec == IQP_LOWORDER_FP32 && (l > INT32_MAX || n > 65536 || cdiv(s, (int64_t)256) > 65535))
        return IQP_ERR_ARG;
    // sparse grid: observables on x (< 2^31), 2048-sample blocks on y (< 65536)
    if (prec == IQP_SPARSE_FP32 && (l > INT32_MAX || cdiv(s, (int64_t)2048) > 65535)) return IQP_ERR_ARG;
    return IQP_OK;
}

iqp_status check_ws(Plan &p, void *ws, size_t ws_bytes) {
    if (ws == nullptr || !aligned(ws, 256)) return IQP_ERR_WORKSPACE;
    if (ws_bytes < p.total) {
        if (ws_bytes < plan_min_bytes(p)) return IQP_ERR_WORKSPACE;
        // The optional regions at the end, in order: each is used only where
        // the workspace reaches its end.
        p.off_skx = 0;  // the two-tile last round runs as single tiles
        if (p.off_gsum != 0 && ws_bytes < p.off_gsum + (size_t)kMaxSplitCtas * kDtSumFloats * 4)
            p.off_gsum = 0;  // one sample tile per tile
        if (p.off_skp != 0 && ws_bytes < p.off_skp + (size_t)round_up((int64_t)kMaxSplitCtas * kSplitSlotFloats * 4 +
                                                                       (int64_t)kMaxSplitCtas * 4, 256))
            p.off_skp = 0;  // phase tiles run whole
    }
    return IQP_OK;
}

template <class T>
T *at(void *ws, size_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

#define IQP_TRY(expr)                                   \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return IQP_ERR_CUDA;     \
    } while (0)

// Parities of A and Z by support gather (P_A, P_A^T, P_Z, P_Z^T) + theta split.
// Independent batches: P_A, every batch of Z transposed, and the gate
// supports (the sample parities are formed inside the row-sparse kernels).
iqp_status prepare(const Plan &p, void *ws, const uint64_t *G, int64_t ldg, const uint64_t *A, int64_t lda,
                   const uint64_t *Z, int64_t ldz, const float *theta, cudaStream_t st) {
    uint64_t *rt = at<uint64_t>(ws, p.off_rt);
    if (p.prec == IQP_LOWORDER_FP32 && !p.indep) {
        // no parity matrices: C, d, the samples transposed and M = C S
        IQP_TRY(launch_theta_prep(theta, p.m, p.mpad, at<float>(ws, p.off_c), nullptr, nullptr, st));
        IQP_TRY(launch_lo_prepare(p.n, G, p.m, ldg, Z, p.s, ldz, at<float>(ws, p.off_c), at<int4>(ws, p.off_sup),
                                  at<uint64_t>(ws, p.off_pzt), p.ldzt, at<float>(ws, p.off_lo_c), p.ldc,
                                  at<float>(ws, p.off_lo_m), p.ldw, at<__nv_bfloat16>(ws, p.off_lo_a),
                                  at<unsigned long long>(ws, p.off_gpart), at<uint32_t>(ws, p.off_status), st));
        return IQP_OK;
    }
    const int4 *sup = at<int4>(ws, p.off_sup);
    if (!p.indep && p.prec != IQP_SPARSE_FP32) {
        // P_A, P_A^T, P_Z, P_Z^T: the support list with both transposes in one launch, both gathers in one
        const ParitySide sides[2] = {
            {A, p.l, lda, at<uint64_t>(ws, p.off_pa), at<uint64_t>(ws, p.off_pat), p.ldlt, rt},
            {Z, p.s, ldz, at<uint64_t>(ws, p.off_pz), at<uint64_t>(ws, p.off_pzt), p.ldzt, rt + p.n * p.ldlt}};
        IQP_TRY(launch_parity_gather_fused(p.n, G, p.m, ldg, at<int4>(ws, p.off_sup), true, p.ldp, sides, 2, st));
        if (p.prec == IQP_SPLIT_BF16) {
            __nv_bfloat16 *hi = at<__nv_bfloat16>(ws, p.off_c);
            IQP_TRY(launch_theta_prep(theta, p.m, p.mpad, nullptr, hi, hi + p.mpad, st));
        } else {
            IQP_TRY(launch_theta_prep(theta, p.m, p.mpad, at<float>(ws, p.off_c), nullptr, nullptr, st));
        }
        return IQP_OK;
    }
    IQP_TRY(launch_support_list(G, p.m, ldg, p.n, at<int4>(ws, p.off_sup), st));
    IQP_TRY(launch_parity_gather(p.n, A, p.l, lda, G, p.m, ldg, at<uint64_t>(ws, p.off_pa), p.ldp,
                                 at<uint64_t>(ws, p.off_pat), p.ldlt, rt, st, sup));
    if (p.indep) {
        IQP_TRY(launch_bit_transpose_batched(Z, p.l, p.s, p.n, ldz, at<uint64_t>(ws, p.off_zt), p.ldzt, st));
        IQP_TRY(launch_theta_prep(theta, p.m, p.mpad, at<float>(ws, p.off_c), nullptr, nullptr, st));
        return IQP_OK;
    }
    // The sparse form reads only P_Z^T (bits over samples).
    IQP_TRY(launch_parity_gather(p.n, Z, p.s, ldz, G, p.m, ldg,
                                 p.prec == IQP_SPARSE_FP32 ? nullptr : at<uint64_t>(ws, p.off_pz), p.ldp,
                                 at<uint64_t>(ws, p.off_pzt), p.ldzt, rt, st, sup));
    if (p.prec == IQP_SPLIT_BF16) {
        __nv_bfloat16 *hi = at<__nv_bfloat16>(ws, p.off_c);
        IQP_TRY(launch_theta_prep(theta, p.m, p.mpad, nullptr, hi, hi + p.mpad, st));
    } else {
        IQP_TRY(launch_theta_prep(theta, p.m, p.mpad, at<float>(ws, p.off_c), nullptr, nullptr, st));
    }
    return IQP_OK;
}

// Phase contraction with the statistics epilogue -> (expval, std_err, S1, S2).
iqp_status forward_stats(const Plan &p, void *ws, double *expval, double *std_err, double *S1, double *S2,
                         cudaStream_t st) {
    double2 *part = at<double2>(ws, p.off_part);
    if (p.prec == IQP_SPLIT_BF16) {
        iqp_status why = IQP_OK;
        if (launch_phase_tc(0, p, ws, nullptr, nullptr, st, &why) != cudaSuccess)
            return why != IQP_OK ? why : IQP_ERR_CUDA;
    } else if (p.prec == IQP_LOWORDER_FP32) {
        IQP_TRY(launch_lo_stats(p.A, p.lda, p.n, p.l, at<uint64_t>(ws, p.off_pzt), p.ldzt, at<float>(ws, p.off_lo_m),
                                p.ldw, at<float>(ws, p.off_lo_c), p.ldc, p.s, part, p.nparts,
                                p.phi_out ? p.phi : nullptr, p.ldphi, at<uint32_t>(ws, p.off_status), st));
    } else if (p.prec == IQP_SPARSE_FP32) {
        const SparseIndep ind{at<int4>(ws, p.off_sup), p.G, p.ldg, p.n};
        IQP_TRY(launch_sparse_stats(at<uint64_t>(ws, p.off_pa), p.ldp,
                                    at<uint64_t>(ws, p.indep ? p.off_zt : p.off_pzt), p.ldzt, at<float>(ws, p.off_c),
                                    p.l, p.s, p.m, part, p.nparts, p.indep ? &ind : nullptr,
                                    p.phi_out ? p.phi : nullptr, p.ldphi, st));
    } else {
        IQP_TRY(launch_phase_simt(0, at<uint64_t>(ws, p.off_pa), at<uint64_t>(ws, p.off_pz), p.ldp,
                                  at<float>(ws, p.off_c), p.l, p.s, p.m, part, p.nparts, nullptr, nullptr, nullptr, 0,
                                  st));
    }
    IQP_TRY(launch_finalize(part, p.nparts, p.pw, p.l, p.s, expval, std_err, S1, S2, st));
    return IQP_OK;
}

// Recompute Phi tile by tile into W, contract against S_Z and mask by P_A.
iqp_status backward(const Plan &p, void *ws, const double *alpha, const double *beta, double *grad,
                    cudaStream_t st) {
    double *gpart = at<double>(ws, p.off_gpart);
    if (p.prec == IQP_LOWORDER_FP32) {
        IQP_TRY(launch_lo_grad(p.A, p.lda, p.n, p.l, at<uint64_t>(ws, p.off_pzt), p.ldzt, at<float>(ws, p.off_lo_m),
                               p.ldw, at<float>(ws, p.off_lo_c), p.ldc, p.s, p.m, at<int4>(ws, p.off_sup), alpha, beta,
                               at<uint64_t>(ws, p.off_rt), p.ldlt, at<float>(ws, p.off_w), at<float>(ws, p.off_lo_v),
                               at<double>(ws, p.off_lo_h), at<double>(ws, p.off_lo_gs),
                               at<unsigned long long>(ws, p.off_gpart), grad, at<__nv_bfloat16>(ws, p.off_lo_a),
                               p.phi_in ? p.phi : nullptr, p.ldphi, at<uint32_t>(ws, p.off_status), st));
        return IQP_OK;
    }
    if (p.prec == IQP_SPARSE_FP32) {
        unsigned long long *gfx = at<unsigned long long>(ws, p.off_gpart);
        const SparseIndep ind{at<int4>(ws, p.off_sup), p.G, p.ldg, p.n};
        IQP_TRY(launch_sparse_grad(at<uint64_t>(ws, p.off_pa), p.ldp,
                                   at<uint64_t>(ws, p.indep ? p.off_zt : p.off_pzt), p.ldzt, at<float>(ws, p.off_c),
                                   p.l, p.s, p.m, p.nparts, alpha, beta, reinterpret_cast<double *>(gfx + p.m), gfx,
                                   grad, p.indep ? &ind : nullptr, p.phi_in ? p.phi : nullptr, p.ldphi, st));
        return IQP_OK;
    }
    if (p.prec == IQP_SPLIT_BF16) {
        iqp_status why = IQP_OK;
        if (p.phi_in) {
            IQP_TRY(launch_w_from_phi(p, ws, alpha, beta, st));
        } else if (launch_phase_tc(1, p, ws, alpha, beta, st, &why) != cudaSuccess) {
            return why != IQP_OK ? why : IQP_ERR_CUDA;
        }
        if (launch_grad_tc(p, ws, st, &why) != cudaSuccess) return why != IQP_OK ? why : IQP_ERR_CUDA;
    } else {
        float *W = at<float>(ws, p.off_w);
        IQP_TRY(launch_phase_simt(1, at<uint64_t>(ws, p.off_pa), at<uint64_t>(ws, p.off_pz), p.ldp,
                                  at<float>(ws, p.off_c), p.l, p.s, p.m, nullptr, 0, alpha, beta, W, p.ldw, st));
        IQP_TRY(launch_grad_simt(W, p.ldw, at<uint64_t>(ws, p.off_pz), at<uint64_t>(ws, p.off_pa), p.ldp, p.l, p.s,
                                 p.m, gpart, st));
    }
    IQP_TRY(launch_grad_reduce(gpart, p.prec == IQP_SPLIT_BF16 ? grad_tc_rows(p) : cdiv(p.l, kATile), p.m, grad, st));
    return IQP_OK;
}

iqp_status mmd_core(int op, int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                    int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const uint64_t *X, int64_t N,
                    int64_t ldx, const float *theta, iqp_precision prec, int flags, double *loss, double *grad,
                    void *ws, size_t ws_bytes, void *stream) {
    iqp_status rc = check_common(n, G, m, ldg, A, l, lda, Z, s, ldz, theta,
                                 (flags & IQP_MMD_INDEP) ? IQP_SPARSE_FP32 : prec);
    if (rc != IQP_OK) return rc;
    if ((rc = check_bits(X, N, ldx, n)) != IQP_OK) return rc;
    if (loss == nullptr || !aligned(loss, 8)) return IQP_ERR_ARG;
    if (op == IQP_OP_MMD_LOSS_GRAD && (grad == nullptr || !aligned(grad, 8))) return IQP_ERR_ARG;
    if (flags & ~(IQP_MMD_UNBIASED | IQP_MMD_SQRT | IQP_MMD_INDEP)) return IQP_ERR_ARG;
    const int unbiased = flags & IQP_MMD_UNBIASED;
    if (unbiased && (s < 2 || N < 2)) return IQP_ERR_ARG;
    const bool indep = (flags & IQP_MMD_INDEP) != 0;
    if (indep && l > INT32_MAX / 2) return IQP_ERR_ARG;
    const bool g = op == IQP_OP_MMD_LOSS_GRAD;
    const int pop = indep ? (g ? IQP_OP_MMD_LOSS_GRAD_INDEP : IQP_OP_MMD_LOSS_INDEP) : op;
    Plan p = make_plan(pop, n, m, l, s, N, prec);
    p.G = G;
    p.ldg = ldg;
    p.A = A;
    p.lda = lda;
    if ((rc = check_ws(p, ws, ws_bytes)) != IQP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = prepare(p, ws, G, ldg, A, lda, Z, ldz, theta, st)) != IQP_OK) return rc;
    double *S1 = at<double>(ws, p.off_s12), *S2 = S1 + l;
    if (g && (p.prec == IQP_LOWORDER_FP32 || p.off_phi != 0)) {  // Phi kept for the gradient pass
        p.phi = at<float>(ws, p.prec == IQP_LOWORDER_FP32 ? p.off_w : p.off_phi);
        p.ldphi = p.ldw;
        p.phi_out = p.phi_in = true;
    }
    if ((rc = forward_stats(p, ws, nullptr, nullptr, S1, S2, st)) != IQP_OK) return rc;
    int64_t *T = at<int64_t>(ws, p.off_T);
    IQP_TRY(launch_parity_sum(n, A, l, lda, X, N, ldx, T, st));
    double *alpha = at<double>(ws, p.off_ab), *beta = alpha + l;
    IQP_TRY(launch_mmd_combine(T, S1, S2, l, s, N, unbiased, (flags & IQP_MMD_SQRT) != 0,
                               at<double>(ws, p.off_terms), alpha, beta, loss, st));
    if (g) return backward(p, ws, alpha, beta, grad, st);
    return IQP_OK;
}

}  // namespace

// The host-side checks iqp_expval runs before it touches the workspace.
iqp_status expval_arg_check(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                            int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                            iqp_precision prec, const double *expval, const double *std_err) {
    const iqp_status rc = check_common(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, prec);
    if (rc != IQP_OK) return rc;
    if ((expval && !aligned(expval, 8)) || (std_err && !aligned(std_err, 8))) return IQP_ERR_ALIGN;
    return IQP_OK;
}

namespace {

uint64_t spin_limit_ns() {
    const char *e = std::getenv("IQP_SPIN_LIMIT_MS");
    double ms = e ? std::atof(e) : 4000.0;
    if (!(ms > 0.0)) ms = 4000.0;
    if (ms > 60000.0) ms = 60000.0;
    return (uint64_t)(ms * 1e6);
}

}  // namespace

uint64_t default_spin_limit_ns() { return spin_limit_ns(); }

}  // namespace iqp

using namespace iqp;

extern "C" {

size_t iqp_workspace_bytes(iqp_op op, int64_t n, int64_t m, int64_t l, int64_t s, int64_t N, iqp_precision prec) {
    if (n < 1 || m < 1 || l < 1 || s < 1) return 0;
    if (op < IQP_OP_EXPVAL || op > IQP_OP_MMD_LOSS_GRAD_INDEP) return 0;
    if (prec != IQP_FP32 && prec != IQP_SPLIT_BF16 && prec != IQP_SPARSE_FP32 && prec != IQP_LOWORDER_FP32) return 0;
    return make_plan(op, n, m, l, s, N, prec).total;
}


iqp_status iqp_parity(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr, const uint64_t *G, int64_t m,
                      int64_t ldg, uint64_t *P, int64_t ldp, void *stream) {
    if (n < 1 || m < 1) return IQP_ERR_ARG;
    iqp_status rc;
    if ((rc = check_bits(R, rows, ldr, n)) != IQP_OK) return rc;
    if ((rc = check_bits(G, m, ldg, n)) != IQP_OK) return rc;
    if (P == nullptr) return IQP_ERR_ARG;
    if (ldp < cdiv(m, 64) || (ldp & 1)) return IQP_ERR_ARG;
    if (!aligned(P, 16)) return IQP_ERR_ALIGN;
    return cuda_status(launch_parity(n, R, rows, ldr, G, m, ldg, P, ldp, nullptr, 0, static_cast<cudaStream_t>(stream)));
}

iqp_status iqp_parity_gather(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr, const uint64_t *G, int64_t m,
                             int64_t ldg, uint64_t *P, int64_t ldp, uint64_t *PT, int64_t ldpt, uint64_t *scratch,
                             void *stream) {
    if (n < 1 || m < 1) return IQP_ERR_ARG;
    iqp_status rc;
    if ((rc = check_bits(R, rows, ldr, n)) != IQP_OK) return rc;
    if ((rc = check_bits(G, m, ldg, n)) != IQP_OK) return rc;
    if (PT == nullptr || scratch == nullptr) return IQP_ERR_ARG;
    if (ldpt < cdiv(rows, 64) || (ldpt & 1)) return IQP_ERR_ARG;
    if (P != nullptr && (ldp < cdiv(m, 64) || (ldp & 1))) return IQP_ERR_ARG;
    if (!aligned(PT, 16) || !aligned(scratch, 16) || (P && !aligned(P, 16))) return IQP_ERR_ALIGN;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (P == nullptr) return cuda_status(launch_parity_gather(n, R, rows, ldr, G, m, ldg, P, ldp, PT, ldpt, scratch, st));
    // the support list after R^T (n * ldpt words, an even count: 16-byte aligned), then the fused pass
    int4 *sup = reinterpret_cast<int4 *>(scratch + n * ldpt);
    cudaError_t e = launch_support_list(G, m, ldg, n, sup, st);
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(launch_parity_gather(n, R, rows, ldr, G, m, ldg, P, ldp, PT, ldpt, scratch, st, sup));
}

iqp_status iqp_parity_sum(int64_t n, const uint64_t *A, int64_t l, int64_t lda, const uint64_t *X, int64_t N,
                          int64_t ldx, int64_t *T, void *stream) {
    if (n < 1) return IQP_ERR_ARG;
    iqp_status rc;
    if ((rc = check_bits(A, l, lda, n)) != IQP_OK) return rc;
    if ((rc = check_bits(X, N, ldx, n)) != IQP_OK) return rc;
    if (T == nullptr) return IQP_ERR_ARG;
    if (!aligned(T, 8)) return IQP_ERR_ALIGN;
    return cuda_status(launch_parity_sum(n, A, l, lda, X, N, ldx, T, static_cast<cudaStream_t>(stream)));
}

iqp_status iqp_expval(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l, int64_t lda,
                      const uint64_t *Z, int64_t s, int64_t ldz, const float *theta, iqp_precision prec,
                      double *expval, double *std_err, void *ws, size_t ws_bytes, void *stream) {
    iqp_status rc = expval_arg_check(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, prec, expval, std_err);
    if (rc != IQP_OK) return rc;
    Plan p = make_plan(IQP_OP_EXPVAL, n, m, l, s, 0, prec);
    p.G = G;
    p.ldg = ldg;
    p.A = A;
    p.lda = lda;
    if ((rc = check_ws(p, ws, ws_bytes)) != IQP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = prepare(p, ws, G, ldg, A, lda, Z, ldz, theta, st)) != IQP_OK) return rc;
    return forward_stats(p, ws, expval, std_err, nullptr, nullptr, st);
}

iqp_status iqp_expval_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                           int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                           const double *alpha, const double *beta, iqp_precision prec, double *grad, void *ws,
                           size_t ws_bytes, void *stream) {
    iqp_status rc = check_common(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, prec);
    if (rc != IQP_OK) return rc;
    if (alpha == nullptr || grad == nullptr) return IQP_ERR_ARG;
    if (!aligned(alpha, 8) || !aligned(grad, 8) || (beta && !aligned(beta, 8))) return IQP_ERR_ALIGN;
    Plan p = make_plan(IQP_OP_EXPVAL_GRAD, n, m, l, s, 0, prec);
    p.G = G;
    p.ldg = ldg;
    p.A = A;
    p.lda = lda;
    if ((rc = check_ws(p, ws, ws_bytes)) != IQP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = prepare(p, ws, G, ldg, A, lda, Z, ldz, theta, st)) != IQP_OK) return rc;
    return backward(p, ws, alpha, beta, grad, st);
}

// Arguments of a caller-owned kept Phi: l x ldphi FP32, ldphi a multiple of
// 64 and >= s, 16-byte aligned; precisions with a Phi-keeping statistics pass.
static iqp_status check_phi(const float *phi, int64_t ldphi, int64_t s, iqp_precision prec) {
    if (phi == nullptr || ldphi < s || ldphi % 64 != 0) return IQP_ERR_ARG;
    if (!aligned(phi, 16)) return IQP_ERR_ALIGN;
    if (prec != IQP_SPLIT_BF16 && prec != IQP_SPARSE_FP32 && prec != IQP_LOWORDER_FP32) return IQP_ERR_UNSUPPORTED;
    return IQP_OK;
}

iqp_status iqp_expval_keep_phi(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                               int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                               iqp_precision prec, double *expval, double *std_err, float *phi, int64_t ldphi,
                               void *ws, size_t ws_bytes, void *stream) {
    iqp_status rc = check_common(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, prec);
    if (rc != IQP_OK) return rc;
    if ((rc = check_phi(phi, ldphi, s, prec)) != IQP_OK) return rc;
    if ((expval && !aligned(expval, 8)) || (std_err && !aligned(std_err, 8))) return IQP_ERR_ALIGN;
    Plan p = make_plan(IQP_OP_EXPVAL, n, m, l, s, 0, prec);
    p.G = G;
    p.ldg = ldg;
    p.A = A;
    p.lda = lda;
    if ((rc = check_ws(p, ws, ws_bytes)) != IQP_OK) return rc;
    p.phi = phi;
    p.ldphi = ldphi;
    p.phi_out = true;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = prepare(p, ws, G, ldg, A, lda, Z, ldz, theta, st)) != IQP_OK) return rc;
    return forward_stats(p, ws, expval, std_err, nullptr, nullptr, st);
}

iqp_status iqp_expval_grad_from_phi(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A,
                                    int64_t l, int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz,
                                    const float *theta, const double *alpha, const double *beta, iqp_precision prec,
                                    const float *phi, int64_t ldphi, double *grad, void *ws, size_t ws_bytes,
                                    void *stream) {
    iqp_status rc = check_common(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, prec);
    if (rc != IQP_OK) return rc;
    if ((rc = check_phi(phi, ldphi, s, prec)) != IQP_OK) return rc;
    if (alpha == nullptr || grad == nullptr) return IQP_ERR_ARG;
    if (!aligned(alpha, 8) || !aligned(grad, 8) || (beta && !aligned(beta, 8))) return IQP_ERR_ALIGN;
    Plan p = make_plan(IQP_OP_EXPVAL_GRAD, n, m, l, s, 0, prec);
    p.G = G;
    p.ldg = ldg;
    p.A = A;
    p.lda = lda;
    if ((rc = check_ws(p, ws, ws_bytes)) != IQP_OK) return rc;
    p.phi = const_cast<float *>(phi);  // read only: phi_in
    p.ldphi = ldphi;
    p.phi_in = true;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = prepare(p, ws, G, ldg, A, lda, Z, ldz, theta, st)) != IQP_OK) return rc;
    return backward(p, ws, alpha, beta, grad, st);
}

iqp_status iqp_expval_value_and_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A,
                                     int64_t l, int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz,
                                     const float *theta, const double *alpha, const double *beta, iqp_precision prec,
                                     double *expval, double *std_err, double *grad, void *ws, size_t ws_bytes,
                                     void *stream) {
    iqp_status rc = check_common(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, prec);
    if (rc != IQP_OK) return rc;
    if (alpha == nullptr || grad == nullptr) return IQP_ERR_ARG;
    if (!aligned(alpha, 8) || !aligned(grad, 8) || (beta && !aligned(beta, 8)) || (expval && !aligned(expval, 8)) ||
        (std_err && !aligned(std_err, 8)))
        return IQP_ERR_ALIGN;
    Plan p = make_plan(IQP_OP_EXPVAL_GRAD, n, m, l, s, 0, prec);
    p.G = G;
    p.ldg = ldg;
    p.A = A;
    p.lda = lda;
    if ((rc = check_ws(p, ws, ws_bytes)) != IQP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = prepare(p, ws, G, ldg, A, lda, Z, ldz, theta, st)) != IQP_OK) return rc;
    if (prec == IQP_SPARSE_FP32) {  // one pass over Phi: statistics, W and the gradient contributions
        unsigned long long *gfx = at<unsigned long long>(ws, p.off_gpart);
        double2 *part = at<double2>(ws, p.off_part);
        IQP_TRY(launch_sparse_value_grad(at<uint64_t>(ws, p.off_pa), p.ldp, at<uint64_t>(ws, p.off_pzt), p.ldzt,
                                         at<float>(ws, p.off_c), p.l, p.s, p.m, p.nparts, part, alpha, beta,
                                         reinterpret_cast<double *>(gfx + p.m), gfx, grad, st));
        IQP_TRY(launch_finalize(part, p.nparts, p.pw, p.l, p.s, expval, std_err, nullptr, nullptr, st));
        return IQP_OK;
    }
    if (prec != IQP_SPLIT_BF16) {
        if (prec == IQP_LOWORDER_FP32) {  // W from the kept Phi (in the W buffer), no second phase pass
            p.phi = at<float>(ws, p.off_w);
            p.ldphi = p.ldw;
            p.phi_out = p.phi_in = true;
        }
        if ((rc = forward_stats(p, ws, expval, std_err, nullptr, nullptr, st)) != IQP_OK) return rc;
        return backward(p, ws, alpha, beta, grad, st);
    }
    iqp_status why = IQP_OK;
    if (launch_phase_tc(2, p, ws, alpha, beta, st, &why) != cudaSuccess) return why != IQP_OK ? why : IQP_ERR_CUDA;
    IQP_TRY(launch_finalize(at<double2>(ws, p.off_part), p.nparts, p.pw, p.l, p.s, expval, std_err, nullptr, nullptr,
                            st));
    if (launch_grad_tc(p, ws, st, &why) != cudaSuccess) return why != IQP_OK ? why : IQP_ERR_CUDA;
    IQP_TRY(launch_grad_reduce(at<double>(ws, p.off_gpart), grad_tc_rows(p), p.m, grad, st));
    return IQP_OK;
}

iqp_status iqp_mmd_loss(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                        int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const uint64_t *X, int64_t N,
                        int64_t ldx, const float *theta, iqp_precision prec, int unbiased, double *loss, void *ws,
                        size_t ws_bytes, void *stream) {
    return mmd_core(IQP_OP_MMD_LOSS, n, G, m, ldg, A, l, lda, Z, s, ldz, X, N, ldx, theta, prec, unbiased, loss,
                    nullptr, ws, ws_bytes, stream);
}

iqp_status iqp_mmd_loss_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                             int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const uint64_t *X, int64_t N,
                             int64_t ldx, const float *theta, iqp_precision prec, int unbiased, double *loss,
                             double *grad, void *ws, size_t ws_bytes, void *stream) {
    return mmd_core(IQP_OP_MMD_LOSS_GRAD, n, G, m, ldg, A, l, lda, Z, s, ldz, X, N, ldx, theta, prec, unbiased, loss,
                    grad, ws, ws_bytes, stream);
}

namespace {

iqp_status indep_core(int op, int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                      int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const float *theta, double *expval,
                      double *std_err, const double *alpha, const double *beta, double *grad, void *ws,
                      size_t ws_bytes, void *stream) {
    iqp_status rc = check_common(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, IQP_SPARSE_FP32);
    if (rc != IQP_OK) return rc;
    if (l > INT32_MAX / 2) return IQP_ERR_ARG;
    Plan p = make_plan(op, n, m, l, s, 0, IQP_SPARSE_FP32);
    p.G = G;
    p.ldg = ldg;
    if ((rc = check_ws(p, ws, ws_bytes)) != IQP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = prepare(p, ws, G, ldg, A, lda, Z, ldz, theta, st)) != IQP_OK) return rc;
    if (op == IQP_OP_EXPVAL_INDEP) return forward_stats(p, ws, expval, std_err, nullptr, nullptr, st);
    return backward(p, ws, alpha, beta, grad, st);
}

}  // namespace

iqp_status iqp_expval_indep(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                            int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                            double *expval, double *std_err, void *ws, size_t ws_bytes, void *stream) {
    if ((expval && !aligned(expval, 8)) || (std_err && !aligned(std_err, 8))) return IQP_ERR_ALIGN;
    return indep_core(IQP_OP_EXPVAL_INDEP, n, G, m, ldg, A, l, lda, Z, s, ldz, theta, expval, std_err, nullptr,
                      nullptr, nullptr, ws, ws_bytes, stream);
}

iqp_status iqp_expval_indep_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                                 int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                                 const double *alpha, const double *beta, double *grad, void *ws, size_t ws_bytes,
                                 void *stream) {
    if (alpha == nullptr || grad == nullptr) return IQP_ERR_ARG;
    if (!aligned(alpha, 8) || !aligned(grad, 8) || (beta && !aligned(beta, 8))) return IQP_ERR_ALIGN;
    return indep_core(IQP_OP_EXPVAL_INDEP_GRAD, n, G, m, ldg, A, l, lda, Z, s, ldz, theta, nullptr, nullptr, alpha,
                      beta, grad, ws, ws_bytes, stream);
}

iqp_status iqp_expand_params(const float *theta_p, int64_t np, const int64_t *start, float *theta_gen, int64_t m,
                             void *stream) {
    if (np < 1 || m < 1 || theta_p == nullptr || start == nullptr || theta_gen == nullptr) return IQP_ERR_ARG;
    if (!aligned(theta_p, 4) || !aligned(theta_gen, 4) || !aligned(start, 8)) return IQP_ERR_ALIGN;
    return cuda_status(launch_expand_params(theta_p, np, start, m, theta_gen, static_cast<cudaStream_t>(stream)));
}

iqp_status iqp_reduce_params(const double *grad_gen, int64_t m, const int64_t *start, int64_t np, double *grad_p,
                             void *stream) {
    if (np < 1 || m < 1 || grad_gen == nullptr || start == nullptr || grad_p == nullptr) return IQP_ERR_ARG;
    if (!aligned(grad_gen, 8) || !aligned(grad_p, 8) || !aligned(start, 8)) return IQP_ERR_ALIGN;
    return cuda_status(launch_reduce_params(grad_gen, m, start, np, grad_p, static_cast<cudaStream_t>(stream)));
}

iqp_status iqp_embed_bits(const uint64_t *src, int64_t rows, int64_t ld_src, const int32_t *wires, int64_t nw,
                          uint64_t *dst, int64_t ld_dst, int64_t n, void *stream) {
    if (nw < 1 || n < 1 || wires == nullptr) return IQP_ERR_ARG;
    iqp_status rc;
    if ((rc = check_bits(src, rows, ld_src, nw)) != IQP_OK) return rc;
    if ((rc = check_bits(dst, rows, ld_dst, n)) != IQP_OK) return rc;
    if (!aligned(wires, 4)) return IQP_ERR_ALIGN;
    return cuda_status(
        launch_embed_bits(src, rows, ld_src, wires, nw, dst, ld_dst, n, static_cast<cudaStream_t>(stream)));
}

iqp_status iqp_uniform_bits(uint64_t seed, uint64_t stream_id, int64_t rows, int64_t n, uint64_t *out, int64_t ld,
                            void *stream) {
    if (n < 1) return IQP_ERR_ARG;
    iqp_status rc;
    if ((rc = check_bits(out, rows, ld, n)) != IQP_OK) return rc;
    return cuda_status(launch_uniform_bits(seed, stream_id, rows, n, ld, out, static_cast<cudaStream_t>(stream)));
}

iqp_status iqp_bernoulli_bits(uint64_t seed, uint64_t stream_id, int64_t rows, int64_t n, double p, uint64_t *out,
                              int64_t ld, void *stream) {
    if (n < 1 || !(p >= 0.0 && p <= 1.0)) return IQP_ERR_ARG;
    iqp_status rc;
    if ((rc = check_bits(out, rows, ld, n)) != IQP_OK) return rc;
    return cuda_status(launch_bernoulli_bits(seed, stream_id, rows, n, p, ld, out, static_cast<cudaStream_t>(stream)));
}

namespace {

iqp_status bitflip_core(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                        int64_t lda, const float *theta, double *expval, const double *w, double *grad, void *ws,
                        size_t ws_bytes, void *stream) {
    if (n < 1 || m < 1 || l < 1) return IQP_ERR_ARG;
    if (m > (int64_t)1 << 36 || l > (int64_t)1 << 31) return IQP_ERR_ARG;
    iqp_status rc;
    if ((rc = check_bits(G, m, ldg, n)) != IQP_OK) return rc;
    if ((rc = check_bits(A, l, lda, n)) != IQP_OK) return rc;
    if (theta == nullptr) return IQP_ERR_ARG;
    if (!aligned(theta, 4)) return IQP_ERR_ALIGN;
    if ((expval && !aligned(expval, 8)) || (w && !aligned(w, 8)) || (grad && !aligned(grad, 8))) return IQP_ERR_ALIGN;
    Plan p = make_plan(IQP_OP_BITFLIP, n, m, l, 1, 0, IQP_FP32);
    if ((rc = check_ws(p, ws, ws_bytes)) != IQP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    IQP_TRY(launch_support_list(G, m, ldg, n, at<int4>(ws, p.off_sup), st));
    IQP_TRY(launch_parity_gather(n, A, l, lda, G, m, ldg, at<uint64_t>(ws, p.off_pa), p.ldp,
                                 at<uint64_t>(ws, p.off_pat), p.ldlt, at<uint64_t>(ws, p.off_rt), st,
                                 at<int4>(ws, p.off_sup)));
    double *c = at<double>(ws, p.off_c), *t = c + p.mpad;
    IQP_TRY(launch_bitflip_gates(theta, m, p.mpad, c, t, st));
    double *ev = expval ? expval : at<double>(ws, p.off_part);
    IQP_TRY(launch_bitflip_rows(at<uint64_t>(ws, p.off_pa), p.ldp, l, c, ev, st));
    if (grad != nullptr) {
        double *v = at<double>(ws, p.off_part) + l;
        IQP_TRY(launch_bitflip_grad(at<uint64_t>(ws, p.off_pat), p.ldlt, m, l, w, ev, v, t, grad, st));
    }
    return IQP_OK;
}

}  // namespace

iqp_status iqp_bitflip_expval(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                              int64_t lda, const float *theta, double *expval, void *ws, size_t ws_bytes,
                              void *stream) {
    if (expval == nullptr) return IQP_ERR_ARG;
    return bitflip_core(n, G, m, ldg, A, l, lda, theta, expval, nullptr, nullptr, ws, ws_bytes, stream);
}

iqp_status iqp_bitflip_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A, int64_t l,
                            int64_t lda, const float *theta, const double *w, double *grad, void *ws,
                            size_t ws_bytes, void *stream) {
    if (w == nullptr || grad == nullptr) return IQP_ERR_ARG;
    return bitflip_core(n, G, m, ldg, A, l, lda, theta, nullptr, w, grad, ws, ws_bytes, stream);
}

iqp_status iqp_read_status(void *ws, size_t ws_bytes, void *stream) {
    if (ws == nullptr || ws_bytes < 256 || !aligned(ws, 256)) return IQP_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t word = 0;
    if (cudaMemcpyAsync(&word, ws, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess) return IQP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return IQP_ERR_CUDA;
    if (cudaMemsetAsync(ws, 0, sizeof(word), st) != cudaSuccess) return IQP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return IQP_ERR_CUDA;
    return static_cast<iqp_status>(word);
}

iqp_status iqp_selftest_timeout(void *ws, size_t ws_bytes, double limit_seconds, void *stream) {
    if (ws == nullptr || ws_bytes < 256 || !aligned(ws, 256)) return IQP_ERR_WORKSPACE;
    if (!(limit_seconds > 0.0) || limit_seconds > 10.0) return IQP_ERR_ARG;
    return cuda_status(launch_timeout_selftest(static_cast<uint32_t *>(ws), (uint64_t)(limit_seconds * 1e9),
                                               static_cast<cudaStream_t>(stream)));
}

const char *iqp_status_string(iqp_status st) {
    switch (st) {
        case IQP_OK: return "ok";
        case IQP_ERR_ARG: return "invalid argument";
        case IQP_ERR_ALIGN: return "misaligned pointer or leading dimension";
        case IQP_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case IQP_ERR_CUDA: return "CUDA error";
        case IQP_ERR_TIMEOUT: return "device-side wait timed out";
        case IQP_ERR_UNSUPPORTED: return "unsupported on this device or build";
    }
    return "unknown status";
}

uint64_t iqp_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void iqp_profile_enable(int on) { g_profiling.store(on ? 1 : 0); }

void iqp_profile_reset(void) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    drain_pending();
    for (int k = 0; k < IQP_KERNEL_COUNT; ++k) {
        g_prof_ms[k] = 0.0;
        g_prof_n[k] = 0;
    }
}

iqp_status iqp_profile_query(iqp_kernel kernel, double *total_ms, uint64_t *launches) {
    if (kernel < 0 || kernel >= IQP_KERNEL_COUNT) return IQP_ERR_ARG;
    std::lock_guard<std::mutex> g(g_prof_mu);
    drain_pending();
    if (total_ms) *total_ms = g_prof_ms[kernel];
    if (launches) *launches = g_prof_n[kernel];
    return IQP_OK;
}

uint32_t iqp_check_status(void) {
    // the first recorded failure of any translation unit (each reads and clears its own word)
    uint32_t first = 0;
    const uint32_t words[] = {check_word_parity(), check_word_simt(), check_word_tc(), check_word_sparse(),
                              check_word_bitflip(), check_word_variants()};
    for (uint32_t w : words)
        if (first == 0 && w != 0) first = w;
    return first;
}

int iqp_checks_enabled(void) {
#ifdef IQP_CHECKS
    return 1;
#else
    return 0;
#endif
}

int iqp_tensor_path_available(void) {
    const int cc = device_cc();
    return cc == 103 ? 1 : 0;
}

}  // extern "C"
