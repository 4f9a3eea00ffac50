/*
 * iqp.h - C ABI of the GB300 (sm_103a) IQP expectation-value library.
 *
 * The library computes, for a parameterised IQP circuit
 *   U(theta) = prod_j exp(i theta_j X_{g_j})  acting on |0>   (Def. 1, Sec. 2),
 * Monte-Carlo estimates of Pauli-Z expectation values
 *   <Z_a> = E_{z ~ U{0,1}^n} [ cos Phi(a,z) ],
 *   Phi(a,z) = sum_j 2 theta_j [g_j.a odd] (1 - 2 [g_j.z odd])
 * (eqs. op_expval and expvalsample, Sec. 2.1; batch form E = C Theta B^T of
 * eq. Emat, Sec. 2.2), their standard errors, the gradient in theta
 * (Sec. 2.4), and the MMD^2 loss of eq. mmd_estimate (Sec. 3.3.1) between the
 * circuit and a data set.
 *
 * Conventions for every call:
 *  - Bit matrices (generators G, observables A, samples Z, data X, parities)
 *    are uint64 words, row-major, `ld` words per row, LSB-first: bit b of word
 *    w is column 64*w + b. `ld` is even and >= ceil(cols/64); base pointers
 *    are 16-byte aligned; padding bits beyond the last column are zero.
 *  - m = rows of G (gates), l = rows of A (observables), s = rows of Z
 *    (samples), N = rows of X (data rows), n = qubits (columns).
 *  - Every pointer except the host status strings is DEVICE memory owned by
 *    the caller. The library allocates nothing: scratch comes from `ws`, sized
 *    by iqp_workspace_bytes(), 256-byte aligned.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and keep no state between calls, so distinct workspaces may be
 *    used from several host threads at once.
 *  - Errors: host-side argument checks run before any launch and return a
 *    status; nothing is launched then. Device-side failures (a bounded wait
 *    that ran out) set a status word inside `ws` (its first 4 bytes, which
 *    must be zero when a workspace is first used: a zeroed allocation, or
 *    after iqp_read_status, which clears it), which iqp_read_status()
 *    returns. Nothing aborts, exits or traps.
 *  - Outputs are float64. theta is float32 on the device.
 */
#ifndef IQP_H
#define IQP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IQP_OK = 0,
    IQP_ERR_ARG = 1,         /* a size, pointer or flag is invalid            */
    IQP_ERR_ALIGN = 2,       /* a pointer or leading dimension is misaligned  */
    IQP_ERR_WORKSPACE = 3,   /* ws is NULL, misaligned or too small           */
    IQP_ERR_CUDA = 4,        /* a CUDA runtime/driver call failed             */
    IQP_ERR_TIMEOUT = 5,     /* a device-side bounded wait ran out            */
    IQP_ERR_UNSUPPORTED = 6  /* the device or build lacks a required feature  */
} iqp_status;

/* Arithmetic of the phase contraction Phi = (2 theta . P_A) S_Z^T.
 * IQP_FP32: FP32 FMA on the SIMT cores (the plain form).
 * IQP_SPLIT_BF16: tcgen05 tensor cores; 2 theta is split into hi + lo BF16
 * parts (hi = RN_bf16(2 theta), lo = RN_bf16(2 theta - hi)), the +-1 and 0/1
 * operands are exact in BF16, and both products accumulate in FP32 in TMEM.
 * IQP_SPARSE_FP32: row-sparse FP32 form on the SIMT cores: for each
 * observable only the gates with [g_j.a odd] are visited, so the work is
 * nnz(P_A) * s instead of l * m * s; the choice when P_A is sparse (density
 * below a few percent, e.g. low-weight observables drawn with small p_sigma).
 * Same tolerances as IQP_FP32; its gradient is bitwise reproducible.
 * IQP_LOWORDER_FP32: for generators of weight <= 2 only (one- and two-body
 * gates, e.g. local_gates of Sec. 3.1.1). With s_q(i) = (-1)^{z_iq} the
 * phase regroups exactly into
 *   Phi[a,i] = sum_{q in a} s_q(i) (d_q + (C S)[q,i]) - 2 sum_{q<r in a} C_qr s_q(i) s_r(i),
 * d_q / C_qr = sums of 2 theta_j over the gates on {q} / {q, r}, so the work
 * is two contractions over the qubit pairs that carry a generator plus
 * O(l |a|^2 s) instead of O(l m s). n <= 65536 (its n x n pair matrices take
 * about 20 n^2 bytes of workspace). FP32 (tolerances of IQP_FP32). A generator of weight > 2 records IQP_ERR_ARG
 * and an observable of weight > 1024 records IQP_ERR_UNSUPPORTED in the
 * device status (iqp_read_status); the outputs are then not meaningful. */
typedef enum { IQP_FP32 = 0, IQP_SPLIT_BF16 = 1, IQP_SPARSE_FP32 = 2, IQP_LOWORDER_FP32 = 3 } iqp_precision;

/* Operation whose scratch iqp_workspace_bytes() sizes. */
typedef enum {
    IQP_OP_EXPVAL = 1,
    IQP_OP_EXPVAL_GRAD = 2,
    IQP_OP_MMD_LOSS = 3,
    IQP_OP_MMD_LOSS_GRAD = 4,
    IQP_OP_BITFLIP = 5,  /* iqp_bitflip_expval and iqp_bitflip_grad */
    IQP_OP_EXPVAL_INDEP = 6,          /* iqp_expval_indep                       */
    IQP_OP_EXPVAL_INDEP_GRAD = 7,     /* iqp_expval_indep_grad                  */
    IQP_OP_MMD_LOSS_INDEP = 8,        /* iqp_mmd_loss with IQP_MMD_INDEP        */
    IQP_OP_MMD_LOSS_GRAD_INDEP = 9    /* iqp_mmd_loss_grad with IQP_MMD_INDEP   */
} iqp_op;

/* Flags of the MMD loss calls (the `unbiased` argument is a bit set). */
#define IQP_MMD_UNBIASED 1 /* U-statistics (else the plug-in form)                     */
#define IQP_MMD_SQRT 2     /* sqrt_loss: return sqrt(max(MMD^2, 0)) and its gradient   */
#define IQP_MMD_INDEP 4    /* one batch per observable: Z has l * s rows (indep_estimates) */

/* Bytes of device scratch `ws` needed by `op` for these sizes (N is ignored
 * except for the MMD ops). Returns 0 for invalid sizes. Host only.
 * With IQP_SPLIT_BF16 its end is optional, in three parts, each used only
 * when `ws_bytes` reaches its end:
 *  - 20.5 MB (160 x 128 KiB plus 640 bytes): a last round of phase tiles that
 *    would leave SMs idle is split along the gates across them (else every
 *    phase tile runs whole);
 *  - 40 MiB (160 x 256 KiB): the running sums of the phase kernels that take
 *    two sample tiles per tile (else one sample tile per tile);
 *  - 80 MiB (640 x 128 KiB plus 640 bytes): the last round of those kernels
 *    is split evenly across the SMs (else it runs as single tiles). */
size_t iqp_workspace_bytes(iqp_op op, int64_t n, int64_t m, int64_t l, int64_t s, int64_t N,
                           iqp_precision prec);

/* GF(2) products of Sec. 2.2 (A.G^T and Z.G^T mod 2):
 *   P[r][j] = (R_r . g_j) mod 2,  r < rows, j < m,
 * written bit-packed: row r of P is ldp words, bit j of the row is parity
 * with gate j; bits j >= m of each written row are set to zero.
 * R: rows x ldr words; G: m x ldg words; n <= 64*min(ldr, ldg).
 * ldp >= ceil(m/64), even. Bit-exact. No scratch. */
iqp_status iqp_parity(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr,
                      const uint64_t *G, int64_t m, int64_t ldg,
                      uint64_t *P, int64_t ldp, void *stream);

/* The same products by support gather, also returning the transpose: with
 * R^T (n x ldpt words) formed in `scratch`, the parities of gate j with 64
 * consecutive rows form one word, the XOR of the rows of R^T at the qubits
 * of supp(g_j); a gate of weight k costs O(k) per 64 rows instead of a fold
 * over all n qubits. Writes PT (m x ldpt words; bit r of row j is
 * (R_r . g_j) mod 2, zero for r >= rows) and, if P != NULL, P exactly as
 * iqp_parity does. With P, the gates' support list is formed first and P^T
 * and P come from one pass (the estimators' own parity step). ldpt >=
 * ceil(rows/64), even. scratch: device memory of n*ldpt*8 bytes, plus 16*m
 * bytes when P != NULL (the support list, after R^T), 16-byte aligned,
 * overwritten. Bit-exact. */
iqp_status iqp_parity_gather(int64_t n, const uint64_t *R, int64_t rows, int64_t ldr,
                             const uint64_t *G, int64_t m, int64_t ldg,
                             uint64_t *P, int64_t ldp, uint64_t *PT, int64_t ldpt,
                             uint64_t *scratch, void *stream);

/* Data parity sums of Sec. 3.3.1: T[a] = sum_{x < N} (-1)^{a.x}, so that
 * <Z_a>_p = T[a]/N for the empirical data distribution. A: l x lda words,
 * X: N x ldx words. T: int64[l], overwritten. Exact. No scratch. */
iqp_status iqp_parity_sum(int64_t n, const uint64_t *A, int64_t l, int64_t lda,
                          const uint64_t *X, int64_t N, int64_t ldx, int64_t *T, void *stream);

/* Estimator of eq. expvalsample for every observable, on the sample batch Z
 * shared by all observables (Sec. 2.2):
 *   expval[a]  = (1/s) sum_i cos Phi(a, z_i),
 *   std_err[a] = sqrt( (1/s) sum_i (cos Phi(a,z_i) - expval[a])^2 ) / sqrt(s)
 * (population variance, ddof = 0). s >= 1. Either output may be NULL.
 * ws: iqp_workspace_bytes(IQP_OP_EXPVAL, ...). */
iqp_status iqp_expval(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                      const uint64_t *A, int64_t l, int64_t lda,
                      const uint64_t *Z, int64_t s, int64_t ldz,
                      const float *theta, iqp_precision prec,
                      double *expval, double *std_err,
                      void *ws, size_t ws_bytes, void *stream);

/* iqp_expval for callers that cannot allocate device memory when they call
 * in (for example a process whose device memory is all owned by another
 * framework's caching pool, or latency-bound code that cannot afford
 * cudaMalloc's device-wide synchronisation). The paper has no counterpart:
 * it is a packaging of iqp_expval, with the same arguments and results
 * minus `ws`. Scratch is one file-scope device array of 64 MiB inside this
 * library, reserved on every GPU that loads the library and held until the
 * process exits; this call allocates nothing. Sizes whose
 * iqp_workspace_bytes(IQP_OP_EXPVAL, ...), less its optional part (see
 * there), exceeds 64 MiB are rejected with IQP_ERR_WORKSPACE before any
 * launch. Where the array holds less than the full workspace, the
 * split-BF16 phase runs the forms whose optional regions fit, so its results
 * may differ in the last bits from iqp_expval's with a full workspace (the
 * same tolerance holds). The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. All calls share the one
 * array: calls that overlap on the GPU (other streams, other host threads)
 * race and corrupt each other's results, so serialise them. Invalid
 * arguments return the status iqp_expval would, before anything is queued.
 * Device-side status (a bounded wait that ran out) is recorded in the array;
 * read it with iqp_noalloc_read_status() before the next call, which
 * clears it. */
iqp_status iqp_expval_noalloc(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                              const uint64_t *A, int64_t l, int64_t lda,
                              const uint64_t *Z, int64_t s, int64_t ldz,
                              const float *theta, iqp_precision prec,
                              double *expval, double *std_err, void *stream);

/* Device-side status of the last iqp_expval_noalloc call on the current
 * device (iqp_read_status for its array): waits for `stream`, returns the
 * status word and clears it. Allocates nothing. */
iqp_status iqp_noalloc_read_status(void *stream);

/* Gradient of the estimator in theta (Sec. 2.4; the estimator is a
 * deterministic function of theta for fixed Z), for losses whose derivative
 * in the samples has the form dL/dPhi(a,z_i) = -sin Phi (alpha[a] + beta[a] cos Phi):
 *   grad[j] = sum_a sum_i sin Phi(a,z_i) (alpha[a] + beta[a] cos Phi(a,z_i))
 *             * 2 [g_j.a odd] (1 - 2 [g_j.z_i odd]).
 * For L = sum_a w_a expval[a] pass alpha[a] = -w_a/s and beta = NULL.
 * Phi is recomputed tile by tile, never stored (iqp_expval_keep_phi and
 * iqp_expval_grad_from_phi keep it instead). alpha: float64[l] (device),
 * beta: float64[l] or NULL. grad: float64[m], overwritten.
 * ws: iqp_workspace_bytes(IQP_OP_EXPVAL_GRAD, ...). */
iqp_status iqp_expval_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                           const uint64_t *A, int64_t l, int64_t lda,
                           const uint64_t *Z, int64_t s, int64_t ldz,
                           const float *theta, const double *alpha, const double *beta,
                           iqp_precision prec, double *grad,
                           void *ws, size_t ws_bytes, void *stream);

/* The forward/backward pair of autograd (Sec. 2.4) without a second phase
 * pass. iqp_expval_keep_phi is iqp_expval that also writes Phi(a, z_i) into
 * phi; iqp_expval_grad_from_phi is iqp_expval_grad that forms
 * W = sin Phi (alpha + beta cos Phi) from that phi instead of recomputing
 * Phi (the same W bit for bit, so the same gradient).
 * phi: l x ldphi float32 on the device, caller-owned, 16-byte aligned,
 * ldphi >= s and a multiple of 64; the order of the samples within a row is
 * the precision's own, so phi is meaningful only to iqp_expval_grad_from_phi
 * with the same n, G, A, Z, theta and prec (not re-checked). The gradient
 * call only reads phi.
 * prec: IQP_SPLIT_BF16, IQP_SPARSE_FP32 or IQP_LOWORDER_FP32
 * (IQP_ERR_UNSUPPORTED for IQP_FP32). Errors: phi NULL, ldphi < s or not a
 * multiple of 64 -> IQP_ERR_ARG; phi not 16-byte aligned -> IQP_ERR_ALIGN.
 * ws: iqp_workspace_bytes(IQP_OP_EXPVAL, ...) for the first,
 * iqp_workspace_bytes(IQP_OP_EXPVAL_GRAD, ...) for the second. */
iqp_status iqp_expval_keep_phi(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                               const uint64_t *A, int64_t l, int64_t lda,
                               const uint64_t *Z, int64_t s, int64_t ldz,
                               const float *theta, iqp_precision prec,
                               double *expval, double *std_err, float *phi, int64_t ldphi,
                               void *ws, size_t ws_bytes, void *stream);
iqp_status iqp_expval_grad_from_phi(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                                    const uint64_t *A, int64_t l, int64_t lda,
                                    const uint64_t *Z, int64_t s, int64_t ldz,
                                    const float *theta, const double *alpha, const double *beta,
                                    iqp_precision prec, const float *phi, int64_t ldphi, double *grad,
                                    void *ws, size_t ws_bytes, void *stream);

/* Estimates and gradient in one call, for a loss whose gradient coefficients
 * alpha, beta (as in iqp_expval_grad) are known before the estimates, e.g.
 * L = sum_a w_a <Z_a> with alpha_a = -w_a / s, beta = NULL. Outputs as
 * iqp_expval plus grad[m]. The parities are formed once. In IQP_SPLIT_BF16
 * and IQP_SPARSE_FP32 a single pass over Phi yields the statistics and W (no
 * recompute); IQP_LOWORDER_FP32 keeps Phi from its statistics pass for W;
 * IQP_FP32 recomputes it. ws: iqp_workspace_bytes(IQP_OP_EXPVAL_GRAD, ...). */
iqp_status iqp_expval_value_and_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                                     const uint64_t *A, int64_t l, int64_t lda,
                                     const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                                     const double *alpha, const double *beta, iqp_precision prec,
                                     double *expval, double *std_err, double *grad,
                                     void *ws, size_t ws_bytes, void *stream);

/* MMD^2 estimate of eq. mmd_estimate (Sec. 3.3.1) over the l observables in
 * A (drawn by the caller, bits i.i.d. Bernoulli(p_sigma) for a Gaussian
 * kernel of bandwidth sigma), with model terms from the estimator on Z and
 * data terms from X:
 *   unbiased != 0:  term_a = (T^2 - N)/(N(N-1)) - 2 (T/N)(S1/s) + (S1^2 - S2)/(s(s-1))
 *   unbiased == 0:  term_a = (T/N - S1/s)^2
 *   loss = (1/l) sum_a term_a,  S1 = sum_i cos Phi, S2 = sum_i cos^2 Phi, T as in
 *   iqp_parity_sum. The unbiased form needs s >= 2 and N >= 2.
 * `unbiased` is a set of IQP_MMD_* flags (1 = unbiased keeps its meaning):
 *   IQP_MMD_SQRT   sqrt_loss (Sec. 3.3.1): loss = sqrt(max(MMD^2, 0)); the
 *                  gradient is (d MMD^2) / (2 loss), zero where loss = 0.
 *   IQP_MMD_INDEP  indep_estimates: observable a uses its own samples, rows
 *                  [a s, (a+1) s) of Z (Z has l * s rows); the estimator runs
 *                  in the row-sparse FP32 arithmetic and `prec` is ignored.
 *                  Workspace op IQP_OP_MMD_LOSS_INDEP.
 * Observables and data on a subset of the qubits (`wires`): embed both with
 * iqp_embed_bits first.
 * loss: one float64 on the device. ws: iqp_workspace_bytes(IQP_OP_MMD_LOSS, ...). */
iqp_status iqp_mmd_loss(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                        const uint64_t *A, int64_t l, int64_t lda,
                        const uint64_t *Z, int64_t s, int64_t ldz,
                        const uint64_t *X, int64_t N, int64_t ldx,
                        const float *theta, iqp_precision prec, int unbiased,
                        double *loss, void *ws, size_t ws_bytes, void *stream);

/* Loss as iqp_mmd_loss and its gradient grad[m] in theta, by the chain rule
 * through S1 and S2 (alpha, beta of iqp_expval_grad formed on the device).
 * With IQP_SPLIT_BF16, IQP_SPARSE_FP32 and IQP_LOWORDER_FP32 (shared
 * batches) the call runs one phase contraction: the statistics pass keeps Phi
 * (l x s FP32, in the workspace) and W is formed from it once alpha, beta are
 * known; IQP_FP32 and independent batches recompute Phi for W.
 * ws: iqp_workspace_bytes(IQP_OP_MMD_LOSS_GRAD, ...). */
iqp_status iqp_mmd_loss_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                             const uint64_t *A, int64_t l, int64_t lda,
                             const uint64_t *Z, int64_t s, int64_t ldz,
                             const uint64_t *X, int64_t N, int64_t ldx,
                             const float *theta, iqp_precision prec, int unbiased,
                             double *loss, double *grad, void *ws, size_t ws_bytes, void *stream);

/* Stochastic bitflip circuit (Sec. 2.5): every gate, instead of acting
 * coherently, flips the bits of g_j with probability sin^2(theta_j). Its
 * expectation values are exact products (eq. expval_bitflip), no sampling:
 *   expval[a] = prod_{j : g_j.a odd} cos(2 theta_j).
 * FP64. ws: iqp_workspace_bytes(IQP_OP_BITFLIP, n, m, l, 1, 0, prec). */
iqp_status iqp_bitflip_expval(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                              const uint64_t *A, int64_t l, int64_t lda, const float *theta,
                              double *expval, void *ws, size_t ws_bytes, void *stream);

/* Gradient of L = sum_a w[a] expval[a] for the bitflip circuit:
 *   grad[j] = -2 tan(2 theta_j) sum_{a : g_j.a odd} w[a] expval[a].
 * w: float64[l] on the device (e.g. dL/d expval). grad: float64[m]. FP64.
 * Same workspace as iqp_bitflip_expval. */
iqp_status iqp_bitflip_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                            const uint64_t *A, int64_t l, int64_t lda, const float *theta,
                            const double *w, double *grad, void *ws, size_t ws_bytes, void *stream);

/* Independent estimates (indep_estimates, Sec. 2.2 and 3.1.2): observable a
 * is estimated on its own sample batch, rows [a s, (a+1) s) of Z (Z has
 * l * s rows of ldz words), so estimates of different observables are
 * uncorrelated, at the cost of l * s * (n-bit) samples and per-observable
 * parities. Outputs as iqp_expval. Arithmetic: the row-sparse FP32 form
 * (work nnz(P_A) * s), with the parity of each (gate, sample) formed from the
 * observable's own samples as the XOR over the gate's support.
 * ws: iqp_workspace_bytes(IQP_OP_EXPVAL_INDEP, n, m, l, s, 0, prec) (prec
 * ignored); it holds every batch transposed (l * n * ceil(s/64) words). */
iqp_status iqp_expval_indep(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                            const uint64_t *A, int64_t l, int64_t lda,
                            const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                            double *expval, double *std_err, void *ws, size_t ws_bytes, void *stream);

/* Gradient of the independent-batch estimator, alpha/beta as in
 * iqp_expval_grad. ws: iqp_workspace_bytes(IQP_OP_EXPVAL_INDEP_GRAD, ...). */
iqp_status iqp_expval_indep_grad(int64_t n, const uint64_t *G, int64_t m, int64_t ldg,
                                 const uint64_t *A, int64_t l, int64_t lda,
                                 const uint64_t *Z, int64_t s, int64_t ldz, const float *theta,
                                 const double *alpha, const double *beta, double *grad,
                                 void *ws, size_t ws_bytes, void *stream);

/* Shared-parameter gates (Sec. 3.1.1): a gate is a tuple of generators with
 * one parameter, exp(i theta_p sum_{g in gate p} X_g). Store G gate by gate:
 * gate p owns generator rows [start[p], start[p+1]), start[0] = 0,
 * start[np] = m, non-decreasing (int64, device). Fixed gates (init_gates with
 * init_coefs) are gates whose parameter the caller does not train.
 * iqp_expand_params: theta_gen[j] = theta_p[p] for j in gate p (float32[m]).
 * iqp_reduce_params: grad_p[p] = sum_{j in gate p} grad_gen[j] (float64, in
 * index order): the gradient in the shared parameters.
 * Ranges outside [0, m) are clamped; rows not covered by a gate are left
 * unwritten. No scratch. */
iqp_status iqp_expand_params(const float *theta_p, int64_t np, const int64_t *start, float *theta_gen, int64_t m,
                             void *stream);
iqp_status iqp_reduce_params(const double *grad_gen, int64_t m, const int64_t *start, int64_t np, double *grad_p,
                             void *stream);

/* `wires` (Sec. 3.3.1): rows on nw wire qubits -> rows on n qubits. Bit k of
 * src row r becomes bit wires[k] of dst row r; every other bit of dst is zero.
 * wires: int32[nw] on the device, distinct, in [0, n) (others are skipped).
 * src: rows x ld_src words (ld_src >= ceil(nw/64)); dst: rows x ld_dst words
 * (ld_dst >= ceil(n/64), even). No scratch. */
iqp_status iqp_embed_bits(const uint64_t *src, int64_t rows, int64_t ld_src, const int32_t *wires, int64_t nw,
                          uint64_t *dst, int64_t ld_dst, int64_t n, void *stream);

/* Random bits on the device for a training loop (fresh samples each step,
 * Sec. 2.4; observables a ~ P_sigma, Sec. 3.3.1), from a counter-based
 * splitmix64 (Steele, Lea and Flood 2014): value k >= 1 of stream t under
 * seed S is mix(S * 0xD1B54A32D192ED03 + t * 0xAEF17502108EF2D9 + k *
 * 0x9E3779B97F4A7C15) with the splitmix64 finaliser.
 * iqp_uniform_bits: word w < ceil(n/64) of row r is value r * L + w + 1, L =
 * ceil(n/64) rounded up to even; bits >= n and words >= ceil(n/64) are zero.
 * iqp_bernoulli_bits: bit q of row r is set iff (value r * n + q + 1 >> 11)
 * * 2^-53 < p (exact in FP64).
 * out: rows x ld words on the device, ld >= ceil(n/64) and even. */
iqp_status iqp_uniform_bits(uint64_t seed, uint64_t stream_id, int64_t rows, int64_t n, uint64_t *out, int64_t ld,
                            void *stream);
iqp_status iqp_bernoulli_bits(uint64_t seed, uint64_t stream_id, int64_t rows, int64_t n, double p, uint64_t *out,
                              int64_t ld, void *stream);

/* Device-side status of the last calls that used `ws`: synchronises
 * `stream`, returns IQP_OK or the first error a kernel recorded (e.g.
 * IQP_ERR_TIMEOUT), and clears it. */
iqp_status iqp_read_status(void *ws, size_t ws_bytes, void *stream);

/* Self-test of the bounded-wait machinery: one CTA waits on an mbarrier that
 * nothing arrives on, gives up after `limit_seconds` (<= 10), records
 * IQP_ERR_TIMEOUT in ws and returns. Read it with iqp_read_status(). */
iqp_status iqp_selftest_timeout(void *ws, size_t ws_bytes, double limit_seconds, void *stream);

/* Device-side self-checks. A library built with -DIQP_CHECKS compares every
 * global index its kernels derive from the caller's shapes with the extent of
 * the buffer before the access; an index outside is skipped and recorded.
 * iqp_check_status() synchronises the device and returns 0 if no index left
 * its buffer since the last call, else 200 + the site of the first that did
 * (the low-order kernels record 100 + site in the workspace status word
 * instead, read by iqp_read_status); it clears what it reports. In the
 * default build the checks are compiled out: iqp_checks_enabled() returns 0
 * and iqp_check_status() returns 0. Not a counterpart of anything in the
 * paper: it stands in for a memory checker. */
uint32_t iqp_check_status(void);
int iqp_checks_enabled(void);

/* Kernels of this library, for iqp_profile_query(). */
typedef enum {
    IQP_KERNEL_PARITY = 0,         /* GF(2) products (P_A, P_Z, P_Z^T)          */
    IQP_KERNEL_PARITY_SUM = 1,     /* data parity sums T                        */
    IQP_KERNEL_THETA_SPLIT = 2,    /* 2 theta, and its hi/lo BF16 split         */
    IQP_KERNEL_PHASE_FP32 = 3,     /* SIMT phase contraction + statistics       */
    IQP_KERNEL_RECOMPUTE_FP32 = 4, /* SIMT phase recompute -> W                 */
    IQP_KERNEL_GRAD_FP32 = 5,      /* SIMT gradient contraction                 */
    IQP_KERNEL_PHASE_TC = 6,       /* tcgen05 phase contraction + statistics    */
    IQP_KERNEL_RECOMPUTE_TC = 7,   /* W (hi/lo): tcgen05 phase recompute, or
                                      from the Phi an MMD statistics pass kept */
    IQP_KERNEL_GRAD_TC = 8,        /* tcgen05 gradient contraction              */
    IQP_KERNEL_FINALIZE = 9,       /* per-observable mean / standard error      */
    IQP_KERNEL_GRAD_REDUCE = 10,   /* fixed-order reduction of gradient parts   */
    IQP_KERNEL_MMD_COMBINE = 11,   /* MMD^2 terms and gradient coefficients     */
    IQP_KERNEL_SELFTEST = 12,      /* iqp_selftest_timeout                      */
    IQP_KERNEL_BITFLIP = 13,       /* bitflip products and gradient sums        */
    IQP_KERNEL_PHASE_SPARSE = 14,  /* row-sparse phase + statistics             */
    IQP_KERNEL_GRAD_SPARSE = 15,   /* row-sparse recompute + gradient           */
    IQP_KERNEL_VARIANTS = 16,      /* shared-parameter expand/reduce, embedding */
    IQP_KERNEL_RNG = 17,           /* on-device random bits                     */
    IQP_KERNEL_LOWORDER = 18,      /* weight <= 2 generators: the low-order form */
    IQP_KERNEL_LOWORDER_GEMM = 19, /* its n x n x s contractions                */
    IQP_KERNEL_COUNT = 20
} iqp_kernel;

/* Per-kernel timing (off by default). When enabled, every launch is
 * bracketed by two CUDA events recorded on the launch's stream; the events
 * add a few microseconds per launch and no synchronisation. Host only;
 * process-wide; thread-safe. */
void iqp_profile_enable(int on);
void iqp_profile_reset(void);
/* Total elapsed milliseconds and launch count of `kernel` since the last
 * reset. Synchronises on the pending events. */
iqp_status iqp_profile_query(iqp_kernel kernel, double *total_ms, uint64_t *launches);

/* Static text for a status. Host only. */
const char *iqp_status_string(iqp_status st);

/* Number of kernels this library has launched in this process (host counter). */
uint64_t iqp_launch_count(void);

/* 1 if the current device supports the IQP_SPLIT_BF16 path (sm_103 family). */
int iqp_tensor_path_available(void);

#ifdef __cplusplus
}
#endif
#endif /* IQP_H */
