// Low-order form: every generator has weight <= 2 (the one- and two-body
// gate sets of Sec. 3.1.1 and Sec. 4). With s_q(i) = (-1)^{z_{i,q}},
// Q_a = supp(a), c_j = 2 theta_j, d_q = sum of c_j over the one-qubit gates
// on q and C_qr = sum of c_j over the gates on {q, r} (symmetric, zero
// diagonal):
//   [g_j.a odd]      = [q in Q_a] for g_j = e_q, [exactly one of q, r in Q_a] for e_q + e_r,
//   1 - 2[g_j.z odd] = s_q(z), or s_q(z) s_r(z),
// so the phase of eq. expvalsample regroups exactly into
//   Phi[a,i] = sum_{q in Q_a} s_q(i) (d_q + M[q,i]) - 2 sum_{q<r in Q_a} C_qr s_q(i) s_r(i),
//   M = C S,  S[r][i] = s_r(i)                              (an n x n x s contraction),
// and with W[a,i] = sin Phi (alpha_a + beta_a cos Phi), V[q,i] = sum_{a : q in Q_a} W[a,i]:
//   grad(gate e_q)       = 2 sum_i s_q(i) V[q,i],
//   grad(gate e_q + e_r) = 2 (H[q,r] + H[r,q]) - 4 K[q,r],
//   H[q,r] = sum_i s_q(i) V[q,i] s_r(i)                     (a second n x n x s contraction),
//   K[q,r] = sum_{a : q, r in Q_a} sum_i W[a,i] s_q(i) s_r(i).
// The work is O(n^2 s + l |Q_a|^2 s) instead of nnz(P_A) s, and nnz(P_A) is
// about l |Q_a| n for all one- and two-body gates. FP32 arithmetic, FP64
// reductions over samples, K accumulated in 64-bit fixed point (integer
// atomics, so the gradient is bitwise reproducible).
//
// Device-side errors: a generator of weight > 2 records IQP_ERR_ARG, an
// observable of weight > 1024 records IQP_ERR_UNSUPPORTED (in the workspace
// status word); the outputs are then not meaningful.
#include "common.cuh"

namespace iqp {

namespace {

constexpr int kQMax = 1024;  // observable weight limit (support list in shared memory)
constexpr int kCQ = 64;      // C restricted to Q_a is staged in shared memory for |Q_a| <= 64
constexpr int kBlk = 256;    // samples per CTA in the per-observable kernels
constexpr unsigned kFull = 0xFFFFFFFFu;

// d_q and C_qr from the support list (q0 < q1 < ... , count).
__global__ void k_lo_build(const int4 *__restrict__ sup, const float *__restrict__ c, int64_t m, float *__restrict__ C,
                           int64_t ldc, float *__restrict__ d, uint32_t *__restrict__ status) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int4 sp = sup[j];
        if (sp.w == 1) {
            atomicAdd(d + sp.x, c[j]);
        } else if (sp.w == 2) {
            atomicAdd(C + (int64_t)sp.x * ldc + sp.y, c[j]);
            atomicAdd(C + (int64_t)sp.y * ldc + sp.x, c[j]);
        } else if (sp.w > 2) {
            record_status(status, IQP_ERR_ARG);
        }
    }
}

// out[p][i] = sum_{k < K} A[p][k] sa(p,k) sb(i,k), sb(i,k) = 1 - 2 bit k of
// row i of Bb, sa likewise from Ab (or 1 when Ab is null). A: P x lda fp32,
// Bb: I x ldb words, Ab: P x ldab words, out: P x ldo fp32. 128 x 128 tiles,
// 8 x 8 per thread, 32-wide K steps; FP32 FMA in k order.
constexpr int GM = 128, GN = 128, GK = 32, GPAD = 4;

__global__ void __launch_bounds__(256) k_lo_gemm(const float *__restrict__ A, int64_t lda,
                                                 const uint32_t *__restrict__ Ab, int64_t ldab32,
                                                 const uint32_t *__restrict__ Bb, int64_t ldb32, int64_t P, int64_t I,
                                                 int64_t K, float *__restrict__ out, int64_t ldo) {
    __shared__ __align__(16) float As[GK][GM + GPAD];
    __shared__ __align__(16) float Bs[GK][GN + GPAD];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * GN, p0 = (int64_t)blockIdx.y * GM;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;
    const int ar = tid & 127, ac = (tid >> 7) * 16;  // A loader: row, first of 16 k's
    const int64_t prow = p0 + ar;
    for (int64_t k0 = 0; k0 < K; k0 += GK) {
        // A tile, transposed to k-major, with the optional sign from Ab.
        uint32_t fl = 0u;
        if (Ab != nullptr && prow < P) fl = Ab[prow * ldab32 + (k0 >> 5)] >> ac;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int64_t k = k0 + ac + q;
            float v = (prow < P && k < K) ? A[prow * lda + k] : 0.f;
            if ((fl >> q) & 1u) v = -v;
            As[ac + q][ar] = v;
        }
        // B tile: +-1 from 32 bits of row i.
        if (tid < GN) {
            const int64_t i = i0 + tid;
            const uint32_t b = i < I ? Bb[i * ldb32 + (k0 >> 5)] : 0u;
#pragma unroll
            for (int q = 0; q < GK; ++q) Bs[q][tid] = ((b >> q) & 1u) ? -1.f : 1.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < GK; ++k) {
            const float4 a_lo = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 a_hi = *reinterpret_cast<const float4 *>(&As[k][64 + ty * 4]);
            const float4 b_lo = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float4 b_hi = *reinterpret_cast<const float4 *>(&Bs[k][64 + tx * 4]);
            const float av[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
            const float bv[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t p = p0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        if (p >= P) continue;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t i = i0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + (q - 4));
            if (i < I) out[p * ldo + i] = acc[r][q];
        }
    }
}

// The support of observable a in increasing qubit order into Q (shared);
// returns |Q_a| capped at kQMax (recording IQP_ERR_UNSUPPORTED beyond it).
// Every thread of the CTA calls it.
__device__ int support_of_row(const uint64_t *__restrict__ arow, int64_t n, int *Q, int *scan,
                              uint32_t *__restrict__ status) {
    const int tid = threadIdx.x;
    const int64_t nw = (n + 63) >> 6;
    int total = 0;
    for (int64_t base = 0; base < nw; base += blockDim.x) {
        uint64_t w = base + tid < nw ? arow[base + tid] : 0ull;
        if (base + tid == nw - 1 && (n & 63)) w &= (1ull << (n & 63)) - 1ull;  // never a qubit >= n
        const int cnt = __popcll(w);
        scan[tid] = cnt;
        __syncthreads();
        // inclusive scan over the CTA (Hillis-Steele)
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            const int v = tid >= off ? scan[tid - off] : 0;
            __syncthreads();
            scan[tid] += v;
            __syncthreads();
        }
        int pos = total + scan[tid] - cnt;
        while (w) {
            const int b = __ffsll((long long)w) - 1;
            w &= w - 1ull;
            if (pos < kQMax) Q[pos] = (int)(64 * (base + tid) + b);
            ++pos;
        }
        total += scan[blockDim.x - 1];
        __syncthreads();
    }
    if (total > kQMax) {
        if (tid == 0) record_status(status, IQP_ERR_UNSUPPORTED);
        total = kQMax;
    }
    return total;
}

// Bits of the lane's sample for qubits Q[t0 .. t0+cnt) (bit t - t0).
__device__ __forceinline__ uint32_t sample_bits(const int *Q, int t0, int cnt, const uint64_t *__restrict__ ZT,
                                                int64_t ldzt, int64_t wi, int bi) {
    uint32_t m = 0u;
    for (int t = 0; t < cnt; ++t) m |= (uint32_t)((ZT[(int64_t)Q[t0 + t] * ldzt + wi] >> bi) & 1ull) << t;
    return m;
}

// Phi for one sample (see the header), the pair term over chunks of 32
// support qubits whose sample bits are gathered once per chunk.
__device__ float lo_phase(const int *Q, int nq, const float *CQ, const float *__restrict__ C, int64_t ldc,
                          const float *__restrict__ d, const float *__restrict__ M, int64_t lds,
                          const uint64_t *__restrict__ ZT, int64_t ldzt, int64_t ic) {
    const int64_t wi = ic >> 6;
    const int bi = (int)(ic & 63);
    float phi = 0.f;
    for (int t = 0; t < nq; ++t) {
        const int q = Q[t];
        const float v = d[q] + M[(int64_t)q * lds + ic];
        phi += ((ZT[(int64_t)q * ldzt + wi] >> bi) & 1ull) ? -v : v;
    }
    float pairs = 0.f;
    const int nch = (nq + 31) >> 5;
    for (int T = 0; T < nch; ++T) {
        const int tn = nq - 32 * T < 32 ? nq - 32 * T : 32;
        const uint32_t mT = sample_bits(Q, 32 * T, tn, ZT, ldzt, wi, bi);
        for (int U = T; U < nch; ++U) {
            const int un = nq - 32 * U < 32 ? nq - 32 * U : 32;
            const uint32_t mU = U == T ? mT : sample_bits(Q, 32 * U, un, ZT, ldzt, wi, bi);
            for (int t = 0; t < tn; ++t) {
                const int tt = 32 * T + t;
                const uint32_t st = (mT >> t) & 1u;
                float acc = 0.f;
                for (int u = (U == T ? t + 1 : 0); u < un; ++u) {
                    const int uu = 32 * U + u;
                    const float cv = nq <= kCQ ? CQ[tt * nq + uu] : C[(int64_t)Q[tt] * ldc + Q[uu]];
                    acc += ((st ^ (mU >> u)) & 1u) ? -cv : cv;
                }
                pairs += acc;
            }
        }
    }
    return phi - 2.f * pairs;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// MODE 0: (sum cos, sum (cos - mean)^2) per (observable, 256 samples) into
// part. MODE 1: W[a][i] = sin Phi (alpha_a + beta_a cos Phi), zero for i >= s.
template <int MODE>
__global__ void __launch_bounds__(kBlk) k_lo_phase(const uint64_t *__restrict__ A, int64_t lda, int64_t n,
                                                   const uint64_t *__restrict__ ZT, int64_t ldzt,
                                                   const float *__restrict__ M, int64_t lds,
                                                   const float *__restrict__ C, int64_t ldc,
                                                   const float *__restrict__ d, int64_t s, int64_t nparts,
                                                   double2 *__restrict__ part, const double *__restrict__ alpha,
                                                   const double *__restrict__ beta, float *__restrict__ W,
                                                   uint32_t *__restrict__ status) {
    __shared__ int Q[kQMax];
    __shared__ float CQ[kCQ * kCQ];
    __shared__ int scan[kBlk];
    __shared__ double red[kBlk / 32];
    const int64_t a = blockIdx.x, blk = blockIdx.y;
    const int nq = support_of_row(A + a * lda, n, Q, scan, status);
    if (nq <= kCQ)
        for (int e = threadIdx.x; e < nq * nq; e += kBlk) CQ[e] = C[(int64_t)Q[e / nq] * ldc + Q[e % nq]];
    __syncthreads();
    const int64_t i = blk * kBlk + threadIdx.x;
    const bool valid = i < s;
    const int64_t ic = valid ? i : s - 1;
    const float phi = lo_phase(Q, nq, CQ, C, ldc, d, M, lds, ZT, ldzt, ic);
    if (MODE == 0) {
        const float cv = valid ? cosf(phi) : 0.f;
        const double S = block_sum((double)cv, red);
        const int64_t nb = s - blk * kBlk < kBlk ? s - blk * kBlk : kBlk;
        const float mean = (float)(S / (double)nb);
        const float dv = cv - mean;
        const double M2 = block_sum(valid ? (double)(dv * dv) : 0.0, red);
        if (threadIdx.x == 0) part[a * nparts + blk] = make_double2(S, M2);
    } else {
        float sn, cn;
        sincosf(phi, &sn, &cn);
        const float al = (float)alpha[a], be = beta ? (float)beta[a] : 0.f;
        if (i < lds) W[a * lds + i] = valid ? sn * (al + be * cn) : 0.f;
    }
}

// V[q][i] = sum over the observables a containing q of W[a][i] (in a order),
// zero for i >= s; gsp[q * nblk + blk] = sum_i s_q(i) V[q][i] over the
// CTA's 256 samples (FP64).
__global__ void __launch_bounds__(kBlk) k_lo_v(const uint64_t *__restrict__ AT, int64_t ldlt,
                                               const uint64_t *__restrict__ ZT, int64_t ldzt,
                                               const float *__restrict__ W, int64_t lds, int64_t s, int64_t nblk,
                                               float *__restrict__ V, double *__restrict__ gsp) {
    __shared__ double red[kBlk / 32];
    const int64_t q = blockIdx.x, blk = blockIdx.y;
    const int64_t i = blk * kBlk + threadIdx.x;
    const bool valid = i < s;
    const int64_t ic = valid ? i : s - 1;
    const uint64_t *row = AT + q * ldlt;
    float v = 0.f;
    for (int64_t w = 0; w < ldlt; ++w) {
        uint64_t bits = row[w];
        while (bits) {
            const int b = __ffsll((long long)bits) - 1;
            bits &= bits - 1ull;
            v += W[(64 * w + b) * lds + ic];
        }
    }
    if (!valid) v = 0.f;
    if (i < lds) V[q * lds + i] = v;
    const float u = ((ZT[q * ldzt + (ic >> 6)] >> (ic & 63)) & 1ull) ? -v : v;
    const double t = block_sum((double)u, red);
    if (threadIdx.x == 0) gsp[q * nblk + blk] = t;
}

__device__ __forceinline__ long long to_fixed(float x, float sc) {
    const float xs = sc * x;  // |xs| < 2^60, exact power-of-two scaling
    const float hi = truncf(xs * 0x1.0p-31f);
    const float lo = fmaf(-hi, 0x1.0p31f, xs);
    return ((long long)__float2int_rz(hi) << 31) + (long long)__float2int_rn(lo);
}

// K[q][r] (q < r in Q_a) += sum_i W[a][i] s_q(i) s_r(i), one warp per pair,
// in 64-bit fixed point with scale `scale`.
__global__ void __launch_bounds__(kBlk) k_lo_pairs(const uint64_t *__restrict__ A, int64_t lda, int64_t n,
                                                   const uint64_t *__restrict__ ZT, int64_t ldzt,
                                                   const float *__restrict__ W, int64_t lds, int64_t s,
                                                   const double *__restrict__ scale,
                                                   unsigned long long *__restrict__ Kfx,
                                                   uint32_t *__restrict__ status) {
    __shared__ int Q[kQMax];
    __shared__ int scan[kBlk];
    const int64_t a = blockIdx.x;
    const int nq = support_of_row(A + a * lda, n, Q, scan, status);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float sc = (float)*scale;
    const int64_t npairs = (int64_t)nq * (nq - 1) / 2;
    const float *wrow = W + a * lds;
    for (int64_t p = warp; p < npairs; p += kBlk / 32) {
        int t = 0;
        int64_t rem = p;
        while (rem >= nq - 1 - t) {
            rem -= nq - 1 - t;
            ++t;
        }
        const int u = t + 1 + (int)rem;
        const uint64_t *zt = ZT + (int64_t)Q[t] * ldzt;
        const uint64_t *zu = ZT + (int64_t)Q[u] * ldzt;
        float acc = 0.f;
        for (int64_t i = lane; i < s; i += 32) {
            const uint64_t x = (zt[i >> 6] ^ zu[i >> 6]) >> (i & 63);
            const float w = wrow[i];
            acc += (x & 1ull) ? -w : w;
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
        if (lane == 0) atomicAdd(Kfx + (int64_t)Q[t] * n + Q[u], (unsigned long long)to_fixed(acc, sc));
    }
}

// grad_j from the parts above (see the header).
__global__ void k_lo_grad_out(const int4 *__restrict__ sup, int64_t m, int64_t n, const double *__restrict__ gsp,
                              int64_t nblk, const float *__restrict__ H, int64_t ldh,
                              const unsigned long long *__restrict__ Kfx, const double *__restrict__ scale,
                              double *__restrict__ grad) {
    const double inv = 1.0 / *scale;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int4 sp = sup[j];
        double g = 0.0;
        if (sp.w == 1) {
            double t = 0.0;
            for (int64_t k = 0; k < nblk; ++k) t += gsp[(int64_t)sp.x * nblk + k];
            g = 2.0 * t;
        } else if (sp.w == 2) {
            const int64_t q = sp.x, r = sp.y;
            const double h = (double)H[q * ldh + r] + (double)H[r * ldh + q];
            const double k = (double)(long long)Kfx[q * n + r] * inv;
            g = 2.0 * h - 4.0 * k;
        }
        grad[j] = g;
    }
}

int grid_1d(int64_t work) {
    int64_t b = cdiv(work, 256);
    if (b < 1) b = 1;
    if (b > 8192) b = 8192;
    return (int)b;
}

}  // namespace

cudaError_t launch_support_list(const uint64_t *G, int64_t m, int64_t ldg, int64_t n, int4 *sup, cudaStream_t st);
cudaError_t launch_bit_transpose_batched(const uint64_t *in, int64_t batch, int64_t in_rows, int64_t in_cols,
                                         int64_t ld_in, uint64_t *out, int64_t ld_out, cudaStream_t st);
cudaError_t launch_fixed_scale(const double *alpha, const double *beta, int64_t l, int64_t s, double *scale,
                               cudaStream_t st);

int64_t lo_part_samples() { return kBlk; }

// C, d and M = C S. C: n x ldc fp32 (+ d: ldc fp32 after it), M: n x lds,
// ZT: n x ldzt words (the samples transposed), sup: m int4.
cudaError_t launch_lo_prepare(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *Z, int64_t s,
                              int64_t ldz, const float *c, int4 *sup, uint64_t *ZT, int64_t ldzt, float *C,
                              int64_t ldc, float *M, int64_t lds, uint32_t *status, cudaStream_t st) {
    cudaError_t e = launch_support_list(G, m, ldg, n, sup, st);
    if (e != cudaSuccess) return e;
    if ((e = launch_bit_transpose_batched(Z, 1, s, n, ldz, ZT, ldzt, st)) != cudaSuccess) return e;
    float *d = C + n * ldc;
    if ((e = cudaMemsetAsync(C, 0, (size_t)(n + 1) * ldc * sizeof(float), st)) != cudaSuccess) return e;
    {
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_build<<<grid_1d(m), 256, 0, st>>>(sup, c, m, C, ldc, d, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    LaunchScope ls(IQP_KERNEL_LOWORDER_GEMM, st);
    // M[q][i] = sum_r C[q][r] s_r(i): A = C, B bits = Z rows (bits over qubits).
    k_lo_gemm<<<dim3((unsigned)cdiv(s, GN), (unsigned)cdiv(n, GM)), 256, 0, st>>>(
        C, ldc, nullptr, 0, reinterpret_cast<const uint32_t *>(Z), 2 * ldz, n, s, n, M, lds);
    return cudaGetLastError();
}

cudaError_t launch_lo_stats(const uint64_t *A, int64_t lda, int64_t n, int64_t l, const uint64_t *ZT, int64_t ldzt,
                            const float *M, int64_t lds, const float *C, int64_t ldc, int64_t s, double2 *part,
                            int64_t nparts, uint32_t *status, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_LOWORDER, st);
    k_lo_phase<0><<<dim3((unsigned)l, (unsigned)nparts), kBlk, 0, st>>>(A, lda, n, ZT, ldzt, M, lds, C, ldc,
                                                                       C + n * ldc, s, nparts, part, nullptr,
                                                                       nullptr, nullptr, status);
    return cudaGetLastError();
}

// AT: n x ldlt words (A transposed), W: l x lds, V: n x lds, H: n x ldc,
// gsp: n x nblk doubles, Kfx: n x n int64 followed by the scale (double).
cudaError_t launch_lo_grad(const uint64_t *A, int64_t lda, int64_t n, int64_t l, const uint64_t *ZT, int64_t ldzt,
                           const float *M, int64_t lds, const float *C, int64_t ldc, int64_t s, int64_t m,
                           const int4 *sup, const double *alpha, const double *beta, uint64_t *AT, int64_t ldlt,
                           float *W, float *V, float *H, double *gsp, unsigned long long *Kfx, double *grad,
                           uint32_t *status, cudaStream_t st) {
    const int64_t nblk = cdiv(s, kBlk);
    double *scale = reinterpret_cast<double *>(Kfx + n * n);
    cudaError_t e = launch_bit_transpose_batched(A, 1, l, n, lda, AT, ldlt, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Kfx, 0, (size_t)n * n * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = launch_fixed_scale(alpha, beta, l, s, scale, st)) != cudaSuccess) return e;
    {
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_phase<1><<<dim3((unsigned)l, (unsigned)nblk), kBlk, 0, st>>>(A, lda, n, ZT, ldzt, M, lds, C, ldc,
                                                                         C + n * ldc, s, nblk, nullptr, alpha, beta,
                                                                         W, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_v<<<dim3((unsigned)n, (unsigned)nblk), kBlk, 0, st>>>(AT, ldlt, ZT, ldzt, W, lds, s, nblk, V, gsp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        // H[q][r] = sum_i (s_q(i) V[q][i]) s_r(i): A = V with signs from ZT, B bits = ZT rows.
        LaunchScope ls(IQP_KERNEL_LOWORDER_GEMM, st);
        const uint32_t *zt32 = reinterpret_cast<const uint32_t *>(ZT);
        k_lo_gemm<<<dim3((unsigned)cdiv(n, GN), (unsigned)cdiv(n, GM)), 256, 0, st>>>(V, lds, zt32, 2 * ldzt, zt32,
                                                                                       2 * ldzt, n, n, s, H, ldc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_pairs<<<(unsigned)l, kBlk, 0, st>>>(A, lda, n, ZT, ldzt, W, lds, s, scale, Kfx, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    LaunchScope ls(IQP_KERNEL_LOWORDER, st);
    k_lo_grad_out<<<grid_1d(m), 256, 0, st>>>(sup, m, n, gsp, nblk, H, ldc, Kfx, scale, grad);
    return cudaGetLastError();
}

}  // namespace iqp
