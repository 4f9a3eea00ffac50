// Plain FP32 form on the SIMT cores, plus the small kernels every form
// shares: theta preparation, the per-observable statistics finalisation, the
// fixed-order gradient reduction and the MMD combine.
//
// Phase contraction (eq. Emat): Phi[a][i] = sum_j c_j P_A[a][j] S_Z[i][j] with
// c_j = 2 theta_j and S_Z = 1 - 2 P_Z, as a 128x128 tile GEMM whose operands
// are expanded from parity bits into shared memory one 32-gate word at a time.
// Gradient (Sec. 2.4): Q[a][j] = sum_i W[a][i] S_Z[i][j], masked by P_A and
// summed over the observables of the tile.
#include "common.cuh"

namespace iqp {

uint32_t check_word_simt() { return take_check_word(); }

namespace {

constexpr int BM = 128, BN = 128, BK = 32, PADF = 4;

// ------------------------------------------------------------ theta split

// c_j = 2 theta_j (exact in FP32); hi = RN_bf16(c), lo = RN_bf16(c - hi)
// (c - hi is exact in FP32). Zero beyond m, up to mpad.
__global__ void k_theta_prep(const float *__restrict__ theta, int64_t m, int64_t mpad, float *__restrict__ c32,
                             __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < mpad; j += (int64_t)gridDim.x * blockDim.x) {
        const float c = j < m ? 2.0f * theta[j] : 0.0f;
        if (!IQP_IN(j, mpad, 20)) continue;
        if (c32) c32[j] = c;
        if (hi) {
            const __nv_bfloat16 h = __float2bfloat16_rn(c);
            hi[j] = h;
            lo[j] = __float2bfloat16_rn(c - __bfloat162float(h));
        }
    }
}

// --------------------------------------------------------- FP32 phase GEMM

// MODE 0: per (observable, 128-sample block) partials (S = sum cos, M2 = sum
// (cos - S/n)^2) into part[a * nparts + blockIdx.x].
// MODE 1: W[a][i] = sin Phi (alpha_a + beta_a cos Phi) into W (fp32, ldw).
template <int MODE>
__global__ void __launch_bounds__(256) k_phase_simt(const uint32_t *__restrict__ PA, const uint32_t *__restrict__ PZ,
                                                     int64_t ldp32, const float *__restrict__ c, int64_t l,
                                                     int64_t s, int64_t kwords, double2 *__restrict__ part,
                                                     int64_t nparts, const double *__restrict__ alpha,
                                                     const double *__restrict__ beta, float *__restrict__ W,
                                                     int64_t ldw) {
    __shared__ __align__(16) float As[2][BK][BM + PADF];
    __shared__ __align__(16) float Bs[2][BK][BN + PADF];
    __shared__ float cs[2][BK];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * BN, a0 = (int64_t)blockIdx.y * BM;

    // Row whose bits this thread expands: A rows for tid < 128, B rows above.
    const bool isA = tid < 128;
    const int er = tid & 127;
    const int64_t grow = isA ? a0 + er : i0 + er;
    const bool rvalid = isA ? grow < l : grow < s;
    const uint32_t *src = (isA ? PA : PZ) + (rvalid ? grow : 0) * ldp32;

    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;

    const int64_t srows = isA ? l : s;  // rows of the matrix this thread reads
    uint32_t bits = rvalid && IQP_IN((src - (isA ? PA : PZ)) + 0, srows * ldp32, 21) ? src[0] : 0u;
    float cnext = tid < BK ? c[tid] : 0.f;
    for (int64_t kw = 0; kw < kwords; ++kw) {
        const int buf = (int)(kw & 1);
        if (tid < BK) cs[buf][tid] = cnext;
        __syncthreads();
        if (isA) {
#pragma unroll
            for (int k = 0; k < BK; ++k) As[buf][k][er] = ((bits >> k) & 1u) ? cs[buf][k] : 0.f;
        } else {
#pragma unroll
            for (int k = 0; k < BK; ++k) Bs[buf][k][er] = ((bits >> k) & 1u) ? -1.f : 1.f;
        }
        __syncthreads();
        if (kw + 1 < kwords) {
            bits = rvalid && IQP_IN((src - (isA ? PA : PZ)) + kw + 1, srows * ldp32, 22) ? src[kw + 1] : 0u;
            cnext = tid < BK && IQP_IN((kw + 1) * BK + tid, kwords * BK, 23) ? c[(kw + 1) * BK + tid] : 0.f;
        }
#pragma unroll 8
        for (int k = 0; k < BK; ++k) {
            const float4 a_lo = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
            const float4 a_hi = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
            const float4 b_lo = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
            const float4 b_hi = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
            const float av[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
            const float bv[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
        }
    }

#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t a = a0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        if (MODE == 0) {
            float cv[8], sum = 0.f;
            bool ok[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t i = i0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + (q - 4));
                ok[q] = i < s;
                cv[q] = ok[q] ? cosf(acc[r][q]) : 0.f;
                sum += cv[q];
            }
#pragma unroll
            for (int off = 8; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
            const int64_t ncol = (s - i0) < BN ? (s - i0) : BN;
            const float mean = sum / (float)ncol;
            float m2 = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float d = cv[q] - mean;
                m2 += ok[q] ? d * d : 0.f;
            }
#pragma unroll
            for (int off = 8; off >= 1; off >>= 1) m2 += __shfl_xor_sync(0xFFFFFFFFu, m2, off);
            if (tx == 0 && a < l && IQP_IN(a * nparts + blockIdx.x, l * nparts, 24))
                part[a * nparts + blockIdx.x] = make_double2((double)sum, (double)m2);
        } else {
            if (a < l) {
                const float al = (float)alpha[a];
                const float be = beta ? (float)beta[a] : 0.f;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int64_t i = i0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + (q - 4));
                    if (i < s && IQP_IN(a * ldw + i, l * ldw, 25)) {
                        float sn, cn;
                        sincosf(acc[r][q], &sn, &cn);
                        W[a * ldw + i] = sn * (al + be * cn);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------- FP32 gradient

// gpart[blockIdx.y * m + j] = sum over the tile's observables a of
//   2 P_A[a][j] * sum_i W[a][i] S_Z[i][j].
__global__ void __launch_bounds__(256) k_grad_simt(const float *__restrict__ W, int64_t ldw,
                                                    const uint32_t *__restrict__ PZ, const uint32_t *__restrict__ PA,
                                                    int64_t ldp32, int64_t l, int64_t s, int64_t m,
                                                    double *__restrict__ gpart) {
    __shared__ __align__(16) float As[BK][BM + PADF];
    __shared__ __align__(16) float Bs[BK][BN + PADF];
    __shared__ float red[16][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t j0 = (int64_t)blockIdx.x * BN, a0 = (int64_t)blockIdx.y * BM;

    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;

    // Loader roles: W row (a0 + tid % 128), columns (tid / 128) * 16 .. +16;
    // sign rows: k = tid / 8, 16 gates at (tid % 8) * 16.
    const int wr = tid & 127, wc = (tid >> 7) * 16;
    const int64_t wrow = a0 + wr;
    const int bk = tid >> 3, bg = tid & 7;

    for (int64_t ib = 0; ib < s; ib += BK) {
        // W tile, transposed into k-major.
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = ib + wc + 4 * q;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (wrow < l && IQP_IN(wrow * ldw + (i + 3 < s ? i + 3 : (i < s ? i : 0)), l * ldw, 26)) {
                if (i + 3 < s) {
                    v = *reinterpret_cast<const float4 *>(W + wrow * ldw + i);
                } else {
                    v.x = i < s ? W[wrow * ldw + i] : 0.f;
                    v.y = i + 1 < s ? W[wrow * ldw + i + 1] : 0.f;
                    v.z = i + 2 < s ? W[wrow * ldw + i + 2] : 0.f;
                }
            }
            As[wc + 4 * q + 0][wr] = v.x;
            As[wc + 4 * q + 1][wr] = v.y;
            As[wc + 4 * q + 2][wr] = v.z;
            As[wc + 4 * q + 3][wr] = v.w;
        }
        // Sign tile from P_Z bits.
        {
            const int64_t i = ib + bk;
            uint32_t b = 0u;
            if (i < s && IQP_IN(i * ldp32 + ((j0 + bg * 16) >> 5), s * ldp32, 27))
                b = (PZ[i * ldp32 + ((j0 + bg * 16) >> 5)] >> ((bg & 1) * 16)) & 0xFFFFu;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 v;
                v.x = ((b >> (4 * q + 0)) & 1u) ? -1.f : 1.f;
                v.y = ((b >> (4 * q + 1)) & 1u) ? -1.f : 1.f;
                v.z = ((b >> (4 * q + 2)) & 1u) ? -1.f : 1.f;
                v.w = ((b >> (4 * q + 3)) & 1u) ? -1.f : 1.f;
                *reinterpret_cast<float4 *>(&Bs[bk][bg * 16 + 4 * q]) = v;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < BK; ++k) {
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

    // Mask by 2 P_A[a][j], sum the thread's 8 rows per column.
    float colsum[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) colsum[q] = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t a = a0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        if (a < l && IQP_IN(a * ldp32 + ((j0 + 64 + tx * 4) >> 5), l * ldp32, 28)) {
            const uint32_t w_lo = PA[a * ldp32 + ((j0 + tx * 4) >> 5)];
            const uint32_t w_hi = PA[a * ldp32 + ((j0 + 64 + tx * 4) >> 5)];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t j = j0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + (q - 4));
                const uint32_t wb = q < 4 ? w_lo : w_hi;
                if ((wb >> (j & 31)) & 1u) colsum[q] += 2.f * acc[r][q];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) red[ty][q < 4 ? tx * 4 + q : 64 + tx * 4 + (q - 4)] = colsum[q];
    __syncthreads();
    if (tid < BN) {
        double t = 0.0;
#pragma unroll
        for (int y = 0; y < 16; ++y) t += (double)red[y][tid];
        const int64_t j = j0 + tid;
        if (j < m && IQP_IN((int64_t)blockIdx.y * m + j, (int64_t)gridDim.y * m, 29)) gpart[(int64_t)blockIdx.y * m + j] = t;
    }
}

// ------------------------------------------------------------ reductions

// Merge the (S, M2) partials of each observable in fixed order (Chan et al.):
// mean = S/s, M2 = sum_k [M2_k + n_k (S_k/n_k - mean)^2].
// Per observable a: the mean of cos Phi over the s samples and its standard
// error from the (sum, M2) partials of pw samples each (Chan's combination),
// plus the sums S1 = sum cos, S2 = sum cos^2 for the MMD loss. One warp per
// observable: lane q takes partials q, q + 32, ... (coalesced 16-byte loads)
// and a fixed xor-shuffle tree combines the lanes, so the result does not
// depend on the launch.
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, w);
    return v;
}

__global__ void __launch_bounds__(256) k_finalize(const double2 *__restrict__ part, int64_t nparts, int64_t pw,
                                                  int64_t l, int64_t s, double *__restrict__ expval,
                                                  double *__restrict__ std_err, double *__restrict__ S1,
                                                  double *__restrict__ S2) {
    const int lane = threadIdx.x & 31;
    const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (a >= l) return;  // whole warps
    if (!IQP_IN(a * nparts + nparts - 1, l * nparts, 30)) return;
    const double2 *p = part + a * nparts;
    double S = 0.0;
    for (int64_t k = lane; k < nparts; k += 32) S += p[k].x;
    S = warp_sum_f64(S);
    const double mean = S / (double)s;
    const double inv_pw = 1.0 / (double)pw;
    double M2 = 0.0;
    for (int64_t k = lane; k < nparts; k += 32) {
        const int64_t nk = (s - k * pw) < pw ? (s - k * pw) : pw;
        const double2 v = p[k];
        const double d = (nk == pw ? v.x * inv_pw : v.x / (double)nk) - mean;
        M2 += v.y + (double)nk * d * d;
    }
    M2 = warp_sum_f64(M2);
    if (lane != 0) return;
    if (expval) expval[a] = mean;
    if (std_err) std_err[a] = sqrt(M2 / (double)s) / sqrt((double)s);
    if (S1) S1[a] = S;
    if (S2) S2[a] = M2 + S * mean;
}

// grad[j] = sum over observable tiles t of gpart[t * m + j], in order.
__global__ void k_grad_reduce(const double *__restrict__ gpart, int64_t ntiles, int64_t m, double *__restrict__ grad) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int64_t k = 0; k < ntiles; ++k) t += gpart[k * m + j];
        grad[j] = t;
    }
}

// MMD^2 of eq. mmd_estimate and the gradient coefficients alpha, beta.
// sqrt_loss: loss' = sqrt(max(loss, 0)) and alpha, beta scaled by 1/(2 loss')
// (chain rule; zero where loss' = 0).
__global__ void __launch_bounds__(1024) k_mmd_combine(const long long *__restrict__ T, const double *__restrict__ S1,
                                                      const double *__restrict__ S2, int64_t l, int64_t s, int64_t N,
                                                      int unbiased, int sqrt_loss, double *__restrict__ terms,
                                                      double *__restrict__ alpha, double *__restrict__ beta,
                                                      double *__restrict__ loss) {
    __shared__ double red[1024];
    const double ds = (double)s, dN = (double)N, dl = (double)l;
    double acc = 0.0;
    for (int64_t a = threadIdx.x; a < l; a += blockDim.x) {
        const double t = (double)T[a];
        const double p = t / dN, q = S1[a] / ds;
        double term, al, be;
        if (unbiased) {
            const double up = (t * t - dN) / (dN * (dN - 1.0));
            const double uq = (S1[a] * S1[a] - S2[a]) / (ds * (ds - 1.0));
            term = up - 2.0 * p * q + uq;
            al = (2.0 * p / ds - 2.0 * S1[a] / (ds * (ds - 1.0))) / dl;
            be = 2.0 / (ds * (ds - 1.0)) / dl;
        } else {
            term = (p - q) * (p - q);
            al = 2.0 * (p - q) / ds / dl;
            be = 0.0;
        }
        if (terms) terms[a] = term;
        if (alpha) alpha[a] = al;
        if (beta) beta[a] = be;
        acc += term;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double L = red[0] / dl;
    if (!sqrt_loss) {
        if (threadIdx.x == 0) *loss = L;
        return;
    }
    const double r = L > 0.0 ? sqrt(L) : 0.0;
    const double f = L > 0.0 ? 0.5 / r : 0.0;
    for (int64_t a = threadIdx.x; a < l; a += blockDim.x) {
        if (alpha) alpha[a] *= f;
        if (beta) beta[a] *= f;
    }
    if (threadIdx.x == 0) *loss = r;
}

// alpha_a = -w_a / s for a linear loss given weights (device helper).
__global__ void k_scale(const double *__restrict__ x, double f, int64_t l, double *__restrict__ y) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a < l) y[a] = f * x[a];
}

}  // namespace

cudaError_t launch_theta_prep(const float *theta, int64_t m, int64_t mpad, float *c32, __nv_bfloat16 *hi,
                              __nv_bfloat16 *lo, cudaStream_t st) {
    int blocks = (int)cdiv(mpad, 256);
    if (blocks > 4096) blocks = 4096;
    LaunchScope ls(IQP_KERNEL_THETA_SPLIT, st);
    k_theta_prep<<<blocks, 256, 0, st>>>(theta, m, mpad, c32, hi, lo);
    return cudaGetLastError();
}

cudaError_t launch_phase_simt(int mode, const uint64_t *PA, const uint64_t *PZ, int64_t ldp, const float *c,
                              int64_t l, int64_t s, int64_t m, double2 *part, int64_t nparts, const double *alpha,
                              const double *beta, float *W, int64_t ldw, cudaStream_t st) {
    const int64_t kwords = cdiv(m, 32);
    const int64_t gy_total = cdiv(l, BM);
    for (int64_t y0 = 0; y0 < gy_total; y0 += 65535) {
        const int64_t ny = gy_total - y0 < 65535 ? gy_total - y0 : 65535;
        const int64_t aoff = y0 * BM;
        dim3 grid((unsigned)cdiv(s, BN), (unsigned)ny);
        const uint32_t *pa = reinterpret_cast<const uint32_t *>(PA + aoff * ldp);
        LaunchScope ls(mode == 0 ? IQP_KERNEL_PHASE_FP32 : IQP_KERNEL_RECOMPUTE_FP32, st);
        if (mode == 0)
            k_phase_simt<0><<<grid, 256, 0, st>>>(pa, reinterpret_cast<const uint32_t *>(PZ), 2 * ldp, c, l - aoff,
                                                  s, kwords, part + aoff * nparts, nparts, nullptr, nullptr, nullptr,
                                                  0);
        else
            k_phase_simt<1><<<grid, 256, 0, st>>>(pa, reinterpret_cast<const uint32_t *>(PZ), 2 * ldp, c, l - aoff,
                                                  s, kwords, nullptr, 0, alpha + aoff, beta ? beta + aoff : nullptr,
                                                  W + aoff * ldw, ldw);
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_simt(const float *W, int64_t ldw, const uint64_t *PZ, const uint64_t *PA, int64_t ldp,
                             int64_t l, int64_t s, int64_t m, double *gpart, cudaStream_t st) {
    const int64_t gy_total = cdiv(l, BM);
    for (int64_t y0 = 0; y0 < gy_total; y0 += 65535) {
        const int64_t ny = gy_total - y0 < 65535 ? gy_total - y0 : 65535;
        const int64_t aoff = y0 * BM;
        dim3 grid((unsigned)cdiv(m, BN), (unsigned)ny);
        LaunchScope ls(IQP_KERNEL_GRAD_FP32, st);
        k_grad_simt<<<grid, 256, 0, st>>>(W + aoff * ldw, ldw, reinterpret_cast<const uint32_t *>(PZ),
                                          reinterpret_cast<const uint32_t *>(PA + aoff * ldp), 2 * ldp, l - aoff, s,
                                          m, gpart + y0 * m);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double2 *part, int64_t nparts, int64_t pw, int64_t l, int64_t s, double *expval,
                            double *std_err, double *S1, double *S2, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_FINALIZE, st);
    k_finalize<<<(unsigned)cdiv(l, 8), 256, 0, st>>>(part, nparts, pw, l, s, expval, std_err, S1, S2);
    return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const double *gpart, int64_t ntiles, int64_t m, double *grad, cudaStream_t st) {
    int blocks = (int)cdiv(m, 256);
    if (blocks > 8192) blocks = 8192;
    LaunchScope ls(IQP_KERNEL_GRAD_REDUCE, st);
    k_grad_reduce<<<blocks, 256, 0, st>>>(gpart, ntiles, m, grad);
    return cudaGetLastError();
}

cudaError_t launch_mmd_combine(const int64_t *T, const double *S1, const double *S2, int64_t l, int64_t s, int64_t N,
                               int unbiased, bool sqrt_loss, double *terms, double *alpha, double *beta, double *loss,
                               cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_MMD_COMBINE, st);
    k_mmd_combine<<<1, 1024, 0, st>>>(reinterpret_cast<const long long *>(T), S1, S2, l, s, N, unbiased,
                                      sqrt_loss ? 1 : 0, terms, alpha, beta, loss);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double *x, double f, int64_t l, double *y, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_FINALIZE, st);
    k_scale<<<(unsigned)cdiv(l, 256), 256, 0, st>>>(x, f, l, y);
    return cudaGetLastError();
}

}  // namespace iqp
