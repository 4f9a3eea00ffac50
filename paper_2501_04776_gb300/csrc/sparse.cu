// Row-sparse form of the phase contraction and of its gradient, for parity
// matrices P_A of low density (Sec. 2.2 notes that C = 1 - (-1)^{A G^T} is
// sparse when observables and generators have small support).
//
// For one observable a, with J_a = { j : P_A[a][j] = 1 } and c_j = 2 theta_j,
//   Phi[a][i] = sum_{j in J_a} c_j (1 - 2 P_Z[i][j])          (eq. Emat)
// and, for W[a][i] = sin Phi (alpha_a + beta_a cos Phi),
//   grad_j    = sum_{a : j in J_a} 2 sum_i W[a][i] (1 - 2 P_Z[i][j]).
// The work is |J_a| * s per observable instead of m * s: the dense forms
// multiply every zero of P_A too.
//
// Layout: one CTA per (observable, block of up to 8 x 2048 samples). Lane q of
// warp r owns the 64 samples of word (32 r + q) of every P_Z^T row, so the
// P_Z^T word of a gate is one coalesced 256-byte load per warp and each term
// is a sign flip and an add in FP32 (no multiply: the operand is +-c_j). The
// set bits of the P_A row are visited in increasing gate order by every warp
// of the CTA (32 words per coalesced load), with the next gate's P_Z^T word
// loaded before the current one is consumed.
//
// Statistics: per-warp (sum cos, sum (cos - mean)^2) partials of 2048 samples
// (FP32 within a lane, FP64 across lanes), merged by the shared finaliser.
// Gradient: the per-warp dot products are added into a 64-bit fixed-point
// accumulator per gate with integer atomics. Integer addition is associative,
// so the result does not depend on the order of the atomics: the gradient is
// bitwise reproducible. The fixed-point scale 2^k is chosen per call from the
// bound B = sum_a 2 s (|alpha_a| + |beta_a|) >= |every partial sum| so that
// B 2^k < 2^61: nothing can overflow, and the rounding error per gate is at
// most (number of contributions) * 2^-k / 2.
#include <cstdlib>

#include "common.cuh"

namespace iqp {

namespace {

constexpr int kWarpSamples = 32 * 64;
constexpr int kMaxWarps = 8;
constexpr unsigned kFull = 0xFFFFFFFFu;

// Two FP32 adds in one instruction (sm_100+ packed FP32): (a.x + b.x, a.y + b.y),
// each rounded to nearest like a scalar add.
__device__ __forceinline__ uint64_t add_f32x2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t pack2(uint32_t lo, uint32_t hi) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(lo), "r"(hi));
    return d;
}

// The lane's 64 accumulators as 32 pairs: pair t holds samples t (low half)
// and 32 + t (high half) of the lane's word.
// acc[t] += (bit t of z ? -c : c, bit 32+t of z ? -c : c).
__device__ __forceinline__ void add_signed(uint64_t (&acc)[32], uint64_t z, uint32_t cb) {
    const uint32_t lo = (uint32_t)z, hi = (uint32_t)(z >> 32);
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const uint32_t a = cb ^ ((lo << (31 - t)) & 0x80000000u);
        const uint32_t b = cb ^ ((hi << (31 - t)) & 0x80000000u);
        acc[t] = add_f32x2(acc[t], pack2(a, b));
    }
}

// sum_k (bit k of z ? -w_k : w_k) over the lane's 64 samples, w paired like
// the accumulators, in 4 interleaved pair sums.
__device__ __forceinline__ float signed_dot(const uint64_t (&w)[32], uint64_t z) {
    const uint32_t lo = (uint32_t)z, hi = (uint32_t)(z >> 32);
    uint64_t p[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const uint32_t a = (uint32_t)w[t] ^ ((lo << (31 - t)) & 0x80000000u);
        const uint32_t b = (uint32_t)(w[t] >> 32) ^ ((hi << (31 - t)) & 0x80000000u);
        p[t & 3] = add_f32x2(p[t & 3], pack2(a, b));
    }
    const uint64_t q = add_f32x2(add_f32x2(p[0], p[1]), add_f32x2(p[2], p[3]));
    return __uint_as_float((uint32_t)q) + __uint_as_float((uint32_t)(q >> 32));
}

// Calls fn(j) for every set bit j of the P_A row, in increasing j, with the
// same j on all lanes of the warp.
template <class F>
__device__ __forceinline__ void for_each_gate(const uint64_t *__restrict__ row, int64_t ldp, int lane, F &fn) {
    uint64_t next = lane < ldp ? __ldg(row + lane) : 0ull;
    for (int64_t w0 = 0; w0 < ldp; w0 += 32) {
        const uint64_t bits = next;
        next = (w0 + 32 + lane < ldp) ? __ldg(row + w0 + 32 + lane) : 0ull;
        uint32_t live = __ballot_sync(kFull, bits != 0ull);
        while (live) {
            const int src = __ffs(live) - 1;
            live &= live - 1u;
            uint64_t wb = __shfl_sync(kFull, bits, src);
            const int64_t jb = (w0 + src) * 64;
            while (wb) {
                const int b = __ffsll((long long)wb) - 1;
                wb &= wb - 1ull;
                fn(jb + b);
            }
        }
    }
}

// The lane's P_Z^T word of gate j. Shared batch: a load from P_Z^T.
// Independent batches: the parity is formed here from the observable's own
// transposed samples ZT (n rows of bits over samples) as the XOR of the rows
// of the gate's support (listed for |supp| <= 3, else read from G).
struct ZSource {
    const uint64_t *PZT;  // shared: P_Z^T; independent: this observable's ZT
    int64_t ldzt;
    int64_t word;
    const int4 *sup;      // independent batches only
    const uint64_t *G;
    int64_t ldg;
    int64_t n;
    int64_t m;            // gates

    template <bool INDEP>
    __device__ __forceinline__ uint64_t get(int64_t j) const {
        if (!IQP_IN(j, m, 70)) return 0ull;  // a set parity bit past the last gate
        if (!INDEP) return __ldg(PZT + j * ldzt + word);
        const int4 sp = __ldg(sup + j);
        if (sp.w <= 3) {
            if (!IQP_IN(sp.w > 0 ? sp.x : 0, n, 71) || !IQP_IN(sp.w > 1 ? sp.y : 0, n, 71) ||
                !IQP_IN(sp.w > 2 ? sp.z : 0, n, 71))
                return 0ull;
            uint64_t z = 0ull;
            if (sp.w > 0) z = __ldg(PZT + (int64_t)sp.x * ldzt + word);
            if (sp.w > 1) z ^= __ldg(PZT + (int64_t)sp.y * ldzt + word);
            if (sp.w > 2) z ^= __ldg(PZT + (int64_t)sp.z * ldzt + word);
            return z;
        }
        uint64_t z = 0ull;
        const uint64_t *g = G + j * ldg;
        const int64_t nw = (n + 63) >> 6;
        for (int64_t w = 0; w < nw; ++w) {
            uint64_t gv = __ldg(g + w);
            while (gv) {
                const int b = __ffsll((long long)gv) - 1;
                gv &= gv - 1ull;
                const int64_t q = 64 * w + b;
                if (q >= n) break;
                z ^= __ldg(PZT + q * ldzt + word);
            }
        }
        return z;
    }
};

// Gates are consumed in batches of kBatch: the batch's P_Z^T words and
// c_j are all loaded before the first is used, so their latencies overlap
// (the batch holds only gate indices while it fills; a register holding an
// in-flight load is never copied, which would wait for it). The gradient
// pass, which also holds W in registers, uses half as many.
constexpr int kPhaseBatch = 8, kGradBatch = 4;

template <class R, int kBatch>
struct GateBatcher {
    int64_t jb[kBatch];
    int nb;
    R &run;
    __device__ __forceinline__ explicit GateBatcher(R &r) : nb(0), run(r) {
#pragma unroll
        for (int t = 0; t < kBatch; ++t) jb[t] = 0;
    }
    __device__ __forceinline__ void operator()(int64_t j) {
#pragma unroll
        for (int t = 0; t + 1 < kBatch; ++t) jb[t] = jb[t + 1];
        jb[kBatch - 1] = j;
        if (++nb == kBatch) {
            run.go(jb);
            nb = 0;
        }
    }
    __device__ __forceinline__ void finish() {
        // warp-uniform: the same gates on every lane
#pragma unroll
        for (int cnt = 1; cnt < kBatch; ++cnt)
            if (nb == cnt) run.go_tail(jb, cnt);
    }
};

template <bool INDEP, int kBatch>
struct PhaseRun {
    uint64_t (&acc)[32];
    const ZSource &zs;
    const float *__restrict__ c;
    __device__ __forceinline__ void go(const int64_t (&jb)[kBatch]) {
        uint64_t z[kBatch];
        uint32_t cv[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            z[t] = zs.get<INDEP>(jb[t]);
            cv[t] = __float_as_uint(__ldg(c + jb[t]));
        }
#pragma unroll
        for (int t = 0; t < kBatch; ++t) add_signed(acc, z[t], cv[t]);
    }
    __device__ __forceinline__ void go_tail(const int64_t (&jb)[kBatch], int cnt) {
#pragma unroll
        for (int t = 0; t < kBatch; ++t)
            if (t >= kBatch - cnt) add_signed(acc, zs.get<INDEP>(jb[t]), __float_as_uint(__ldg(c + jb[t])));
    }
};

// Phi for the lane's 64 samples (sum over J_a, increasing j), paired as in
// add_signed.
template <bool INDEP>
__device__ __forceinline__ void phase_row(uint64_t (&acc)[32], const uint64_t *__restrict__ parow, int64_t ldp,
                                          const ZSource &zs, const float *__restrict__ c, int lane) {
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0ull;
    PhaseRun<INDEP, kPhaseBatch> run{acc, zs, c};
    GateBatcher<PhaseRun<INDEP, kPhaseBatch>, kPhaseBatch> batch(run);
    for_each_gate(parow, ldp, lane, batch);
    batch.finish();
}

// Gradient contributions of a batch of gates: per gate the lane's signed
// dot product of W with the gate's P_Z^T word, reduced over the warp, added
// in fixed point to the gate's accumulator.
template <bool INDEP, int kBatch>
struct GradRun {
    const uint64_t (&w)[32];
    const ZSource &zs;
    unsigned long long *__restrict__ gfx;
    float sc;  // 2 * scale, a power of two in [2^-119, 2^119]: exact scaling in FP32
    int lane;
    // Fixed-point value of one contribution without FP64 (slow on this GPU):
    // x = sc d, |x| < 2^61, split exactly into hi 2^31 + lo.
    __device__ __forceinline__ void emit(uint64_t z, int64_t j) {
        float d = signed_dot(w, z);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) d += __shfl_xor_sync(kFull, d, off);
        if (lane == 0 && IQP_IN(j, zs.m, 72)) {
            const float x = sc * d;
            const float hi = truncf(x * 0x1.0p-31f);
            const float lo = fmaf(-hi, 0x1.0p31f, x);
            const long long q = ((long long)__float2int_rz(hi) << 31) + (long long)__float2int_rn(lo);
            atomicAdd(gfx + j, (unsigned long long)q);
        }
    }
    __device__ __forceinline__ void go(const int64_t (&jb)[kBatch]) {
        uint64_t z[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) z[t] = zs.get<INDEP>(jb[t]);
#pragma unroll
        for (int t = 0; t < kBatch; ++t) emit(z[t], jb[t]);
    }
    __device__ __forceinline__ void go_tail(const int64_t (&jb)[kBatch], int cnt) {
#pragma unroll
        for (int t = 0; t < kBatch; ++t)
            if (t >= kBatch - cnt) emit(zs.get<INDEP>(jb[t]), jb[t]);
    }
};

// MODE 0: statistics partials, and Phi itself into phi (l x ldphi FP32) when
// phi is not null (a gradient pass follows). MODE 1: W from Phi (read from
// phi when not null, else recomputed), then the gradient contributions of
// every gate of J_a. MODE 2: both from one Phi (gradient coefficients known
// in advance), the statistics and W as MODE 0 and MODE 1 form them. Independent batches always recompute (keeping Phi there
// would push the statistics pass past its register budget).
// INDEP: PZT holds every observable's transposed samples (n x ldzt words
// each, observable a at PZT + a n ldzt) and the parities are formed on the fly.
template <int MODE, bool INDEP>
__global__ void __launch_bounds__(256, 2)
    k_sparse(const uint64_t *__restrict__ PA, int64_t ldp, const uint64_t *__restrict__ PZT, int64_t ldzt,
             int64_t m, const float *__restrict__ c, int64_t s, int64_t nparts, double2 *__restrict__ part,
             const double *__restrict__ alpha, const double *__restrict__ beta, const double *__restrict__ scale,
             unsigned long long *__restrict__ gfx, const int4 *__restrict__ sup, const uint64_t *__restrict__ G,
             int64_t ldg, int64_t n, float *__restrict__ phi, int64_t ldphi) {
    const int lane = threadIdx.x & 31;
    const int64_t a = blockIdx.x;
    const int64_t r = (int64_t)blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);  // 2048-sample range
    if (r >= nparts) return;  // warp-uniform; no block-level barriers below
    const int64_t vwords = cdiv(s, 64);
    const int64_t word_raw = r * 32 + lane;
    const bool wvalid = word_raw < vwords;
    const int64_t word = wvalid ? word_raw : vwords - 1;  // in-bounds load, result masked
    const int64_t i0 = word_raw * 64;
    const int nvalid = !wvalid ? 0 : (s - i0 >= 64 ? 64 : (int)(s - i0));
    const uint64_t *parow = PA + a * ldp;
    const ZSource zs{INDEP ? PZT + a * n * ldzt : PZT, ldzt, word, sup, G, ldg, n, m};
    [[maybe_unused]] const int64_t l = gridDim.x;  // one observable per CTA column

    uint64_t acc2[32];
    // The lane's 64 samples i0 .. i0 + 63 lie inside a row of phi (ldphi is a
    // multiple of 64) whenever the lane's word is valid; they are kept in the
    // accumulators' pair order (pair t: samples t and 32 + t), 256 bytes a lane.
    if (MODE == 1 && !INDEP && phi != nullptr) {
        const bool pin = IQP_IN(a * ldphi + (wvalid ? i0 + 63 : 0), l * ldphi, 73);
        const uint4 *prow = reinterpret_cast<const uint4 *>(phi + a * ldphi + (wvalid && pin ? i0 : 0));
#pragma unroll
        for (int v = 0; v < 16; ++v) {
            const uint4 q = wvalid && pin ? prow[v] : make_uint4(0u, 0u, 0u, 0u);
            acc2[2 * v] = (uint64_t)q.x | ((uint64_t)q.y << 32);
            acc2[2 * v + 1] = (uint64_t)q.z | ((uint64_t)q.w << 32);
        }
    } else {
        phase_row<INDEP>(acc2, parow, ldp, zs, c, lane);
        if (MODE == 0 && !INDEP && phi != nullptr && wvalid && IQP_IN(a * ldphi + i0 + 63, l * ldphi, 74)) {
            uint4 *prow = reinterpret_cast<uint4 *>(phi + a * ldphi + i0);
#pragma unroll
            for (int v = 0; v < 16; ++v)
                prow[v] = make_uint4((uint32_t)acc2[2 * v], (uint32_t)(acc2[2 * v] >> 32), (uint32_t)acc2[2 * v + 1],
                                     (uint32_t)(acc2[2 * v + 1] >> 32));
        }
    }
    float acc[64];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        acc[t] = __uint_as_float((uint32_t)acc2[t]);
        acc[32 + t] = __uint_as_float((uint32_t)(acc2[t] >> 32));
    }

    if (MODE == 0 || MODE == 2) {
        // MODE 2 keeps Phi in acc for W below and takes the cosines twice.
        float sum = 0.f;
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            const float cv = k < nvalid ? cosf(acc[k]) : 0.f;
            if (MODE == 0) acc[k] = cv;
            sum += cv;
        }
        double ds = (double)sum;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) ds += __shfl_xor_sync(kFull, ds, off);
        const int64_t nr = (s - r * kWarpSamples) < kWarpSamples ? (s - r * kWarpSamples) : kWarpSamples;
        const float mean = (float)(ds / (double)nr);
        float m2 = 0.f;
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            const float d = (MODE == 0 ? acc[k] : (k < nvalid ? cosf(acc[k]) : 0.f)) - mean;
            m2 += k < nvalid ? d * d : 0.f;
        }
        double dm = (double)m2;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) dm += __shfl_xor_sync(kFull, dm, off);
        if (lane == 0 && IQP_IN(a * nparts + r, l * nparts, 75)) part[a * nparts + r] = make_double2(ds, dm);
    }
    if (MODE != 0) {
        const float al = (float)alpha[a];
        const float be = beta ? (float)beta[a] : 0.f;
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            float sn, cn;
            sincosf(acc[k], &sn, &cn);
            acc[k] = k < nvalid ? sn * (al + be * cn) : 0.f;
        }
#pragma unroll
        for (int t = 0; t < 32; ++t) acc2[t] = pack2(__float_as_uint(acc[t]), __float_as_uint(acc[32 + t]));
        const float sc = (float)(2.0 * *scale);
        GradRun<INDEP, kGradBatch> run{acc2, zs, gfx, sc, lane};
        GateBatcher<GradRun<INDEP, kGradBatch>, kGradBatch> batch(run);
        for_each_gate(parow, ldp, lane, batch);
        batch.finish();
    }
}

// scale = 2^k with B 2^k < 2^61, B = sum_a 2 s (|alpha_a| + |beta_a|)
// (fixed-order FP64 sum).
__global__ void __launch_bounds__(256) k_sparse_scale(const double *__restrict__ alpha,
                                                      const double *__restrict__ beta, int64_t l, int64_t s,
                                                      double *__restrict__ scale) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t a = threadIdx.x; a < l; a += 256) acc += fabs(alpha[a]) + (beta ? fabs(beta[a]) : 0.0);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // B in [2^e, 2^(e+1)); scale = 2^(60-e) gives B scale < 2^61. e is
        // clamped to [-58, 180] so that 2 scale is a normal FP32 number.
        const double B = 2.0 * (double)s * red[0];
        int e = (B > 0.0 && B < 1e300) ? ilogb(B) : 0;
        if (e < -58) e = -58;
        if (e > 180) e = 180;
        *scale = ldexp(1.0, 60 - e);
    }
}

// grad[j] = fixed-point accumulator / scale.
__global__ void k_sparse_grad_out(const unsigned long long *__restrict__ gfx, int64_t m,
                                  const double *__restrict__ scale, double *__restrict__ grad) {
    const double inv = 1.0 / *scale;  // a power of two: exact
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        grad[j] = (double)(long long)gfx[j] * inv;
}

// Warps per CTA (IQP_SPARSE_WARPS, 1..8, default 1): every warp scans its
// observable's P_A row on its own, so larger CTAs share nothing and only
// coarsen the scheduling; single-warp CTAs balance observables of unequal
// |J_a| best and, ordered observable-fastest, keep the P_Z^T segments of one
// 2048-sample range hot in L2 across observables.
int sparse_warps() {
    static int w = -1;
    if (w < 0) {
        const char *e = std::getenv("IQP_SPARSE_WARPS");
        const int v = e ? std::atoi(e) : 1;
        w = (v >= 1 && v <= kMaxWarps) ? v : 1;
    }
    return w;
}

dim3 sparse_grid(int64_t l, int64_t nparts, int *threads) {
    const int cap = sparse_warps();
    const int nw = nparts < cap ? (int)nparts : cap;
    *threads = 32 * nw;
    return dim3((unsigned)l, (unsigned)cdiv(nparts, nw));
}

}  // namespace

int64_t sparse_part_samples() { return kWarpSamples; }
uint32_t check_word_sparse() { return take_check_word(); }

// Statistics partials and the gradient from one pass over Phi (shared
// batches; alpha, beta known before the estimates): k_sparse<2>.
cudaError_t launch_sparse_value_grad(const uint64_t *PA, int64_t ldp, const uint64_t *PZT, int64_t ldzt,
                                     const float *c, int64_t l, int64_t s, int64_t m, int64_t nparts, double2 *part,
                                     const double *alpha, const double *beta, double *scale, unsigned long long *gfx,
                                     double *grad, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(gfx, 0, (size_t)m * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    {
        LaunchScope ls(IQP_KERNEL_GRAD_SPARSE, st);
        k_sparse_scale<<<1, 256, 0, st>>>(alpha, beta, l, s, scale);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        int threads = 0;
        const dim3 grid = sparse_grid(l, nparts, &threads);
        LaunchScope ls(IQP_KERNEL_PHASE_SPARSE, st);
        k_sparse<2, false><<<grid, threads, 0, st>>>(PA, ldp, PZT, ldzt, m, c, s, nparts, part, alpha, beta, scale, gfx,
                                                     nullptr, nullptr, 0, 0, nullptr, 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    int blocks = (int)cdiv(m, 256);
    if (blocks > 8192) blocks = 8192;
    LaunchScope ls(IQP_KERNEL_GRAD_SPARSE, st);
    k_sparse_grad_out<<<blocks, 256, 0, st>>>(gfx, m, scale, grad);
    return cudaGetLastError();
}

// scale (one double) = 2^k with sum_a 2 s (|alpha_a| + |beta_a|) 2^k < 2^61;
// used by every fixed-point gradient accumulation.
cudaError_t launch_fixed_scale(const double *alpha, const double *beta, int64_t l, int64_t s, double *scale,
                               cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_GRAD_SPARSE, st);
    k_sparse_scale<<<1, 256, 0, st>>>(alpha, beta, l, s, scale);
    return cudaGetLastError();
}

// indep != nullptr: independent batches (PZT = every observable's ZT).
// phi != nullptr: Phi is kept there (l x ldphi FP32, ldphi a multiple of 64).
cudaError_t launch_sparse_stats(const uint64_t *PA, int64_t ldp, const uint64_t *PZT, int64_t ldzt, const float *c,
                                int64_t l, int64_t s, int64_t m, double2 *part, int64_t nparts,
                                const SparseIndep *indep, float *phi, int64_t ldphi, cudaStream_t st) {
    int threads = 0;
    const dim3 grid = sparse_grid(l, nparts, &threads);
    LaunchScope ls(IQP_KERNEL_PHASE_SPARSE, st);
    if (indep)
        k_sparse<0, true><<<grid, threads, 0, st>>>(PA, ldp, PZT, ldzt, m, c, s, nparts, part, nullptr, nullptr,
                                                    nullptr, nullptr, indep->sup, indep->G, indep->ldg, indep->n,
                                                    phi, ldphi);
    else
        k_sparse<0, false><<<grid, threads, 0, st>>>(PA, ldp, PZT, ldzt, m, c, s, nparts, part, nullptr, nullptr,
                                                     nullptr, nullptr, nullptr, nullptr, 0, 0, phi, ldphi);
    return cudaGetLastError();
}

cudaError_t launch_sparse_grad(const uint64_t *PA, int64_t ldp, const uint64_t *PZT, int64_t ldzt, const float *c,
                               int64_t l, int64_t s, int64_t m, int64_t nparts, const double *alpha,
                               const double *beta, double *scale, unsigned long long *gfx, double *grad,
                               const SparseIndep *indep, const float *phi, int64_t ldphi, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(gfx, 0, (size_t)m * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    {
        LaunchScope ls(IQP_KERNEL_GRAD_SPARSE, st);
        k_sparse_scale<<<1, 256, 0, st>>>(alpha, beta, l, s, scale);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        int threads = 0;
        const dim3 grid = sparse_grid(l, nparts, &threads);
        LaunchScope ls(IQP_KERNEL_GRAD_SPARSE, st);
        if (indep)
            k_sparse<1, true><<<grid, threads, 0, st>>>(PA, ldp, PZT, ldzt, m, c, s, nparts, nullptr, alpha, beta, scale,
                                                        gfx, indep->sup, indep->G, indep->ldg, indep->n,
                                                        const_cast<float *>(phi), ldphi);
        else
            k_sparse<1, false><<<grid, threads, 0, st>>>(PA, ldp, PZT, ldzt, m, c, s, nparts, nullptr, alpha, beta,
                                                         scale, gfx, nullptr, nullptr, 0, 0, const_cast<float *>(phi),
                                                         ldphi);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    int blocks = (int)cdiv(m, 256);
    if (blocks > 8192) blocks = 8192;
    LaunchScope ls(IQP_KERNEL_GRAD_SPARSE, st);
    k_sparse_grad_out<<<blocks, 256, 0, st>>>(gfx, m, scale, grad);
    return cudaGetLastError();
}

}  // namespace iqp
