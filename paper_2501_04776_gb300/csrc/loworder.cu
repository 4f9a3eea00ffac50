// Low-order form: every generator has weight <= 2 (the one- and two-body
// gate sets of Sec. 3.1.1 and Sec. 4). With s_q(i) = (-1)^{z_{i,q}},
// Q_a = supp(a), c_j = 2 theta_j, d_q = sum of c_j over the one-qubit gates
// on q and C_qr = sum of c_j over the gates on {q, r} (symmetric, zero
// diagonal):
//   [g_j.a odd]      = [q in Q_a] for g_j = e_q, [exactly one of q, r in Q_a] for e_q + e_r,
//   1 - 2[g_j.z odd] = s_q(z), or s_q(z) s_r(z),
// so the phase of eq. expvalsample regroups exactly into
//   Phi[a,i] = sum_{q in Q_a} s_q(i) (d_q + M[q,i]) - 2 sum_{q<r in Q_a} C_qr s_q(i) s_r(i),
//   M = C S,  S[r][i] = s_r(i)        (an n x n x s contraction over the pairs with a generator),
// and with W[a,i] = sin Phi (alpha_a + beta_a cos Phi), V[q,i] = sum_{a : q in Q_a} W[a,i]:
//   grad(gate e_q)       = 2 sum_i s_q(i) V[q,i],
//   grad(gate e_q + e_r) = 2 (H[q,r] + H[r,q]) - 4 K[q,r],
//   H[q,r] = sum_i s_q(i) V[q,i] s_r(i)   (needed only for the pairs with a generator),
//   K[q,r] = sum_{a : q, r in Q_a} sum_i W[a,i] s_q(i) s_r(i).
// The work is O(p s + l |Q_a|^2 s), p = number of qubit pairs carrying a
// generator, instead of nnz(P_A) s, and nnz(P_A) is about l |Q_a| n for all
// one- and two-body gates. FP32 arithmetic, FP64
// reductions over samples; C, d and K accumulated in 64-bit fixed point
// (integer atomics, so repeated supports and the gradient are bitwise
// reproducible).
//
// Device-side errors: a generator of weight > 2 records IQP_ERR_ARG, an
// observable of weight > 1024 records IQP_ERR_UNSUPPORTED (in the workspace
// status word); the outputs are then not meaningful.
#include <cstdlib>

#include "common.cuh"

namespace iqp {

namespace {

constexpr int kQMax = 1024;  // observable weight limit (support list in shared memory)
constexpr int kPairMax = 512;  // pairs of Q_a held in shared memory per round
constexpr int kBlk = 256;    // samples per CTA in the per-observable kernels
constexpr int kQ4 = 256;     // supports up to this size take four sample blocks per pass in k_lo_phase
constexpr unsigned kFull = 0xFFFFFFFFu;

// Optional self-checks (-DIQP_LO_CHECKS, or the library-wide -DIQP_CHECKS):
// an index out of its buffer records status 100 + site in the workspace status
// word and the access is skipped.
#if defined(IQP_CHECKS) && !defined(IQP_LO_CHECKS)
#define IQP_LO_CHECKS
#endif
#ifdef IQP_LO_CHECKS
#define LO_OK(cond, site) ((cond) ? true : (record_status(status_dbg, 100u + (site)), false))
#else
#define LO_OK(cond, site) true
#endif

// d_q, C_qr and E (bits r of row q and q of row r set iff some generator
// acts on {q, r}) from the support list (q0 < q1 < ..., count). Repeated
// supports add their coefficients: each c_j is rounded to a multiple of
// 2^-k, the sums are formed exactly in 64-bit fixed point (integer atomics,
// so their order does not matter) and each is rounded to FP32 once, which
// keeps every result bitwise reproducible.
//
// Scale 2^k of the fixed point, from the largest |c_j| (its float bits, taken
// by an integer atomicMax) and m: m max|c_j| 2^k < 2^62, so no partial sum
// overflows; k is clamped to [-60, 100].
__device__ __forceinline__ int lo_fx_exp(unsigned cmax_bits, int64_t m) {
    const float cm = __uint_as_float(cmax_bits);
    if (!(cm > 0.f) || !(cm < INFINITY)) return 40;
    int e = 0;
    frexp((double)cm * (double)(m > 0 ? m : 1), &e);  // the bound is < 2^e
    const int k = 62 - e;
    return k < -60 ? -60 : (k > 100 ? 100 : k);
}

__global__ void k_lo_cmax(const int4 *__restrict__ sup, const float *__restrict__ c, int64_t m,
                          unsigned *__restrict__ cmax) {
    unsigned v = 0u;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int w = sup[j].w;
        if (w == 1 || w == 2) {
            const unsigned b = __float_as_uint(fabsf(c[j]));  // non-negative floats order like their bits
            v = b > v ? b : v;
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const unsigned o = __shfl_xor_sync(kFull, v, off);
        v = o > v ? o : v;
    }
    if ((threadIdx.x & 31) == 0 && v != 0u) atomicMax(cmax, v);
}

// Cfx (n x n) and dfx (n): fixed-point sums of c_j; E bits.
__global__ void k_lo_build(const int4 *__restrict__ sup, const float *__restrict__ c, int64_t m, int64_t n,
                           unsigned long long *__restrict__ Cfx, unsigned long long *__restrict__ dfx,
                           const unsigned *__restrict__ cmax, unsigned long long *__restrict__ E, int64_t lde,
                           uint32_t *__restrict__ status) {
    [[maybe_unused]] uint32_t *status_dbg = status;
    const int k = lo_fx_exp(*cmax, m);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int4 sp = sup[j];
        if (!LO_OK(sp.w <= 0 || (sp.x >= 0 && sp.x < n && (sp.w < 2 || (sp.y > sp.x && sp.y < n))), 8)) continue;
        if (sp.w == 1 || sp.w == 2) {
            const unsigned long long v = (unsigned long long)llrint(ldexp((double)c[j], k));
            if (sp.w == 1) {
                atomicAdd(dfx + sp.x, v);
            } else {
                atomicAdd(Cfx + (int64_t)sp.x * n + sp.y, v);
                atomicAdd(Cfx + (int64_t)sp.y * n + sp.x, v);
                atomicOr(E + (int64_t)sp.x * lde + (sp.y >> 6), 1ull << (sp.y & 63));
                atomicOr(E + (int64_t)sp.y * lde + (sp.x >> 6), 1ull << (sp.x & 63));
            }
        } else if (sp.w > 2) {
            record_status(status, IQP_ERR_ARG);
        }
    }
}

// C (n x ldc, zero in columns >= n) and d (n) from their fixed-point sums,
// each rounded to FP32 once.
__global__ void k_lo_fx_float(const unsigned long long *__restrict__ Cfx, const unsigned long long *__restrict__ dfx,
                              const unsigned *__restrict__ cmax, int64_t m, int64_t n, float *__restrict__ C,
                              int64_t ldc, float *__restrict__ d) {
    const float inv = ldexpf(1.0f, -lo_fx_exp(*cmax, m));
    const int64_t total = n * ldc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total + n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < total) {
            const int64_t q = i / ldc, r = i - q * ldc;
            C[i] = r < n ? __ll2float_rn((long long)Cfx[q * n + r]) * inv : 0.f;
        } else {
            d[i - total] = __ll2float_rn((long long)dfx[i - total]) * inv;
        }
    }
}

// ------------------------------------------------ pair contractions
// Both n x n x s contractions visit only the pairs that carry a generator
// (the set bits of E): one warp per (qubit q, range of 2048 samples), lane
// l owning the 64 samples of word 32 range + l of every ZT row, each term a
// sign flip and an FP32 add (as in the row-sparse form).

constexpr int kCsBatch = 8;

// fn(r) for every set bit r of E row q, in increasing r, warp-uniformly.
template <class F>
__device__ __forceinline__ void for_each_bit(const unsigned long long *__restrict__ row, int64_t nw, int lane, F &fn) {
    for (int64_t w0 = 0; w0 < nw; w0 += 32) {
        const uint64_t bits = w0 + lane < nw ? row[w0 + lane] : 0ull;
        uint32_t live = __ballot_sync(kFull, bits != 0ull);
        while (live) {
            const int src = __ffs(live) - 1;
            live &= live - 1u;
            uint64_t wb = __shfl_sync(kFull, bits, src);
            const int64_t rb = (w0 + src) * 64;
            while (wb) {
                const int b = __ffsll((long long)wb) - 1;
                wb &= wb - 1ull;
                fn(rb + b);
            }
        }
    }
}

// M[q][i] = sum_{r in E_q} C_qr s_r(i) (M = C S restricted to the pairs with
// a generator, which is all of C's nonzeros). Grid (n, ranges) x 32 threads.
__global__ void __launch_bounds__(32) k_lo_cs(const unsigned long long *__restrict__ E, int64_t lde,
                                              const float *__restrict__ C, int64_t ldc,
                                              const uint64_t *__restrict__ ZT, int64_t ldzt, int64_t s,
                                              float *__restrict__ M, int64_t lds) {
    const int lane = threadIdx.x;
    const int64_t q = blockIdx.x, r0 = blockIdx.y;
    const int64_t vwords = cdiv(s, 64);
    const int64_t wraw = r0 * 32 + lane;
    const int64_t word = wraw < vwords ? wraw : vwords - 1;  // in-bounds load, result unused
    float acc[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) acc[k] = 0.f;
    const float *crow = C + q * ldc;
    auto add = [&](uint64_t z, uint32_t cb) {
        const uint32_t lo = (uint32_t)z, hi = (uint32_t)(z >> 32);
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] += __uint_as_float(cb ^ ((lo << (31 - k)) & 0x80000000u));
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[32 + k] += __uint_as_float(cb ^ ((hi << (31 - k)) & 0x80000000u));
    };
    // Pairs are consumed in batches of kCsBatch: the batch's loads are all
    // issued before the first is used (only indices are held while a batch
    // fills), so their latencies overlap.
    int64_t rb[kCsBatch];
    int nb = 0;
#pragma unroll
    for (int t = 0; t < kCsBatch; ++t) rb[t] = 0;
    auto visit = [&](int64_t r) {
#pragma unroll
        for (int t = 0; t + 1 < kCsBatch; ++t) rb[t] = rb[t + 1];
        rb[kCsBatch - 1] = r;
        if (++nb == kCsBatch) {
            uint64_t z[kCsBatch];
            uint32_t cb[kCsBatch];
#pragma unroll
            for (int t = 0; t < kCsBatch; ++t) {
                z[t] = __ldg(ZT + rb[t] * ldzt + word);
                cb[t] = __float_as_uint(__ldg(crow + rb[t]));
            }
#pragma unroll
            for (int t = 0; t < kCsBatch; ++t) add(z[t], cb[t]);
            nb = 0;
        }
    };
    for_each_bit(E + q * lde, lde, lane, visit);
#pragma unroll
    for (int t = 0; t < kCsBatch; ++t)
        if (t >= kCsBatch - nb) add(__ldg(ZT + rb[t] * ldzt + word), __float_as_uint(__ldg(crow + rb[t])));
    if (wraw < vwords) {
        float *mrow = M + q * lds + wraw * 64;  // lds is a multiple of 64
#pragma unroll
        for (int k = 0; k < 64; k += 4) *reinterpret_cast<float4 *>(mrow + k) = make_float4(acc[k], acc[k + 1], acc[k + 2], acc[k + 3]);
    }
}

// H[q][r] = sum_i s_q(i) V[q][i] s_r(i) for r in E_q. Warp (q, k) takes
// every kHSplit-th set bit of E_q starting at the k-th (listed in shared
// memory, kRMax at a time) and walks the sample ranges in order, so each
// H[q][r] is accumulated by one warp alone (fixed order, FP32 per range,
// FP64 across ranges).
constexpr int kHSplit = 8;
constexpr int kRMax = 1024;
constexpr int kHPre = 4;

__global__ void __launch_bounds__(32) k_lo_h(const unsigned long long *__restrict__ E, int64_t lde,
                                             const uint64_t *__restrict__ ZT, int64_t ldzt,
                                             const float *__restrict__ V, int64_t lds, int64_t s,
                                             double *__restrict__ Hd, int64_t ldh) {
    __shared__ int rl[kRMax];
    const int lane = threadIdx.x;
    const int64_t q = blockIdx.x;
    const int split = blockIdx.y;
    const int64_t vwords = cdiv(s, 64);
    const int64_t nranges = cdiv(vwords, 32);
    double *hrow = Hd + q * ldh;
    const unsigned long long *erow = E + q * lde;
    int seen = 0;        // set bits of E_q visited so far
    int64_t w0 = 0;      // next E word to scan
    while (w0 < lde) {
        // list this warp's next pairs
        int nr = 0;
        while (w0 < lde && nr <= kRMax - 64) {
            const uint64_t bits0 = erow[w0];
            uint64_t bits = bits0;
            // bit b of the word is this warp's when (seen + rank of b) % kHSplit == split
            const int rank_start = seen;
            const int cnt = __popcll(bits0);
            if (lane == 0) {
                int rk = rank_start;
                while (bits) {
                    const int b = __ffsll((long long)bits) - 1;
                    bits &= bits - 1ull;
                    if (rk % kHSplit == split) rl[nr++] = (int)(64 * w0 + b);
                    ++rk;
                }
            }
            nr = __shfl_sync(kFull, nr, 0);
            seen += cnt;
            ++w0;
        }
        __syncwarp();
        for (int64_t r0 = 0; r0 < nranges; ++r0) {
            const int64_t wraw = r0 * 32 + lane;
            const bool wvalid = wraw < vwords;
            const int64_t word = wvalid ? wraw : vwords - 1;
            float u[64];
            const uint64_t zq = __ldg(ZT + q * ldzt + word);
            const float *vrow = V + q * lds + word * 64;
#pragma unroll
            for (int k = 0; k < 64; k += 4) {
                const float4 v4 = wvalid ? *reinterpret_cast<const float4 *>(vrow + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                u[k] = v4.x;
                u[k + 1] = v4.y;
                u[k + 2] = v4.z;
                u[k + 3] = v4.w;
            }
#pragma unroll
            for (int k = 0; k < 64; ++k) u[k] = ((zq >> k) & 1ull) ? -u[k] : u[k];
            // loads of the next kHPre pairs are issued ahead of their use
            uint64_t zn[kHPre];
#pragma unroll
            for (int t = 0; t < kHPre; ++t) zn[t] = t < nr ? __ldg(ZT + (int64_t)rl[t] * ldzt + word) : 0ull;
            for (int e0 = 0; e0 < nr; e0 += kHPre) {
                uint64_t zc[kHPre];
#pragma unroll
                for (int t = 0; t < kHPre; ++t) {
                    zc[t] = zn[t];
                    const int en = e0 + kHPre + t;
                    zn[t] = en < nr ? __ldg(ZT + (int64_t)rl[en] * ldzt + word) : 0ull;
                }
#pragma unroll
                for (int t = 0; t < kHPre; ++t) {
                const int e = e0 + t;
                if (e >= nr) break;
                const int64_t r = rl[e];
                const uint64_t z = zc[t];
                const uint32_t lo = (uint32_t)z, hi = (uint32_t)(z >> 32);
                float p[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    p[k & 7] += __uint_as_float(__float_as_uint(u[k]) ^ ((lo << (31 - k)) & 0x80000000u));
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    p[k & 7] += __uint_as_float(__float_as_uint(u[32 + k]) ^ ((hi << (31 - k)) & 0x80000000u));
                float dsum = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) dsum += __shfl_xor_sync(kFull, dsum, off);
                if (lane == 0) hrow[r] = r0 == 0 ? (double)dsum : hrow[r] + (double)dsum;
                }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------- the contractions on the tensor cores
// With the tensor cores both contractions are dense GEMMs with one +-1
// operand from bits, M = C S (K = the n qubits r) and H = (s o V) S^T
// (K = the s samples), like the phase contraction; the FP32 operand goes in
// as a hi + lo BF16 split. k_lo_split writes that split: element (q, k) of
// a rows x cols FP32 matrix, multiplied by s_q(k) = (-1)^(bit k of zt row q)
// when zt is given, into rows x kpad BF16 matrices (zero for k >= cols).
// One thread per 8 consecutive elements.
__global__ void k_lo_split(const float *__restrict__ in, int64_t ld_in, int64_t rows, int64_t cols,
                           const uint64_t *__restrict__ zt, int64_t ldzt, int64_t kpad, __nv_bfloat16 *__restrict__ hi,
                           __nv_bfloat16 *__restrict__ lo) {
    const int64_t per_row = kpad / 8, total = rows * per_row;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / per_row, k0 = (e - q * per_row) * 8;
        const uint32_t sb = zt ? (uint32_t)(zt[q * ldzt + (k0 >> 6)] >> (k0 & 63)) & 0xFFu : 0u;
        uint32_t ph[4], pl[4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            float x0 = k0 + t < cols ? in[q * ld_in + k0 + t] : 0.f;
            float x1 = k0 + t + 1 < cols ? in[q * ld_in + k0 + t + 1] : 0.f;
            if ((sb >> t) & 1u) x0 = -x0;
            if ((sb >> (t + 1)) & 1u) x1 = -x1;
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
            ph[t / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            pl[t / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        *reinterpret_cast<uint4 *>(hi + q * kpad + k0) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
        *reinterpret_cast<uint4 *>(lo + q * kpad + k0) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
    }
}

// Exclusive prefix sum of v over the CTA (every thread calls it); *total
// receives the sum.
__device__ int block_scan(int v, int *scan, int *total) {
    const int tid = threadIdx.x;
    scan[tid] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // inclusive (Hillis-Steele)
        const int u = tid >= off ? scan[tid - off] : 0;
        __syncthreads();
        scan[tid] += u;
        __syncthreads();
    }
    const int incl = scan[tid];
    *total = scan[blockDim.x - 1];
    __syncthreads();
    return incl - v;
}

// The support of observable a in increasing qubit order into Q (shared);
// returns |Q_a| capped at kQMax (recording IQP_ERR_UNSUPPORTED beyond it).
// Every thread of the CTA calls it.
__device__ int support_of_row(const uint64_t *__restrict__ arow, int64_t n, int *Q, int *scan,
                              uint32_t *__restrict__ status) {
    [[maybe_unused]] uint32_t *status_dbg = status;
    const int tid = threadIdx.x;
    const int64_t nw = (n + 63) >> 6;
    int total = 0;
    for (int64_t base = 0; base < nw; base += blockDim.x) {
        uint64_t w = base + tid < nw ? arow[base + tid] : 0ull;
        if (base + tid == nw - 1 && (n & 63)) w &= (1ull << (n & 63)) - 1ull;  // never a qubit >= n
        int sum = 0;
        int pos = total + block_scan(__popcll(w), scan, &sum);
        while (w) {
            const int b = __ffsll((long long)w) - 1;
            w &= w - 1ull;
            if (pos < kQMax && LO_OK(64 * (base + tid) + b < n, 1)) Q[pos] = (int)(64 * (base + tid) + b);
            ++pos;
        }
        total += sum;
    }
    __syncthreads();  // Q is complete before anyone reads it
    if (total > kQMax) {
        if (tid == 0) record_status(status, IQP_ERR_UNSUPPORTED);
        total = kQMax;
    }
    return total;
}

// Shared state of the per-(observable, 256-sample block) kernels.
struct LoShared {
    int Q[kQMax];              // support of the observable
    union alignas(16) {
        uint32_t bits[kQMax][8];    // one 256-sample block: bit (i - i0) of word i/32 for qubit Q[t]
        uint32_t bits4[kQ4][32];    // four blocks at once, for supports of at most kQ4 qubits
    };
    int pr[kPairMax];          // pairs t | u << 16 (t < u) with a generator on {Q[t], Q[u]}
    float pc[kPairMax];        // C restricted to those pairs
    int scan[kBlk];
    int wsum[kBlk / 32];
    float redf[kBlk / 32];
};

// Sample blocks handled by one CTA: the support and, when it fits, the
// pair list are built once and reused for every block.
constexpr int kGroup = 8;    // sample blocks per CTA of k_lo_v (its per-block sums live in registers)
constexpr int kPGroup = 16;  // sample blocks per CTA of k_lo_phase and k_lo_pairs (support and pair list built once)
constexpr int kObsMax = 4096;  // observables of one qubit listed per pass in k_lo_v

// The sample bits of block blk for every support qubit.
__device__ void lo_load_bits(LoShared &sh, int nq, int64_t n, const uint64_t *__restrict__ ZT, int64_t ldzt,
                             int64_t blk, [[maybe_unused]] uint32_t *__restrict__ status_dbg) {
    __syncthreads();  // previous readers of bits are done
    for (int e = threadIdx.x; e < nq * 4; e += kBlk) {
        const int t = e >> 2, k = e & 3;
        const int64_t w = blk * 4 + k;
        const bool okq = LO_OK(t < kQMax && sh.Q[t] >= 0 && sh.Q[t] < n, 2);
        const uint64_t z = (w < ldzt && okq) ? ZT[(int64_t)sh.Q[t] * ldzt + w] : 0ull;
        sh.bits[t][2 * k] = (uint32_t)z;
        sh.bits[t][2 * k + 1] = (uint32_t)(z >> 32);
    }
    __syncthreads();
}

// Appends to the pair list, in (t, u) order, the pairs with a generator
// among the candidates c = t nq + u from *c0 on, 256 per round (compacted
// with warp ballots), until the list holds more than kPairMax - kBlk
// entries or the candidates run out. Returns the list length; every thread
// calls it and gets the same value.
__device__ int lo_fill_pairs(LoShared &sh, int nq, int64_t *c0, const unsigned long long *__restrict__ E,
                             int64_t lde, const float *__restrict__ C, int64_t ldc, int64_t n,
                             [[maybe_unused]] uint32_t *__restrict__ status_dbg) {
    (void)n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ncand = (int64_t)nq * nq;
    int np = 0;
    while (*c0 < ncand && np <= kPairMax - kBlk) {
        const int64_t c = *c0 + threadIdx.x;
        int t = 0, u = 0;
        bool ok = false;
        if (c < ncand) {
            t = (int)(c / nq);
            u = (int)(c - (int64_t)t * nq);
            if (u > t && LO_OK(t < nq && u < nq, 3)) {
                const int q = sh.Q[t], r = sh.Q[u];
                if (LO_OK(q >= 0 && q < n && r >= 0 && r < n, 4)) ok = (E[(int64_t)q * lde + (r >> 6)] >> (r & 63)) & 1ull;
            }
        }
        const uint32_t bal = __ballot_sync(kFull, ok);
        if (lane == 0) sh.wsum[warp] = __popc(bal);
        __syncthreads();
        int off = np, tot = 0;
#pragma unroll
        for (int w = 0; w < kBlk / 32; ++w) {
            const int v = sh.wsum[w];
            off += w < warp ? v : 0;
            tot += v;
        }
        const int pos = off + __popc(bal & ((1u << lane) - 1u));
        if (ok && LO_OK(pos >= 0 && pos < kPairMax, 5)) {
            sh.pr[pos] = t | (u << 16);
            sh.pc[pos] = C[(int64_t)sh.Q[t] * ldc + sh.Q[u]];
        }
        np += tot;
        *c0 += kBlk;
        __syncthreads();
    }
    return np;
}

// v with its sign flipped when bit 31 of y is set.
__device__ __forceinline__ float flip_if(float v, uint32_t y) {
    return __int_as_float(__float_as_int(v) ^ (int)(y & 0x80000000u));
}

// Sum of v over the CTA in FP32 (warp shuffles, then the warps' sums in
// fixed order); every thread gets it. The partial sums of one 256-sample
// block are kept in FP32 and combined across blocks in FP64, as in the
// tensor-core epilogue (FP64 arithmetic runs at 1/64 of the FP32 rate here).
__device__ __forceinline__ float block_sum_f(float v, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kBlk / 32; ++w) t += red[w];
    return t;
}

// The sample bits of blocks blk0 .. blk0 + 3 for every support qubit:
// bits4[t][w] holds samples 32 w .. 32 w + 31 of the 1024. No barriers.
__device__ __forceinline__ void lo_fill_bits4(LoShared &sh, int nq, int64_t n, const uint64_t *__restrict__ ZT,
                                              int64_t ldzt, int64_t blk0,
                                              [[maybe_unused]] uint32_t *__restrict__ status_dbg) {
    for (int e = threadIdx.x; e < nq * 16; e += kBlk) {
        const int t = e >> 4, k = e & 15;
        const int64_t w = blk0 * 4 + k;
        const bool okq = LO_OK(t < kQ4 && sh.Q[t] >= 0 && sh.Q[t] < n, 2);
        const uint64_t z = (w < ldzt && okq) ? ZT[(int64_t)sh.Q[t] * ldzt + w] : 0ull;
        sh.bits4[t][2 * k] = (uint32_t)z;
        sh.bits4[t][2 * k + 1] = (uint32_t)(z >> 32);
    }
}

// lo_fill_bits4 between barriers: previous readers of bits4 are done before
// it, every word is in place after it.
__device__ void lo_load_bits4(LoShared &sh, int nq, int64_t n, const uint64_t *__restrict__ ZT, int64_t ldzt,
                              int64_t blk0, uint32_t *__restrict__ status_dbg) {
    __syncthreads();
    lo_fill_bits4(sh, nq, n, ZT, ldzt, blk0, status_dbg);
    __syncthreads();
}

// MODE 0: (sum cos, sum (cos - mean)^2) per (observable, 256 samples) into
// part, and Phi itself into phi (row stride ldphi >= lds, columns < lds) when
// phi is not null (a gradient pass follows). MODE 1: W[a][i] = sin Phi
// (alpha_a + beta_a cos Phi), zero for i >= s.
// The pair term visits only the pairs of Q_a that carry a generator (C_qr is
// zero on the others). CTA (a, g) takes sample blocks kPGroup g ..
// kPGroup g + kPGroup - 1. For |Q_a| <= kQ4 a thread owns four consecutive
// samples of a 1024-sample pass (four blocks; block b is warps 2b, 2b + 1),
// so every support qubit costs one 16-byte load of M and every pair one
// word pair of sample bits for four samples; larger supports take one block
// per pass, one sample per thread.
template <int MODE>
__global__ void __launch_bounds__(kBlk) k_lo_phase(const uint64_t *__restrict__ A, int64_t lda, int64_t n,
                                                   const uint64_t *__restrict__ ZT, int64_t ldzt,
                                                   const float *__restrict__ M, int64_t lds,
                                                   const float *__restrict__ C, int64_t ldc,
                                                   const float *__restrict__ d, const unsigned long long *__restrict__ E,
                                                   int64_t lde, int64_t s, int64_t nparts, double2 *__restrict__ part,
                                                   const double *__restrict__ alpha, const double *__restrict__ beta,
                                                   float *__restrict__ W, float *__restrict__ phi, int64_t ldphi,
                                                   uint32_t *__restrict__ status) {
    [[maybe_unused]] uint32_t *status_dbg = status;
    __shared__ LoShared sh;
    __shared__ const float *mrow[kQ4];  // M + Q[t] lds (four-block form)
    __shared__ float dq[kQ4];           // d[Q[t]] (four-block form)
    const int64_t a = blockIdx.x;
    const int nq = support_of_row(A + a * lda, n, sh.Q, sh.scan, status);
    const int tid = threadIdx.x, w = tid >> 5, bit = tid & 31;
    const int64_t ncand = (int64_t)nq * nq;
    int64_t c0 = 0;
    int np = lo_fill_pairs(sh, nq, &c0, E, lde, C, ldc, n, status);
    const bool complete = c0 >= ncand;  // the whole list fits: reuse it for every block
    const float al = MODE == 1 ? (float)alpha[a] : 0.f;
    const float be = (MODE == 1 && beta) ? (float)beta[a] : 0.f;
    const int64_t bstart = blockIdx.y * (int64_t)kPGroup;
    const int64_t b1 = bstart + kPGroup < nparts ? bstart + kPGroup : nparts;
    if (nq <= kQ4) {
        for (int t = tid; t < nq; t += kBlk) {
            const int q = sh.Q[t];
            const bool ok = LO_OK(q >= 0 && q < n, 7);
            mrow[t] = M + (ok ? (int64_t)q * lds : 0);
            dq[t] = ok ? d[q] : 0.f;
        }
        const int word = tid >> 3;              // bits4 word of this thread's samples
        const int sh4 = 28 - 4 * (tid & 7);     // moves their four bits to bits 28 .. 31
        for (int64_t blk0 = bstart; blk0 < b1; blk0 += 4) {
            lo_load_bits4(sh, nq, n, ZT, ldzt, blk0, status);  // also orders the mrow/dq stores
            const int64_t i0 = blk0 * kBlk + 4 * (int64_t)tid;
            const int64_t blk = blk0 + (tid >> 6);  // this thread's block
            const int64_t i0c = i0 < lds ? i0 : lds - 4;  // lds is a multiple of 64
            float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
            for (int t = 0; t < nq; ++t) {
                if (!LO_OK(i0c >= 0 && i0c + 3 < lds, 8)) break;
                const float4 mv = *reinterpret_cast<const float4 *>(mrow[t] + i0c);
                const float dv = dq[t];
                const uint32_t y = sh.bits4[t][word] << sh4;
                p0 = p0 + flip_if(dv + mv.x, y << 3);
                p1 = p1 + flip_if(dv + mv.y, y << 2);
                p2 = p2 + flip_if(dv + mv.z, y << 1);
                p3 = p3 + flip_if(dv + mv.w, y);
            }
            float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
            if (!complete && blk0 != bstart) {
                c0 = 0;  // the list is rebuilt round by round for every pass
                np = lo_fill_pairs(sh, nq, &c0, E, lde, C, ldc, n, status);
            }
            while (true) {
                for (int p = 0; p < np; ++p) {
                    const int pr = sh.pr[p];
                    if (!LO_OK((pr & 0xFFFF) < nq && (pr >> 16) < nq && p < kPairMax, 6)) continue;
                    const uint32_t y = (sh.bits4[pr & 0xFFFF][word] ^ sh.bits4[pr >> 16][word]) << sh4;
                    const float cv = sh.pc[p];
                    q0 = q0 + flip_if(cv, y << 3);
                    q1 = q1 + flip_if(cv, y << 2);
                    q2 = q2 + flip_if(cv, y << 1);
                    q3 = q3 + flip_if(cv, y);
                }
                if (complete || c0 >= ncand) break;
                __syncthreads();
                np = lo_fill_pairs(sh, nq, &c0, E, lde, C, ldc, n, status);
            }
            const float ph[4] = {p0 - 2.f * q0, p1 - 2.f * q1, p2 - 2.f * q2, p3 - 2.f * q3};
            bool valid[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) valid[k] = i0 + k < s && blk < b1;
            if (MODE == 0) {
                float cv[4], S1 = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    cv[k] = valid[k] ? cosf(ph[k]) : 0.f;
                    S1 += cv[k];
                }
                // Block b's sums: its two warps' shuffle sums, in warp order.
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) S1 += __shfl_xor_sync(kFull, S1, off);
                __syncthreads();
                if (bit == 0) sh.redf[w] = S1;
                __syncthreads();
                const float S = sh.redf[w & ~1] + sh.redf[w | 1];
                const int64_t nb = s - blk * kBlk < kBlk ? s - blk * kBlk : kBlk;
                const float mean = nb > 0 ? S / (float)nb : 0.f;
                float M2 = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float dv = cv[k] - mean;
                    M2 += valid[k] ? dv * dv : 0.f;
                }
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) M2 += __shfl_xor_sync(kFull, M2, off);
                __syncthreads();
                if (bit == 0) sh.redf[w] = M2;
                __syncthreads();
                if ((tid & 63) == 0 && blk < b1)
                    part[a * nparts + blk] = make_double2((double)S, (double)(sh.redf[w] + sh.redf[w + 1]));
                if (phi != nullptr && i0 < lds && blk < b1)
                    *reinterpret_cast<float4 *>(phi + a * ldphi + i0) = make_float4(ph[0], ph[1], ph[2], ph[3]);
            } else if (i0 < lds && blk < b1) {
                float o[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float sn, cn;
                    sincosf(ph[k], &sn, &cn);
                    o[k] = valid[k] ? sn * (al + be * cn) : 0.f;
                }
                *reinterpret_cast<float4 *>(W + a * lds + i0) = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
        return;
    }
    for (int64_t blk = bstart; blk < b1; ++blk) {
        lo_load_bits(sh, nq, n, ZT, ldzt, blk, status);
        const int64_t i = blk * kBlk + tid;
        const bool valid = i < s;
        const int64_t ic = valid ? i : s - 1;
        float ph = 0.f;
        for (int t = 0; t < nq; ++t) {
            const int q = sh.Q[t];
            if (!LO_OK(q >= 0 && q < n && ic >= 0 && ic < lds, 7)) continue;
            const float v = d[q] + M[(int64_t)q * lds + ic];
            ph += ((sh.bits[t][w] >> bit) & 1u) ? -v : v;
        }
        float pairs = 0.f;
        if (!complete && blk != bstart) {
            c0 = 0;  // the list is rebuilt round by round for every block
            np = lo_fill_pairs(sh, nq, &c0, E, lde, C, ldc, n, status);
        }
        while (true) {
            for (int p = 0; p < np; ++p) {
                const int pr = sh.pr[p];
                if (!LO_OK((pr & 0xFFFF) < nq && (pr >> 16) < nq && p < kPairMax, 6)) continue;
                const uint32_t x = sh.bits[pr & 0xFFFF][w] ^ sh.bits[pr >> 16][w];
                const float cv = sh.pc[p];
                pairs += ((x >> bit) & 1u) ? -cv : cv;
            }
            if (complete || c0 >= ncand) break;
            __syncthreads();
            np = lo_fill_pairs(sh, nq, &c0, E, lde, C, ldc, n, status);
        }
        ph -= 2.f * pairs;
        if (MODE == 0) {
            const float cv = valid ? cosf(ph) : 0.f;
            const float S = block_sum_f(cv, sh.redf);
            const int64_t nb = s - blk * kBlk < kBlk ? s - blk * kBlk : kBlk;
            const float mean = S / (float)nb;
            const float dv = cv - mean;
            const float M2 = block_sum_f(valid ? dv * dv : 0.f, sh.redf);
            if (tid == 0) part[a * nparts + blk] = make_double2((double)S, (double)M2);
            if (phi != nullptr && i < lds) phi[a * ldphi + i] = ph;
        } else {
            float sn, cn;
            sincosf(ph, &sn, &cn);
            if (i < lds) W[a * lds + i] = valid ? sn * (al + be * cn) : 0.f;
        }
    }
}

// V[q][i] = sum over the observables a containing q of W[a][i] (in a order),
// zero for i >= s; gsp[q * nblk + blk] = sum_i s_q(i) V[q][i] over the
// CTA's 256 samples (FP64). A thread owns four consecutive samples of each
// 1024-sample pass (block b of the pass is warps 2b, 2b + 1), so every
// observable costs one 16-byte load of W per thread and pass.
__global__ void __launch_bounds__(kBlk) k_lo_v(const uint64_t *__restrict__ AT, int64_t ldlt,
                                               const uint64_t *__restrict__ ZT, int64_t ldzt,
                                               const float *__restrict__ W, int64_t lds, int64_t s, int64_t nblk,
                                               float *__restrict__ V, double *__restrict__ gsp) {
    __shared__ float red[kBlk / 32];
    __shared__ int obs[kObsMax];
    __shared__ int wsum[kBlk / 32];
    constexpr int kPass = kGroup / 4;  // 1024-sample passes per CTA
    const int64_t q = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t *row = AT + q * ldlt;
    const int64_t b0 = blockIdx.y * (int64_t)kGroup;
    const int64_t b1 = b0 + kGroup < nblk ? b0 + kGroup : nblk;
    float4 v[kPass];
#pragma unroll
    for (int g = 0; g < kPass; ++g) v[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    // The observables containing q, kObsMax at a time, in increasing order
    // (each thread compacts one 64-observable word; warps in order).
    for (int64_t w0 = 0; w0 < ldlt; w0 += kObsMax / 64) {
        int no = 0;
        for (int64_t wb = w0; wb < w0 + kObsMax / 64 && wb < ldlt; wb += kBlk) {
            const int64_t wi = wb + threadIdx.x;
            uint64_t bits = (wi < w0 + kObsMax / 64 && wi < ldlt) ? row[wi] : 0ull;
            const int cnt = __popcll(bits);
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int u = __shfl_up_sync(kFull, incl, off);
                if (lane >= off) incl += u;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            int off = no, tot = 0;
#pragma unroll
            for (int k = 0; k < kBlk / 32; ++k) {
                off += k < warp ? wsum[k] : 0;
                tot += wsum[k];
            }
            int pos = off + incl - cnt;
            while (bits) {
                const int b = __ffsll((long long)bits) - 1;
                bits &= bits - 1ull;
                obs[pos++] = (int)(64 * wi + b);
            }
            no += tot;
            __syncthreads();
        }
#pragma unroll
        for (int g = 0; g < kPass; ++g) {
            if (b0 + 4 * g < b1) {  // uniform
                const int64_t i0 = (b0 + 4 * g) * kBlk + 4 * (int64_t)threadIdx.x;
                const int64_t i0c = i0 < lds ? i0 : lds - 4;  // lds is a multiple of 64
                float4 acc = v[g];
                for (int k = 0; k < no; ++k) {
                    const float4 x = *reinterpret_cast<const float4 *>(W + (int64_t)obs[k] * lds + i0c);
                    acc.x += x.x;
                    acc.y += x.y;
                    acc.z += x.z;
                    acc.w += x.w;
                }
                v[g] = acc;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int g = 0; g < kPass; ++g) {
        if (b0 + 4 * g >= b1) continue;  // uniform
        const int64_t i0 = (b0 + 4 * g) * kBlk + 4 * (int64_t)threadIdx.x;
        const int64_t blk = b0 + 4 * g + (threadIdx.x >> 6);
        const bool in = blk < b1 && i0 < lds;
        const float vv[4] = {in && i0 < s ? v[g].x : 0.f, in && i0 + 1 < s ? v[g].y : 0.f,
                             in && i0 + 2 < s ? v[g].z : 0.f, in && i0 + 3 < s ? v[g].w : 0.f};
        if (in) *reinterpret_cast<float4 *>(V + q * lds + i0) = make_float4(vv[0], vv[1], vv[2], vv[3]);
        // lds <= 64 ldzt, so the word of i0 is inside row q of ZT when i0 < lds.
        const uint32_t nib = in ? (uint32_t)(ZT[q * ldzt + (i0 >> 6)] >> (i0 & 63)) : 0u;
        float u = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) u += ((nib >> k) & 1u) ? -vv[k] : vv[k];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) u += __shfl_xor_sync(kFull, u, off);
        __syncthreads();
        if (lane == 0) red[warp] = u;
        __syncthreads();
        if ((threadIdx.x & 63) == 0 && blk < b1) gsp[q * nblk + blk] = (double)(red[warp] + red[warp + 1]);
    }
}

// W[a][i] = sin Phi (alpha_a + beta_a cos Phi) (zero for i >= s) from the
// Phi the statistics pass kept (l x ldphi; phi may be W itself: each
// element is read before it is written, by the same thread), four samples
// per thread: the arithmetic of k_lo_phase<1>, without recomputing Phi.
__global__ void __launch_bounds__(256) k_lo_w(const float *phi, int64_t ldphi, float *W, int64_t lds, int64_t l,
                                             int64_t s, const double *__restrict__ alpha,
                                             const double *__restrict__ beta) {
    const int64_t per_row = lds / 4;
    const int64_t total = l * per_row;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = g / per_row, i0 = (g - a * per_row) * 4;
        const float al = (float)alpha[a];
        const float be = beta ? (float)beta[a] : 0.f;
        const float4 f = *reinterpret_cast<const float4 *>(phi + a * ldphi + i0);
        const float v[4] = {f.x, f.y, f.z, f.w};
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float sn, cn;
            sincosf(v[k], &sn, &cn);
            o[k] = i0 + k < s ? sn * (al + be * cn) : 0.f;
        }
        *reinterpret_cast<float4 *>(W + a * lds + i0) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

__device__ __forceinline__ long long to_fixed(float x, float sc) {
    const float xs = sc * x;  // |xs| < 2^60, exact power-of-two scaling
    const float hi = truncf(xs * 0x1.0p-31f);
    const float lo = fmaf(-hi, 0x1.0p31f, xs);
    return ((long long)__float2int_rz(hi) << 31) + (long long)__float2int_rn(lo);
}

// K[q][r] += sum over the samples of W[a][i] s_q(i) s_r(i) for the pairs
// q < r of Q_a that carry a generator (the only K entries the gradient
// reads). The pair list is taken kPairPass pairs at a time; warp w owns
// pairs w, w + 8, ... of the pass, each lane eight samples of every block,
// with a running sum per (pair, lane) in registers over the CTA's blocks,
// then one shuffle reduction and one fixed-point atomic per (pair, CTA).
// For supports of at most kQ4 qubits the sample bits and W of four blocks
// are staged per pair of barriers (one block at a time otherwise).
// CTA (a, g) takes blocks kPGroup g ...
constexpr int kPairPass = 128;
__global__ void __launch_bounds__(kBlk) k_lo_pairs(const uint64_t *__restrict__ A, int64_t lda, int64_t n,
                                                   const uint64_t *__restrict__ ZT, int64_t ldzt,
                                                   const float *__restrict__ C, int64_t ldc,
                                                   const unsigned long long *__restrict__ E, int64_t lde,
                                                   const float *__restrict__ W, int64_t lds, int64_t s,
                                                   int64_t nblk, const double *__restrict__ scale,
                                                   unsigned long long *__restrict__ Kfx,
                                                   uint32_t *__restrict__ status) {
    [[maybe_unused]] uint32_t *status_dbg = status;
    __shared__ LoShared sh;
    __shared__ __align__(16) float wb[4 * kBlk];
    constexpr int kPerWarp = kPairPass / (kBlk / 32);
    const int64_t a = blockIdx.x;
    const int nq = support_of_row(A + a * lda, n, sh.Q, sh.scan, status);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sa = 31 - lane;  // moves this lane's sample bit to bit 31
    const float sc = (float)*scale;
    const int64_t ncand = (int64_t)nq * nq;
    const int64_t b0 = blockIdx.y * (int64_t)kPGroup;
    const int64_t b1 = b0 + kPGroup < nblk ? b0 + kPGroup : nblk;
    int64_t c0 = 0;
    while (c0 < ncand) {
        const int np = lo_fill_pairs(sh, nq, &c0, E, lde, C, ldc, n, status);
        for (int p0 = 0; p0 < np; p0 += kPairPass) {
            float acc[kPerWarp];
#pragma unroll
            for (int j = 0; j < kPerWarp; ++j) acc[j] = 0.f;
            // One block's sample-bit rows (8 words per support qubit, at
            // word stride ws of the shared rows) against the lane's 8 W values.
            auto block_pairs = [&](const uint32_t *rows, int ws, const float (&wv)[8]) {
#pragma unroll
                for (int j = 0; j < kPerWarp; ++j) {
                    const int p = p0 + warp + (kBlk / 32) * j;
                    if (p < np) {  // uniform in the warp
                        const int pr = sh.pr[p];
                        const int t = pr & 0xFFFF, u = pr >> 16;
                        if (!LO_OK(t < nq && u < nq && t < kQMax && u < kQMax && p < kPairMax, 9)) continue;
                        const uint4 t0 = *reinterpret_cast<const uint4 *>(rows + t * ws);
                        const uint4 t1 = *reinterpret_cast<const uint4 *>(rows + t * ws + 4);
                        const uint4 u0 = *reinterpret_cast<const uint4 *>(rows + u * ws);
                        const uint4 u1 = *reinterpret_cast<const uint4 *>(rows + u * ws + 4);
                        float v = acc[j];
                        v += flip_if(wv[0], (t0.x ^ u0.x) << sa);
                        v += flip_if(wv[1], (t0.y ^ u0.y) << sa);
                        v += flip_if(wv[2], (t0.z ^ u0.z) << sa);
                        v += flip_if(wv[3], (t0.w ^ u0.w) << sa);
                        v += flip_if(wv[4], (t1.x ^ u1.x) << sa);
                        v += flip_if(wv[5], (t1.y ^ u1.y) << sa);
                        v += flip_if(wv[6], (t1.z ^ u1.z) << sa);
                        v += flip_if(wv[7], (t1.w ^ u1.w) << sa);
                        acc[j] = v;
                    }
                }
            };
            if (nq <= kQ4) {
                for (int64_t blk0 = b0; blk0 < b1; blk0 += 4) {
                    __syncthreads();  // previous readers of bits4 and wb are done
                    lo_fill_bits4(sh, nq, n, ZT, ldzt, blk0, status);
                    {
                        const int64_t i0 = blk0 * kBlk + 4 * (int64_t)threadIdx.x;
                        const bool in = blk0 + (threadIdx.x >> 6) < b1 && i0 < lds;  // lds: a multiple of 64
                        float4 w4 = in ? *reinterpret_cast<const float4 *>(W + a * lds + i0)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                        if (i0 >= s) w4.x = 0.f;
                        if (i0 + 1 >= s) w4.y = 0.f;
                        if (i0 + 2 >= s) w4.z = 0.f;
                        if (i0 + 3 >= s) w4.w = 0.f;
                        *reinterpret_cast<float4 *>(&wb[4 * threadIdx.x]) = w4;
                    }
                    __syncthreads();
                    for (int b = 0; b < 4 && blk0 + b < b1; ++b) {  // uniform
                        float wv[8];
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) wv[kk] = wb[kBlk * b + 32 * kk + lane];
                        block_pairs(&sh.bits4[0][8 * b], 32, wv);
                    }
                }
            } else {
                for (int64_t blk = b0; blk < b1; ++blk) {
                    lo_load_bits(sh, nq, n, ZT, ldzt, blk, status);
                    const int64_t i = blk * kBlk + threadIdx.x;
                    wb[threadIdx.x] = i < s ? W[a * lds + i] : 0.f;
                    __syncthreads();
                    float wv[8];
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) wv[kk] = wb[32 * kk + lane];
                    block_pairs(&sh.bits[0][0], 8, wv);
                }
            }
#pragma unroll
            for (int j = 0; j < kPerWarp; ++j) {
                const int p = p0 + warp + (kBlk / 32) * j;
                if (p < np) {  // uniform in the warp
                    float v = acc[j];
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
                    const int pr = sh.pr[p];
                    if (lane == 0)
                        atomicAdd(Kfx + (int64_t)sh.Q[pr & 0xFFFF] * n + sh.Q[pr >> 16],
                                  (unsigned long long)to_fixed(v, sc));
                }
            }
        }
        __syncthreads();  // the list is read before the next round rebuilds it
    }
}

// grad_j from the parts above (see the header).
__global__ void k_lo_grad_out(const int4 *__restrict__ sup, int64_t m, int64_t n, const double *__restrict__ gsp,
                              int64_t nblk, const double *__restrict__ H, int64_t ldh,
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
            const double h = H[q * ldh + r] + H[r * ldh + q];
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

// The pair contractions on the tensor cores (split BF16) unless IQP_LO_TC=0.
bool lo_tensor() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("IQP_LO_TC");
        v = (e != nullptr && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Elements of the split-BF16 operand buffer (hi and lo) the tensor-core
// contractions need: the larger of C's (n x round_up(n, 64)) and s o V's
// (n x lds), twice.
int64_t lo_split_elems(int64_t n, int64_t lds) {
    const int64_t kc = round_up(n, 64);
    return 2 * n * (kc > lds ? kc : lds);
}

namespace {
cudaError_t launch_split(const float *in, int64_t ld_in, int64_t rows, int64_t cols, const uint64_t *zt,
                         int64_t ldzt, int64_t kpad, __nv_bfloat16 *hi, __nv_bfloat16 *lo, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_LOWORDER, st);
    k_lo_split<<<grid_1d(rows * (kpad / 8)), 256, 0, st>>>(in, ld_in, rows, cols, zt, ldzt, kpad, hi, lo);
    return cudaGetLastError();
}
}  // namespace

// C, d and M = C S. C: n x ldc fp32 (+ d: ldc fp32 after it), M: n x lds,
// ZT: n x ldzt words (the samples transposed), sup: m int4.
int64_t lo_lde(int64_t n) { return cdiv(n, 64); }

// C, d, E and M = C S. C: n x ldc fp32 (+ d: ldc fp32 after it), E: n x
// lo_lde(n) words right after d, M: n x lds, ZT: n x ldzt words (the samples
// transposed), sup: m int4.
cudaError_t launch_lo_prepare(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *Z, int64_t s,
                              int64_t ldz, const float *c, int4 *sup, uint64_t *ZT, int64_t ldzt, float *C,
                              int64_t ldc, float *M, int64_t lds, __nv_bfloat16 *split, unsigned long long *fx,
                              uint32_t *status, cudaStream_t st) {
    cudaError_t e = launch_support_list(G, m, ldg, n, sup, st);
    if (e != cudaSuccess) return e;
    if ((e = launch_bit_transpose_batched(Z, 1, s, n, ldz, ZT, ldzt, st)) != cudaSuccess) return e;
    float *d = C + n * ldc;
    unsigned long long *E = reinterpret_cast<unsigned long long *>(d + ldc);
    const int64_t lde = lo_lde(n);
    // fx: Cfx (n x n), dfx (n), then the largest |c_j| (float bits).
    unsigned long long *Cfx = fx, *dfx = fx + n * n;
    unsigned *cmax = reinterpret_cast<unsigned *>(dfx + n);
    if ((e = cudaMemsetAsync(E, 0, (size_t)n * lde * 8, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(fx, 0, (size_t)(n * n + n) * 8 + 16, st)) != cudaSuccess) return e;
    {
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_cmax<<<grid_1d(m), 256, 0, st>>>(sup, c, m, cmax);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_lo_build<<<grid_1d(m), 256, 0, st>>>(sup, c, m, n, Cfx, dfx, cmax, E, lde, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_lo_fx_float<<<grid_1d(n * ldc + n), 256, 0, st>>>(Cfx, dfx, cmax, m, n, C, ldc, d);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // M = C S: rows q, columns the samples (Z's rows), K the qubits r.
    const int64_t kc = round_up(n, 64);
    bool done = false;
    if (lo_tensor() && split != nullptr && ldz >= 4 && ldz % 2 == 0 && (reinterpret_cast<uintptr_t>(Z) & 15) == 0) {
        __nv_bfloat16 *hi = split, *lo = split + n * kc;
        if ((e = launch_split(C, ldc, n, n, nullptr, 0, kc, hi, lo, st)) != cudaSuccess) return e;
        e = launch_tc_dense(hi, lo, n, kc, n, Z, s, ldz, M, lds, false, status, st);
        if (e != cudaSuccess && e != cudaErrorNotSupported) return e;
        done = e == cudaSuccess;
    }
    if (!done) {
        LaunchScope ls(IQP_KERNEL_LOWORDER_GEMM, st);
        k_lo_cs<<<dim3((unsigned)n, (unsigned)cdiv(s, 2048)), 32, 0, st>>>(E, lde, C, ldc, ZT, ldzt, s, M, lds);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_lo_stats(const uint64_t *A, int64_t lda, int64_t n, int64_t l, const uint64_t *ZT, int64_t ldzt,
                            const float *M, int64_t lds, const float *C, int64_t ldc, int64_t s, double2 *part,
                            int64_t nparts, float *phi, int64_t ldphi, uint32_t *status, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_LOWORDER, st);
    const float *d = C + n * ldc;
    const unsigned long long *E = reinterpret_cast<const unsigned long long *>(d + ldc);
    k_lo_phase<0><<<dim3((unsigned)l, (unsigned)cdiv(nparts, kPGroup)), kBlk, 0, st>>>(A, lda, n, ZT, ldzt, M, lds, C, ldc, d, E,
                                                                       lo_lde(n), s, nparts, part, nullptr, nullptr,
                                                                       nullptr, phi, ldphi, status);
    return cudaGetLastError();
}

// AT: n x ldlt words (A transposed), W: l x lds, V: n x lds, H: n x ldc,
// gsp: n x nblk doubles, Kfx: n x n int64 followed by the scale (double).
cudaError_t launch_lo_grad(const uint64_t *A, int64_t lda, int64_t n, int64_t l, const uint64_t *ZT, int64_t ldzt,
                           const float *M, int64_t lds, const float *C, int64_t ldc, int64_t s, int64_t m,
                           const int4 *sup, const double *alpha, const double *beta, uint64_t *AT, int64_t ldlt,
                           float *W, float *V, double *H, double *gsp, unsigned long long *Kfx, double *grad,
                           __nv_bfloat16 *split, const float *phi, int64_t ldphi, uint32_t *status,
                           cudaStream_t st) {
    const int64_t nblk = cdiv(s, kBlk);
    double *scale = reinterpret_cast<double *>(Kfx + n * n);
    const float *d = C + n * ldc;
    const unsigned long long *E = reinterpret_cast<const unsigned long long *>(d + ldc);
    const int64_t lde = lo_lde(n);
    cudaError_t e = launch_bit_transpose_batched(A, 1, l, n, lda, AT, ldlt, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Kfx, 0, (size_t)n * n * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = launch_fixed_scale(alpha, beta, l, s, scale, st)) != cudaSuccess) return e;
    if (phi != nullptr) {  // Phi kept by the statistics pass (possibly in W itself)
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_w<<<grid_1d(l * (lds / 4)), 256, 0, st>>>(phi, ldphi, W, lds, l, s, alpha, beta);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_phase<1><<<dim3((unsigned)l, (unsigned)cdiv(nblk, kPGroup)), kBlk, 0, st>>>(A, lda, n, ZT, ldzt, M, lds, C, ldc, d,
                                                                         E, lde, s, nblk, nullptr, alpha, beta, W, nullptr, 0,
                                                                         status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_v<<<dim3((unsigned)n, (unsigned)cdiv(nblk, kGroup)), kBlk, 0, st>>>(AT, ldlt, ZT, ldzt, W, lds, s, nblk,
                                                                                  V, gsp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // H = (s o V) S^T: rows q, columns r (ZT's rows), K the samples.
    bool h_done = false;
    if (lo_tensor() && split != nullptr) {
        __nv_bfloat16 *hi = split, *lo = split + n * lds;
        if ((e = launch_split(V, lds, n, s, ZT, ldzt, lds, hi, lo, st)) != cudaSuccess) return e;
        e = launch_tc_dense(hi, lo, n, lds, s, ZT, n, ldzt, H, ldc, true, status, st);
        if (e != cudaSuccess && e != cudaErrorNotSupported) return e;
        h_done = e == cudaSuccess;
    }
    if (!h_done) {
        LaunchScope ls(IQP_KERNEL_LOWORDER_GEMM, st);
        k_lo_h<<<dim3((unsigned)n, (unsigned)kHSplit), 32, 0, st>>>(E, lde, ZT, ldzt, V, lds, s, H, ldc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        LaunchScope ls(IQP_KERNEL_LOWORDER, st);
        k_lo_pairs<<<dim3((unsigned)l, (unsigned)cdiv(nblk, kPGroup)), kBlk, 0, st>>>(A, lda, n, ZT, ldzt, C, ldc, E,
                                                                                     lde, W, lds, s, nblk, scale, Kfx,
                                                                                     status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    LaunchScope ls(IQP_KERNEL_LOWORDER, st);
    k_lo_grad_out<<<grid_1d(m), 256, 0, st>>>(sup, m, n, gsp, nblk, H, ldc, Kfx, scale, grad);
    return cudaGetLastError();
}

}  // namespace iqp
