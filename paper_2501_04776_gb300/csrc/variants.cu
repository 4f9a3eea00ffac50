// Options around the estimator: shared-parameter gates (Sec. 3.1.1), the
// `wires` embedding of the MMD loss (Sec. 3.3.1), and counter-based random
// bits for samples z ~ U{0,1}^n and observables a ~ P_sigma (bitwise
// Bernoulli) drawn on the device inside a training loop (Sec. 2.4: fresh
// samples every step).
//
// Random bits: splitmix64 (Steele, Lea and Flood, OOPSLA 2014) used as a
// counter-based generator: value k (k = 1, 2, ...) of stream t under seed S is
//   mix(S * PHI + t * PSI + k * GAMMA),
// mix = the splitmix64 finaliser (variant 13 of Stafford's mixers), with the
// odd constants GAMMA (the golden-ratio increment of splitmix64) and PHI, PSI
// selecting the seed and stream. Uniform doubles take the top 53 bits.
#include "common.cuh"

namespace iqp {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhi = 0xD1B54A32D192ED03ull;
constexpr uint64_t kPsi = 0xAEF17502108EF2D9ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// theta_gen[j] = theta_p[p] for j in [start[p], start[p+1]) (clamped to [0, m)).
__global__ void k_expand_params(const float *__restrict__ theta_p, int64_t np, const int64_t *__restrict__ start,
                                int64_t m, float *__restrict__ theta_gen) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t j0 = start[p], j1 = start[p + 1];
        j0 = j0 < 0 ? 0 : j0;
        j1 = j1 > m ? m : j1;
        const float t = theta_p[p];
        for (int64_t j = j0; j < j1; ++j)
            if (IQP_IN(j, m, 102)) theta_gen[j] = t;
    }
}

// grad_p[p] = sum of grad_gen over the gate's generators, in index order.
__global__ void k_reduce_params(const double *__restrict__ grad_gen, int64_t m, const int64_t *__restrict__ start,
                                int64_t np, double *__restrict__ grad_p) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t j0 = start[p], j1 = start[p + 1];
        j0 = j0 < 0 ? 0 : j0;
        j1 = j1 > m ? m : j1;
        double acc = 0.0;
        for (int64_t j = j0; j < j1; ++j)
            if (IQP_IN(j, m, 103)) acc += grad_gen[j];
        grad_p[p] = acc;
    }
}

// dst row r: bit wires[k] = bit k of src row r; all other bits zero. One
// thread per row; wires outside [0, 64 ld_dst) and outside [0, n) are skipped.
__global__ void k_embed_bits(const uint64_t *__restrict__ src, int64_t rows, int64_t ld_src,
                             const int32_t *__restrict__ wires, int64_t nw, uint64_t *__restrict__ dst,
                             int64_t ld_dst, int64_t n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        uint64_t *d = dst + r * ld_dst;
        for (int64_t w = 0; w < ld_dst; ++w) d[w] = 0ull;
        const uint64_t *s = src + r * ld_src;
        for (int64_t k = 0; k < nw; ++k) {
            const int64_t q = wires[k];
            if (q < 0 || q >= n) continue;
            if (!IQP_IN(k >> 6, ld_src, 100) || !IQP_IN(q >> 6, ld_dst, 101)) continue;
            if ((s[k >> 6] >> (k & 63)) & 1ull) d[q >> 6] |= 1ull << (q & 63);
        }
    }
}

// Uniform bits: word w (< ceil(n/64)) of row r is value r * ldgen + w + 1 of
// the stream, ldgen = ceil(n/64) rounded up to even; bits >= n and words
// >= ceil(n/64) are zero.
__global__ void k_uniform_bits(uint64_t seed, uint64_t stream, int64_t rows, int64_t n, int64_t ld,
                               uint64_t *__restrict__ out) {
    const int64_t full = n >> 6, rem = n & 63, used = full + (rem ? 1 : 0);
    const int64_t ldgen = used + (used & 1);
    const uint64_t base = seed * kPhi + stream * kPsi;
    const int64_t total = rows * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / ld, w = e - r * ld;
        uint64_t v = 0ull;
        if (w < used) {
            v = mix64(base + (uint64_t)(r * ldgen + w + 1) * kGamma);
            if (w == full && rem) v &= (1ull << rem) - 1ull;
        }
        out[e] = v;
    }
}

// Bernoulli(p) bits: bit q of row r is set iff uniform value r * n + q + 1 of
// the stream is < p, the uniform being (value >> 11) * 2^-53 in FP64 (exact).
__global__ void k_bernoulli_bits(uint64_t seed, uint64_t stream, int64_t rows, int64_t n, double p, int64_t ld,
                                 uint64_t *__restrict__ out) {
    const uint64_t base = seed * kPhi + stream * kPsi;
    const int64_t total = rows * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / ld, w = e - r * ld;
        uint64_t v = 0ull;
        const int64_t q0 = w * 64;
        const int64_t q1 = q0 + 64 < n ? q0 + 64 : n;
        for (int64_t q = q0; q < q1; ++q) {
            const uint64_t x = mix64(base + (uint64_t)(r * n + q + 1) * kGamma);
            const double u = (double)(x >> 11) * 0x1.0p-53;
            if (u < p) v |= 1ull << (q - q0);
        }
        out[e] = v;
    }
}

}  // namespace

uint32_t check_word_variants() { return take_check_word(); }

namespace {

int grid_for(int64_t work) {
    int64_t b = cdiv(work, 256);
    if (b < 1) b = 1;
    if (b > 8192) b = 8192;
    return (int)b;
}

}  // namespace

cudaError_t launch_expand_params(const float *theta_p, int64_t np, const int64_t *start, int64_t m, float *theta_gen,
                                 cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_VARIANTS, st);
    k_expand_params<<<grid_for(np), 256, 0, st>>>(theta_p, np, start, m, theta_gen);
    return cudaGetLastError();
}

cudaError_t launch_reduce_params(const double *grad_gen, int64_t m, const int64_t *start, int64_t np,
                                 double *grad_p, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_VARIANTS, st);
    k_reduce_params<<<grid_for(np), 256, 0, st>>>(grad_gen, m, start, np, grad_p);
    return cudaGetLastError();
}

cudaError_t launch_embed_bits(const uint64_t *src, int64_t rows, int64_t ld_src, const int32_t *wires, int64_t nw,
                              uint64_t *dst, int64_t ld_dst, int64_t n, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_VARIANTS, st);
    k_embed_bits<<<grid_for(rows), 256, 0, st>>>(src, rows, ld_src, wires, nw, dst, ld_dst, n);
    return cudaGetLastError();
}

cudaError_t launch_uniform_bits(uint64_t seed, uint64_t stream, int64_t rows, int64_t n, int64_t ld, uint64_t *out,
                                cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_RNG, st);
    k_uniform_bits<<<grid_for(rows * ld), 256, 0, st>>>(seed, stream, rows, n, ld, out);
    return cudaGetLastError();
}

cudaError_t launch_bernoulli_bits(uint64_t seed, uint64_t stream, int64_t rows, int64_t n, double p, int64_t ld,
                                  uint64_t *out, cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_RNG, st);
    k_bernoulli_bits<<<grid_for(rows * ld), 256, 0, st>>>(seed, stream, rows, n, p, ld, out);
    return cudaGetLastError();
}

}  // namespace iqp
