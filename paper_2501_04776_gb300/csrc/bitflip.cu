// Stochastic bitflip circuits (Sec. 2.5): each gate flips the bits of g_j
// with probability sin^2(theta_j) instead of acting coherently, and the
// expectation values are exact products (eq. expval_bitflip):
//   <Z_a> = prod_{j in J_a} cos(2 theta_j),  J_a = { j : g_j.a odd }.
// For L = sum_a w_a <Z_a>:
//   dL/dtheta_j = -2 tan(2 theta_j) * sum_a [g_j.a odd] w_a <Z_a>.
// Both are FP64 reductions over the bit-packed parities: a product over the
// set bits of each P_A row, and a sum over the set bits of each P_A^T row.
// The reduction order is fixed (lane-strided, then a shuffle tree), so the
// results are deterministic.
#include "common.cuh"

namespace iqp {

uint32_t check_word_bitflip() { return take_check_word(); }

namespace {

// c_j = cos(2 theta_j), t_j = -2 tan(2 theta_j), zero beyond m.
__global__ void k_bitflip_gates(const float *__restrict__ theta, int64_t m, int64_t mpad, double *__restrict__ c,
                                double *__restrict__ t) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < mpad; j += (int64_t)gridDim.x * blockDim.x) {
        if (j < m) {
            const double x = 2.0 * (double)theta[j];
            double sn, cs;
            sincos(x, &sn, &cs);
            c[j] = cs;
            t[j] = -2.0 * sn / cs;
        } else {
            c[j] = 1.0;
            t[j] = 0.0;
        }
    }
}

// expval[a] = product of c_j over the set bits j of P_A row a. One warp per row.
__global__ void __launch_bounds__(256) k_bitflip_rows(const uint64_t *__restrict__ PA, int64_t ldp, int64_t l,
                                                       const double *__restrict__ c, double *__restrict__ expval) {
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (a >= l) return;
    const uint64_t *row = PA + a * ldp;
    double prod = 1.0;
    for (int64_t w = lane; w < ldp; w += 32) {
        uint64_t bits = row[w];
        while (bits) {
            const int b = __ffsll((long long)bits) - 1;
            bits &= bits - 1ull;
            if (IQP_IN(w * 64 + b, ldp * 64, 90)) prod *= c[w * 64 + b];
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) prod *= __shfl_xor_sync(0xFFFFFFFFu, prod, off);
    if (lane == 0) expval[a] = prod;
}

// v[a] = w[a] * expval[a].
__global__ void k_bitflip_weights(const double *__restrict__ w, const double *__restrict__ ev, int64_t l,
                                  double *__restrict__ v) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a < l) v[a] = w[a] * ev[a];
}

// grad[j] = t_j * sum of v[a] over the set bits a of P_A^T row j. One warp per gate.
__global__ void __launch_bounds__(256) k_bitflip_grad(const uint64_t *__restrict__ PAT, int64_t ldlt, int64_t m,
                                                       [[maybe_unused]] int64_t l, const double *__restrict__ v,
                                                       const double *__restrict__ t, double *__restrict__ grad) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= m) return;
    const uint64_t *row = PAT + j * ldlt;
    double acc = 0.0;
    for (int64_t w = lane; w < ldlt; w += 32) {
        uint64_t bits = row[w];
        while (bits) {
            const int b = __ffsll((long long)bits) - 1;
            bits &= bits - 1ull;
            if (IQP_IN(w * 64 + b, l, 91)) acc += v[w * 64 + b];  // bits past the last observable are zero
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (lane == 0) grad[j] = t[j] * acc;
}

}  // namespace

cudaError_t launch_bitflip_gates(const float *theta, int64_t m, int64_t mpad, double *c, double *t, cudaStream_t st) {
    int blocks = (int)cdiv(mpad, 256);
    if (blocks > 4096) blocks = 4096;
    LaunchScope ls(IQP_KERNEL_BITFLIP, st);
    k_bitflip_gates<<<blocks, 256, 0, st>>>(theta, m, mpad, c, t);
    return cudaGetLastError();
}

cudaError_t launch_bitflip_rows(const uint64_t *PA, int64_t ldp, int64_t l, const double *c, double *expval,
                                cudaStream_t st) {
    LaunchScope ls(IQP_KERNEL_BITFLIP, st);
    k_bitflip_rows<<<(unsigned)cdiv(l, 8), 256, 0, st>>>(PA, ldp, l, c, expval);
    return cudaGetLastError();
}

cudaError_t launch_bitflip_grad(const uint64_t *PAT, int64_t ldlt, int64_t m, int64_t l, const double *w,
                                const double *ev, double *v, const double *t, double *grad, cudaStream_t st) {
    {
        LaunchScope ls(IQP_KERNEL_BITFLIP, st);
        k_bitflip_weights<<<(unsigned)cdiv(l, 256), 256, 0, st>>>(w, ev, l, v);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    LaunchScope ls(IQP_KERNEL_BITFLIP, st);
    k_bitflip_grad<<<(unsigned)cdiv(m, 8), 256, 0, st>>>(PAT, ldlt, m, l, v, t, grad);
    return cudaGetLastError();
}

}  // namespace iqp
