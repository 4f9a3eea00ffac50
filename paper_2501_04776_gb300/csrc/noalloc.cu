// iqp_expval without a caller-supplied workspace.
//
// Some callers cannot allocate device memory when they call in: a host
// process whose device memory is entirely owned by another framework's
// caching pool, or latency-bound code for which cudaMalloc's implicit
// device-wide synchronisation and unbounded run time are not acceptable.
// For them this file keeps the forward estimator's scratch in one file-scope
// device array of fixed size, reserved when the GPU loads this library and
// held until the process exits. Nothing here calls cudaMalloc or cudaFree.
#include <mutex>

#include "common.cuh"

namespace iqp {

namespace {

constexpr size_t kNoAllocBytes = (size_t)64 << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

// The scratch itself. In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
iqp_status noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IQP_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return IQP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return IQP_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return IQP_OK;
}

}  // namespace

}  // namespace iqp

extern "C" iqp_status iqp_expval_noalloc(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, const uint64_t *A,
                                         int64_t l, int64_t lda, const uint64_t *Z, int64_t s, int64_t ldz,
                                         const float *theta, iqp_precision prec, double *expval, double *std_err,
                                         void *stream) {
    // The checks iqp_expval runs come first, so invalid arguments give the
    // same status as there and nothing is queued for them.
    iqp_status rc = iqp::expval_arg_check(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, prec, expval, std_err);
    if (rc != IQP_OK) return rc;
    // The array must hold the op's workspace; the optional split-tile scratch
    // at its end is used only when it fits as well.
    const size_t need = iqp::workspace_min_bytes(IQP_OP_EXPVAL, n, m, l, s, 0, prec);
    if (need == 0) return IQP_ERR_ARG;
    if (need > iqp::kNoAllocBytes) return IQP_ERR_WORKSPACE;
    void *ws = nullptr;
    if ((rc = iqp::noalloc_scratch(&ws)) != IQP_OK) return rc;
    // The array keeps the previous call's contents; the device status word at
    // its start must begin at zero. Every other region is fully rewritten.
    if (cudaMemsetAsync(ws, 0, 256, static_cast<cudaStream_t>(stream)) != cudaSuccess) return IQP_ERR_CUDA;
    return iqp_expval(n, G, m, ldg, A, l, lda, Z, s, ldz, theta, prec, expval, std_err, ws, iqp::kNoAllocBytes,
                      stream);
}

extern "C" iqp_status iqp_noalloc_read_status(void *stream) {
    void *ws = nullptr;
    const iqp_status rc = iqp::noalloc_scratch(&ws);
    if (rc != IQP_OK) return rc;
    return iqp_read_status(ws, iqp::kNoAllocBytes, stream);
}
