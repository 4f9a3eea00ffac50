// Host-side interface of the fused parity step (parity.cu), shared with the
// estimators' preparation in api.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace iqp {

// One row matrix R (rows x ldr words) of a fused parity call: its R^T scratch
// (n x ldpt words), P^T (m x ldpt) and P (rows x ldp).
struct ParitySide {
    const uint64_t *R;
    int64_t rows, ldr;
    uint64_t *P, *PT;
    int64_t ldpt;
    uint64_t *RT;
};

// Fused support-gather parities of one or two row matrices sharing the gates
// G (m x ldg words over n qubits) and their support list `sup` (formed here
// first if form_sup, in the same launch as both R^T where rows are short):
// both R^T in one launch, then P^T and P of both in one launch. ldp even,
// each ldpt even.
cudaError_t launch_parity_gather_fused(int64_t n, const uint64_t *G, int64_t m, int64_t ldg, int4 *sup,
                                       bool form_sup, int64_t ldp, const ParitySide *side, int nside,
                                       cudaStream_t st);

}  // namespace iqp
