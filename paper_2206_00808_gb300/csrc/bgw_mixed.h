// Mixed-precision contraction (split-BF16, three products, FP32 accumulation
// on tcgen05 tensor cores; FP64 weights and FP64 reduction across k).
// Internal; declared for the C-ABI layer.
#pragma once
#include <cuda_runtime.h>

namespace bgw {

// Bytes of workspace herk_mixed needs for P pairs, ng G-vectors, nfreq
// frequencies.
size_t mixed_workspace_bytes(long P, int ng, int nfreq);

// acc[j][g][g'] (complex128, lower block triangle) += sum_p w[j][p]
// conj(M[p][g]) M[p][g'] with M complex64 [P][ng] and w FP64 [nfreq][P].
// *nkernels receives the number of kernels launched.  A device-side wait
// that gives up writes a non-zero code to the device int *err (the host
// reports BGW_E_TIMEOUT when it reads it back).
cudaError_t herk_mixed(const void *M, int P, int ng, const double *w, int nfreq, void *ws,
                       void *acc, cudaStream_t st, int *nkernels, int *err);

}  // namespace bgw
