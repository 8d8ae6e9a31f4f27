// FP64-accurate contraction of chi0 on tcgen05 tensor cores (BF16 digit
// slices with exact integer accumulation).  Internal; declared for the
// C-ABI layer.
#pragma once
#include <cuda_runtime.h>

namespace bgw {

constexpr int F64TC_ERR_SIGN = 16;

// Bytes of workspace f64tc_contract needs for P pairs, ng G-vectors, nfreq
// frequencies (digit planes and per-row exponents).
size_t f64tc_workspace_bytes(long P, int ng, int nfreq);

// acc[j][g][g'] (complex128, lower block triangle) += sum_p w[j][p]
// conj(M[p][g]) M[p][g'] for M complex128 [P][ng] and w FP64 [nfreq][P]
// (every w < 0 or = 0), to FP64 accuracy: per frequency the rows of
// Y = sqrt(-w) (Re M, Im M) are scaled by a power of two per row and cut into
// five signed base-256 digits, and the 15 digit products of total order <= 4
// run on tcgen05 in BF16 with exact integer sums.  Launches the exponent
// pass, the digit split and ONE persistent contraction of at most sm_count
// blocks.  A device-side wait that gives up writes a non-zero code to *err;
// a positive weight (an occupied band above an empty one) writes
// F64TC_ERR_SIGN there and its pair is left out (the digit form takes
// -Y Y^T with Y = sqrt(-w) (Re M, Im M)).
cudaError_t f64tc_contract(const void *M, int P, int ng, const double *w, int nfreq, void *acc, void *ws,
                           int sm_count, cudaStream_t st, int *err);

}  // namespace bgw
