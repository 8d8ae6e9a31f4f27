// Mixed-precision contraction (split-BF16 or split-TF32 with three products,
// or one TF32 product; FP32 accumulation on tcgen05 tensor cores; FP64
// weights and FP64 reduction across k).  Internal; declared for the C-ABI
// layer.
#pragma once
#include <cuda_runtime.h>

namespace bgw {

// Operand formats (the values of the matching bgw_precision entries).
enum MixedFormat { kMixedBF16x3 = 1, kMixedTF32x3 = 2, kMixedTF32 = 3 };

// Bytes of workspace the mixed contraction needs for P pairs, ng G-vectors, nfreq
// frequencies in format fmt.
size_t mixed_workspace_bytes(long P, int ng, int nfreq, int fmt);

// Operand split: M complex64 [P][ng] and w FP64 [nfreq][P] -> the hi/lo
// planes (BF16 or TF32; hi only for kMixedTF32) of X = interleaved (Re, Im)
// rows and of w_j X in ws.
cudaError_t mixed_split(const void *M, int P, int ng, const double *w, int nfreq, void *ws, int fmt,
                        cudaStream_t st);

// One q-point of a grouped contraction: its split planes (from mixed_split),
// pair count and accumulator.
struct MixedQ {
    void *ws;
    int P, ng;
    void *acc;
};

// Largest number of q-points one grouped launch takes.
int mixed_max_group();

// For every q of the group, acc[j][g][g'] (complex128, lower block triangle)
// += sum_p w[j][p] conj(M[p][g]) M[p][g'] from its planes, on tcgen05 tensor
// cores, in ONE persistent launch of at most sm_count blocks.  A device-side
// wait that gives up writes a non-zero code to the device int *err (the host
// reports BGW_E_TIMEOUT when it reads it back).
// drop_first_load (tests only): block 0 skips its first TMA stage so the
// consumers' bounded waits expire and the error path runs.
cudaError_t mixed_gemm(const MixedQ *qs, int nq, int nfreq, int fmt, int sm_count, cudaStream_t st, int *err,
                       int drop_first_load = 0);

}  // namespace bgw
