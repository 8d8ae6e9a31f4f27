// FP64 instantiation of the real-space grid and matrix-element kernels.
#define BGW_REAL double
#define BGW_SUFFIX f64
#include "bgw_grid_impl.cuh"

namespace bgw {
cudaError_t grid_tables_init_f64() { return f64::upload_tables(); }
cudaError_t wfn_to_grid_f64(const double *coeff, int ngw, int B, const int *cube_map,
                            const Axes &a, void *S, void *R, void *U, cudaStream_t st, int path) {
    return f64::wfn_to_grid(coeff, ngw, B, cube_map, a, S, R, U, st, path);
}
cudaError_t wfn_to_grid_batch_f64(const K1Job *jobs, int n, int B, cudaStream_t st, bool *batched) {
    return f64::wfn_to_grid_batch(jobs, n, B, st, batched);
}
cudaError_t mtxel_f64(const void *Uv, const void *Uc, int nv, int nc, const Axes &a,
                      const int *gmap, int ng, void *A, void *Bs, void *M, long ldm,
                      cudaStream_t st, int tv, int tc, int lanes, int zy, const XPassHook *hook, int *err,
                      int drop) {
    return f64::mtxel(Uv, Uc, nv, nc, a, gmap, ng, A, Bs, M, ldm, st, tv, tc, lanes, zy, hook, err, drop);
}
cudaError_t bounds_take_grid_f64(unsigned *word) { return bgw_bounds_take(word); }
}  // namespace bgw
