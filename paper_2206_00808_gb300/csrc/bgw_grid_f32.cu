// FP32 instantiation of the real-space grid and matrix-element kernels
// (the mixed-precision path: complex64 grids and M).
#define BGW_REAL float
#define BGW_SUFFIX f32
#include "bgw_grid_impl.cuh"

namespace bgw {
cudaError_t grid_tables_init_f32() { return f32::upload_tables(); }
cudaError_t wfn_to_grid_f32(const double *coeff, int ngw, int B, const int *cube_map,
                            const Axes &a, void *S, void *R, void *U, cudaStream_t st, int path) {
    return f32::wfn_to_grid(coeff, ngw, B, cube_map, a, S, R, U, st, path);
}
cudaError_t wfn_to_grid_batch_f32(const K1Job *jobs, int n, int B, cudaStream_t st, bool *batched) {
    return f32::wfn_to_grid_batch(jobs, n, B, st, batched);
}
cudaError_t mtxel_f32(const void *Uv, const void *Uc, int nv, int nc, const Axes &a,
                      const int *gmap, int ng, void *A, void *Bs, void *M, long ldm,
                      cudaStream_t st, int tv, int tc, int lanes, int zy, const XPassHook *hook, int *err,
                      int drop) {
    return f32::mtxel(Uv, Uc, nv, nc, a, gmap, ng, A, Bs, M, ldm, st, tv, tc, lanes, zy, hook, err, drop);
}
int plane_tile_candidates(int nv, int nc, const Axes &a, int *tv, int *tc, int max) {
    return f32::plane_tile_list(nv, nc, a, tv, tc, max);
}
cudaError_t bounds_take_grid_f32(unsigned *word) { return bgw_bounds_take(word); }
}  // namespace bgw
