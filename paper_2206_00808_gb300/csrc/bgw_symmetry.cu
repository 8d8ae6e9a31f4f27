// Spinor symmetry unfolding (arXiv:2206.00808, Sec. "Spinor wavefunctions and
// symmetries").
//
// A symmetry {R|tau} takes the plane-wave coefficients of a spinor Bloch state
// at k to those at Rk:
//     c'_{n,Rk,a}(G') = e^{-i G'.tau} sum_b U_ab c_{n,k,b}(R^-1 G')
// (the unfolding relation of the no-spin subsection, with the common phase
// e^{-i Rk.tau} dropped, and the SU(2) matrix of the spinor subsection).  The
// rotated sphere is the image of the sphere at k, so entry i of the output is
// entry i of the input with Miller index h'_i = R_lat^-T h_i: no gather.
//
// U comes from the rotation's axis n and angle theta,
//     U = cos(theta/2) I - i sin(theta/2) n.sigma,
// which turns spin expectation values with the active Cartesian rotation R.
// (n, theta) are read from a unit quaternion found by Markley's modification
// of Shepperd's algorithm: the 4 x 4 matrix X of the attitude matrix R^T,
// its column of largest norm, normalised, positive branch; then
// theta = 2 atan2(|q_vec|, q4), n = q_vec / |q_vec|.  The lattice-basis
// rotation goes to Cartesian as A R_lat A^-1 (A: lattice vectors as columns);
// an improper operation (det = -1) turns the spinor by its proper part -R.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/bgw_chi.h"

void bgw_set_global_error(const std::string &msg);

namespace {

struct Mat3 {
    double m[3][3];
};

double det3(const Mat3 &a) {
    return a.m[0][0] * (a.m[1][1] * a.m[2][2] - a.m[1][2] * a.m[2][1]) -
           a.m[0][1] * (a.m[1][0] * a.m[2][2] - a.m[1][2] * a.m[2][0]) +
           a.m[0][2] * (a.m[1][0] * a.m[2][1] - a.m[1][1] * a.m[2][0]);
}

// Inverse by the adjugate (3 x 3, det != 0).
Mat3 inv3(const Mat3 &a) {
    const double d = det3(a);
    Mat3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
            r.m[i][j] = (a.m[i1][j1] * a.m[i2][j2] - a.m[i1][j2] * a.m[i2][j1]) / d;
        }
    return r;
}

Mat3 mul3(const Mat3 &a, const Mat3 &b) {
    Mat3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += a.m[i][k] * b.m[k][j];
            r.m[i][j] = s;
        }
    return r;
}

// U (row-major complex [2][2]) and (n, theta) of a lattice-basis operation.
bgw_status su2_of(const double *avec, const int *rot_lat, double *U, double *axis_angle, std::string &err) {
    Mat3 A, Rl;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A.m[i][j] = avec[3 * j + i];   // column j = lattice vector a_j
            Rl.m[i][j] = rot_lat[3 * i + j];
        }
    const double dl = det3(Rl);
    if (std::fabs(std::fabs(dl) - 1.0) > 1e-12) {
        err = "symmetry: the lattice-basis rotation is not unimodular";
        return BGW_E_ARG;
    }
    const double da = det3(A);
    if (!(std::fabs(da) > 0.0) || !std::isfinite(da)) {
        err = "symmetry: singular cell";
        return BGW_E_ARG;
    }
    Mat3 R = mul3(mul3(A, Rl), inv3(A));
    // must be orthogonal: the operation has to be a symmetry of the lattice metric
    double worst = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += R.m[k][i] * R.m[k][j];
            worst = std::fmax(worst, std::fabs(s - (i == j ? 1.0 : 0.0)));
        }
    if (worst > 1e-8) {
        err = "symmetry: the operation is not a rotation of this cell (R^T R != I)";
        return BGW_E_ARG;
    }
    if (det3(R) < 0)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) R.m[i][j] = -R.m[i][j];
    // attitude matrix T = R^T and Shepperd's 4 x 4 matrix (Markley's form)
    double T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] = R.m[j][i];
    const double tr = T[0][0] + T[1][1] + T[2][2];
    const double X[4][4] = {
        {1 + 2 * T[0][0] - tr, T[1][0] + T[0][1], T[2][0] + T[0][2], T[1][2] - T[2][1]},
        {T[0][1] + T[1][0], 1 + 2 * T[1][1] - tr, T[2][1] + T[1][2], T[2][0] - T[0][2]},
        {T[0][2] + T[2][0], T[1][2] + T[2][1], 1 + 2 * T[2][2] - tr, T[0][1] - T[1][0]},
        {T[1][2] - T[2][1], T[2][0] - T[0][2], T[0][1] - T[1][0], 1 + tr}};
    int best = 0;
    double bn = -1;
    for (int c = 0; c < 4; ++c) {
        double s = 0;
        for (int r = 0; r < 4; ++r) s += X[r][c] * X[r][c];
        if (s > bn) {
            bn = s;
            best = c;
        }
    }
    bn = std::sqrt(bn);
    double q[4];
    for (int r = 0; r < 4; ++r) q[r] = X[r][best] / bn;
    const double vn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    const double theta = 2.0 * std::atan2(vn, q[3]);
    double n[3] = {0.0, 0.0, 1.0};
    if (vn > 0)
        for (int i = 0; i < 3; ++i) n[i] = q[i] / vn;
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    // cos(theta/2) I - i sin(theta/2) (n_x sigma_x + n_y sigma_y + n_z sigma_z)
    const double u[8] = {c, -s * n[2], -s * n[1], -s * n[0], s * n[1], -s * n[0], c, s * n[2]};
    if (U)
        for (int i = 0; i < 8; ++i) U[i] = u[i];
    if (axis_angle) {
        axis_angle[0] = n[0];
        axis_angle[1] = n[1];
        axis_angle[2] = n[2];
        axis_angle[3] = theta;
    }
    return BGW_OK;
}

// One thread per (plane wave i, chunk of kBandChunk bands): the phase
// e^{-2 pi i h'.tau} is formed once per thread from the rotated Miller index
// h' = M h (M = R_lat^-T), then applied to its bands; reads and writes are
// coalesced along i.
constexpr int kBandChunk = 16;

struct Op {
    int M[3][3];
    double tau[3];
    double2 u[4];   // U row-major
};

__global__ void k8_unfold(const double2 *__restrict__ in, double2 *__restrict__ out, int nb, int ngw,
                          const int *__restrict__ gvec, Op op) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ngw) return;
    const int h0 = gvec[3 * i], h1 = gvec[3 * i + 1], h2 = gvec[3 * i + 2];
    double f = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r) f += (double)(op.M[r][0] * h0 + op.M[r][1] * h1 + op.M[r][2] * h2) * op.tau[r];
    f -= floor(f);                                        // turns in [0, 1)
    double sn, cs;
    sincospi(-2.0 * f, &sn, &cs);
    // the phase folded into this plane wave's copy of U: V = e^{-i G'.tau} U
    // (the 2 x 2 complex product is the whole per-band cost, on the FP64 pipe)
    double2 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        v[k] = make_double2(cs * op.u[k].x - sn * op.u[k].y, cs * op.u[k].y + sn * op.u[k].x);
    const int n1 = min(nb, (int)(blockIdx.y + 1) * kBandChunk);
#pragma unroll 4
    for (int n = blockIdx.y * kBandChunk; n < n1; ++n) {
        const double2 a = in[(2L * n) * ngw + i], b = in[(2L * n + 1) * ngw + i];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const double2 u0 = v[2 * r], u1 = v[2 * r + 1];
            const double x = fma(u0.x, a.x, fma(-u0.y, a.y, fma(u1.x, b.x, -u1.y * b.y)));
            const double y = fma(u0.x, a.y, fma(u0.y, a.x, fma(u1.x, b.y, u1.y * b.x)));
            out[(2L * n + r) * ngw + i] = make_double2(x, y);
        }
    }
}

}  // namespace

extern "C" bgw_status bgw_symmetry_su2(const double *avec, const int *rot_lat, double *U, double *axis_angle) {
    if (!avec || !rot_lat) {
        bgw_set_global_error("symmetry_su2: null pointer argument");
        return BGW_E_ARG;
    }
    std::string err;
    const bgw_status st = su2_of(avec, rot_lat, U, axis_angle, err);
    if (st != BGW_OK) bgw_set_global_error(err);
    return st;
}

extern "C" bgw_status bgw_unfold_spinor(const double *avec, const int *rot_lat, const double *tau, int nb,
                                        int ngw, const int *gvec_in, int *gvec_out, const void *c_in,
                                        void *c_out, void *stream) {
    auto fail = [](bgw_status s, const std::string &m) {
        bgw_set_global_error(m);
        return s;
    };
    if (!avec || !rot_lat || !tau || !gvec_in || !gvec_out || !c_in || !c_out)
        return fail(BGW_E_ARG, "unfold_spinor: null pointer argument");
    if (nb < 0 || ngw < 1) return fail(BGW_E_ARG, "unfold_spinor: nb >= 0 and ngw >= 1 required");
    if (c_in == c_out) return fail(BGW_E_ARG, "unfold_spinor: input and output must not alias");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(tau[a])) return fail(BGW_E_ARG, "unfold_spinor: non-finite tau");
    double U[8];
    std::string err;
    bgw_status st = su2_of(avec, rot_lat, U, nullptr, err);
    if (st != BGW_OK) return fail(st, err);
    // Miller indices transform with R_lat^-T (integer for a unimodular R_lat)
    Mat3 Rl;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rl.m[i][j] = rot_lat[3 * i + j];
    const Mat3 Ri = inv3(Rl);
    int M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = (int)std::lround(Ri.m[j][i]);
    for (int g = 0; g < ngw; ++g)
        for (int i = 0; i < 3; ++i)
            gvec_out[3 * g + i] =
                M[i][0] * gvec_in[3 * g] + M[i][1] * gvec_in[3 * g + 1] + M[i][2] * gvec_in[3 * g + 2];
    if (nb == 0) return BGW_OK;
    if ((long)nb > 65535L * kBandChunk) return fail(BGW_E_ARG, "unfold_spinor: too many bands for one call");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *g_dev = nullptr;
    const size_t gbytes = sizeof(int) * 3 * (size_t)ngw;
    cudaError_t e = cudaMallocAsync(&g_dev, gbytes, s);
    // a pageable source: the copy has read gvec_in when it returns
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_dev, gvec_in, gbytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        Op op;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) op.M[i][j] = M[i][j];
            op.tau[i] = tau[i];
        }
        for (int i = 0; i < 4; ++i) op.u[i] = make_double2(U[2 * i], U[2 * i + 1]);
        const dim3 grid((unsigned)((ngw + 255) / 256), (unsigned)((nb + kBandChunk - 1) / kBandChunk));
        k8_unfold<<<grid, 256, 0, s>>>(static_cast<const double2 *>(c_in), static_cast<double2 *>(c_out), nb,
                                       ngw, static_cast<const int *>(g_dev), op);
        e = cudaGetLastError();
    }
    if (g_dev) {
        const cudaError_t f = cudaFreeAsync(g_dev, s);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? BGW_E_NOMEM : BGW_E_CUDA,
                    std::string("unfold_spinor: ") + cudaGetErrorString(e));
    return BGW_OK;
}
