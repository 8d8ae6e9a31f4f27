"""Spinor symmetry unfolding, plain numpy (TEST INFRASTRUCTURE ONLY).

Only `tests/` may import this module; the product path never does.  It
follows arXiv:2206.00808, Sec. "Spinor wavefunctions and symmetries":

  * a symmetry {R|tau} maps c_{n,k}(G) to c~_{n,Rk}(G') = c_{n,k}(R^-1 G')
    e^{-i G'.tau} (the unfolding relation of the no-spin subsection, the
    common phase e^{-i Rk.tau} dropped);
  * the two spinor components are then mixed by the SU(2) matrix of the
    rotation's axis n and angle theta, cos(theta/2) - i sin(theta/2) n.sigma
    (the 2 x 2 matrix of the spinor subsection; see the readings below);
  * (n, theta) come from a unit quaternion found by Markley's version of
    Shepperd's algorithm (the auxiliary 4 x 4 matrix X, its largest column,
    the positive branch), then theta = 2 arctan(|q_vec| / q_4) and
    n = q_vec / |q_vec|;
  * lattice-basis rotations are taken to Cartesian by A R_lat A^-1 (A has the
    lattice vectors as columns); an improper operation S (det = -1) rotates
    the spinor by its proper part -S.

Readings where the printed text is garbled or ambiguous:
  * the quaternion form of the matrix and the matrix X are written for the
    attitude (passive) matrix, the transpose of the active rotation
    R(n, theta) printed first; X is built here from R^T of the active R, so
    that the quaternion's vector part is n sin(theta/2) of the active R;
  * in X the (1,3) entry is R_31 + R_13 (printed R_31 + R_12), the (2,2)
    entry of the quaternion form is -q1^2 + q2^2 - q3^2 + q4^2 (printed with
    "q^2"), and theta needs the square root of q1^2 + q2^2 + q3^2;
  * the (2,1) entry of the printed SU(2) matrix carries a sign error (as
    printed the matrix is not unitary); the matrix used is
    exp(-i theta/2 n.sigma), which satisfies U sigma_j U^+ = sum_k R_kj sigma_k
    for the active R, i.e. it rotates spin expectation values with R.

Parity status: pinned by tests/test_oracle_symmetry.py (round trips over the
48 cubic operations, SU(2) homomorphism and adjoint action, unitarity, and a
brute-force real-space evaluation of the unfolded spinor).
"""
from __future__ import annotations

import numpy as np

SIGMA = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def axis_angle_matrix(n, theta) -> np.ndarray:
    """The active rotation by theta about the unit vector n (the Euler
    axis/angle matrix of the paper)."""
    n = np.asarray(n, float)
    c, s = np.cos(theta), np.sin(theta)
    nx, ny, nz = n
    return np.array([
        [c + nx * nx * (1 - c), -nz * s + nx * ny * (1 - c), ny * s + nx * nz * (1 - c)],
        [nz * s + ny * nx * (1 - c), c + ny * ny * (1 - c), -nx * s + ny * nz * (1 - c)],
        [-ny * s + nz * nx * (1 - c), nx * s + nz * ny * (1 - c), c + nz * nz * (1 - c)],
    ])


def quaternion(R) -> np.ndarray:
    """Unit quaternion (q1, q2, q3, q4) = (n sin(theta/2), cos(theta/2)) of the
    proper active rotation R, by Markley's modification of Shepperd's
    algorithm applied to the attitude matrix A = R^T; positive branch."""
    A = np.asarray(R, float).T
    tr = np.trace(A)
    X = np.array([
        [1 + 2 * A[0, 0] - tr, A[1, 0] + A[0, 1], A[2, 0] + A[0, 2], A[1, 2] - A[2, 1]],
        [A[0, 1] + A[1, 0], 1 + 2 * A[1, 1] - tr, A[2, 1] + A[1, 2], A[2, 0] - A[0, 2]],
        [A[0, 2] + A[2, 0], A[1, 2] + A[2, 1], 1 + 2 * A[2, 2] - tr, A[0, 1] - A[1, 0]],
        [A[1, 2] - A[2, 1], A[2, 0] - A[0, 2], A[0, 1] - A[1, 0], 1 + tr],
    ])
    norms = np.linalg.norm(X, axis=0)
    i = int(np.argmax(norms))
    return X[:, i] / norms[i]


def axis_angle(q) -> tuple[np.ndarray, float]:
    """(n, theta) from a unit quaternion: theta = 2 arctan(|q_vec| / q4) with
    the two-argument arctangent (theta in [0, 2 pi]); n = (0, 0, 1) for the
    identity."""
    v = np.asarray(q[:3], float)
    s = np.linalg.norm(v)
    theta = 2.0 * np.arctan2(s, q[3])
    n = v / s if s > 0 else np.array([0.0, 0.0, 1.0])
    return n, float(theta)


def su2(n, theta) -> np.ndarray:
    """exp(-i theta/2 n.sigma) = cos(theta/2) I - i sin(theta/2) n.sigma."""
    n = np.asarray(n, float)
    return np.cos(theta / 2) * np.eye(2) - 1j * np.sin(theta / 2) * np.einsum("i,ijk->jk", n, SIGMA)


def cartesian(avec, rot_lat) -> np.ndarray:
    """R_cart = A R_lat A^-1 with A the lattice vectors as columns (avec has
    them as rows)."""
    A = np.asarray(avec, float).T
    return A @ np.asarray(rot_lat, float) @ np.linalg.inv(A)


def spin_matrix(avec, rot_lat) -> np.ndarray:
    """SU(2) matrix of a lattice-basis symmetry: the proper part of its
    Cartesian rotation (times -1 if det = -1) through its quaternion."""
    R = cartesian(avec, rot_lat)
    if np.linalg.det(R) < 0:
        R = -R
    n, theta = axis_angle(quaternion(R))
    return su2(n, theta)


def unfold(coeff, gvec, avec, rot_lat, tau):
    """c~(G') for the symmetry {R|tau}: coeff [nb][2][ngw] on the Miller list
    gvec [ngw][3] at k; returns (coeff', gvec') at Rk with gvec'_i = R h_i in
    Miller indices (h' = R_lat^-T h) and
        coeff'[n][a][i] = e^{-2 pi i h'_i . tau} sum_b U[a][b] coeff[n][b][i],
    tau in crystal coordinates."""
    M = np.rint(np.linalg.inv(np.asarray(rot_lat, float)).T).astype(np.int64)
    g2 = np.asarray(gvec, np.int64) @ M.T
    phase = np.exp(-2j * np.pi * (g2 @ np.asarray(tau, float)))
    U = spin_matrix(avec, rot_lat)
    out = np.einsum("ab,nbi->nai", U, np.asarray(coeff, np.complex128)) * phase[None, None, :]
    return out, g2.astype(np.int32)


def cubic_operations() -> list[np.ndarray]:
    """The 48 operations of the cube (signed permutation matrices), Cartesian."""
    import itertools
    ops = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3))
            for i, j in enumerate(perm):
                R[i, j] = signs[i]
            ops.append(R)
    return ops
