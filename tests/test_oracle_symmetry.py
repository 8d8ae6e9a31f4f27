"""Pins of the oracle's spinor symmetry unfolding (oracle/symmetry.py): the
quaternion / axis-angle round trip over the 48 cubic operations and random
rotations, unitarity, the SU(2) homomorphism and adjoint action, the lattice
to Cartesian change of basis, and a brute-force real-space evaluation of an
unfolded spinor Bloch function."""
import numpy as np
import pytest

from oracle import symmetry as sym
from paper_2206_00808_gb300 import synthetic as syn


def proper(R):
    return -R if np.linalg.det(R) < 0 else R


def random_rotation(rng):
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    return sym.axis_angle_matrix(n, rng.uniform(0, 2 * np.pi))


def test_round_trip_cubic_operations():
    ops = sym.cubic_operations()
    assert len(ops) == 48
    for R in ops:
        P = proper(R)
        q = sym.quaternion(P)
        assert abs(np.linalg.norm(q) - 1) < 1e-15
        n, theta = sym.axis_angle(q)
        assert 0 <= theta <= 2 * np.pi
        assert np.abs(sym.axis_angle_matrix(n, theta) - P).max() < 1e-14


def test_round_trip_random_and_singular_angles():
    rng = np.random.default_rng(4)
    cases = [random_rotation(rng) for _ in range(200)]
    cases += [np.eye(3), np.diag([1.0, -1.0, -1.0]), np.diag([-1.0, 1.0, -1.0]),
              sym.axis_angle_matrix([1 / np.sqrt(2), 1 / np.sqrt(2), 0], np.pi),
              sym.axis_angle_matrix([0, 0, 1], 1e-9), sym.axis_angle_matrix([0, 1, 0], np.pi - 1e-9)]
    for R in cases:
        n, theta = sym.axis_angle(sym.quaternion(R))
        assert np.abs(sym.axis_angle_matrix(n, theta) - R).max() < 1e-13


def test_su2_unitary_and_adjoint_action():
    rng = np.random.default_rng(5)
    for R in [proper(R) for R in sym.cubic_operations()] + [random_rotation(rng) for _ in range(50)]:
        U = sym.su2(*sym.axis_angle(sym.quaternion(R)))
        assert np.abs(U @ U.conj().T - np.eye(2)).max() < 1e-14
        assert abs(np.linalg.det(U) - 1) < 1e-14
        # a spin's expectation vector turns with R: U sigma_j U^+ = sum_k R_kj sigma_k
        for j in range(3):
            lhs = U @ sym.SIGMA[j] @ U.conj().T
            rhs = np.einsum("k,kab->ab", R[:, j], sym.SIGMA)
            assert np.abs(lhs - rhs).max() < 1e-14


def test_su2_homomorphism_on_the_rotation_group_of_the_cube():
    ops = [proper(R) for R in sym.cubic_operations()]
    U = {i: sym.su2(*sym.axis_angle(sym.quaternion(R))) for i, R in enumerate(ops)}
    for i, R1 in enumerate(ops):
        for j, R2 in enumerate(ops):
            U12 = sym.su2(*sym.axis_angle(sym.quaternion(R1 @ R2)))
            prod = U[i] @ U[j]
            assert min(np.abs(U12 - prod).max(), np.abs(U12 + prod).max()) < 1e-13


def test_fcc_lattice_operations_map_back_to_cartesian():
    avec = syn.fcc_cell(10.26)
    A = avec.T
    for R in sym.cubic_operations():
        R_lat = np.linalg.inv(A) @ R @ A
        assert np.abs(R_lat - np.rint(R_lat)).max() < 1e-12       # FCC has the full cubic group
        assert np.abs(sym.cartesian(avec, np.rint(R_lat)) - R).max() < 1e-12
        S = sym.spin_matrix(avec, np.rint(R_lat))
        Uref = sym.su2(*sym.axis_angle(sym.quaternion(proper(R))))
        assert np.abs(S - Uref).max() < 1e-13


def _bloch(coeff, gvec, k, B, r):
    """psi[n][alpha](r) = sum_G c(G) e^{i (k+G).r} at Cartesian points r (npt, 3)."""
    kc = (np.asarray(gvec, float) + k) @ B                       # (ngw, 3) Cartesian k+G
    ph = np.exp(1j * r @ kc.T)                                   # (npt, ngw)
    return np.einsum("pi,nai->pna", ph, coeff)


@pytest.mark.parametrize("op_index", [1, 7, 13, 22, 30, 47])
def test_unfolded_spinor_by_real_space_brute_force(op_index):
    """psi'_{Rk}(R r + tau) = e^{i Rk.tau} U psi_k(r) for the unfolded
    coefficients (the dropped common phase put back)."""
    rng = np.random.default_rng(op_index)
    avec = syn.fcc_cell(10.26)
    A = avec.T
    B = syn.reciprocal(avec)                                     # rows b_i
    R = sym.cubic_operations()[op_index]
    R_lat = np.rint(np.linalg.inv(A) @ R @ A)
    tau = np.array([0.25, 0.25, 0.25])                           # crystal coordinates
    k = np.array([0.25, 0.0, 0.5])
    gvec = syn.wfn_sphere(B, k, 3.0)
    c = rng.normal(size=(2, 2, len(gvec))) + 1j * rng.normal(size=(2, 2, len(gvec)))
    c2, g2 = sym.unfold(c, gvec, avec, R_lat, tau)
    k2 = np.linalg.inv(R_lat).T @ k                              # Rk in crystal coordinates of B
    r = rng.uniform(-5, 5, size=(7, 3))
    tau_c = A @ tau
    lhs = _bloch(c2, g2, k2, B, r @ R.T + tau_c)
    kc2 = k2 @ B
    U = sym.spin_matrix(avec, R_lat)
    rhs = np.exp(1j * kc2 @ tau_c) * np.einsum("ab,pnb->pna", U, _bloch(c, gvec, k, B, r))
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(rhs).max()
