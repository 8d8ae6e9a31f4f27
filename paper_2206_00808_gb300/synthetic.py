"""Seeded synthetic inputs for the spinor polarizability chi0.

This module builds *inputs* only: a crystal cell, a Gamma-centred k-grid,
plane-wave G-spheres, spinor plane-wave coefficients, band energies and
imaginary-axis frequencies.  It holds none of the method's arithmetic (no
matrix element, no FFT, no energy denominator, no contraction): both the CUDA
path and the CPU oracle consume what it returns.

Shapes follow the paper's statement of the problem:
  * spinor states psi_nk = sum_alpha phi_nk,alpha |alpha>, normalised over both
    components together (Sec. II);
  * plane-wave form u_nk,alpha(r) = sum_G c_nk,alpha(G) e^{iG.r} (Sec. III.A);
  * the polarizability needs occupied bands at one k and empty bands at
    another, band energies, a momentum transfer q and a dielectric G-sphere
    (Sec. II, the polarizability formula and Eq. matrix_el).

Recipe (all seeded through numpy's SeedSequence([config_id, k_index, stream])):
  * coefficients: complex128 Gaussians of shape (2*N_w(k), N_v + N_c),
    orthonormalised column-wise by a thin QR over the stacked [up; down]
    components, so every band is unit-normalised over both spinor components
    and the bands at one k are mutually orthonormal;
  * energies (eV): valence U[-12, 0], conduction U[1.1, 30], each sorted;
  * frequencies (eV): omega_j = linspace(0, 40, N_omega) on the imaginary axis
    (omega = 0 alone for a static run).
Cell sizes come from the paper's parameter table (Si-like FCC a = 10.26 bohr;
GaSb-like FCC a = 6.10 Angstrom = 11.53 bohr); the paper's DFT wavefunctions
are not available, so these seeded states stand in for them.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

__all__ = [
    "Problem", "fcc_cell", "rhombohedral_cell", "reciprocal", "kgrid_points",
    "wfn_sphere", "eps_sphere", "spinor_coefficients", "band_energies",
    "make_problem", "make_batched_problem", "make_bi2se3_problem", "spinor_coefficients_device",
    "CONFIGS", "spinless_to_spinor", "rotate_spin",
    "plane_wave_bands", "fill_coefficients",
]


# ----------------------------------------------------------------- geometry --

def fcc_cell(a: float) -> np.ndarray:
    """FCC primitive vectors (rows, bohr) for cubic lattice constant a."""
    return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


def rhombohedral_cell(a_hex: float, c_hex: float) -> np.ndarray:
    """Rhombohedral primitive vectors (rows, bohr) from hexagonal a and c."""
    a, c = a_hex, c_hex
    return np.array([
        [a / 2.0, -a / (2.0 * np.sqrt(3.0)), c / 3.0],
        [0.0, a / np.sqrt(3.0), c / 3.0],
        [-a / 2.0, -a / (2.0 * np.sqrt(3.0)), c / 3.0],
    ])


def reciprocal(avec: np.ndarray) -> np.ndarray:
    """Reciprocal vectors (rows, 1/bohr): B = 2 pi A^{-T}."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(avec, float)).T


def kgrid_points(n) -> np.ndarray:
    """Gamma-centred grid j_i/n_i in crystal coordinates, lexicographic order."""
    n1, n2, n3 = (int(x) for x in n)
    pts = [(i / n1, j / n2, l / n3) for i in range(n1) for j in range(n2) for l in range(n3)]
    return np.array(pts, dtype=np.float64)


def _miller_box(bvec: np.ndarray, radius2: float, center: np.ndarray) -> np.ndarray:
    """All Miller triples that can lie within |center + h| B < sqrt(radius2):
    h_i = (center + h).a_i / 2pi - center_i, so |h_i| <= r |a_i| / 2pi + |center_i|."""
    alen = np.linalg.norm(2.0 * np.pi * np.linalg.inv(np.asarray(bvec, float)).T, axis=1)
    r = int(np.ceil(np.sqrt(radius2) * alen.max() / (2.0 * np.pi) + np.abs(center).max())) + 1
    rng = range(-r, r + 1)
    return np.array(list(itertools.product(rng, rng, rng)), dtype=np.int64)


def wfn_sphere(bvec: np.ndarray, k: np.ndarray, ecut_ry: float) -> np.ndarray:
    """Miller indices h with |(k + h) B|^2 < ecut (Rydberg), lexicographic."""
    h = _miller_box(bvec, ecut_ry, np.asarray(k))
    e = (((np.asarray(k)[None, :] + h) @ bvec) ** 2).sum(1)
    s = h[e < ecut_ry]
    order = np.lexsort((s[:, 2], s[:, 1], s[:, 0]))
    return np.ascontiguousarray(s[order].astype(np.int32))


def eps_sphere(bvec: np.ndarray, q: np.ndarray, ng: int) -> np.ndarray:
    """The ng Miller vectors with the smallest |(q + h) B|^2; ties broken by
    lexicographic h, so a shell-closing ng equals the |q+G|^2 < Ecut sphere."""
    radius2 = 1.0
    while True:
        h = _miller_box(bvec, radius2, np.asarray(q))
        e = (((np.asarray(q)[None, :] + h) @ bvec) ** 2).sum(1)
        if (e < radius2).sum() >= ng:
            break
        radius2 *= 2.0
    e = np.round(e, 10)
    order = np.lexsort((h[:, 2], h[:, 1], h[:, 0], e))
    return np.ascontiguousarray(h[order[:ng]].astype(np.int32))


# ------------------------------------------------------------ wavefunctions --

def _rng(config_id: int, ik: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(config_id), int(ik), int(stream)]))


def spinor_coefficients(config_id: int, ik: int, ngw: int, nbands: int) -> np.ndarray:
    """Orthonormal spinor coefficients, complex128 [nbands][2][ngw]."""
    rng = _rng(config_id, ik, 0)
    z = rng.standard_normal((2 * ngw, nbands)) + 1j * rng.standard_normal((2 * ngw, nbands))
    qmat, _ = np.linalg.qr(z, mode="reduced")
    return np.ascontiguousarray(qmat.T.reshape(nbands, 2, ngw))


def band_energies(config_id: int, ik: int, nv: int, nc: int) -> np.ndarray:
    """Sorted band energies in eV: valence U[-12,0], conduction U[1.1,30]."""
    rng = _rng(config_id, ik, 1)
    ev = np.sort(rng.uniform(-12.0, 0.0, nv))
    ec = np.sort(rng.uniform(1.1, 30.0, nc))
    return np.concatenate([ev, ec]).astype(np.float64)


def spinless_to_spinor(phi: np.ndarray) -> np.ndarray:
    """Spinless orbitals phi [nb][ngw] -> spinors [2nb][2][ngw]: phi x |up>
    for band 2i and phi x |down> for band 2i+1."""
    nb, ngw = phi.shape
    out = np.zeros((2 * nb, 2, ngw), dtype=np.complex128)
    out[0::2, 0, :] = phi
    out[1::2, 1, :] = phi
    return out


def rotate_spin(coeff: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Apply one 2x2 unitary to the (up, down) components of every band."""
    return np.einsum("ab,nbg->nag", u, coeff)


def plane_wave_bands(gvec: np.ndarray, picks) -> np.ndarray:
    """Bands that are single plane waves: picks = [(sphere index, alpha), ...]."""
    out = np.zeros((len(picks), 2, len(gvec)), dtype=np.complex128)
    for n, (ig, a) in enumerate(picks):
        out[n, a, ig] = 1.0
    return out


# ----------------------------------------------------------------- problems --

@dataclasses.dataclass
class Problem:
    """One chi0(q, i omega) workload: everything the C-ABI takes."""
    name: str
    avec: np.ndarray            # (3,3) bohr, rows a_i
    box: tuple                  # FFT box (N1, N2, N3)
    kgrid: tuple                # (n1, n2, n3)
    kcrys: np.ndarray           # (Nk, 3) crystal coordinates
    nv: int
    nc: int                     # conduction bands per k held (nc_max)
    gvec: list                  # per k: (N_w(k), 3) int32 Miller indices
    coeff: list                 # per k: complex128 [nv+nc][2][N_w(k)]
    energy: list                # per k: float64 [nv+nc] eV
    qs: list                    # list of (q crystal (3,), eps sphere (N_G,3) int32, nc(q))
    freq: np.ndarray            # (N_omega,) eV, imaginary-axis magnitudes
    precision: str = "fp64"
    config_id: int = -1         # seed of the coefficient generator (fill_coefficients)

    @property
    def nk(self) -> int:
        return len(self.kcrys)

    @property
    def nbands(self) -> int:
        return self.nv + self.nc

    def pairs(self, iq: int = 0) -> int:
        return self.nk * self.nv * self.qs[iq][2]


def _coefficients(config_id, ik, ngw, nbands, on):
    """Coefficients of one k: numpy ("host"), torch on a CUDA device ("cuda"),
    or None (generated later by fill_coefficients)."""
    if on is None:
        return None
    if on == "host":
        return spinor_coefficients(config_id, ik, ngw, nbands)
    return spinor_coefficients_device(config_id, ik, ngw, nbands, on)


def fill_coefficients(p: "Problem", ks, on="host"):
    """Generate the coefficients of k-points `ks` of a problem made with
    coeff_on=None (or replace them), on the host or a CUDA device."""
    for ik in ks:
        p.coeff[ik] = _coefficients(p.config_id, ik, len(p.gvec[ik]), p.nbands, on)
    return p


def _fcc_problem(name, config_id, a, box, ecut_wfn, ng, kgrid, nv, nc, q, nfreq,
                 precision, coeff_on="host"):
    avec = fcc_cell(a)
    bvec = reciprocal(avec)
    kc = kgrid_points(kgrid)
    gvec, coeff, energy = [], [], []
    for ik in range(len(kc)):
        g = wfn_sphere(bvec, kc[ik], ecut_wfn)
        gvec.append(g)
        coeff.append(_coefficients(config_id, ik, len(g), nv + nc, coeff_on))
        energy.append(band_energies(config_id, ik, nv, nc))
    q = np.asarray(q, float)
    qs = [(q, eps_sphere(bvec, q, ng), nc)]
    freq = np.linspace(0.0, 40.0, nfreq) if nfreq > 1 else np.zeros(1)
    return Problem(name, avec, tuple(box), tuple(kgrid), kc, nv, nc, gvec, coeff, energy,
                   qs, freq, precision, config_id)


# Workloads: Si-like (FCC 10.26 bohr) and GaSb-like (FCC 11.53 bohr) cells from
# the paper's parameter table; sizes as listed in the module docstring.
CONFIGS = {
    "si16_q0": dict(config_id=0, a=10.26, box=(16, 16, 16), ecut_wfn=28.1, ng=137,
                    kgrid=(2, 2, 2), nv=8, nc=24, q=(0, 0, 0), nfreq=1, precision="fp64"),
    "si18_qx": dict(config_id=0, a=10.26, box=(18, 18, 18), ecut_wfn=28.1, ng=137,
                    kgrid=(2, 2, 2), nv=8, nc=24, q=(0.5, 0, 0), nfreq=1, precision="fp64"),
    "si24": dict(config_id=1, a=10.26, box=(24, 24, 24), ecut_wfn=58.0, ng=350,
                 kgrid=(4, 4, 4), nv=8, nc=200, q=(0.25, 0, 0), nfreq=5, precision="fp64"),
    "gasb32": dict(config_id=2, a=11.53, box=(32, 32, 32), ecut_wfn=85.0, ng=800,
                   kgrid=(6, 6, 6), nv=18, nc=400, q=(1 / 6, 0, 0), nfreq=16, precision="mixed"),
}


def make_batched_problem(config_id: int = 3, a: float = 11.53, box=(32, 32, 32),
                         ecut_wfn: float = 85.0, kgrid=(6, 6, 6), nv: int = 18, nq: int = 40,
                         ng_range=(700, 900), nc_range=(300, 500), nfreq: int = 16,
                         precision: str = "mixed") -> Problem:
    """Many q-points of one k-grid with ragged sizes: q = the first nq grid
    vectors after Gamma in lexicographic order; per q a dielectric sphere of
    N_G(q) ~ U{ng_range} smallest |q+G|^2 and N_c(q) ~ U{nc_range} conduction
    bands (seeded).  Bands are generated for the largest N_c."""
    rng = _rng(config_id, 0, 2)
    ngs = rng.integers(ng_range[0], ng_range[1] + 1, nq)
    ncs = rng.integers(nc_range[0], nc_range[1] + 1, nq)
    nc_max = int(ncs.max())
    p = _fcc_problem(f"batch{nq}", config_id, a, box, ecut_wfn, int(ngs[0]), kgrid, nv, nc_max,
                     (0.0, 0.0, 0.0), nfreq, precision)
    bvec = reciprocal(p.avec)
    qpts = kgrid_points(kgrid)[1:nq + 1]
    p.qs = [(q, eps_sphere(bvec, q, int(ng)), int(nc)) for q, ng, nc in zip(qpts, ngs, ncs)]
    return p


BOHR_PER_ANGSTROM = 1.0 / 0.529177210903


def spinor_coefficients_device(config_id: int, ik: int, ngw: int, nbands: int, device="cuda"):
    """Orthonormal spinor coefficients generated on a CUDA device with torch
    (complex128 [nbands][2][ngw]); same recipe as spinor_coefficients, for
    sizes whose host QR would take too long.  Seeded per (config, k)."""
    import torch
    seed = int(np.random.SeedSequence([int(config_id), int(ik), 0]).generate_state(1)[0])
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    z = torch.randn((2 * ngw, nbands), dtype=torch.complex128, generator=g, device=device)
    q, _ = torch.linalg.qr(z, mode="reduced")
    return q.T.reshape(nbands, 2, ngw).contiguous()


def make_bi2se3_problem(config_id: int = 4, box=(64, 64, 64), ecut_wfn: float = 67.9, ng: int = 2000,
                        kgrid=(6, 6, 6), nv: int = 48, nc: int = 1000, q=(1 / 6, 0, 0),
                        nfreq: int = 8, device="cuda") -> Problem:
    """Bi2Se3-like rhombohedral cell (hexagonal a = 4.143 A, c = 28.636 A),
    64^3 box, ~9000 plane waves per spinor component, N_G = 2000; the
    coefficients are generated on the device (torch tensors), or not at all
    with device=None (fill_coefficients makes them per k)."""
    avec = rhombohedral_cell(4.143 * BOHR_PER_ANGSTROM, 28.636 * BOHR_PER_ANGSTROM)
    bvec = reciprocal(avec)
    kc = kgrid_points(kgrid)
    gvec, coeff, energy = [], [], []
    for ik in range(len(kc)):
        gk = wfn_sphere(bvec, kc[ik], ecut_wfn)
        gvec.append(gk)
        coeff.append(None if device is None else spinor_coefficients_device(config_id, ik, len(gk), nv + nc,
                                                                            device))
        energy.append(band_energies(config_id, ik, nv, nc))
    qv = np.asarray(q, float)
    freq = np.linspace(0.0, 40.0, nfreq) if nfreq > 1 else np.zeros(1)
    p = Problem("bi2se3", avec, tuple(box), tuple(kgrid), kc, nv, nc, gvec, coeff, energy,
                [(qv, eps_sphere(bvec, qv, ng), nc)], freq, "mixed", config_id)
    return p


def make_problem(name: str, **overrides) -> Problem:
    """Build a named workload; `overrides` change any of its sizes, and
    coeff_on = "host" (default, numpy), "cuda" (torch on the device) or None
    (no coefficients yet: fill_coefficients) says where the coefficients are
    made."""
    spec = dict(CONFIGS[name])
    spec.update(overrides)
    return _fcc_problem(name, **spec)
