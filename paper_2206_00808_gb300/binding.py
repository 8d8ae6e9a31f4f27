"""Thin ctypes binding of libbgwchi.so (include/bgw_chi.h), same names.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch CUDA tensors (their data_ptr is passed);
host buffers are numpy arrays or CPU tensors.  Importing this module fails
loudly when the library has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# BGW_LIBRARY=bounds loads the index-checking build (libbgwchi_bounds.so)
LIB_PATH = _build.LIB_BOUNDS if os.environ.get("BGW_LIBRARY") == "bounds" else _build.LIB
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2206_00808_gb300.build.build()")
_lib = ctypes.CDLL(LIB_PATH)

BGW_OK, BGW_E_ARG, BGW_E_STATE, BGW_E_CUDA, BGW_E_NOMEM, BGW_E_GRID, BGW_E_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
BGW_W_ALIAS = 1
BGW_FP64, BGW_MIXED_BF16X3, BGW_MIXED_TF32X3, BGW_MIXED_TF32 = 0, 1, 2, 3
PRECISIONS = {"fp64": BGW_FP64, "mixed": BGW_MIXED_BF16X3, "tf32x3": BGW_MIXED_TF32X3, "tf32": BGW_MIXED_TF32}

EXPORTED = ["bgw_version", "bgw_create", "bgw_wfn_upload", "bgw_mtxel_spinor", "bgw_chi0_reset",
            "bgw_chi0_accumulate", "bgw_chi0_finalize", "bgw_profile", "bgw_profile_read",
            "bgw_mtxel_spinor_noalloc", "bgw_set_option", "bgw_get_option", "bgw_autotune",
            "bgw_graph_begin", "bgw_graph_end", "bgw_graph_launch", "bgw_chi0_progress",
            "bgw_chi0_checkpoint_bytes", "bgw_chi0_checkpoint", "bgw_chi0_resume", "bgw_coulomb_sqrt",
            "bgw_epsinv_workspace_bytes", "bgw_epsinv", "bgw_symmetry_su2", "bgw_unfold_spinor",
            "bgw_mtxel_bands", "bgw_sigma_cohsex", "bgw_bse_kernel", "bgw_bounds_check", "bgw_destroy",
            "bgw_last_error"]
BGW_OPT_KCHUNK, BGW_OPT_PAIR_TILE_V, BGW_OPT_PAIR_TILE_C, BGW_OPT_GRID_SLOTS = 1, 2, 3, 4
BGW_OPT_TEST_DROP_LOAD, BGW_OPT_TEST_FAIL_ALLOC, BGW_OPT_K1_PATH, BGW_OPT_MTXEL_LANES = 5, 6, 7, 8
BGW_OPT_DEFER_K1, BGW_OPT_COPY_AHEAD, BGW_OPT_OVERLAP, BGW_OPT_FP64_CONTRACTION = 9, 10, 11, 12
BGW_OPT_MTXEL_ZY = 13
STAGES = ["wfn_to_grid", "mtxel", "weights", "contraction", "finalize", "operand_split", "mtxel_x"]


class bgw_q(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double * 3), ("ng", ctypes.c_int), ("gvec", ctypes.c_void_p),
                ("nc", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_lib.bgw_version.argtypes, _lib.bgw_version.restype = [], ctypes.c_char_p
_lib.bgw_create.argtypes = [ctypes.POINTER(_P), _P, _I, _P, _I, _I, _I, _P]
_lib.bgw_wfn_upload.argtypes = [_P, _I, _I, _P, _P, _P, _I]
_lib.bgw_mtxel_spinor.argtypes = [_P, ctypes.POINTER(bgw_q), _I, _I, _I, _I, _I, _P]
_lib.bgw_chi0_reset.argtypes = [_P]
_lib.bgw_chi0_accumulate.argtypes = [_P, _I, ctypes.POINTER(bgw_q), _I, _P, _I, _I]
_lib.bgw_chi0_finalize.argtypes = [_P, _I, _P, _I]
_lib.bgw_profile.argtypes = [_P, _I]
_lib.bgw_profile_read.argtypes = [_P, _P, _P, _P, _I]
_lib.bgw_mtxel_spinor_noalloc.argtypes = [_P, _P, _P, _I, _I, _P, _I, _P, _P, _P]
_lib.bgw_set_option.argtypes = [_P, _I, ctypes.c_long]
_lib.bgw_get_option.argtypes = [_P, _I, ctypes.POINTER(ctypes.c_long)]
_lib.bgw_autotune.argtypes = [_P, _I, ctypes.POINTER(bgw_q), _I, _P, _I, _I, ctypes.c_char_p]
for _f in ["bgw_graph_begin", "bgw_graph_end", "bgw_graph_launch"]:
    getattr(_lib, _f).argtypes = [_P]
    getattr(_lib, _f).restype = ctypes.c_int
_lib.bgw_chi0_progress.argtypes = [_P, _P]
_lib.bgw_chi0_checkpoint_bytes.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t)]
_lib.bgw_chi0_checkpoint.argtypes = [_P, _P, ctypes.c_size_t]
_lib.bgw_chi0_resume.argtypes = [_P, _I, ctypes.POINTER(bgw_q), _I, _P, _P, ctypes.c_size_t]
_lib.bgw_coulomb_sqrt.argtypes, _lib.bgw_coulomb_sqrt.restype = [_P, _P, _I, _P, _P], ctypes.c_int
_lib.bgw_epsinv_workspace_bytes.argtypes = [_I, _I]
_lib.bgw_epsinv_workspace_bytes.restype = ctypes.c_size_t
_lib.bgw_epsinv.argtypes = [_I, _I, _P, _P, _I, _P, ctypes.c_size_t, _P]
_lib.bgw_epsinv.restype = ctypes.c_int
_lib.bgw_symmetry_su2.argtypes, _lib.bgw_symmetry_su2.restype = [_P, _P, _P, _P], ctypes.c_int
_lib.bgw_unfold_spinor.argtypes = [_P, _P, _P, _I, _I, _P, _P, _P, _P, _P]
_lib.bgw_unfold_spinor.restype = ctypes.c_int
_lib.bgw_mtxel_bands.argtypes = [_P, ctypes.POINTER(bgw_q), _I, _I, _I, _I, _I, _P]
_lib.bgw_sigma_cohsex.argtypes = [_P, ctypes.POINTER(bgw_q), _I, _I, _I, _P, _P, _P, _P]
_lib.bgw_bse_kernel.argtypes = [_P, _I, _I, ctypes.POINTER(bgw_q), _P, ctypes.POINTER(bgw_q), _P, _I, _I, _I, _I,
                                _P, _P]
_lib.bgw_bounds_check.argtypes, _lib.bgw_bounds_check.restype = [ctypes.POINTER(ctypes.c_uint)], ctypes.c_int
for _f in ["bgw_mtxel_bands", "bgw_sigma_cohsex", "bgw_bse_kernel"]:
    getattr(_lib, _f).restype = ctypes.c_int
_lib.bgw_destroy.argtypes, _lib.bgw_destroy.restype = [_P], None
_lib.bgw_last_error.argtypes, _lib.bgw_last_error.restype = [_P], ctypes.c_char_p
for _f in ["bgw_create", "bgw_wfn_upload", "bgw_mtxel_spinor", "bgw_chi0_reset",
           "bgw_chi0_accumulate", "bgw_chi0_finalize", "bgw_profile", "bgw_profile_read",
           "bgw_mtxel_spinor_noalloc", "bgw_set_option", "bgw_get_option", "bgw_autotune",
           "bgw_chi0_progress", "bgw_chi0_checkpoint_bytes", "bgw_chi0_checkpoint", "bgw_chi0_resume"]:
    getattr(_lib, _f).restype = ctypes.c_int


class BgwError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"bgw status {status}: {message}")
        self.status = status


def _check(status: int, ctx) -> int:
    if status < 0:
        raise BgwError(status, bgw_last_error(ctx))
    return status


def _host_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ptr_and_device(x):
    """(pointer, on_device) for a numpy array or a torch tensor."""
    if isinstance(x, np.ndarray):
        return _host_ptr(x), 0
    import torch
    if isinstance(x, torch.Tensor):
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_handle(stream):
    """cudaStream_t of a torch stream (None: torch's current stream when CUDA
    is up, else the default stream)."""
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return ctypes.c_void_p(0)
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def make_q(q, gvec: np.ndarray, nc: int):
    """A bgw_q struct plus the array that must outlive the call using it."""
    g = np.ascontiguousarray(gvec, dtype=np.int32)
    s = bgw_q((ctypes.c_double * 3)(*[float(x) for x in q]), len(g), _host_ptr(g), int(nc))
    return s, g


def bgw_version() -> str:
    return _lib.bgw_version().decode()


def bgw_last_error(ctx) -> str:
    m = _lib.bgw_last_error(ctx)
    return m.decode() if m else ""


def bgw_create(fft, kcrys, nv: int, nc_max: int, precision="fp64", stream=None):
    fft = np.ascontiguousarray(fft, dtype=np.int32)
    kc = np.ascontiguousarray(kcrys, dtype=np.float64)
    prec = PRECISIONS.get(precision, precision)
    ctx = ctypes.c_void_p()
    _check(_lib.bgw_create(ctypes.byref(ctx), _host_ptr(fft), len(kc), _host_ptr(kc), nv, nc_max,
                           prec, _stream_handle(stream)), None)
    return ctx


def bgw_wfn_upload(ctx, ik: int, gvec, coeff, energy) -> int:
    """coeff complex128 [nb][2][ngw] and energy float64 [nb], both host or both device."""
    g = np.ascontiguousarray(gvec, dtype=np.int32)
    pc, dc = _ptr_and_device(coeff)
    pe, de = _ptr_and_device(energy)
    if dc != de:
        raise ValueError("coeff and energy must both be host or both be device buffers")
    return _check(_lib.bgw_wfn_upload(ctx, ik, len(g), _host_ptr(g), pc, pe, dc), ctx)


def bgw_mtxel_spinor(ctx, q, gvec, ik: int, v0: int, nv: int, c0: int, nc: int, M_dev) -> int:
    s, keep = make_q(q, gvec, nc if nc > 0 else 1)
    pm, dm = _ptr_and_device(M_dev)
    if not dm:
        raise ValueError("M_dev must be a device tensor")
    st = _lib.bgw_mtxel_spinor(ctx, ctypes.byref(s), ik, v0, nv, c0, nc, pm)
    del keep
    return _check(st, ctx)


def bgw_chi0_reset(ctx) -> int:
    return _check(_lib.bgw_chi0_reset(ctx), ctx)


def bgw_chi0_accumulate(ctx, qs, freq, k_begin: int, k_end: int) -> int:
    """qs: list of (q, gvec, nc)."""
    structs, keep = [], []
    for q, g, nc in qs:
        s, a = make_q(q, g, nc)
        structs.append(s)
        keep.append(a)
    arr = (bgw_q * len(structs))(*structs)
    f = np.ascontiguousarray(freq, dtype=np.float64)
    return _check(_lib.bgw_chi0_accumulate(ctx, len(structs), arr, len(f), _host_ptr(f),
                                           k_begin, k_end), ctx)


def bgw_chi0_finalize(ctx, iq: int, out) -> int:
    """out: complex128 [nfreq][ng][ng], a device tensor (async) or host array (blocking)."""
    p, d = _ptr_and_device(out)
    return _check(_lib.bgw_chi0_finalize(ctx, iq, p, d), ctx)


def bgw_chi0_progress(ctx, nk: int) -> np.ndarray:
    """Per-k count of accumulate calls in the running sum."""
    out = np.zeros(nk, dtype=np.int32)
    _check(_lib.bgw_chi0_progress(ctx, _host_ptr(out)), ctx)
    return out


def bgw_chi0_checkpoint(ctx) -> bytes:
    """The running sum as a checkpoint (bytes)."""
    n = ctypes.c_size_t(0)
    _check(_lib.bgw_chi0_checkpoint_bytes(ctx, ctypes.byref(n)), ctx)
    buf = np.empty(n.value, dtype=np.uint8)
    _check(_lib.bgw_chi0_checkpoint(ctx, _host_ptr(buf), n.value), ctx)
    return buf.tobytes()


def bgw_chi0_resume(ctx, qs, freq, data: bytes) -> int:
    """Start the running sum from a checkpoint of the same problem and q-set."""
    structs, keep = [], []
    for q, g, nc in qs:
        s, a = make_q(q, g, nc)
        structs.append(s)
        keep.append(a)
    arr = (bgw_q * len(structs))(*structs)
    f = np.ascontiguousarray(freq, dtype=np.float64)
    b = np.frombuffer(data, dtype=np.uint8)
    return _check(_lib.bgw_chi0_resume(ctx, len(structs), arr, len(f), _host_ptr(f), _host_ptr(b),
                                       len(b)), ctx)


EPSINV_MODES = {"epsinv_sym": 0, "W": 1, "epsinv": 2}


def bgw_coulomb_sqrt(avec, q, gvec) -> np.ndarray:
    """sqrt(v(q+G)) in eV^1/2 for the sphere gvec (ng, 3), cell rows avec (bohr)."""
    a = np.ascontiguousarray(np.asarray(avec, dtype=np.float64).reshape(9))
    qq = np.ascontiguousarray(q, dtype=np.float64)
    g = np.ascontiguousarray(gvec, dtype=np.int32)
    s = np.zeros(len(g), dtype=np.float64)
    _check(_lib.bgw_coulomb_sqrt(_host_ptr(a), _host_ptr(qq), len(g), _host_ptr(g), _host_ptr(s)), None)
    return s


def bgw_epsinv_workspace_bytes(ng: int, nfreq: int) -> int:
    return int(_lib.bgw_epsinv_workspace_bytes(ng, nfreq))


def bgw_epsinv(chi_dev, s, mode="W", work=None, stream=None) -> int:
    """In place on the device tensor chi_dev (complex128 [nfreq][ng][ng]):
    eps~^-1 ("epsinv_sym"), W ("W") or the paper's eps^-1 ("epsinv")."""
    nf, ng = int(chi_dev.shape[0]), int(chi_dev.shape[1])
    sv = np.ascontiguousarray(s, dtype=np.float64)
    pw, wb = (None, 0) if work is None else (work.data_ptr(), work.numel() * work.element_size())
    return _check(_lib.bgw_epsinv(ng, nf, _host_ptr(sv), ctypes.c_void_p(chi_dev.data_ptr()),
                                  EPSINV_MODES[mode], ctypes.c_void_p(pw), wb, _stream_handle(stream)), None)


def bgw_symmetry_su2(avec, rot_lat):
    """(U complex [2][2], n [3], theta) of a lattice-basis symmetry operation."""
    a = np.ascontiguousarray(np.asarray(avec, dtype=np.float64).reshape(9))
    r = np.ascontiguousarray(np.asarray(rot_lat).reshape(9), dtype=np.int32)
    u = np.zeros(8, dtype=np.float64)
    na = np.zeros(4, dtype=np.float64)
    _check(_lib.bgw_symmetry_su2(_host_ptr(a), _host_ptr(r), _host_ptr(u), _host_ptr(na)), None)
    return u.view(np.complex128).reshape(2, 2), na[:3].copy(), float(na[3])


def bgw_unfold_spinor(avec, rot_lat, tau, gvec, c_in, c_out, stream=None) -> np.ndarray:
    """Coefficients at Rk into the device tensor c_out from c_in ([nb][2][ngw]
    complex128 on the device); returns the rotated Miller list (host)."""
    a = np.ascontiguousarray(np.asarray(avec, dtype=np.float64).reshape(9))
    r = np.ascontiguousarray(np.asarray(rot_lat).reshape(9), dtype=np.int32)
    t = np.ascontiguousarray(tau, dtype=np.float64)
    g = np.ascontiguousarray(gvec, dtype=np.int32)
    g2 = np.zeros_like(g)
    nb, ngw = int(c_in.shape[0]), int(c_in.shape[2])
    _check(_lib.bgw_unfold_spinor(_host_ptr(a), _host_ptr(r), _host_ptr(t), nb, ngw, _host_ptr(g), _host_ptr(g2),
                                  ctypes.c_void_p(c_in.data_ptr()), ctypes.c_void_p(c_out.data_ptr()),
                                  _stream_handle(stream)), None)
    return g2


def bgw_profile(ctx, enable: bool) -> int:
    return _check(_lib.bgw_profile(ctx, int(bool(enable))), ctx)


def bgw_profile_read(ctx) -> dict:
    """{stage: (device ms, launch groups, kernels)} since bgw_profile(ctx, True)."""
    n = len(STAGES)
    ms = np.zeros(n, dtype=np.float64)
    calls = np.zeros(n, dtype=np.int64)
    kern = np.zeros(n, dtype=np.int64)
    _check(_lib.bgw_profile_read(ctx, _host_ptr(ms), _host_ptr(calls), _host_ptr(kern), n), ctx)
    return {s: (float(ms[i]), int(calls[i]), int(kern[i])) for i, s in enumerate(STAGES)}


def bgw_mtxel_spinor_noalloc(fft, Uv, Uc, nv: int, nc: int, G0, gvec, M_dev, stream=None) -> int:
    """Allocation-free FP64 matrix elements from device grids Uv [nv][2][N^3]
    and Uc [nc][2][N^3] (complex128 tensors) into M_dev [nv][nc][ng]."""
    import torch
    f = np.ascontiguousarray(fft, dtype=np.int32)
    g0 = np.ascontiguousarray(G0, dtype=np.int32)
    g = np.ascontiguousarray(gvec, dtype=np.int32)
    nbox = int(np.prod(f))
    cur = torch.cuda.current_device()
    for name, t, n in (("Uv", Uv, nv * 2 * nbox), ("Uc", Uc, nc * 2 * nbox), ("M_dev", M_dev, nv * nc * len(g))):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.complex128 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous complex128 tensor")
        if t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} elements, the call needs {n}")
        if t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    pv, _ = _ptr_and_device(Uv)
    pc, _ = _ptr_and_device(Uc)
    pm, _ = _ptr_and_device(M_dev)
    return _check(_lib.bgw_mtxel_spinor_noalloc(_host_ptr(f), pv, pc, nv, nc, _host_ptr(g0), len(g),
                                                _host_ptr(g), pm, _stream_handle(stream)), None)


def bgw_mtxel_bands(ctx, q, gvec, ik: int, n0: int, nn: int, m0: int, nm: int, M_dev) -> int:
    """M_{n m}(k, q, G) for bands n0..n0+nn-1 at k and m0..m0+nm-1 at k+q
    (indices over all uploaded bands) into the device tensor M_dev [nn][nm][ng]."""
    s, keep = make_q(q, gvec, 1)
    pm, dm = _ptr_and_device(M_dev)
    if not dm:
        raise ValueError("M_dev must be a device tensor")
    st = _lib.bgw_mtxel_bands(ctx, ctypes.byref(s), ik, n0, nn, m0, nm, pm)
    del keep
    return _check(st, ctx)


def bgw_sigma_cohsex(ctx, q, gvec, ik: int, n0: int, nn: int, W_dev, vq, sx=None, coh=None):
    """Adds one q-point's static screened-exchange and Coulomb-hole shares to
    sx, coh (float64 [nn], zeros when not given) for bands n0.. at k; returns
    (sx, coh)."""
    s, keep = make_q(q, gvec, 1)
    v = np.ascontiguousarray(vq, dtype=np.float64)
    sx = np.zeros(nn) if sx is None else sx
    coh = np.zeros(nn) if coh is None else coh
    assert sx.dtype == np.float64 and coh.dtype == np.float64 and len(sx) >= nn and len(coh) >= nn
    pw, dw = _ptr_and_device(W_dev)
    if not dw:
        raise ValueError("W_dev must be a device tensor")
    _check(_lib.bgw_sigma_cohsex(ctx, ctypes.byref(s), ik, n0, nn, pw, _host_ptr(v), _host_ptr(sx), _host_ptr(coh)),
           ctx)
    del keep
    return sx, coh


def bgw_bse_kernel(ctx, ik: int, jk: int, q0, gvec0, v0_coul, qd, gvecd, W_dev, v0: int, nv: int, c0: int, nc: int,
                   KX_dev=None, KD_dev=None) -> int:
    """One (k_i, k_j) block of the exchange (KX_dev) and direct (KD_dev) BSE
    kernels, device complex128 [nv*nc][nv*nc] tensors (either may be None)."""
    s0, k0 = make_q(q0, gvec0, 1)
    sd, kd = make_q(qd, gvecd, 1)
    v = np.ascontiguousarray(v0_coul, dtype=np.float64)
    pw = ctypes.c_void_p(W_dev.data_ptr()) if W_dev is not None else None
    px = ctypes.c_void_p(KX_dev.data_ptr()) if KX_dev is not None else None
    pd = ctypes.c_void_p(KD_dev.data_ptr()) if KD_dev is not None else None
    st = _lib.bgw_bse_kernel(ctx, ik, jk, ctypes.byref(s0), _host_ptr(v), ctypes.byref(sd), pw, v0, nv, c0, nc, px,
                             pd)
    del k0, kd
    return _check(st, ctx)


def bgw_bounds_check():
    """(status, word): the index-check status word of the bounds-checking
    build, read and cleared (status BGW_E_STATE in the default build)."""
    w = ctypes.c_uint(0)
    st = _lib.bgw_bounds_check(ctypes.byref(w))
    return st, w.value


def bgw_set_option(ctx, option: int, value: int) -> int:
    return _check(_lib.bgw_set_option(ctx, option, int(value)), ctx)


def bgw_get_option(ctx, option: int) -> int:
    v = ctypes.c_long()
    _check(_lib.bgw_get_option(ctx, option, ctypes.byref(v)), ctx)
    return v.value


def bgw_autotune(ctx, qs, freq, k_begin: int, k_end: int, cache_path=None) -> dict:
    """Time candidate tiles / k-chunks, set the fastest; returns the choice."""
    structs, keep = [], []
    for q, g, nc in qs:
        s, a = make_q(q, g, nc)
        structs.append(s)
        keep.append(a)
    arr = (bgw_q * len(structs))(*structs)
    f = np.ascontiguousarray(freq, dtype=np.float64)
    cp = cache_path.encode() if cache_path else None
    _check(_lib.bgw_autotune(ctx, len(structs), arr, len(f), _host_ptr(f), k_begin, k_end, cp), ctx)
    return {"kchunk": bgw_get_option(ctx, BGW_OPT_KCHUNK),
            "pair_tile": (bgw_get_option(ctx, BGW_OPT_PAIR_TILE_V), bgw_get_option(ctx, BGW_OPT_PAIR_TILE_C)),
            "mtxel_zy": bgw_get_option(ctx, BGW_OPT_MTXEL_ZY)}


def bgw_graph_begin(ctx) -> int:
    return _check(_lib.bgw_graph_begin(ctx), ctx)


def bgw_graph_end(ctx) -> int:
    return _check(_lib.bgw_graph_end(ctx), ctx)


def bgw_graph_launch(ctx) -> int:
    return _check(_lib.bgw_graph_launch(ctx), ctx)


def bgw_destroy(ctx) -> None:
    _lib.bgw_destroy(ctx)


class Chi0Context:
    """Owns one bgw context for a synthetic Problem (marshalling helper)."""

    def __init__(self, problem, precision=None, stream=None):
        self.p = problem
        self.stream = stream
        self.precision = precision or problem.precision
        self.ctx = bgw_create(problem.box, problem.kcrys, problem.nv, problem.nc, self.precision,
                              stream)

    def upload(self, device_inputs=None, ks=None):
        """Upload every k (host numpy inputs, or device tensors given as a
        list of (coeff, energy) pairs)."""
        for ik in (range(self.p.nk) if ks is None else ks):
            if device_inputs is None:
                c = np.ascontiguousarray(self.p.coeff[ik])
                e = np.ascontiguousarray(self.p.energy[ik])
            else:
                c, e = device_inputs[ik]
            bgw_wfn_upload(self.ctx, ik, self.p.gvec[ik], c, e)

    def qlist(self):
        return [(q, g, nc) for q, g, nc in self.p.qs]

    def accumulate(self, k_begin=0, k_end=None, freq=None):
        return bgw_chi0_accumulate(self.ctx, self.qlist(), self.p.freq if freq is None else freq,
                                   k_begin, self.p.nk if k_end is None else k_end)

    def finalize(self, iq=0, out=None):
        ng = len(self.p.qs[iq][1])
        if out is None:
            out = np.zeros((len(self.p.freq), ng, ng), dtype=np.complex128)
        bgw_chi0_finalize(self.ctx, iq, out)
        return out

    def reset(self):
        bgw_chi0_reset(self.ctx)

    def autotune(self, k_begin=0, k_end=None, cache_path=None):
        return bgw_autotune(self.ctx, self.qlist(), self.p.freq, k_begin,
                            self.p.nk if k_end is None else k_end, cache_path)

    def close(self):
        if self.ctx is not None:
            bgw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
