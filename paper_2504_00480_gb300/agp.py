"""Thin Python binding of the C ABI in include/agp.h (ctypes).

Only argument marshalling happens here: torch tensors are passed to the
library as raw device pointers with their row stride, on the current torch
CUDA stream. Every step of the computation runs in the CUDA kernels of
libagp.so; if that library is missing or fails to load, every call raises.

Module-level functions carry the C names (``agp_plan_create``,
``agp_matvec``, ...). ``Plan`` bundles them for convenience.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_int32, c_int64, c_void_p

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libagp.so")

AGP_OK, AGP_EINVAL, AGP_EDOMAIN, AGP_ECUDA, AGP_ENOMEM, AGP_NOT_CONVERGED, AGP_TIMEOUT, AGP_ENAN = range(8)
AGP_F32, AGP_F64 = 0, 1
KERNELS = {"gauss": 0, "matern12": 1, "matern32": 2, "imq": 3, "sinc": 4}
PARAMS = {"ell": 0, "sigma_f": 1, "sigma_eps": 2}


class AgpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [
        ("n", c_int64), ("p", c_int), ("X", c_void_p), ("ldx", c_int64), ("P", c_int),
        ("win_ptr", POINTER(c_int)), ("win_feat", POINTER(c_int)), ("N", POINTER(c_int)),
        ("cutoff", c_int), ("sigma_os", c_int), ("kernel", c_int),
        ("ell", c_double), ("sigma_f", c_double), ("sigma_eps", c_double), ("prec", c_int),
    ]


class Profile(ctypes.Structure):
    _fields_ = [("ms", c_double * 4), ("launches", c_int64 * 4),
                ("ms_by_dim", (c_double * 4) * 4), ("timed_by_dim", (c_int64 * 4) * 4)]


STAGES = ("spread", "fft", "interp", "other")

_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "agp_plan_create": (c_int, [POINTER(c_void_p), POINTER(_Desc), c_void_p]),
    "agp_plan_destroy": (c_int, [c_void_p]),
    "agp_set_hyper": (c_int, [c_void_p, c_double, c_double, c_double, c_void_p]),
    "agp_matvec": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int, c_int, c_void_p]),
    "agp_deriv_matvec": (c_int, [c_void_p, c_int, c_void_p, c_int64, c_void_p, c_int64, c_int,
                                 c_void_p]),
    "agp_adjoint_nfft": (c_int, [c_void_p, c_int, c_void_p, c_int64, c_int, c_void_p, c_void_p]),
    "agp_nfft_real": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_int64, c_void_p]),
    "agp_plan_bins": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "agp_plan_coeffs": (c_int, [c_void_p, c_int, c_int, POINTER(c_double), c_void_p]),
    "agp_plan_query": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int), c_int, POINTER(c_int),
                               POINTER(c_int), POINTER(c_int64)]),
    "agp_pcg_solve": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int, c_double,
                              c_int, c_int, POINTER(c_int), POINTER(c_double), c_void_p]),
    "agp_nlml_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int, c_double,
                              c_int, POINTER(c_double), POINTER(c_double), c_void_p]),
    "agp_nlml_grad_seed": (c_int, [c_void_p, c_void_p, c_int, c_int, ctypes.c_uint64, c_double,
                                   c_int, POINTER(c_double), POINTER(c_double), c_void_p]),
    "agp_rademacher": (c_int, [c_int, c_int64, c_int, ctypes.c_uint64, c_void_p, c_int64,
                               c_void_p]),
    "agp_plan_landmarks": (c_int, [c_void_p, c_int, c_void_p, c_int, POINTER(c_int), c_void_p]),
    "agp_plan_set_item_points": (c_int, [c_void_p, c_int, c_void_p]),
    "agp_plan_set_tensor_cores": (c_int, [c_void_p, c_int]),
    "agp_plan_set_boundary": (c_int, [c_void_p, c_double, c_int, c_void_p]),
    "agp_plan_check": (c_int, [c_void_p, c_void_p]),
    "agp_plan_tensor_cores": (c_int, [c_void_p, POINTER(c_int)]),
    "agp_plan_kernel_families": (c_int, [c_void_p, c_int, ctypes.c_int64, POINTER(c_int),
                                         POINTER(c_int)]),
    "agp_autotune_clear_cache": (c_int, []),
    "agp_plan_autotune": (c_int, [c_void_p, c_int, c_int, POINTER(c_int), POINTER(c_double),
                                  c_void_p]),
    "agp_nlml_grad_pc": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, POINTER(c_double), c_int,
                                 c_int, c_int, c_double, c_int, POINTER(c_double),
                                 POINTER(c_double), c_void_p]),
    "agp_afn_create": (c_int, [POINTER(c_void_p), c_void_p, c_int, c_int, c_void_p]),
    "agp_afn_destroy": (c_int, [c_void_p]),
    "agp_afn_apply": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int, c_void_p]),
    "agp_afn_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int64), POINTER(c_double)]),
    "agp_afn_pattern": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "agp_pcg_solve_afn": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int,
                                  c_double, c_int, POINTER(c_int), POINTER(c_double), c_void_p]),
    "agp_nlml_grad_afn": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int,
                                  c_double, c_int, POINTER(c_double), POINTER(c_double),
                                  c_void_p]),
    "agp_dot_columns": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int,
                                POINTER(c_double), c_void_p]),
    "agp_dot_columns_static": (c_int, [c_int, c_void_p, c_int64, c_void_p, c_int64, c_int64, c_int,
                                       c_void_p, c_void_p]),
    "agp_batch_create": (c_int, [POINTER(c_void_p), POINTER(c_void_p), c_int, c_void_p]),
    "agp_batch_destroy": (c_int, [c_void_p]),
    "agp_batch_bind": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_int64), POINTER(c_void_p),
                               POINTER(c_int64), c_int, c_void_p]),
    "agp_batch_matvec": (c_int, [c_void_p, c_int, c_void_p]),
    "agp_spectra_size": (c_int, [c_void_p, c_int, POINTER(c_int64)]),
    "agp_matvec_spectra": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_int, c_int,
                                   c_void_p, c_void_p]),
    "agp_spectral_form": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p,
                                  c_void_p]),
    "agp_profile_enable": (c_int, [c_void_p, c_int]),
    "agp_profile_read": (c_int, [c_void_p, POINTER(Profile), c_int, c_void_p]),
    "agp_plan_set_wait_limit": (c_int, [c_void_p, ctypes.c_int64]),
    "agp_status_string": (ctypes.c_char_p, [c_int]),
    "agp_last_error": (ctypes.c_char_p, []),
}


def load_library(path: str = LIB_PATH):
    """Load libagp.so (built by ``paper_2504_00480_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2504_00480_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(status: int):
    if status != AGP_OK:
        lib = load_library()
        raise AgpError(status, f"{lib.agp_status_string(status).decode()}: "
                               f"{lib.agp_last_error().decode()}")


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _block(t: torch.Tensor, dtype, what: str):
    """(pointer, leading dimension, R) of an [n][R] RHS-minor block."""
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{what} must be {dtype}, got {t.dtype}")
    if t.dim() == 1:
        if t.stride(0) != 1:
            raise ValueError(f"{what} must be contiguous")
        return t.data_ptr(), 1, 1
    if t.dim() != 2 or (t.stride(1) != 1 and t.shape[1] != 1):
        raise ValueError(f"{what} must be 2-D with unit column stride")
    return t.data_ptr(), t.stride(0), t.shape[1]


# ---------------------------------------------------------------------------
# C-named functions
# ---------------------------------------------------------------------------

def agp_plan_create(X: torch.Tensor, windows, N, cutoff: int, kernel: str = "gauss",
                    ell: float = 1.0, sigma_f: float = 1.0, sigma_eps: float = 0.0,
                    sigma_os: int = 2) -> c_void_p:
    lib = load_library()
    if not X.is_cuda or X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a 2-D CUDA tensor with unit column stride")
    if X.dtype not in (torch.float32, torch.float64):
        raise ValueError("X must be float32 or float64")
    P = len(windows)
    Ns = [int(N)] * P if np.isscalar(N) else [int(v) for v in N]
    ptr = [0]
    feat = []
    for w in windows:
        feat += [int(f) for f in w]
        ptr.append(len(feat))
    wp = (c_int * len(ptr))(*ptr)
    wf = (c_int * max(1, len(feat)))(*feat)
    Na = (c_int * P)(*Ns)
    d = _Desc(n=X.shape[0], p=X.shape[1], X=X.data_ptr(), ldx=X.stride(0), P=P,
              win_ptr=wp, win_feat=wf, N=Na, cutoff=int(cutoff), sigma_os=int(sigma_os),
              kernel=KERNELS[kernel], ell=float(ell), sigma_f=float(sigma_f),
              sigma_eps=float(sigma_eps), prec=0 if X.dtype == torch.float32 else 1)
    h = c_void_p()
    _check(lib.agp_plan_create(byref(h), byref(d), _stream()))
    return h


def agp_plan_destroy(plan: c_void_p):
    _check(load_library().agp_plan_destroy(plan))


def agp_set_hyper(plan: c_void_p, ell: float, sigma_f: float, sigma_eps: float):
    _check(load_library().agp_set_hyper(plan, float(ell), float(sigma_f), float(sigma_eps),
                                        _stream()))


def agp_matvec(plan: c_void_p, V: torch.Tensor, Out: torch.Tensor, add_noise: bool = True):
    vp, ldv, R = _block(V, V.dtype, "V")
    op, ldo, Ro = _block(Out, V.dtype, "Out")
    if Ro != R or Out.shape[0] != V.shape[0]:
        raise ValueError("Out must have V's shape")
    _check(load_library().agp_matvec(plan, vp, ldv, op, ldo, R, int(bool(add_noise)), _stream()))


def agp_deriv_matvec(plan: c_void_p, which: str, V: torch.Tensor, Out: torch.Tensor):
    vp, ldv, R = _block(V, V.dtype, "V")
    op, ldo, Ro = _block(Out, V.dtype, "Out")
    if Ro != R or Out.shape[0] != V.shape[0]:
        raise ValueError("Out must have V's shape")
    _check(load_library().agp_deriv_matvec(plan, PARAMS[which], vp, ldv, op, ldo, R, _stream()))


def agp_spectra_size(plan: c_void_p, R: int) -> int:
    e = c_int64()
    _check(load_library().agp_spectra_size(plan, int(R), byref(e)))
    return e.value


def agp_matvec_spectra(plan: c_void_p, V: torch.Tensor, Out: torch.Tensor | None,
                       spec: torch.Tensor, add_noise: bool = True):
    """Out = K_hat V (skipped when Out is None) and the forward spectra of V
    into spec (complex tensor of agp_spectra_size(R) elements)."""
    vp, ldv, R = _block(V, V.dtype, "V")
    if Out is None:
        op, ldo = None, R
    else:
        op, ldo, Ro = _block(Out, V.dtype, "Out")
        if Ro != R or Out.shape[0] != V.shape[0]:
            raise ValueError("Out must have V's shape")
    cdt = torch.complex64 if V.dtype == torch.float32 else torch.complex128
    if spec.dtype != cdt or not spec.is_contiguous() or spec.numel() < agp_spectra_size(plan, R):
        raise ValueError("spec must be a contiguous complex tensor of agp_spectra_size(R) elements")
    _check(load_library().agp_matvec_spectra(plan, vp, ldv, op, ldo, R, int(bool(add_noise)),
                                             spec.data_ptr(), _stream()))


def agp_spectral_form(plan: c_void_p, which: str | None, A: torch.Tensor, B: torch.Tensor,
                      R: int) -> torch.Tensor:
    """Device float64 [R]: G_r^T Op V_r from the spectra A (of G) and B (of V);
    Op = sigma_f^2 sum_s K_s (which None), its ell-derivative ("ell") or
    2 sigma_f sum_s K_s ("sigma_f")."""
    out = torch.empty(R, dtype=torch.float64, device=A.device)
    w = -1 if which is None else PARAMS[which]
    _check(load_library().agp_spectral_form(plan, w, A.data_ptr(), B.data_ptr(), int(R),
                                            out.data_ptr(), _stream()))
    return out


def agp_adjoint_nfft(plan: c_void_p, window: int, V: torch.Tensor, chat: torch.Tensor):
    vp, ldv, R = _block(V, V.dtype, "V")
    if not chat.is_cuda or not chat.is_contiguous():
        raise ValueError("chat must be a contiguous CUDA tensor")
    _check(load_library().agp_adjoint_nfft(plan, window, vp, ldv, R, chat.data_ptr(), _stream()))


def agp_nfft_real(plan: c_void_p, window: int, fhat: torch.Tensor, Out: torch.Tensor):
    op, ldo, R = _block(Out, Out.dtype, "Out")
    if not fhat.is_cuda or not fhat.is_contiguous():
        raise ValueError("fhat must be a contiguous CUDA tensor")
    _check(load_library().agp_nfft_real(plan, window, fhat.data_ptr(), R, op, ldo, _stream()))


def agp_plan_bins(plan: c_void_p, window: int, bins: torch.Tensor):
    if bins.dtype != torch.int32 or not bins.is_cuda or not bins.is_contiguous():
        raise ValueError("bins must be a contiguous int32 CUDA tensor")
    _check(load_library().agp_plan_bins(plan, window, bins.data_ptr(), _stream()))


def agp_plan_coeffs(plan: c_void_p, window: int, deriv: bool, out: np.ndarray):
    if out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array")
    _check(load_library().agp_plan_coeffs(plan, window, int(bool(deriv)),
                                          out.ctypes.data_as(POINTER(c_double)), _stream()))


def agp_plan_query(plan: c_void_p, window: int = 0):
    n, P, d, N, it = c_int64(), c_int(), c_int(), c_int(), c_int64()
    _check(load_library().agp_plan_query(plan, byref(n), byref(P), window, byref(d), byref(N),
                                         byref(it)))
    return {"n": n.value, "P": P.value, "d": d.value, "N": N.value, "n_items": it.value}


def agp_pcg_solve(plan: c_void_p, B: torch.Tensor, Xsol: torch.Tensor, rtol: float = 1e-4,
                  maxit: int = 200, n_landmarks: int = 0, raise_not_converged: bool = True):
    """Batched CG for K_hat X = B. Returns (iters, relres) as numpy arrays."""
    bp, ldb, R = _block(B, B.dtype, "B")
    xp, ldx, Rx = _block(Xsol, B.dtype, "Xsol")
    if Rx != R or Xsol.shape[0] != B.shape[0]:
        raise ValueError("Xsol must have B's shape")
    it = (c_int * R)()
    rel = (c_double * R)()
    st = load_library().agp_pcg_solve(plan, bp, ldb, xp, ldx, R, float(rtol), int(maxit),
                                      int(n_landmarks), it, rel, _stream())
    if st != AGP_NOT_CONVERGED or raise_not_converged:
        _check(st)
    return np.array(it[:], dtype=np.int64), np.array(rel[:], dtype=np.float64)


def agp_nlml_grad_pc(plan: c_void_p, y: torch.Tensor, Wn: torch.Tensor, Wk: np.ndarray,
                     n_landmarks: int, lanczos_steps: int = 20, rtol: float = 0.0, maxit: int = 0):
    """Preconditioned (nlml, grads) with probe vectors Wn (device [n][nz]) and
    Wk (host [k][nz], k = len(landmarks(n_landmarks)))."""
    if y.dim() != 1 or not y.is_contiguous():
        raise ValueError("y must be a contiguous 1-D tensor")
    wp, ldw, nz = _block(Wn, y.dtype, "Wn")
    wk = np.ascontiguousarray(np.asarray(Wk, dtype=np.float64))
    if wk.ndim != 2 or wk.shape[1] != nz:
        raise ValueError("Wk must be [k][nz]")
    nl = c_double()
    g = (c_double * 3)()
    _check(load_library().agp_nlml_grad_pc(plan, y.data_ptr(), wp, ldw,
                                           wk.ctypes.data_as(POINTER(c_double)), nz,
                                           int(n_landmarks), int(lanczos_steps), float(rtol),
                                           int(maxit), byref(nl), g, _stream()))
    return nl.value, {"ell": g[0], "sigma_f": g[1], "sigma_eps": g[2]}


def agp_plan_set_item_points(plan: c_void_p, points: int):
    _check(load_library().agp_plan_set_item_points(plan, int(points), _stream()))


def agp_plan_set_boundary(plan: c_void_p, eps_b: float, p: int):
    """Outer boundary smoothing of kappa_R (layer width eps_b, order p; 0
    switches it off); the points must lie in the ball |x| <= 1/4 - eps_b/2."""
    _check(load_library().agp_plan_set_boundary(plan, float(eps_b), int(p), _stream()))


def agp_plan_autotune(plan: c_void_p, R: int = 32, reps: int = 3):
    """(chosen points per work item, mean ms per matvec at that size)."""
    pts = c_int()
    ms = c_double()
    _check(load_library().agp_plan_autotune(plan, int(R), int(reps), byref(pts), byref(ms),
                                            _stream()))
    return pts.value, ms.value


def agp_plan_landmarks(plan: c_void_p, n_landmarks: int) -> np.ndarray:
    """The landmark indices agp_pcg_solve uses for n_landmarks (sorted)."""
    P = c_int()
    _check(load_library().agp_plan_query(plan, None, byref(P), 0, None, None, None))
    cap = P.value * (-(-int(n_landmarks) // P.value))
    idx = (c_int32 * max(cap, 1))()
    cnt = c_int()
    _check(load_library().agp_plan_landmarks(plan, int(n_landmarks), idx, cap, byref(cnt),
                                             _stream()))
    return np.array(idx[:cnt.value], dtype=np.int64)


def agp_afn_create(plan: c_void_p, n_landmarks: int, fill: int) -> c_void_p:
    h = c_void_p()
    _check(load_library().agp_afn_create(byref(h), plan, int(n_landmarks), int(fill), _stream()))
    return h


def agp_afn_destroy(afn: c_void_p):
    _check(load_library().agp_afn_destroy(afn))


def agp_afn_apply(afn: c_void_p, V: torch.Tensor, Y: torch.Tensor):
    """Y = M^{-1} V (float64 CUDA blocks [n][R])."""
    vp, ldv, R = _block(V, torch.float64, "V")
    yp, ldy, Ry = _block(Y, torch.float64, "Y")
    if Ry != R or Y.shape[0] != V.shape[0]:
        raise ValueError("Y must have V's shape")
    _check(load_library().agp_afn_apply(afn, vp, ldv, yp, ldy, R, _stream()))


def agp_afn_info(afn: c_void_p):
    """(landmark count, nonzeros of G, log det M)."""
    k = c_int()
    nnz = c_int64()
    ld = c_double()
    _check(load_library().agp_afn_info(afn, byref(k), byref(nnz), byref(ld)))
    return k.value, nnz.value, ld.value


def agp_afn_pattern(afn: c_void_p, n: int, fill: int):
    """(landmarks [k], pattern [n - k][fill]) as numpy int arrays."""
    k, _, _ = agp_afn_info(afn)
    lm = np.zeros(max(k, 1), dtype=np.int32)
    J = np.zeros((max(n - k, 1), fill), dtype=np.int32)
    _check(load_library().agp_afn_pattern(afn, lm.ctypes.data_as(c_void_p),
                                          J.ctypes.data_as(c_void_p), _stream()))
    return lm[:k].astype(np.int64), J[:n - k].astype(np.int64)


def agp_pcg_solve_afn(plan: c_void_p, afn: c_void_p, B: torch.Tensor, Xsol: torch.Tensor,
                      rtol: float = 1e-4, maxit: int = 200, raise_not_converged: bool = True):
    """CG for K_hat X = B preconditioned by the AFN object. Returns (iters, relres)."""
    bp, ldb, R = _block(B, B.dtype, "B")
    xp, ldx, Rx = _block(Xsol, B.dtype, "Xsol")
    if Rx != R or Xsol.shape[0] != B.shape[0]:
        raise ValueError("Xsol must have B's shape")
    it = (c_int * R)()
    rel = (c_double * R)()
    st = load_library().agp_pcg_solve_afn(plan, afn, bp, ldb, xp, ldx, R, float(rtol), int(maxit),
                                          it, rel, _stream())
    if st != AGP_NOT_CONVERGED or raise_not_converged:
        _check(st)
    return np.array(it[:], dtype=np.int64), np.array(rel[:], dtype=np.float64)


def agp_nlml_grad_afn(plan: c_void_p, afn: c_void_p, y: torch.Tensor, Wn: torch.Tensor,
                      lanczos_steps: int = 20, rtol: float = 0.0, maxit: int = 0):
    """(nlml, grads) with the AFN preconditioner; Wn: device [n][nz] vectors
    with covariance I in the plan precision."""
    if y.dim() != 1 or not y.is_contiguous():
        raise ValueError("y must be a contiguous 1-D tensor")
    wp, ldw, nz = _block(Wn, y.dtype, "Wn")
    nl = c_double()
    g = (c_double * 3)()
    _check(load_library().agp_nlml_grad_afn(plan, afn, y.data_ptr(), wp, ldw, nz,
                                            int(lanczos_steps), float(rtol), int(maxit), byref(nl),
                                            g, _stream()))
    return nl.value, {"ell": g[0], "sigma_f": g[1], "sigma_eps": g[2]}


class Afn:
    """The additive AFN preconditioner of a plan at its current hyperparameters."""

    def __init__(self, plan: "Plan", n_landmarks: int, fill: int):
        self.plan = plan
        self.fill = int(fill)
        self._h = agp_afn_create(plan.handle, n_landmarks, fill)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            agp_afn_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, V: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = torch.empty_like(V) if out is None else out
        agp_afn_apply(self._h, V, out)
        return out

    def info(self):
        return agp_afn_info(self._h)

    def pattern(self):
        return agp_afn_pattern(self._h, self.plan.n, self.fill)

    def nlml_grad(self, y: torch.Tensor, Wn: torch.Tensor, lanczos_steps: int = 20,
                  rtol: float = 0.0, maxit: int = 0):
        return agp_nlml_grad_afn(self.plan.handle, self._h, y, Wn, lanczos_steps, rtol, maxit)

    def solve(self, B: torch.Tensor, rtol: float = 1e-4, maxit: int = 200,
              raise_not_converged: bool = True):
        X = torch.empty_like(B)
        it, rel = agp_pcg_solve_afn(self.plan.handle, self._h, B, X, rtol, maxit,
                                    raise_not_converged)
        return X, it, rel


def agp_nlml_grad(plan: c_void_p, y: torch.Tensor, Z: torch.Tensor, lanczos_steps: int = 20,
                  rtol: float = 0.0, maxit: int = 0):
    """(nlml, {"ell": g, "sigma_f": g, "sigma_eps": g}) with probes Z [n][nz]."""
    if y.dim() != 1 or not y.is_contiguous():
        raise ValueError("y must be a contiguous 1-D tensor")
    zp, ldz, nz = _block(Z, y.dtype, "Z")
    nl = c_double()
    g = (c_double * 3)()
    _check(load_library().agp_nlml_grad(plan, y.data_ptr(), zp, ldz, nz, int(lanczos_steps),
                                        float(rtol), int(maxit), byref(nl), g, _stream()))
    return nl.value, {"ell": g[0], "sigma_f": g[1], "sigma_eps": g[2]}


def agp_nlml_grad_seed(plan: c_void_p, y: torch.Tensor, n_probes: int, seed: int,
                       lanczos_steps: int = 20, rtol: float = 0.0, maxit: int = 0):
    """agp_nlml_grad with Rademacher probes drawn on the device from `seed`."""
    if y.dim() != 1 or not y.is_contiguous():
        raise ValueError("y must be a contiguous 1-D tensor")
    nl = c_double()
    g = (c_double * 3)()
    _check(load_library().agp_nlml_grad_seed(plan, y.data_ptr(), int(n_probes),
                                             int(lanczos_steps), int(seed), float(rtol),
                                             int(maxit), byref(nl), g, _stream()))
    return nl.value, {"ell": g[0], "sigma_f": g[1], "sigma_eps": g[2]}


def agp_rademacher(n: int, R: int, seed: int, dtype=torch.float32, device="cuda") -> torch.Tensor:
    """n x R Rademacher block from the library's counter-based generator."""
    Z = torch.empty((n, R), dtype=dtype, device=device)
    prec = AGP_F32 if dtype == torch.float32 else AGP_F64
    _check(load_library().agp_rademacher(prec, int(n), int(R), int(seed), Z.data_ptr(), R,
                                         _stream()))
    return Z


def agp_dot_columns(plan: c_void_p, A: torch.Tensor, B: torch.Tensor) -> np.ndarray:
    """FP64 column dot products of two [n][R] blocks (library kernels)."""
    ap, lda, R = _block(A, A.dtype, "A")
    bp, ldb, Rb = _block(B, A.dtype, "B")
    if Rb != R or A.shape[0] != B.shape[0]:
        raise ValueError("A and B must have the same shape")
    out = (c_double * R)()
    _check(load_library().agp_dot_columns(plan, ap, lda, bp, ldb, R, out, _stream()))
    return np.array(out[:], dtype=np.float64)


def agp_dot_columns_static(A: torch.Tensor, B: torch.Tensor, out: torch.Tensor):
    """Column dot products into out (float64 CUDA tensor [R]) without any
    device allocation by the library: for callers that must not allocate
    (see include/agp.h). Calls that overlap on the GPU share one scratch
    array and race; the first call on a device must precede stream capture."""
    if A.dtype not in (torch.float32, torch.float64):
        raise ValueError("A must be float32 or float64")
    ap, lda, R = _block(A, A.dtype, "A")
    bp, ldb, Rb = _block(B, A.dtype, "B")
    if Rb != R or A.shape[0] != B.shape[0]:
        raise ValueError("A and B must have the same shape")
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < R or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 CUDA tensor with R entries")
    prec = 0 if A.dtype == torch.float32 else 1
    _check(load_library().agp_dot_columns_static(prec, ap, lda, bp, ldb, A.shape[0], R,
                                                 out.data_ptr(), _stream()))


def agp_batch_create(plans) -> c_void_p:
    hs = (c_void_p * len(plans))(*[p.handle.value for p in plans])
    b = c_void_p()
    _check(load_library().agp_batch_create(byref(b), hs, len(plans), _stream()))
    return b


def agp_batch_destroy(batch: c_void_p):
    _check(load_library().agp_batch_destroy(batch))


def agp_batch_bind(batch: c_void_p, Vs, Outs):
    """Bind per-problem right-hand sides and outputs ([n_q][R] blocks)."""
    if len(Vs) != len(Outs):
        raise ValueError("need one output per right-hand side block")
    ptrs_v, lds_v, ptrs_o, lds_o, Rs = [], [], [], [], set()
    for V, O in zip(Vs, Outs):
        vp, ldv, R = _block(V, V.dtype, "V")
        op, ldo, Ro = _block(O, V.dtype, "Out")
        if Ro != R or O.shape[0] != V.shape[0]:
            raise ValueError("Out must have V's shape")
        ptrs_v.append(vp), lds_v.append(ldv), ptrs_o.append(op), lds_o.append(ldo), Rs.add(R)
    if len(Rs) != 1:
        raise ValueError("every problem of a batch needs the same number of columns")
    k = len(Vs)
    _check(load_library().agp_batch_bind(batch, (c_void_p * k)(*ptrs_v), (c_int64 * k)(*lds_v),
                                         (c_void_p * k)(*ptrs_o), (c_int64 * k)(*lds_o),
                                         Rs.pop(), _stream()))


def agp_batch_matvec(batch: c_void_p, which: str | None = None):
    w = -1 if which is None else PARAMS[which]
    _check(load_library().agp_batch_matvec(batch, w, _stream()))


class Batch:
    """Independent plans applied together, one launch per stage."""

    def __init__(self, plans):
        self.plans = list(plans)          # the batch refers to them: keep them alive
        self._h = agp_batch_create(self.plans)

    def bind(self, Vs, Outs):
        self._bound = (list(Vs), list(Outs))
        agp_batch_bind(self._h, Vs, Outs)

    def matvec(self, which: str | None = None):
        agp_batch_matvec(self._h, which)

    def close(self):
        if self._h is not None and self._h.value:
            agp_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def agp_profile_enable(plan: c_void_p, enable: bool = True):
    _check(load_library().agp_profile_enable(plan, int(bool(enable))))


def agp_profile_read(plan: c_void_p, reset: bool = True) -> dict:
    p = Profile()
    _check(load_library().agp_profile_read(plan, byref(p), int(bool(reset)), _stream()))
    return {s: {"ms": p.ms[i], "launches": p.launches[i],
                "ms_by_dim": [p.ms_by_dim[i][d] for d in range(4)],
                "timed_by_dim": [p.timed_by_dim[i][d] for d in range(4)]}
            for i, s in enumerate(STAGES)}


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class Plan:
    """A plan over fixed points X (CUDA tensor [n][p], float32 or float64)."""

    def __init__(self, X: torch.Tensor, windows, N, cutoff: int, kernel: str = "gauss",
                 ell: float = 1.0, sigma_f: float = 1.0, sigma_eps: float = 0.0,
                 sigma_os: int = 2):
        self.windows = [list(w) for w in windows]
        self.N = [int(N)] * len(windows) if np.isscalar(N) else [int(v) for v in N]
        self.cutoff = int(cutoff)
        self.kernel = kernel
        self.dtype = X.dtype
        self.device = X.device
        self.n = X.shape[0]
        self.ell, self.sigma_f, self.sigma_eps = float(ell), float(sigma_f), float(sigma_eps)
        self._h = agp_plan_create(X, windows, N, cutoff, kernel, ell, sigma_f, sigma_eps, sigma_os)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            agp_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_hyper(self, ell: float, sigma_f: float, sigma_eps: float):
        agp_set_hyper(self._h, ell, sigma_f, sigma_eps)
        self.ell, self.sigma_f, self.sigma_eps = float(ell), float(sigma_f), float(sigma_eps)

    def ensure_hyper(self, ell: float, sigma_f: float, sigma_eps: float):
        """set_hyper, skipped when the plan already holds these values."""
        if (float(ell), float(sigma_f), float(sigma_eps)) != (self.ell, self.sigma_f,
                                                                self.sigma_eps):
            self.set_hyper(ell, sigma_f, sigma_eps)

    def matvec(self, V: torch.Tensor, out: torch.Tensor | None = None, add_noise: bool = True):
        out = torch.empty_like(V) if out is None else out
        agp_matvec(self._h, V, out, add_noise)
        return out

    def spectra(self, V: torch.Tensor, out: torch.Tensor | None = None,
                add_noise: bool = True) -> tuple:
        """(K_hat V or None, spectra of V): with `out` (a tensor, or True for a
        new one) the matvec is applied too."""
        R = V.shape[1]
        cdt = torch.complex64 if self.dtype == torch.float32 else torch.complex128
        spec = torch.empty(agp_spectra_size(self._h, R), dtype=cdt, device=V.device)
        if out is True:
            out = torch.empty_like(V)
        agp_matvec_spectra(self._h, V, out if out is not None else None, spec, add_noise)
        return out, spec

    def spectral_form(self, which: str | None, A: torch.Tensor, B: torch.Tensor, R: int):
        return agp_spectral_form(self._h, which, A, B, R)

    def deriv_matvec(self, which: str, V: torch.Tensor, out: torch.Tensor | None = None):
        out = torch.empty_like(V) if out is None else out
        agp_deriv_matvec(self._h, which, V, out)
        return out

    def adjoint_nfft(self, window: int, V: torch.Tensor) -> torch.Tensor:
        d = len(self.windows[window])
        N = self.N[window]
        R = 1 if V.dim() == 1 else V.shape[1]
        cdt = torch.complex64 if self.dtype == torch.float32 else torch.complex128
        chat = torch.empty((R,) + (N,) * d, dtype=cdt, device=V.device)
        agp_adjoint_nfft(self._h, window, V, chat)
        return chat

    def nfft_real(self, window: int, fhat: torch.Tensor, out: torch.Tensor | None = None):
        R = fhat.shape[0]
        if out is None:
            out = torch.empty((self.n, R), dtype=self.dtype, device=fhat.device)
        agp_nfft_real(self._h, window, fhat.contiguous(), out)
        return out

    def bins(self, window: int) -> torch.Tensor:
        d = len(self.windows[window])
        b = torch.empty((self.n, d), dtype=torch.int32, device=self.device)
        agp_plan_bins(self._h, window, b)
        return b

    def coeffs(self, window: int, deriv: bool = False) -> np.ndarray:
        d = len(self.windows[window])
        out = np.empty((self.N[window],) * d, dtype=np.float64)
        agp_plan_coeffs(self._h, window, deriv, out)
        return out

    def solve(self, B: torch.Tensor, rtol: float = 1e-4, maxit: int = 200,
              raise_not_converged: bool = True, n_landmarks: int = 0):
        X = torch.empty_like(B)
        it, rel = agp_pcg_solve(self._h, B, X, rtol, maxit, n_landmarks, raise_not_converged)
        return X, it, rel

    def nlml_grad_pc(self, y: torch.Tensor, Wn: torch.Tensor, Wk, n_landmarks: int,
                     lanczos_steps: int = 20, rtol: float = 0.0, maxit: int = 0):
        return agp_nlml_grad_pc(self._h, y, Wn, Wk, n_landmarks, lanczos_steps, rtol, maxit)

    def afn(self, n_landmarks: int, fill: int) -> Afn:
        return Afn(self, n_landmarks, fill)

    def set_tensor_cores(self, enable: int = 3):
        """3: both persistent tensor-memory kernels (the default), 1:
        tensor-memory spreading with shared-memory interpolation, 2: both with
        operands in shared memory, 0: FMA pipes only."""
        _check(load_library().agp_plan_set_tensor_cores(self._h, int(enable)))

    def set_boundary(self, eps_b: float, p: int):
        agp_plan_set_boundary(self._h, eps_b, p)

    def check(self):
        """Raise AgpError (AGP_TIMEOUT) if a bounded device wait expired."""
        _check(load_library().agp_plan_check(self._h, _stream()))

    def set_wait_limit(self, polls: int = 0):
        """Polls per bounded tensor-core wait (0: the library default)."""
        _check(load_library().agp_plan_set_wait_limit(self._h, int(polls)))

    def autotune(self, R: int = 32, reps: int = 3):
        """(points per work item, ms per matvec) of the fastest choice; the
        chosen kernel family is tensor_cores()."""
        return agp_plan_autotune(self._h, R, reps)

    def tensor_cores(self) -> int:
        m = c_int()
        _check(load_library().agp_plan_tensor_cores(self._h, byref(m)))
        return m.value

    def kernel_families(self, R: int, ldv: int | None = None) -> tuple[int, int]:
        """(spreading, interpolation) kernel family of the d = 3 windows for an
        R-column application: 3 tensor-memory, 2 shared-memory tensor-core
        over cell runs, 1 tensor-core over work items, 0 FMA, -1 no d = 3
        window."""
        sp, ip = c_int(), c_int()
        _check(load_library().agp_plan_kernel_families(self._h, int(R), int(ldv or R),
                                                       byref(sp), byref(ip)))
        return sp.value, ip.value

    def set_item_points(self, points: int):
        agp_plan_set_item_points(self._h, points)

    def landmarks(self, n_landmarks: int) -> np.ndarray:
        return agp_plan_landmarks(self._h, n_landmarks)

    def nlml_grad(self, y: torch.Tensor, Z: torch.Tensor, lanczos_steps: int = 20,
                  rtol: float = 0.0, maxit: int = 0):
        return agp_nlml_grad(self._h, y, Z, lanczos_steps, rtol, maxit)

    def nlml_grad_seed(self, y: torch.Tensor, n_probes: int, seed: int, lanczos_steps: int = 20,
                       rtol: float = 0.0, maxit: int = 0):
        return agp_nlml_grad_seed(self._h, y, n_probes, seed, lanczos_steps, rtol, maxit)

    def profile(self, enable: bool = True):
        agp_profile_enable(self._h, enable)

    def profile_read(self, reset: bool = True) -> dict:
        return agp_profile_read(self._h, reset)

    def query(self, window: int = 0):
        return agp_plan_query(self._h, window)
