"""Thin Python binding of libseedcg (include/seedcg.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the CUDA
library.  Device memory for inputs and outputs comes from PyTorch tensors
(complex128, on the GPU); host numpy arrays are also accepted where the C
ABI accepts host pointers.  There is no CPU fallback: if the library or a
GPU is missing, loading or the first call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

SEEDCG_OK = 0
SEEDCG_ERR_ARG = -1
SEEDCG_ERR_OOM = -2
SEEDCG_ERR_CUDA = -3
SEEDCG_ERR_NOT_CONVERGED = -4
SEEDCG_ERR_BREAKDOWN = -5
SEEDCG_ERR_NAN = -6
SEEDCG_ERR_TIMEOUT = -7

SEEDCG_FP64 = 0
SEEDCG_MIXED_V32 = 1
SEEDCG_MIXED_VBF16 = 2
PRECISIONS = {"fp64": SEEDCG_FP64, "mixed_v32": SEEDCG_MIXED_V32, "mixed_vbf16": SEEDCG_MIXED_VBF16}

OP_D, OP_DDAG, OP_M = 0, 1, 2


class seedcg_options(ctypes.Structure):
    _fields_ = [("m_max", ctypes.c_int), ("past_factor", ctypes.c_double),
                ("precision", ctypes.c_int), ("reliable_delta", ctypes.c_double),
                ("po_passes", ctypes.c_int), ("seed_mode", ctypes.c_int),
                ("x0_given", ctypes.c_int), ("cg_maxiter", ctypes.c_int),
                ("stop_after_seed", ctypes.c_int), ("poll_every", ctypes.c_int),
                ("use_tensor_cores", ctypes.c_int), ("use_guess", ctypes.c_int),
                ("resid_mode", ctypes.c_int), ("po_guard", ctypes.c_int)]


class seedcg_info(ctypes.Structure):
    _fields_ = [("m_conv", ctypes.c_int), ("m", ctypes.c_int), ("po_count", ctypes.c_int),
                ("cg_iters_max", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("iters", ctypes.POINTER(ctypes.c_int)),
                ("matvecs", ctypes.POINTER(ctypes.c_int)),
                ("true_resid", ctypes.POINTER(ctypes.c_double)),
                ("ms_total", ctypes.c_float), ("ms_lanczos", ctypes.c_float),
                ("ms_po", ctypes.c_float), ("ms_seed", ctypes.c_float), ("ms_cg", ctypes.c_float),
                ("true_resid_D", ctypes.POINTER(ctypes.c_double))]


_lib = None

# every entry point of include/seedcg.h, for the export check
EXPORTS = ["seedcg_default_options", "seedcg_create", "seedcg_set_options", "seedcg_solve",
           "seedcg_apply", "seedcg_get_lanczos", "seedcg_get_basis", "seedcg_last_error",
           "seedcg_destroy", "seedcg_kernel_launches", "seedcg_time_dslash",
           "seedcg_project_basis", "seedcg_batch_solve", "seedcg_guess_set_weights",
           "seedcg_guess_get_weights", "seedcg_guess_loss_grad", "seedcg_guess_train",
           "seedcg_guess_predict", "seedcg_apply_noalloc", "seedcg_selftest_bounded_wait",
           "seedcg_apply_eo", "seedcg_eo_source", "seedcg_eo_reconstruct", "seedcg_tridiag_lowest",
           "seedcg_deflate_guess", "seedcg_solve_eo"]
GUESS_NW = 11520


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libseedcg.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or (build_if_missing and not _build.up_to_date()):
        if not build_if_missing:
            raise RuntimeError(f"libseedcg not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    hpp = ctypes.POINTER(ctypes.c_void_p)
    lib.seedcg_default_options.argtypes = [ctypes.POINTER(seedcg_options)]
    lib.seedcg_default_options.restype = None
    lib.seedcg_create.argtypes = [hpp, ip, vp, ctypes.c_double, ctypes.POINTER(seedcg_options)]
    lib.seedcg_set_options.argtypes = [vp, ctypes.POINTER(seedcg_options)]
    lib.seedcg_solve.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, ctypes.POINTER(seedcg_info), vp]
    lib.seedcg_apply.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 vp, vp, vp]
    lib.seedcg_get_lanczos.argtypes = [vp, ctypes.c_int, dp, dp, dp, ip]
    lib.seedcg_get_basis.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    lib.seedcg_last_error.argtypes = [vp]
    lib.seedcg_last_error.restype = ctypes.c_char_p
    lib.seedcg_time_dslash.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_float), vp]
    lib.seedcg_time_dslash.restype = ctypes.c_int
    lib.seedcg_batch_solve.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ip,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(seedcg_info), vp]
    lib.seedcg_batch_solve.restype = ctypes.c_int
    lib.seedcg_solve_eo.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(seedcg_info), vp]
    lib.seedcg_solve_eo.restype = ctypes.c_int
    lib.seedcg_tridiag_lowest.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, vp, vp]
    lib.seedcg_tridiag_lowest.restype = ctypes.c_int
    lib.seedcg_deflate_guess.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
    lib.seedcg_deflate_guess.restype = ctypes.c_int
    lib.seedcg_apply_eo.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.seedcg_eo_source.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.seedcg_eo_reconstruct.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp]
    for name in ("seedcg_apply_eo", "seedcg_eo_source", "seedcg_eo_reconstruct"):
        getattr(lib, name).restype = ctypes.c_int
    lib.seedcg_selftest_bounded_wait.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
    lib.seedcg_selftest_bounded_wait.restype = ctypes.c_int
    lib.seedcg_apply_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         vp, vp, vp]
    lib.seedcg_apply_noalloc.restype = ctypes.c_int
    lib.seedcg_guess_set_weights.argtypes = [vp, vp]
    lib.seedcg_guess_get_weights.argtypes = [vp, vp]
    lib.seedcg_guess_loss_grad.argtypes = [vp, ctypes.c_int, vp, vp, dp, vp, vp]
    lib.seedcg_guess_train.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, dp, vp]
    lib.seedcg_guess_predict.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    for name in ("seedcg_guess_set_weights", "seedcg_guess_get_weights", "seedcg_guess_loss_grad",
                 "seedcg_guess_train", "seedcg_guess_predict"):
        getattr(lib, name).restype = ctypes.c_int
    lib.seedcg_project_basis.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp]
    lib.seedcg_project_basis.restype = ctypes.c_int
    lib.seedcg_kernel_launches.argtypes = []
    lib.seedcg_kernel_launches.restype = ctypes.c_ulonglong
    lib.seedcg_destroy.argtypes = [vp]
    lib.seedcg_destroy.restype = None
    for name in ("seedcg_create", "seedcg_set_options", "seedcg_solve", "seedcg_apply",
                 "seedcg_get_lanczos", "seedcg_get_basis"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class SeedCGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"seedcg status {code}: {msg}")
        self.code = code


def _ptr(a) -> int:
    """Data pointer of a torch tensor (device or host) or a numpy array."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError("expected a torch tensor or numpy array")


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def seedcg_default_options() -> seedcg_options:
    o = seedcg_options()
    load().seedcg_default_options(ctypes.byref(o))
    return o


def seedcg_last_error(h) -> str:
    m = load().seedcg_last_error(h)
    return m.decode() if m else ""


def _check(h, code: int, allow=()):
    if code != SEEDCG_OK and code not in allow:
        raise SeedCGError(code, seedcg_last_error(h))
    return code


def seedcg_create(dims: Sequence[int], gauge, kappa: float, opt: Optional[seedcg_options] = None):
    lib = load()
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    code = lib.seedcg_create(ctypes.byref(h), d, ctypes.c_void_p(_ptr(gauge)), float(kappa),
                             ctypes.byref(opt) if opt is not None else None)
    if code != SEEDCG_OK:
        raise SeedCGError(code, seedcg_last_error(None))
    return h


def seedcg_set_options(h, opt: seedcg_options):
    _check(h, load().seedcg_set_options(h, ctypes.byref(opt)))


def seedcg_solve(h, nrhs: int, B, X, tol: float, extra_iters: int, reorth_period: int,
                 stream=None, allow_not_converged: bool = False):
    """Returns (status, info dict).  B, X: complex128 [nrhs][V][4][3], host or device."""
    info = seedcg_info()
    iters = (ctypes.c_int * nrhs)()
    mv = (ctypes.c_int * nrhs)()
    tr = (ctypes.c_double * nrhs)()
    trd = (ctypes.c_double * nrhs)(*([float("nan")] * nrhs))
    info.iters = iters
    info.matvecs = mv
    info.true_resid = tr
    info.true_resid_D = trd
    code = load().seedcg_solve(h, int(nrhs), ctypes.c_void_p(_ptr(B)), ctypes.c_void_p(_ptr(X)),
                               float(tol), int(extra_iters), int(reorth_period),
                               ctypes.byref(info), _stream_ptr(stream))
    _check(h, code, allow=(SEEDCG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    out = {"status": code, "m_conv": info.m_conv, "m": info.m, "po_count": info.po_count,
           "cg_iters_max": info.cg_iters_max, "reliable_updates": info.reliable_updates,
           "iters": list(iters), "matvecs": list(mv), "true_resid": list(tr),
           "true_resid_D": list(trd),
           "ms_total": info.ms_total, "ms_lanczos": info.ms_lanczos, "ms_po": info.ms_po,
           "ms_seed": info.ms_seed, "ms_cg": info.ms_cg}
    return code, out


def seedcg_batch_solve(hs, Bs, Xs, tol: float, extra_iters: int, reorth_period: int, stream=None,
                       allow_not_converged: bool = False):
    """One call for several fields: returns (status, [info dict per field])."""
    nf = len(hs)
    harr = (ctypes.c_void_p * nf)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])
    nrhs = (ctypes.c_int * nf)(*[int(b.shape[0]) for b in Bs])
    barr = (ctypes.c_void_p * nf)(*[_ptr(b) for b in Bs])
    xarr = (ctypes.c_void_p * nf)(*[_ptr(x) for x in Xs])
    infos = (seedcg_info * nf)()
    keep = []
    for f in range(nf):
        k = int(nrhs[f])
        it, mv, tr = (ctypes.c_int * k)(), (ctypes.c_int * k)(), (ctypes.c_double * k)()
        keep.append((it, mv, tr))
        infos[f].iters, infos[f].matvecs, infos[f].true_resid = it, mv, tr
    code = load().seedcg_batch_solve(harr, nf, nrhs, barr, xarr, float(tol), int(extra_iters),
                                     int(reorth_period), infos, _stream_ptr(stream))
    _check(hs[0], code, allow=(SEEDCG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    out = []
    for f in range(nf):
        it, mv, tr = keep[f]
        i = infos[f]
        out.append({"m_conv": i.m_conv, "m": i.m, "po_count": i.po_count,
                    "cg_iters_max": i.cg_iters_max, "reliable_updates": i.reliable_updates,
                    "iters": list(it), "matvecs": list(mv), "true_resid": list(tr),
                    "ms_total": i.ms_total, "ms_lanczos": i.ms_lanczos, "ms_po": i.ms_po,
                    "ms_seed": i.ms_seed, "ms_cg": i.ms_cg})
    return code, out


def seedcg_apply(h, op: int, prec: int, multi: int, n: int, inp, out, stream=None):
    _check(h, load().seedcg_apply(h, int(op), int(prec), int(multi), int(n),
                                  ctypes.c_void_p(_ptr(inp)), ctypes.c_void_p(_ptr(out)),
                                  _stream_ptr(stream)))


def seedcg_apply_noalloc(h, op: int, prec: int, multi: int, n: int, inp, out, stream=None):
    """seedcg_apply without any device allocation (fixed 16 MiB scratch)."""
    _check(h, load().seedcg_apply_noalloc(h, int(op), int(prec), int(multi), int(n),
                                          ctypes.c_void_p(_ptr(inp)), ctypes.c_void_p(_ptr(out)),
                                          _stream_ptr(stream)))


NOALLOC_SCRATCH_BYTES = 16 << 20

EO_A, EO_ADAG, EO_MEO = 0, 1, 2


def seedcg_tridiag_lowest(alpha, beta, nev: int):
    """Host: the nev smallest eigenpairs of tridiag(beta, alpha, beta); returns
    (theta [nev], S [m][nev])."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    m = a.size
    b = np.ascontiguousarray(beta, dtype=np.float64)[:max(m - 1, 1)]
    theta = np.zeros(nev)
    S = np.zeros((m, nev))
    code = load().seedcg_tridiag_lowest(int(m), ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(b.ctypes.data),
                                        int(nev), ctypes.c_void_p(theta.ctypes.data),
                                        ctypes.c_void_p(S.ctypes.data))
    if code != SEEDCG_OK:
        raise SeedCGError(code, "tridiagonal eigensolve rejected its arguments")
    return theta, S


def seedcg_deflate_guess(h, nev: int, B, X0, stream=None):
    """Deflated initial guesses X0 for the right-hand sides B from the last
    solve's Ritz vectors; returns the nev Ritz values."""
    theta = np.zeros(nev)
    _check(h, load().seedcg_deflate_guess(h, int(nev), int(B.shape[0]), ctypes.c_void_p(_ptr(B)),
                                          ctypes.c_void_p(_ptr(X0)), ctypes.c_void_p(theta.ctypes.data),
                                          _stream_ptr(stream)))
    return theta


def seedcg_apply_eo(h, op: int, prec: int, inp, out, stream=None):
    """Even-odd operator on half-lattice (odd-site) vectors: A, A^dag or A^dag A."""
    n = inp.shape[0]
    _check(h, load().seedcg_apply_eo(h, int(op), int(prec), int(n), ctypes.c_void_p(_ptr(inp)),
                                     ctypes.c_void_p(_ptr(out)), _stream_ptr(stream)))


def seedcg_solve_eo(h, eta, X, tol: float, extra_iters: int, reorth_period: int, stream=None,
                    allow_not_converged: bool = False):
    """Even-odd preconditioned Improved Seed-CG for D x = eta (full-lattice eta and X on the device)."""
    nrhs = int(eta.shape[0])
    info = seedcg_info()
    iters = (ctypes.c_int * nrhs)()
    mv = (ctypes.c_int * nrhs)()
    tr = (ctypes.c_double * nrhs)()
    trd = (ctypes.c_double * nrhs)(*([float("nan")] * nrhs))
    info.iters, info.matvecs, info.true_resid, info.true_resid_D = iters, mv, tr, trd
    code = load().seedcg_solve_eo(h, nrhs, ctypes.c_void_p(_ptr(eta)), ctypes.c_void_p(_ptr(X)), float(tol),
                                  int(extra_iters), int(reorth_period), ctypes.byref(info), _stream_ptr(stream))
    _check(h, code, allow=(SEEDCG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return code, {"status": code, "m_conv": info.m_conv, "m": info.m, "po_count": info.po_count,
                  "cg_iters_max": info.cg_iters_max, "reliable_updates": info.reliable_updates,
                  "iters": list(iters), "matvecs": list(mv), "true_resid": list(tr),
                  "true_resid_D": list(trd), "ms_total": info.ms_total, "ms_lanczos": info.ms_lanczos,
                  "ms_po": info.ms_po, "ms_seed": info.ms_seed, "ms_cg": info.ms_cg}


def seedcg_eo_source(h, eta, phi, stream=None):
    """phi = eta_o + kappa H_oe eta_e (full eta -> half phi)."""
    _check(h, load().seedcg_eo_source(h, int(eta.shape[0]), ctypes.c_void_p(_ptr(eta)),
                                      ctypes.c_void_p(_ptr(phi)), _stream_ptr(stream)))


def seedcg_eo_reconstruct(h, x_odd, eta, x, stream=None):
    """Full solution from the odd sites: x_e = eta_e + kappa H_eo x_o."""
    _check(h, load().seedcg_eo_reconstruct(h, int(eta.shape[0]), ctypes.c_void_p(_ptr(x_odd)),
                                           ctypes.c_void_p(_ptr(eta)), ctypes.c_void_p(_ptr(x)),
                                           _stream_ptr(stream)))


def seedcg_selftest_bounded_wait(limit_ms: float = 20.0) -> int:
    """Run the bounded-wait self-check; returns the kernel's status
    (SEEDCG_ERR_TIMEOUT when the wait gave up as it must)."""
    st = ctypes.c_int(0)
    code = load().seedcg_selftest_bounded_wait(float(limit_ms), ctypes.byref(st))
    if code != SEEDCG_OK:
        raise SeedCGError(code, "bounded-wait self-check could not run")
    return st.value


def seedcg_get_lanczos(h, cap: int):
    a = np.zeros(cap)
    b = np.zeros(cap)
    d = np.zeros(cap)
    m = ctypes.c_int()
    dp = ctypes.POINTER(ctypes.c_double)
    _check(h, load().seedcg_get_lanczos(h, int(cap), a.ctypes.data_as(dp), b.ctypes.data_as(dp),
                                        d.ctypes.data_as(dp), ctypes.byref(m)))
    k = min(cap, m.value)
    return a[:k], b[:k], d[:k], m.value


def seedcg_get_basis(h, first: int, count: int, out):
    _check(h, load().seedcg_get_basis(h, int(first), int(count), ctypes.c_void_p(_ptr(out))))


def seedcg_time_dslash(h, prec: int, n: int, reps: int, flush_l2: int = 1, stream=None) -> float:
    ms = ctypes.c_float()
    _check(h, load().seedcg_time_dslash(h, int(prec), int(n), int(reps), int(flush_l2),
                                        ctypes.byref(ms), _stream_ptr(stream)))
    return float(ms.value)


def seedcg_project_basis(h, rows: int, nvec: int, X, use_tensor_cores: int = 1, stream=None):
    """C[a][j] = v_a^dag x_j against the stored basis; returns complex128 [rows][nvec]."""
    C = np.zeros((rows, nvec), dtype=np.complex128)
    _check(h, load().seedcg_project_basis(h, int(rows), int(nvec), ctypes.c_void_p(_ptr(X)),
                                          ctypes.c_void_p(C.ctypes.data), int(use_tensor_cores),
                                          _stream_ptr(stream)))
    return C


def _weights_flat(Ws):
    w = np.concatenate([np.asarray(W, dtype=np.complex128).reshape(-1) for W in Ws])
    if w.size != GUESS_NW:
        raise ValueError("guess weights must hold 11520 complex entries")
    return np.ascontiguousarray(w)


def seedcg_guess_set_weights(h, Ws):
    w = _weights_flat(Ws) if isinstance(Ws, (list, tuple)) else np.ascontiguousarray(Ws, dtype=np.complex128)
    _check(h, load().seedcg_guess_set_weights(h, ctypes.c_void_p(w.ctypes.data)))


def seedcg_guess_get_weights(h):
    w = np.zeros(GUESS_NW, dtype=np.complex128)
    _check(h, load().seedcg_guess_get_weights(h, ctypes.c_void_p(w.ctypes.data)))
    return w


def seedcg_guess_loss_grad(h, B, X, want_grad=True, stream=None):
    loss = ctypes.c_double()
    g = np.zeros(GUESS_NW, dtype=np.complex128) if want_grad else None
    _check(h, load().seedcg_guess_loss_grad(h, int(B.shape[0]), ctypes.c_void_p(_ptr(B)),
                                            ctypes.c_void_p(_ptr(X)), ctypes.byref(loss),
                                            ctypes.c_void_p(g.ctypes.data) if want_grad else None,
                                            _stream_ptr(stream)))
    return loss.value, g


def seedcg_guess_train(h, B, X, epochs, batch, lr, stream=None):
    loss = ctypes.c_double()
    _check(h, load().seedcg_guess_train(h, int(B.shape[0]), ctypes.c_void_p(_ptr(B)),
                                        ctypes.c_void_p(_ptr(X)), int(epochs), int(batch), float(lr),
                                        ctypes.byref(loss), _stream_ptr(stream)))
    return loss.value


def seedcg_guess_predict(h, B, X0, stream=None):
    _check(h, load().seedcg_guess_predict(h, int(B.shape[0]), ctypes.c_void_p(_ptr(B)),
                                          ctypes.c_void_p(_ptr(X0)), _stream_ptr(stream)))


def split_weights(w):
    """Flat complex128 [11520] -> the three layer arrays [9][C_out][C_in][4][4]."""
    w = np.asarray(w)
    a, b = 9 * 8 * 16, 9 * 64 * 16
    return [w[:a].reshape(9, 8, 1, 4, 4), w[a:a + b].reshape(9, 8, 8, 4, 4),
            w[a + b:].reshape(9, 1, 8, 4, 4)]


def seedcg_kernel_launches() -> int:
    return int(load().seedcg_kernel_launches())


def seedcg_destroy(h):
    if h:
        load().seedcg_destroy(h)


def make_options(**kw) -> seedcg_options:
    """Defaults of the C library, with fields overridden by keyword."""
    o = seedcg_default_options()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Solver:
    """Convenience owner of one handle (one gauge field)."""

    def __init__(self, dims, gauge, kappa, **opts):
        self.dims = tuple(int(d) for d in dims)
        self.vol = int(np.prod(self.dims))
        self.h = seedcg_create(self.dims, gauge, kappa, make_options(**opts) if opts else None)

    def set_options(self, **opts):
        seedcg_set_options(self.h, make_options(**opts))

    def solve(self, B, X, tol=1e-8, extra_iters=0, reorth_period=10, stream=None,
              allow_not_converged=False):
        nrhs = B.shape[0]
        return seedcg_solve(self.h, nrhs, B, X, tol, extra_iters, reorth_period, stream,
                            allow_not_converged)

    def apply(self, op, inp, out, prec=0, multi=0, stream=None):
        n = inp.shape[0] if len(inp.shape) == 4 else 1
        seedcg_apply(self.h, op, prec, multi, n, inp, out, stream)

    def time_dslash(self, prec=1, n=12, reps=20, flush_l2=1, stream=None):
        return seedcg_time_dslash(self.h, prec, n, reps, flush_l2, stream)

    def close(self):
        if self.h:
            seedcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
