"""Oracle Wilson operator: Python face of the plain-C FP64 definition.

Test infrastructure only.  See `oracle/__init__.py` for who may use it.

Paper, Section 3 (Wilson fermions; normal equations A^dag A x = A^dag phi):
this module gives D, D^dag = g5 D g5 and M = D^dag D on the full lattice,
periodic in space and antiperiodic in time.  The arithmetic lives in
`wilson_ref.c`, compiled with gcc on first use (or by `build_oracle()`).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_wilson.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the plain-C oracle operator (gcc, OpenMP).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_wilson_apply.argtypes = [ctypes.POINTER(ctypes.c_int), dp, ctypes.c_double,
                                                ctypes.c_int, dp, dp, dp]
            lib.oracle_wilson_apply.restype = None
            lib.oracle_gamma.argtypes = [ctypes.c_int, dp]
            lib.oracle_gamma5.argtypes = [dp]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gamma(mu: int) -> np.ndarray:
    """The 4x4 gamma matrix g_{mu+1} the operator uses (mu = 0..3 <-> x,y,z,t)."""
    out = np.zeros((4, 4), dtype=np.complex128)
    _load().oracle_gamma(mu, _dp(out))
    return out


def gamma5() -> np.ndarray:
    out = np.zeros((4, 4), dtype=np.complex128)
    _load().oracle_gamma5(_dp(out))
    return out


class WilsonOperator:
    """D = 1 - kappa H on one gauge field.  Vectors are complex128 arrays of
    V*12 entries (any shape that flattens to [site][spin][colour])."""

    OP_D, OP_DDAG, OP_M = 0, 1, 2

    def __init__(self, dims, gauge: np.ndarray, kappa: float):
        self.dims = tuple(int(d) for d in dims)
        self.vol = int(np.prod(self.dims))
        self.n = 12 * self.vol
        g = np.ascontiguousarray(gauge, dtype=np.complex128)
        if g.size != self.vol * 36:
            raise ValueError("gauge field has the wrong size for these dims")
        self.gauge = g
        self.kappa = float(kappa)
        self._dims_c = (ctypes.c_int * 4)(*self.dims)
        self.matvecs = 0  # applications of D or D^dag

    def _apply(self, op: int, x: np.ndarray) -> np.ndarray:
        xin = np.ascontiguousarray(x, dtype=np.complex128).reshape(-1)
        if xin.size != self.n:
            raise ValueError("vector has the wrong size")
        out = np.empty_like(xin)
        tmp = np.empty_like(xin)
        _load().oracle_wilson_apply(self._dims_c, _dp(self.gauge), self.kappa, op,
                                    _dp(xin), _dp(out), _dp(tmp))
        self.matvecs += 2 if op == self.OP_M else 1
        return out.reshape(np.shape(x))

    def D(self, x):
        return self._apply(self.OP_D, x)

    def Ddag(self, x):
        return self._apply(self.OP_DDAG, x)

    def M(self, x):
        """M = D^dag D (Hermitian positive definite)."""
        return self._apply(self.OP_M, x)

    def dense(self, op: int = OP_D) -> np.ndarray:
        """Dense matrix of D / D^dag / M by applying it to unit vectors (tiny lattices)."""
        if self.n > 4096:
            raise ValueError("dense operator only for tiny lattices")
        mat = np.empty((self.n, self.n), dtype=np.complex128)
        e = np.zeros(self.n, dtype=np.complex128)
        for k in range(self.n):
            e[k] = 1.0
            mat[:, k] = self._apply(op, e)
            e[k] = 0.0
        return mat
