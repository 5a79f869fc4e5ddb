"""Seeded synthetic inputs: gauge fields, sources and the workload table.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It holds NO arithmetic of the method itself (no Dirac
operator, no Krylov step, no projection): only the recipe that draws the
inputs from fixed seeds, so that both sides see the same numbers.

Layouts (the library boundary uses the same ones):
  * site index  s = x + Lx*(y + Ly*(z + Lz*t)), mu = 0..3 <-> x, y, z, t
  * gauge field complex128 [site][mu][3][3]  (U_mu(x), row index = colour a)
  * spinor      complex128 [site][spin 4][colour 3]

Recipe for the gauge links (stands in for the quenched 20^3x32 beta=6.0
configuration of the paper's Section 3, which is not public):
  U_mu(x) = exp(i * eps * A),  A = sum_{a=1..8} c_a lambda_a,
  c_a ~ N(0, 1) drawn from numpy's PCG64 stream `default_rng(seed)` in the
  order (site, mu, a); lambda_a are the Gell-Mann matrices.  The exponential
  is taken through the Hermitian eigendecomposition of A in float64.

Sources (Section 3 uses point sources with Dirac/colour indices (1,1),(1,2)):
  * point: eta^j = delta_{x,0} e_{(s,c)}, j-1 = 3*s + c, j = 1..12
  * z2:    each complex component is +1 or -1 (imaginary part 0) with
           probability 1/2, from `default_rng(seed + 1000*(field + 1) + stream)`.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

Dims = Tuple[int, int, int, int]


def volume(dims: Dims) -> int:
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3), complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1.0
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1.0, -1.0
    lam[3][0, 2] = lam[3][2, 0] = 1.0
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1.0
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1.0 / np.sqrt(3.0)
    lam[7][2, 2] = -2.0 / np.sqrt(3.0)
    return lam


def gauge_field(dims: Dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) links U_mu(x) = exp(i eps A), complex128 [V][4][3][3]."""
    vol = volume(dims)
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((vol, 4, 8))
    a = np.einsum("sma,aij->smij", c, gell_mann())
    a = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))  # exactly Hermitian
    w, q = np.linalg.eigh(a)
    ph = np.exp(1j * eps * w)
    u = np.einsum("smik,smk,smjk->smij", q, ph, np.conj(q))
    return np.ascontiguousarray(u)


def unit_gauge(dims: Dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    u = np.zeros((volume(dims), 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def point_sources(dims: Dims, n: int = 12) -> np.ndarray:
    """Unit point sources at the origin, one per (spin, colour), [n][V][4][3]."""
    if not 1 <= n <= 12:
        raise ValueError("point sources come in at most 12 spin-colour indices")
    eta = np.zeros((n, volume(dims), 4, 3), dtype=np.complex128)
    for j in range(n):
        eta[j, 0, j // 3, j % 3] = 1.0
    return eta


def z2_sources(dims: Dims, n: int, seed: int, field_index: int = 0,
               stream: int = 0) -> np.ndarray:
    """Real Z2 noise (+-1 per complex component), [n][V][4][3]."""
    rng = np.random.default_rng(seed + 1000 * (field_index + 1) + stream)
    bits = rng.integers(0, 2, size=(n, volume(dims), 4, 3))
    return (2.0 * bits - 1.0).astype(np.complex128)


def guess_weights(seed: int, scale: float = 0.1) -> np.ndarray:
    """Seeded starting weights of the learned-guess network (flat complex128 [11520]:
    layers 1 -> 8, 8 -> 8, 8 -> 1, each [9 directions][C_out][C_in][4][4]), complex
    Gaussian with standard deviation scale / sqrt(9 * C_in * 4) per part."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in ((1, 8), (8, 8), (8, 1)):
        sd = scale / np.sqrt(9 * ci * 4)
        shape = (9, co, ci, 4, 4)
        parts.append((sd * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))).reshape(-1))
    return np.concatenate(parts)


def random_spinors(dims: Dims, n: int, seed: int) -> np.ndarray:
    """Complex Gaussian spinors for operator tests, [n][V][4][3]."""
    rng = np.random.default_rng(seed)
    shape = (n, volume(dims), 4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_su3(n: int, seed: int) -> np.ndarray:
    """Haar-ish random SU(3) matrices (QR of a complex Gaussian), [n][3][3]."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q[:, :, 0] /= det[:, None]
    return q


# --------------------------------------------------------------------------
# Workload table.  kappa values live in kappa.json beside this file; they are
# tuned once (so that cond(M) reaches the target) by the oracle's tuning
# script and are set-up data, not results.
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class FieldSpec:
    name: str
    dims: Dims
    eps: float
    seed: int
    cond_target: float
    field_index: int = 0

    def gauge(self) -> np.ndarray:
        return gauge_field(self.dims, self.eps, self.seed)


@dataclass(frozen=True)
class Workload:
    name: str
    fields: Tuple[FieldSpec, ...]
    nrhs: Tuple[int, ...]
    sources: str            # "point" | "z2"
    tol: float = 1e-8
    past_factor: float = 2.0
    reorth_period: int = 10
    precision: str = "fp64"  # fp64 | mixed_v32 | mixed_vbf16

    def sources_for(self, i: int) -> np.ndarray:
        f = self.fields[i]
        if self.sources == "point":
            return point_sources(f.dims, self.nrhs[i])
        return z2_sources(f.dims, self.nrhs[i], f.seed, f.field_index)


_F_TINY = FieldSpec("tiny_4x4x4x4_eps0.3", (4, 4, 4, 4), 0.3, 0, 1e3)
_F_SMALL = FieldSpec("small_8x8x8x16_eps0.5", (8, 8, 8, 16), 0.5, 1, 1e4)
_F_LARGE = FieldSpec("large_16x16x16x32_eps0.5", (16, 16, 16, 32), 0.5, 2, 1e5)
_F_B1 = FieldSpec("batch_8x8x8x16_eps0.5", (8, 8, 8, 16), 0.5, 3, 1e4, 0)
_F_B2 = FieldSpec("batch_12x12x12x24_eps0.5", (12, 12, 12, 24), 0.5, 4, 1e4, 1)
_F_B3 = FieldSpec("batch_16x16x16x32_eps0.5", (16, 16, 16, 32), 0.5, 5, 1e4, 2)

FIELDS: Dict[str, FieldSpec] = {f.name: f for f in
                                (_F_TINY, _F_SMALL, _F_LARGE, _F_B1, _F_B2, _F_B3)}

WORKLOADS: Dict[str, Workload] = {
    # plain FP64 Improved Seed-CG, Z2 sources, 1.5x past convergence
    "tiny_4x4x4x4_nrhs4": Workload("tiny_4x4x4x4_nrhs4", (_F_TINY,), (4,), "z2",
                                   past_factor=1.5),
    # 12 point sources, full V, 2x past convergence
    "small_8x8x8x16_nrhs12": Workload("small_8x8x8x16_nrhs12", (_F_SMALL,), (12,),
                                      "point"),
    # the headline: 16^3x32, 12 point sources, mixed precision
    "large_16x16x16x32_nrhs12": Workload("large_16x16x16x32_nrhs12", (_F_LARGE,),
                                         (12,), "point", precision="mixed_vbf16"),
    # three uneven lattices in one batched launch
    "batch3_uneven_nrhs24_12_6": Workload("batch3_uneven_nrhs24_12_6",
                                          (_F_B1, _F_B2, _F_B3), (24, 12, 6), "z2",
                                          precision="mixed_v32"),
}

_KAPPA_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kappa.json")


def kappa_table() -> Dict[str, dict]:
    if not os.path.exists(_KAPPA_FILE):
        return {}
    with open(_KAPPA_FILE) as fh:
        return json.load(fh)


def kappa_for(field_name: str) -> float:
    tab = kappa_table()
    if field_name not in tab:
        raise KeyError(f"no tuned kappa for {field_name}; run the oracle's tuning script")
    return float(tab[field_name]["kappa"])
