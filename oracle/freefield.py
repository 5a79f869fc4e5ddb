"""Oracle pin: the free-field (all links = 1) Wilson operator in momentum space.

Test infrastructure only.  For U = 1 a plane wave psi(x) = exp(i p.x) u is an
eigenvector of the hopping term, so

  D(p) = 1 - 2 kappa sum_mu cos p_mu + 2 i kappa sum_mu g_mu sin p_mu,
  M(p) = D(p)^dag D(p) = (1 - 2 kappa sum cos p_mu)^2 + 4 kappa^2 sum sin^2 p_mu,

the latter a multiple of the 12x12 identity (the g_mu anticommute), with
p_k = 2 pi n_k / L_k in space and p_t = (2 pi n_t + pi) / L_t (antiperiodic).
"""
from __future__ import annotations

import itertools

import numpy as np


def momenta(dims):
    lx, ly, lz, lt = dims
    for nt, nz, ny, nx in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        yield (2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz,
               (2 * np.pi * nt + np.pi) / lt)


def spectrum_M(dims, kappa: float) -> np.ndarray:
    """All 12*V eigenvalues of M = D^dag D on the free field, sorted."""
    ev = []
    for p in momenta(dims):
        c = sum(np.cos(q) for q in p)
        s2 = sum(np.sin(q) ** 2 for q in p)
        ev.extend([(1 - 2 * kappa * c) ** 2 + 4 * kappa ** 2 * s2] * 12)
    return np.sort(np.array(ev))


def cond_M(dims, kappa: float) -> float:
    ev = spectrum_M(dims, kappa)
    return ev[-1] / ev[0]


def D_of_p(p, kappa: float, gammas) -> np.ndarray:
    """The 4x4 spin matrix D(p) (colour-diagonal) for momentum p."""
    d = (1 - 2 * kappa * sum(np.cos(q) for q in p)) * np.eye(4, dtype=np.complex128)
    for mu in range(4):
        d = d + 2j * kappa * np.sin(p[mu]) * gammas[mu]
    return d


def plane_wave(dims, p, u: np.ndarray) -> np.ndarray:
    """psi(x) = exp(i p.x) u for a spin-colour vector u [4][3]; [V][4][3]."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t)).reshape(-1)
    return phase[:, None, None] * u[None, :, :]
