"""Ritz vectors from a stored Lanczos basis and deflated initial guesses for later
right-hand sides on the same field: test infrastructure, like the rest of oracle/.

The paper's premise (Section 1, and the choice of m in Section 2) is that the Krylov
subspace built past convergence holds accurate eigenvectors with small eigenvalues.
With V = [v_1 .. v_m] orthonormal and T_m = V^dag M V tridiagonal (alpha on the
diagonal, beta_1 .. beta_{m-1} beside it), an eigenpair (theta, s) of T_m gives the
Ritz pair (theta, y = V s), and Lanczos' relation M V = V T_m + beta_m v_{m+1} e_m^T
makes ||M y - theta y|| = |beta_m s_m|.  A new right-hand side b is deflated by the
Galerkin projection onto Y = span(y_1 .. y_k): x_0 = Y c with (Y^dag M Y) c = Y^dag b.
"""
import numpy as np
from scipy.linalg import eigh_tridiagonal


def ritz_pairs(V: np.ndarray, alpha: np.ndarray, beta: np.ndarray, nev: int):
    """The nev smallest Ritz values theta, the Ritz vectors as the rows of Y
    ([nev][N]) and the residual estimates |beta_m s_m|."""
    m = len(alpha)
    nev = min(nev, m)
    theta, S = eigh_tridiagonal(np.asarray(alpha, dtype=float), np.asarray(beta[:m - 1], dtype=float),
                                select="i", select_range=(0, nev - 1))
    Y = S.T @ np.asarray(V)[:m]
    est = np.abs(beta[m - 1] * S[m - 1, :])
    return theta, Y, est


def deflated_guess(M, Y: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x_0 = Y c with (Y^dag M Y) c = Y^dag b (Galerkin projection onto span Y)."""
    MY = np.stack([M(y) for y in Y])
    G = Y.conj() @ MY.T
    c = np.linalg.solve(G, Y.conj() @ b)
    return c @ Y
