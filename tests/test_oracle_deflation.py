"""Pins for Ritz extraction and deflated initial guesses (oracle/deflation.py,
CPU): the Ritz residuals equal Lanczos' |beta_m s_m| estimate, converged Ritz
values are eigenvalues of the dense M, the deflated guess satisfies its Galerkin
condition, and on a near-critical field it saves a later system CG iterations."""
import numpy as np

from oracle.deflation import deflated_guess, ritz_pairs
from oracle.seedcg import cg, improved_seed_cg
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import workloads as W

DIMS = (4, 4, 4, 4)


def _run(kappa, seed=7):
    op = WilsonOperator(DIMS, W.gauge_field(DIMS, 0.5, seed), kappa)
    eta = W.point_sources(DIMS, 3).reshape(3, -1)
    B = np.stack([op.Ddag(e) for e in eta])
    r = improved_seed_cg(op.M, B[:1], None, 1e-10, 4000, 10, past_factor=2.0)
    return op, B, r.seed


def test_ritz_residuals_and_values():
    op, B, s = _run(0.2)
    theta, Y, est = ritz_pairs(s.V, s.alpha, s.beta, 12)
    lam = np.linalg.eigvalsh(op.dense(WilsonOperator.OP_M))
    scale = lam[-1]
    assert np.all(np.diff(theta) >= 0)
    for i in range(len(theta)):
        res = np.linalg.norm(op.M(Y[i]) - theta[i] * Y[i])
        assert abs(res - est[i]) <= 1e-7 * scale, (i, res, est[i])
        assert abs(np.linalg.norm(Y[i]) - 1.0) <= 1e-8
        # a Ritz value is within its residual of an eigenvalue of M
        assert np.abs(lam - theta[i]).min() <= res + 1e-10 * scale
    assert abs(theta[0] - lam[0]) <= 1e-8 * scale


def test_deflated_guess_galerkin_condition_and_gain():
    op, B, s = _run(0.23)
    theta, Y, est = ritz_pairs(s.V, s.alpha, s.beta, 16)
    b = B[2]
    x0 = deflated_guess(op.M, Y, b)
    g = Y.conj() @ (b - op.M(x0))
    assert np.abs(g).max() <= 1e-9 * np.linalg.norm(b)
    cold = cg(op.M, b, None, 1e-8, 20000).iters
    warm = cg(op.M, b, x0, 1e-8, 20000).iters
    assert warm < 0.7 * cold, (warm, cold)


def test_deflated_guess_galerkin_condition_for_any_basis():
    """The Galerkin projection holds for a general basis too (a Gram matrix that
    is neither diagonal nor real), not only for Ritz vectors."""
    op = WilsonOperator(DIMS, W.gauge_field(DIMS, 0.5, 8), 0.2)
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((3, op.n)) + 1j * rng.standard_normal((3, op.n))
    b = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    x0 = deflated_guess(op.M, Y, b)
    g = Y.conj() @ (b - op.M(x0))
    assert np.abs(g).max() <= 1e-9 * np.linalg.norm(b) * np.linalg.norm(Y[0])
