"""Ritz deflation on the GPU against the oracle (oracle/deflation.py): after a
past-convergence solve of one system, the library's 16 lowest Ritz values and
its Galerkin-deflated guess for a later system match the oracle's, and the guess
saves that system CG iterations."""
import numpy as np
import pytest

from oracle.deflation import deflated_guess, ritz_pairs
from oracle.seedcg import cg, improved_seed_cg
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu


def test_deflated_guess_matches_oracle_and_saves_iterations():
    need_gpu()
    dims, kappa, nev = (4, 4, 4, 4), 0.23, 16
    u = W.gauge_field(dims, 0.5, 7)
    op = WilsonOperator(dims, u, kappa)
    eta = W.point_sources(dims, 3)
    B = np.stack([op.Ddag(e) for e in eta.reshape(3, -1)]).reshape(eta.shape)
    ref = improved_seed_cg(op.M, B[:1].reshape(1, -1), None, 1e-10, 4000, 10, past_factor=2.0).seed
    theta_ref, Y, _ = ritz_pairs(ref.V, ref.alpha, ref.beta, nev)
    x0_ref = deflated_guess(op.M, Y, B[2].reshape(-1))
    s = seedcg.Solver(dims, u, kappa, precision="fp64", past_factor=2.0)
    X = dev(np.zeros_like(B[:1]))
    code, info = s.solve(dev(B[:1]), X, 1e-10, 0, 10)
    assert code == seedcg.SEEDCG_OK
    X0 = dev(np.zeros_like(B[2:3]))
    theta = seedcg.seedcg_deflate_guess(s.h, nev, dev(B[2:3]), X0)
    assert np.allclose(theta, theta_ref, rtol=1e-8, atol=0)
    x0 = host(X0).reshape(-1)
    assert rel(x0, x0_ref) <= 1e-6
    cold = cg(op.M, B[2].reshape(-1), None, 1e-8, 20000).iters
    warm = cg(op.M, B[2].reshape(-1), x0, 1e-8, 20000).iters
    assert warm < 0.7 * cold, (warm, cold)
    # the guess goes straight into a solve (x0_given)
    s.set_options(precision="fp64", past_factor=1.0, x0_given=1)
    code, info2 = s.solve(dev(B[2:3]), X0, 1e-8, 0, 10)
    assert code == seedcg.SEEDCG_OK and info2["true_resid"][0] <= 1e-8
    assert info2["iters"][0] < 0.7 * cold
    s.close()
