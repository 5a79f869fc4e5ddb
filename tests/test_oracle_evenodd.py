"""Pins for the even-odd preconditioned system of Section 3 (oracle/evenodd.py,
CPU): the hopping term couples opposite parities only, the Schur-complement
route reproduces the dense solution of D x = eta, A^dag = gamma5 A gamma5 is
A's adjoint, the seed method on A^dag A solves the odd-site system, and the
preconditioned system is better conditioned than D^dag D."""
import numpy as np

from oracle.evenodd import EvenOddOperator, parity
from oracle.seedcg import improved_seed_cg
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import workloads as W

DIMS = (4, 4, 4, 4)


def _eo(kappa=0.2, seed=11):
    op = WilsonOperator(DIMS, W.gauge_field(DIMS, 0.5, seed), kappa)
    return op, EvenOddOperator(op)


def test_parity_checkerboard():
    par = parity(DIMS)
    assert par.sum() * 2 == par.size
    assert par[0] == 0 and par[1] == 1 and par[DIMS[0]] == 1 and par[DIMS[0] + 1] == 0


def test_hopping_couples_opposite_parities_only():
    op, eo = _eo()
    psi = W.random_spinors(DIMS, 1, 3)[0]
    h_from_even = eo.hop(eo.embed_even(psi[eo.even]))
    h_from_odd = eo.hop(eo.embed_odd(psi[eo.odd]))
    assert np.abs(h_from_even[eo.even]).max() == 0.0
    assert np.abs(h_from_odd[eo.odd]).max() == 0.0
    assert np.abs(h_from_even[eo.odd]).max() > 0.1


def test_schur_complement_route_solves_d_x_eq_eta():
    op, eo = _eo()
    eta = W.random_spinors(DIMS, 1, 4)[0]
    Dd = op.dense(WilsonOperator.OP_D)
    x_ref = np.linalg.solve(Dd, eta.reshape(-1))
    Ad = np.empty((eo.n, eo.n), dtype=np.complex128)
    e = np.zeros(eo.n, dtype=np.complex128)
    for k in range(eo.n):
        e[k] = 1.0
        Ad[:, k] = eo.A(e)
        e[k] = 0.0
    x_o = np.linalg.solve(Ad, eo.source(eta).reshape(-1))
    x = eo.reconstruct(x_o, eta).reshape(-1)
    assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
    # A^dag really is the adjoint, and A^dag A is Hermitian positive definite
    rng = np.random.default_rng(5)
    a = rng.standard_normal(eo.n) + 1j * rng.standard_normal(eo.n)
    b = rng.standard_normal(eo.n) + 1j * rng.standard_normal(eo.n)
    assert abs(np.vdot(b, eo.A(a)) - np.vdot(eo.Adag(b), a)) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(b) * 10
    Md = Ad.conj().T @ Ad
    ev = np.linalg.eigvalsh(Md)
    assert ev[0] > 0
    # the preconditioned system is better conditioned than D^dag D
    evf = np.linalg.eigvalsh(Dd.conj().T @ Dd)
    assert ev[-1] / ev[0] < evf[-1] / evf[0]


def test_seed_method_on_the_odd_site_system():
    op, eo = _eo(kappa=0.21, seed=12)
    etas = W.point_sources(DIMS, 2)
    phis = np.stack([eo.source(e).reshape(-1) for e in etas])
    B = np.stack([eo.Adag(p) for p in phis])
    r = improved_seed_cg(eo.M, B, None, 1e-10, 4000, 10, past_factor=1.5)
    assert r.true_resid.max() <= 1e-10
    for j in range(2):
        x = eo.reconstruct(r.X[j], etas[j]).reshape(-1)
        rd = np.linalg.norm(etas[j].reshape(-1) - op.D(x)) / np.linalg.norm(etas[j])
        assert rd <= 1e-6, (j, rd)
