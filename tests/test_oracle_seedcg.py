"""Pins for the oracle's Improved Seed-CG (CPU only).

Each check ties the oracle to something other than itself: the LU
factorisation of Eq. (2), textbook CG (the D-Lanczos equivalence the paper
cites), the closed form of Eq. (1), dense solves and dense eigensolves on tiny
lattices, and the orthogonality that re-orthogonalisation must restore.
"""
import math

import numpy as np
import pytest

from oracle import freefield
from oracle.seedcg import (cg, classic_seed_cg, galerkin_seed, improved_seed_cg, lanczos_extremes, lu_factors,
                           seed_lanczos, tridiag)
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import workloads as W

DIMS = (4, 2, 2, 4)          # 64 sites, N = 768


def _problem(dims=DIMS, kappa=0.2, eps=0.5, seed=7, nrhs=4):
    op = WilsonOperator(dims, W.gauge_field(dims, eps, seed), kappa)
    eta = W.z2_sources(dims, nrhs, seed).reshape(nrhs, -1)
    B = np.stack([op.Ddag(e) for e in eta])
    return op, eta, B


def _textbook_cg_iterates(M, b, n):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    out = []
    for _ in range(n):
        q = M(p)
        a = rr / np.vdot(p, q).real
        x = x + a * p
        r = r - a * q
        rn = np.vdot(r, r).real
        p = r + (rn / rr) * p
        rr = rn
        out.append(x.copy())
    return out


def test_lu_of_T_reconstructs_T():
    op, _, B = _problem()
    res = seed_lanczos(op.M, B, None, 1e-30, 40, 0)
    T = tridiag(res.alpha, res.beta)
    L, U, gam, dlt = lu_factors(res.alpha, res.beta)
    assert np.abs(L @ U - T).max() <= 1e-14 * np.abs(T).max()
    # the recurrence inside Algorithm 1 (step 6) gives the same factors
    assert np.allclose(res.delta, dlt, rtol=1e-13, atol=0)
    assert np.allclose(res.gamma, gam, rtol=1e-13, atol=0)
    # tridiagonal solve by the factors equals a dense solve
    rhs = np.arange(1.0, len(res.alpha) + 1)
    y = np.linalg.solve(U, np.linalg.solve(L, rhs))
    assert np.allclose(y, np.linalg.solve(T, rhs), rtol=1e-9)


def test_lanczos_first_rhs_equals_textbook_cg():
    """D-Lanczos is CG: x^1 after i steps equals the i-th CG iterate, and
    beta_i |zeta_i/delta_i| equals the true residual norm."""
    op, _, B = _problem()
    n = 20
    res = seed_lanczos(op.M, B[:1], None, 1e-30, n, 0, keep_x1_history=True)
    ref = _textbook_cg_iterates(op.M, B[0], n)
    for i in range(n):
        x = res.x1_history[i]
        assert np.linalg.norm(x - ref[i]) <= 1e-10 * np.linalg.norm(ref[i])
        true_r = np.linalg.norm(B[0] - op.M(x))
        assert abs(res.resid_est[i] - true_r) <= 1e-8 * np.linalg.norm(B[0])


def test_literal_seed_equals_eq1():
    """Steps 4 and 7 (incremental LU update) reproduce x_0 + V T^{-1} V^dag r_0."""
    op, _, B = _problem()
    rng = np.random.default_rng(3)
    X0 = 0.01 * (rng.standard_normal(B.shape) + 1j * rng.standard_normal(B.shape))
    res = seed_lanczos(op.M, B, X0, 1e-30, 30, 0)
    Xb = galerkin_seed(res.V, res.alpha, res.beta, res.R0, X0)
    # dense T^{-1} as a second route to Eq. (1)
    T = tridiag(res.alpha, res.beta)
    Xd = X0 + (res.V.T @ np.linalg.solve(T, res.V.conj() @ res.R0.T)).T
    for j in range(B.shape[0]):
        nrm = np.linalg.norm(Xd[j])
        assert np.linalg.norm(res.X[j] - Xd[j]) <= 1e-10 * nrm
        assert np.linalg.norm(Xb[j] - Xd[j]) <= 1e-12 * nrm
    # R0 really is b - M x0
    assert np.linalg.norm(res.R0[1] - (B[1] - op.M(X0[1]))) < 1e-14 * np.linalg.norm(B[1])


def test_galerkin_condition_with_po():
    """x^j from Eq. (1) makes the residual orthogonal to span(V)."""
    op, _, B = _problem()
    res = seed_lanczos(op.M, B, None, 1e-30, 60, 1)
    X = galerkin_seed(res.V, res.alpha, res.beta, res.R0)
    for j in range(1, B.shape[0]):
        g = res.V.conj() @ (B[j] - op.M(X[j]))
        assert np.linalg.norm(g) <= 1e-8 * np.linalg.norm(res.V.conj() @ res.R0[j])


def test_periodic_reorthogonalisation_restores_orthogonality():
    """Plain Lanczos loses orthogonality once Ritz values converge (Section 2);
    PO every k steps keeps V orthonormal to ~1e-10 right after each PO step."""
    op, _, B = _problem(kappa=0.22)
    m = 200
    plain = seed_lanczos(op.M, B[:1], None, 1e-30, m, 0)
    loss = np.abs(plain.V.conj() @ plain.V.T - np.eye(plain.m)).max()
    assert loss > 1e-4
    k = 10
    po = seed_lanczos(op.M, B[:1], None, 1e-30, m, k)
    assert po.po_count == m // k
    for i in range(k, po.m + 1, k):
        Vi = po.V[:i]
        assert np.abs(Vi.conj() @ Vi.T - np.eye(i)).max() <= 1e-10
    full = seed_lanczos(op.M, B[:1], None, 1e-30, m, 1, po_passes=2)
    assert np.abs(full.V.conj() @ full.V.T - np.eye(full.m)).max() <= 1e-12


def test_T_extreme_ritz_values_match_dense_spectrum():
    """Past convergence, T_m holds the extreme eigenvalues of M (Section 2:
    the subspace contains accurate low eigenvectors)."""
    dims = (4, 4, 4, 4)
    op = WilsonOperator(dims, W.gauge_field(dims, 0.3, 0), 0.2)
    ev = np.linalg.eigvalsh(op.dense(WilsonOperator.OP_M))
    b = op.Ddag(W.z2_sources(dims, 1, 0).reshape(-1))
    res = seed_lanczos(op.M, b[None], None, 1e-10, 600, 10, past_factor=2.0)
    assert res.m_conv > 0 and res.m >= 2 * res.m_conv - 1
    ritz = np.linalg.eigvalsh(tridiag(res.alpha, res.beta))
    assert abs(ritz[0] - ev[0]) <= 1e-8 * ev[0]
    assert abs(ritz[-1] - ev[-1]) <= 1e-8 * ev[-1]


@pytest.mark.parametrize("seed_mode", ["literal", "blocked"])
def test_whole_method_against_dense_solve(seed_mode):
    op, _, B = _problem(nrhs=5)
    Md = op.dense(WilsonOperator.OP_M)
    ev = np.linalg.eigvalsh(Md)
    cond = ev[-1] / ev[0]
    tol = 1e-8
    out = improved_seed_cg(op.M, B, None, tol, 2000, 10, past_factor=1.5, seed_mode=seed_mode)
    Xd = np.linalg.solve(Md, B.T).T
    for j in range(B.shape[0]):
        assert out.true_resid[j] <= tol
        assert np.linalg.norm(B[j] - Md @ out.X[j]) <= tol * np.linalg.norm(B[j])
        assert np.linalg.norm(out.X[j] - Xd[j]) <= cond * tol * np.linalg.norm(Xd[j])
    # seeding pays: the seeded systems need fewer CG iterations than from zero
    plain = [cg(op.M, B[j], None, tol, 5000).iters for j in range(1, B.shape[0])]
    assert max(out.cg_iters[1:]) < min(plain)


def test_brute_force_2x2x2x2():
    dims = (2, 2, 2, 2)
    op = WilsonOperator(dims, W.gauge_field(dims, 0.8, 5), 0.19)
    B = W.random_spinors(dims, 3, 1).reshape(3, -1)
    d = op.dense(WilsonOperator.OP_D)
    Md = d.conj().T @ d
    out = improved_seed_cg(op.M, B, None, 1e-10, 500, 5, past_factor=2.0)
    Xd = np.linalg.solve(Md, B.T).T
    cond = np.linalg.cond(Md)
    for j in range(3):
        assert np.linalg.norm(out.X[j] - Xd[j]) <= cond * 1e-10 * np.linalg.norm(Xd[j])


def test_m_rule_past_convergence_and_extra_iters():
    op, _, B = _problem(nrhs=2)
    a = seed_lanczos(op.M, B, None, 1e-8, 5000, 10, past_factor=1.5)
    assert a.m == math.ceil(1.5 * a.m_conv)
    b = seed_lanczos(op.M, B, None, 1e-8, 5000, 10, past_factor=1.0, extra_iters=7)
    assert b.m_conv == a.m_conv and b.m == a.m_conv + 7
    c = seed_lanczos(op.M, B, None, 1e-8, a.m_conv + 3, 10, past_factor=2.0)
    assert c.m == a.m_conv + 3
    # m_conv is the first i whose residual estimate is below tol ||b^1||
    bn = np.linalg.norm(B[0])
    assert a.resid_est[a.m_conv - 1] <= 1e-8 * bn < a.resid_est[a.m_conv - 2]


def test_edge_cases():
    op, _, B = _problem(nrhs=3)
    # zero first right-hand side: no Lanczos, others go straight to CG
    Bz = B.copy()
    Bz[0] = 0
    out = improved_seed_cg(op.M, Bz, None, 1e-8, 100, 10)
    assert out.seed.m == 0 and np.all(out.X[0] == 0)
    assert out.true_resid[1] <= 1e-8 and out.true_resid[2] <= 1e-8
    # one right-hand side
    out1 = improved_seed_cg(op.M, B[:1], None, 1e-8, 2000, 10, past_factor=1.0)
    assert out1.true_resid[0] <= 1e-8
    # exact initial guess for RHS 1
    x_exact = np.linalg.solve(op.dense(WilsonOperator.OP_M), B[0])
    X0 = np.zeros_like(B)
    X0[0] = x_exact
    res = seed_lanczos(op.M, B, X0, 1e-8, 100, 10)
    assert res.beta0 <= 1e-10 * np.linalg.norm(B[0])


def test_breakdown_on_eigenvector():
    """b^1 an eigenvector of M: beta_1 = 0, x^1 = b/lambda is exact at i = 1."""
    dims = (4, 2, 2, 4)
    op = WilsonOperator(dims, W.unit_gauge(dims), 0.1)
    p = (np.pi / 2, 0.0, np.pi, np.pi / 4)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((4, 3)) + 0j
    b = freefield.plane_wave(dims, p, u).reshape(-1)
    res = seed_lanczos(op.M, b[None], None, 1e-8, 50, 10)
    assert res.breakdown and res.m == 1
    lam = (1 - 2 * 0.1 * sum(np.cos(q) for q in p)) ** 2 + 4 * 0.01 * sum(np.sin(q) ** 2 for q in p)
    assert np.linalg.norm(res.X[0] - b / lam) <= 1e-13 * np.linalg.norm(b / lam)


def test_lanczos_extremes_free_field_cond():
    """Set-up pin: the tuning's Lanczos cond estimate equals the closed form."""
    dims = (8, 8, 4, 8)
    kappa = 0.124
    op = WilsonOperator(dims, W.unit_gauge(dims), kappa)
    lo, hi, _ = lanczos_extremes(op.M, op.n, max_iters=3000, rtol=1e-6)
    ev = freefield.spectrum_M(dims, kappa)
    assert abs(lo - ev[0]) <= 1e-4 * ev[0]
    assert abs(hi - ev[-1]) <= 1e-6 * ev[-1]


@pytest.mark.parametrize("passes", [1, 2])
def test_step8_reorth_against_every_previous_vector(passes):
    """Step 8 in isolation: v_i leaves orthogonal to ALL of v_1..v_{i-1} (even
    when it leans on v_{i-1}), with unit norm and in span(V, v_i); f leaves
    orthogonal to v_1..v_i."""
    rng = np.random.default_rng(4)
    n, i = 300, 9
    q, _ = np.linalg.qr(rng.standard_normal((n, i - 1)) + 1j * rng.standard_normal((n, i - 1)))
    V = np.zeros((i + 2, n), dtype=np.complex128)
    V[:i - 1] = q.T
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v = 0.1 * z + 3.0 * V[i - 2] + 0.5 * V[0]
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n) + 2.0 * V[i - 2]
    from oracle.seedcg import periodic_reorth
    v2, f2 = periodic_reorth(V, i, v, f, passes)
    assert abs(np.linalg.norm(v2) - 1) < 1e-14
    assert np.abs(V[:i - 1].conj() @ v2).max() < 1e-14
    assert np.abs(V[:i].conj() @ f2).max() < 1e-13
    assert np.array_equal(V[i - 1], v2)
    # v2 is (z's part outside span V_{i-1}) normalised: the only admissible result
    zp = z - (V[:i - 1].conj() @ z) @ V[:i - 1]
    assert np.linalg.norm(v2 - zp / np.linalg.norm(zp)) < 1e-13


def _near_critical(nrhs=2):
    """4^4, eps 0.5, kappa 0.23: cond(M) ~ 4e4 with a few isolated low modes
    (dense spectrum: lambda_2 / lambda_1 ~ 1.9, lambda_8 / lambda_1 ~ 9), the
    near-critical regime of the paper's example (Section 3)."""
    dims = (4, 4, 4, 4)
    op = WilsonOperator(dims, W.gauge_field(dims, 0.5, 7), 0.23)
    eta = W.point_sources(dims, nrhs).reshape(nrhs, -1)
    return op, np.stack([op.Ddag(e) for e in eta])


def test_seeding_gain_near_critical():
    """Section 3: the seeded second system needs far fewer CG iterations
    (matvecs) than CG from zero, and running RHS 1 further past convergence
    does not make it worse."""
    op, B = _near_critical()
    plain = cg(op.M, B[1], None, 1e-8, 20000).iters
    r12 = improved_seed_cg(op.M, B, None, 1e-8, 20000, 10, past_factor=1.2)
    r20 = improved_seed_cg(op.M, B, None, 1e-8, 20000, 10, past_factor=2.0)
    assert r20.seed.m == math.ceil(2.0 * r20.seed.m_conv)
    assert r20.cg_iters[1] < 0.4 * plain
    assert r20.cg_iters[1] <= r12.cg_iters[1] < plain
    assert max(r12.true_resid.max(), r20.true_resid.max()) <= 1e-8


def test_po_guard_when_orthogonality_is_lost_between_po_steps():
    """With k = 100 on N = 3072 the basis loses orthogonality between PO
    steps; a PO step then lengthens f (impossible for an orthogonal
    projection) and the guard of step 8 ends Lanczos at i - 1, i a multiple of
    k.  The stored basis is then far from orthonormal, which is what the
    guard detects, and CG still brings every system to tol."""
    op, B = _near_critical(3)
    r = improved_seed_cg(op.M, B, None, 1e-8, 20000, 100, past_factor=2.0)
    s = r.seed
    assert s.breakdown and s.m % 100 == 99 and s.po_count == (s.m + 1) // 100 - 1
    V = s.V
    assert np.abs(V.conj() @ V.T - np.eye(len(V))).max() > 0.1
    assert np.all(np.isfinite(r.X)) and r.true_resid.max() <= 1e-8
    # the guard never fires while PO keeps the basis orthonormal (k = 10)
    r10 = improved_seed_cg(op.M, B[:2], None, 1e-8, 20000, 10, past_factor=1.0)
    assert not r10.seed.breakdown and r10.seed.m == r10.seed.m_conv


def test_po_guard_reading_from_projection_geometry():
    """The two tests of the step-8 guard follow from the geometry of one
    classical Gram-Schmidt pass v' = v - V c, c = V^dag v:
        ||v'||^2 = ||v||^2 - ||c||^2 + c^dag (G - I) c,   G = V^dag V.
    (a) For an orthonormal V (G = I) this is Pythagoras: the pass never
        lengthens a vector, and ||v'|| = ||v|| sin(theta), theta the angle
        between v and span V.  A pass that lengthens f therefore proves
        c^dag (G - I) c > ||c||^2: G has an eigenvalue above 2, i.e. some
        direction is stored twice (a ghost copy) and V is no basis of the
        Krylov space T describes.  The 1 % margin lies far above the rounding
        of an orthonormal V in any stored precision (relative 2^-9 in bf16).
    (b) ||v'|| < 1/2 for a unit v_i means theta < 30 degrees: the Lanczos
        vector has mostly re-entered the stored space (in exact arithmetic
        theta = 90 degrees), so the orthogonality lost since the previous PO
        step is of order one, not of rounding size."""
    from oracle.seedcg import periodic_reorth
    rng = np.random.default_rng(21)
    n, i = 400, 12
    q, _ = np.linalg.qr(rng.standard_normal((n, i - 1)) + 1j * rng.standard_normal((n, i - 1)))
    V = np.zeros((i + 1, n), dtype=np.complex128)
    V[:i - 1] = q.T
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    zp = z - (V[:i - 1].conj() @ z) @ V[:i - 1]
    zp /= np.linalg.norm(zp)
    y = V[3] * np.exp(0.4j)                      # a unit vector inside span V
    for theta_deg in (10.0, 25.0, 29.0, 31.0, 45.0, 80.0):
        th = np.deg2rad(theta_deg)
        v = np.sin(th) * zp + np.cos(th) * y          # unit vector at angle theta to span V
        f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        Vw = V.copy()
        v2, f2, ok = periodic_reorth(Vw, i, v, f, 1, guard=True)
        c = V[:i - 1].conj() @ v
        # Pythagoras for the orthonormal basis, and ||v'|| = sin(theta)
        vp = v - c @ V[:i - 1]
        assert abs(np.linalg.norm(vp) ** 2 - (1.0 - np.linalg.norm(c) ** 2)) < 1e-13
        assert abs(np.linalg.norm(vp) - np.sin(th)) < 1e-13
        assert ok == (theta_deg > 30.0), theta_deg
        if ok:   # an orthonormal basis never lengthens f
            assert np.linalg.norm(f2) <= np.linalg.norm(f) * (1 + 1e-14)
    # a direction stored twice (G's top eigenvalue 2) is the borderline: along it the
    # pass keeps the length; stored three times (eigenvalue 3) the pass lengthens f
    f = 2.0 * V[0] + 0.05 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    for copies, grows in ((2, False), (3, True)):
        Vd = V.copy()
        for k in range(1, copies):
            Vd[i - 1 - k] = V[0]
        fd = f - (Vd[:i - 1].conj() @ f) @ Vd[:i - 1]
        G = Vd[:i - 1].conj() @ Vd[:i - 1].T
        assert abs(np.linalg.eigvalsh(G).max() - copies) < 1e-12
        assert (np.linalg.norm(fd) > 1.01 * np.linalg.norm(f)) == grows, copies


def test_classic_repeated_seeding():
    """The comparison variant (Section 1): every round's seed system runs D-Lanczos
    from its seeded guess, which is textbook CG from that guess (same iteration
    count within one); later systems start closer and need fewer iterations than CG
    from zero; the solutions are the dense solve's within cond(M) * tol."""
    op, eta, B = _problem(nrhs=4)
    tol = 1e-9
    Md = op.dense(WilsonOperator.OP_M)
    ev = np.linalg.eigvalsh(Md)
    Xd = np.linalg.solve(Md, B.T).T
    for mode in ("blocked", "literal"):
        r = classic_seed_cg(op.M, B, None, tol, 4000, 10, seed_mode=mode)
        assert r.true_resid.max() <= tol
        # every system is converged by its own round; the final CG only mops up
        assert r.cg_iters.max() <= 5, r.cg_iters
        for j in range(4):
            assert np.linalg.norm(r.X[j] - Xd[j]) <= ev[-1] / ev[0] * tol * np.linalg.norm(Xd[j])
    # round by round, without PO (D-Lanczos is then CG): the seeded guesses of round j,
    # then textbook CG from them needs the same number of iterations
    nopo = classic_seed_cg(op.M, B, None, tol, 4000, 0)
    X = np.zeros_like(B)
    for j in range(4):
        start = X[j:] if j > 0 else None
        res = seed_lanczos(op.M, B[j:], start, tol, 4000, 0, 1.0)
        textbook = cg(op.M, B[j], None if start is None else start[0], tol, 4000).iters
        assert abs(res.m - textbook) <= 2, (j, res.m, textbook)
        assert res.m == nopo.lanczos_iters[j]
        X[j:] = galerkin_seed(res.V, res.alpha, res.beta, res.R0, start)
    plain = [cg(op.M, B[j], None, tol, 4000).iters for j in range(4)]
    assert all(nopo.lanczos_iters[j] < plain[j] for j in range(1, 4))
