"""Parity of the CUDA Improved Seed-CG with the oracle (Section 2, Algorithm 1
and Eq. 1-2), through the C-ABI.

Bars (from the method's specification): FP64 GPU vs FP64 oracle solutions
within 1e-6 relative at tol = 1e-8, every true residual <= tol recomputed in
FP64, iteration counts within 2%.  The Lanczos scalars of T and the seeded
guesses are compared before CG as well.  Mixed-precision modes must meet the
same residual bar; their distance to the oracle is bounded by cond(M) * tol
(several correct solutions exist within that distance)."""
import functools
import math

import numpy as np
import pytest

from oracle.seedcg import cg, classic_seed_cg, improved_seed_cg, seed_lanczos, galerkin_seed
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu, recompute_slack, rel

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _tiny():
    wl = W.WORKLOADS["tiny_4x4x4x4_nrhs4"]
    f = wl.fields[0]
    u = f.gauge()
    kappa = W.kappa_for(f.name)
    op = WilsonOperator(f.dims, u, kappa)
    eta = wl.sources_for(0)
    B = np.stack([op.Ddag(e) for e in eta]).reshape(len(eta), -1)
    return f.dims, u, kappa, op, eta, B, wl


def _gpu_B(s, eta):
    out = dev(np.zeros_like(eta))
    s.apply(seedcg.OP_DDAG, dev(eta), out, prec=0, multi=1)
    return out


def _within(a, b, frac=0.02):
    return abs(a - b) <= max(1, math.ceil(frac * max(a, b)))


@pytest.mark.parametrize("seed_mode", [0, 1])
def test_tiny_fp64_lanczos_scalars_and_seeds(seed_mode):
    need_gpu()
    dims, u, kappa, op, eta, B, wl = _tiny()
    ref = seed_lanczos(op.M, B, None, TOL, 4000, wl.reorth_period, wl.past_factor)
    s = seedcg.Solver(dims, u, kappa, past_factor=wl.past_factor, seed_mode=seed_mode,
                      stop_after_seed=1, precision="fp64")
    Bd = _gpu_B(s, eta)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(Bd, X, TOL, 0, wl.reorth_period)
    assert info["m_conv"] == ref.m_conv and info["m"] == ref.m
    assert info["po_count"] == ref.po_count
    a, b, d, m = seedcg.seedcg_get_lanczos(s.h, 10000)
    k = min(40, m)
    assert np.allclose(a[:k], ref.alpha[:k], rtol=1e-10, atol=0)
    assert np.allclose(b[:k], ref.beta[:k], rtol=1e-10, atol=0)
    assert np.allclose(d[:k], ref.delta[:k], rtol=1e-10, atol=0)
    want = ref.X.copy()
    if seed_mode == 1:   # Eq. (1) for j >= 2; x^1 by the LU recurrence of steps 3 and 6
        want[1:] = galerkin_seed(ref.V, ref.alpha, ref.beta, ref.R0)[1:]
    got = host(X).reshape(len(eta), -1)
    for j in range(len(eta)):
        assert rel(got[j], want[j]) <= 1e-8, (j, rel(got[j], want[j]))
    # the stored basis is the oracle's, and orthonormal after the last PO step
    Vg = dev(np.zeros((m,) + eta.shape[1:], dtype=np.complex128))
    seedcg.seedcg_get_basis(s.h, 0, m, Vg)
    Vg = host(Vg).reshape(m, -1)
    assert rel(Vg[:20], ref.V[:20]) <= 1e-10
    last = (m // wl.reorth_period) * wl.reorth_period
    G = Vg[:last].conj() @ Vg[:last].T
    assert np.abs(G - np.eye(last)).max() <= 1e-10
    s.close()


@pytest.mark.parametrize("seed_mode", [0, 1])
def test_tiny_fp64_full_solve_matches_oracle(seed_mode):
    need_gpu()
    dims, u, kappa, op, eta, B, wl = _tiny()
    ref = improved_seed_cg(op.M, B, None, TOL, 4000, wl.reorth_period, wl.past_factor,
                           seed_mode="literal" if seed_mode == 0 else "blocked")
    s = seedcg.Solver(dims, u, kappa, past_factor=wl.past_factor, seed_mode=seed_mode)
    Bd = _gpu_B(s, eta)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(Bd, X, TOL, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK
    got = host(X).reshape(len(eta), -1)
    for j in range(len(eta)):
        assert info["true_resid"][j] <= TOL
        tr = np.linalg.norm(B[j] - op.M(got[j])) / np.linalg.norm(B[j])
        assert tr <= TOL, (j, tr)
        assert rel(got[j], ref.X[j]) <= 1e-6
        assert _within(info["iters"][j], int(ref.iters[j])), (j, info["iters"], ref.iters)
    s.close()


@pytest.mark.parametrize("precision,tc", [("mixed_v32", 1), ("mixed_vbf16", 1), ("mixed_vbf16", 0),
                                          ("mixed_vbf16", 2)])
def test_tiny_mixed_meets_residual_bar(precision, tc):
    """tc: use_tensor_cores (bf16 basis: 1 tcgen05 for the seeds only, 2 also for
    the PO projection, 0 never)."""
    need_gpu()
    dims, u, kappa, op, eta, B, wl = _tiny()
    Md = op.dense(WilsonOperator.OP_M)
    ev = np.linalg.eigvalsh(Md)
    cond = ev[-1] / ev[0]
    Xd = np.linalg.solve(Md, B.T).T
    s = seedcg.Solver(dims, u, kappa, past_factor=wl.past_factor, precision=precision,
                      use_tensor_cores=tc)
    Bd = _gpu_B(s, eta)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(Bd, X, TOL, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK
    got = host(X).reshape(len(eta), -1)
    for j in range(len(eta)):
        tr = np.linalg.norm(B[j] - Md @ got[j]) / np.linalg.norm(B[j])
        assert tr <= TOL
        assert rel(got[j], Xd[j]) <= cond * TOL
    assert info["reliable_updates"] >= len(eta)
    s.close()


def test_edge_cases_ragged_lattice():
    """Ragged 6x4x4x6 lattice; nrhs = 1; a zero first right-hand side; a given x0."""
    need_gpu()
    dims = (6, 4, 4, 6)
    u = W.gauge_field(dims, 0.5, 8)
    kappa = 0.19
    op = WilsonOperator(dims, u, kappa)
    eta = W.z2_sources(dims, 3, 8)
    B = np.stack([op.Ddag(e) for e in eta])
    s = seedcg.Solver(dims, u, kappa, past_factor=1.2)
    # nrhs = 1
    X = dev(np.zeros_like(B[:1]))
    code, info = s.solve(dev(B[:1]), X, TOL, 0, 10)
    assert code == 0 and info["true_resid"][0] <= TOL
    ref = improved_seed_cg(op.M, B[:1].reshape(1, -1), None, TOL, 4000, 10, 1.2)
    assert info["m"] == ref.seed.m and rel(host(X), ref.X) <= 1e-6
    # zero first right-hand side: no Lanczos, the others solved by CG from zero
    Bz = B.copy()
    Bz[0] = 0
    X = dev(np.zeros_like(Bz))
    code, info = s.solve(dev(Bz), X, TOL, 0, 10)
    assert code == 0 and info["m"] == 0
    got = host(X)
    assert np.all(got[0] == 0)
    for j in (1, 2):
        assert np.linalg.norm(B[j] - op.M(got[j])) <= TOL * np.linalg.norm(B[j])
    # x0 given (a perturbed solution): r0 = b - M x0
    from oracle.seedcg import cg
    Xs = np.stack([cg(op.M, b.reshape(-1), None, 1e-12, 20000).x for b in B])
    X0 = (Xs * (1 + 1e-3)).reshape(B.shape)
    s.set_options(past_factor=1.2, x0_given=1)
    X = dev(X0)
    code, info = s.solve(dev(B), X, TOL, 0, 10)
    assert code == 0
    got = host(X)
    for j in range(3):
        assert np.linalg.norm(B[j] - op.M(got[j])) <= TOL * np.linalg.norm(B[j])
    # host (numpy) buffers work through the same entry point
    s.set_options(past_factor=1.2)
    Xh = np.zeros_like(B)
    code, info = s.solve(np.ascontiguousarray(B), Xh, TOL, 0, 10)
    assert code == 0 and info["true_resid"][2] <= TOL
    s.close()


@functools.lru_cache(maxsize=1)
def _small_oracle():
    """The 8^3x16, 12-point-source workload solved by the oracle (blocked
    seeds), shared by the tests of every precision mode."""
    wl = W.WORKLOADS["small_8x8x8x16_nrhs12"]
    f = wl.fields[0]
    u = f.gauge()
    kappa = W.kappa_for(f.name)
    op = WilsonOperator(f.dims, u, kappa)
    eta = wl.sources_for(0)
    B = np.stack([op.Ddag(e) for e in eta]).reshape(len(eta), -1)
    ref = improved_seed_cg(op.M, B, None, TOL, 6000, wl.reorth_period, wl.past_factor,
                           seed_mode="blocked")
    return wl, f, u, kappa, op, eta, B, ref


@pytest.mark.parametrize("precision", ["fp64", "mixed_v32", "mixed_vbf16"])
def test_small_8x8x8x16_point_sources(precision):
    """The 8^3x16, 12-point-source workload at full size against the oracle.
    FP64: solutions within 1e-6 and iterations within 2 %.  Mixed modes (bf16
    with the tcgen05 seed projection, as the benchmark runs): every residual,
    recomputed by the oracle, meets tol and the solutions are within the
    distance 2 cond(M) tol that two such residuals allow.  Every mode: x^1
    after the Lanczos run (steps 3 and 6, before any CG) is the oracle's x^1
    within cond(M) times the sum of the two residuals, and RHS 1 is not
    iterated again when its residual after Lanczos already meets tol."""
    need_gpu()
    wl, f, u, kappa, op, eta, B, ref = _small_oracle()
    cond = W.kappa_table()[f.name]["cond"]
    lam_max = W.kappa_table()[f.name]["lam_max"]
    s = seedcg.Solver(f.dims, u, kappa, past_factor=wl.past_factor, precision=precision,
                      m_max=6000, stop_after_seed=1)
    Bd = dev(B.reshape(eta.shape))
    X = dev(np.zeros_like(eta))
    code, info = s.solve(Bd, X, TOL, 0, wl.reorth_period)
    x1 = host(X).reshape(len(eta), -1)[0]
    b1 = np.linalg.norm(B[0])
    r1 = np.linalg.norm(B[0] - op.M(x1)) / b1
    r1_ref = np.linalg.norm(B[0] - op.M(ref.seed.X[0])) / b1
    assert rel(x1, ref.seed.X[0]) <= 2 * cond * (r1 + r1_ref), (r1, r1_ref)
    if precision == "fp64":
        assert rel(x1, ref.seed.X[0]) <= 1e-8
    s.set_options(past_factor=wl.past_factor, precision=precision, m_max=6000)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(Bd, X, TOL, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK
    if r1 <= TOL:
        assert info["iters"][0] == info["m"], (r1, info["iters"])
    got = host(X).reshape(len(eta), -1)
    for j in range(len(eta)):
        assert info["true_resid"][j] <= TOL
        rd = np.linalg.norm(B[j] - op.M(got[j])) / np.linalg.norm(B[j])
        slack = recompute_slack(lam_max, np.linalg.norm(got[j]), np.linalg.norm(B[j]))
        assert rd <= TOL + slack, (j, rd)
        assert rel(got[j], ref.X[j]) <= 2 * cond * (TOL + slack)
    if precision == "fp64":
        assert _within(info["m_conv"], ref.seed.m_conv)
        for j in range(len(eta)):
            assert rel(got[j], ref.X[j]) <= 1e-6
            assert _within(info["iters"][j], int(ref.iters[j])), (j, info["iters"], ref.iters)
    print(f"{precision}: x^1 residual after Lanczos {r1:.2e} (oracle {r1_ref:.2e}); "
          f"m_conv {info['m_conv']} m {info['m']} iters {info['iters']}")
    s.close()


def test_cg_only_matches_textbook_cg():
    """seed_mode = 3 (no seeding: standard CG from zero for every system, the
    baseline of Section 3) against the oracle's textbook CG: iterations within
    2 % and solutions within 1e-6 in FP64; no Lanczos run."""
    need_gpu()
    dims, u, kappa, op, eta, B, wl = _tiny()
    s = seedcg.Solver(dims, u, kappa, precision="fp64", seed_mode=3)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(_gpu_B(s, eta), X, TOL, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK and info["m"] == 0 and info["po_count"] == 0
    got = host(X).reshape(len(eta), -1)
    for j in range(len(eta)):
        ref = cg(op.M, B[j], None, TOL, 100000)
        assert rel(got[j], ref.x) <= 1e-6
        assert _within(info["iters"][j], ref.iters), (j, info["iters"][j], ref.iters)
        assert np.linalg.norm(B[j] - op.M(got[j])) <= TOL * np.linalg.norm(B[j])
    s.set_options(precision="mixed_vbf16", seed_mode=3)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(_gpu_B(s, eta), X, TOL, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK and info["m"] == 0
    got = host(X).reshape(len(eta), -1)
    lam_max = np.linalg.eigvalsh(op.dense(WilsonOperator.OP_M))[-1]
    for j in range(len(eta)):
        rd = np.linalg.norm(B[j] - op.M(got[j])) / np.linalg.norm(B[j])
        assert rd <= TOL + recompute_slack(lam_max, np.linalg.norm(got[j]), np.linalg.norm(B[j]))
    s.close()


def _near_critical(nrhs):
    """4^4, eps 0.5, kappa 0.23 (cond ~ 4e4, a few isolated low modes)."""
    dims = (4, 4, 4, 4)
    u = W.gauge_field(dims, 0.5, 7)
    op = WilsonOperator(dims, u, 0.23)
    eta = W.point_sources(dims, nrhs)
    B = np.stack([op.Ddag(e) for e in eta.reshape(nrhs, -1)])
    return dims, u, op, eta, B


def test_near_critical_seeding_gain_matches_oracle():
    """Past-convergence seeding in the regime where it pays (Section 3): the
    GPU reproduces the oracle's iteration counts, including the seeded
    system's gain over CG from zero, and its solutions."""
    need_gpu()
    dims, u, op, eta, B = _near_critical(2)
    ref = improved_seed_cg(op.M, B, None, TOL, 8000, 10, past_factor=2.0)
    s = seedcg.Solver(dims, u, 0.23, past_factor=2.0, precision="fp64")
    X = dev(np.zeros_like(eta))
    code, info = s.solve(_gpu_B(s, eta), X, TOL, 0, 10)
    assert code == seedcg.SEEDCG_OK
    assert _within(info["m_conv"], ref.seed.m_conv) and _within(info["m"], ref.seed.m)
    got = host(X).reshape(2, -1)
    for j in range(2):
        assert info["true_resid"][j] <= TOL
        assert rel(got[j], ref.X[j]) <= 1e-6
        assert _within(info["iters"][j], int(ref.iters[j])), (j, info["iters"], ref.iters)
    assert info["iters"][1] < 0.4 * info["m_conv"]
    s.close()


def test_po_guard_when_orthogonality_is_lost():
    """k = 100 on N = 3072: the basis loses orthogonality between PO steps and
    the step-8 guard ends Lanczos at i - 1, i a multiple of k, as in the
    oracle.  Past the loss of orthogonality the Lanczos trajectory depends on
    rounding, so only what is unique is compared with the oracle (the first
    hundred Lanczos scalars); the rest must be valid: the guard position,
    finite solutions and every true residual <= tol."""
    need_gpu()
    dims, u, op, eta, B = _near_critical(3)
    ref = seed_lanczos(op.M, B, None, TOL, 8000, 100, 2.0)
    assert ref.breakdown
    s = seedcg.Solver(dims, u, 0.23, past_factor=2.0, precision="fp64")
    X = dev(np.zeros_like(eta))
    code, info = s.solve(_gpu_B(s, eta), X, TOL, 0, 100)
    assert code == seedcg.SEEDCG_OK
    assert info["m_conv"] == 0 and info["m"] % 100 == 99 and info["m"] < 2000
    a, b, d, m = seedcg.seedcg_get_lanczos(s.h, 10000)
    assert np.allclose(a[:100], ref.alpha[:100], rtol=1e-8, atol=0)
    assert np.allclose(b[:100], ref.beta[:100], rtol=1e-8, atol=0)
    got = host(X).reshape(3, -1)
    assert np.all(np.isfinite(got))
    for j in range(3):
        tr = np.linalg.norm(B[j] - op.M(got[j])) / np.linalg.norm(B[j])
        assert info["true_resid"][j] <= TOL and tr <= TOL
    s.close()


def test_po_step8_as_printed_without_the_guard():
    """po_guard = 0 runs step 8 as printed at k = 100 on the near-critical 4^4
    field: the basis loses orthogonality between PO steps, the oracle's run
    continues far past where the guard would stop it and never converges.  As
    with the guard, past the loss of orthogonality the trajectory depends on
    rounding, so only the first hundred Lanczos scalars are compared with the
    oracle; the rest must be valid: finite solutions, every true residual <=
    tol, and a run that did not converge by the recurrence (m_conv = 0) but
    went past the guard's stopping point."""
    need_gpu()
    dims, u, op, eta, B = _near_critical(2)
    ref = seed_lanczos(op.M, B, None, TOL, 8000, 100, 2.0, po_guard=False)
    assert ref.m_conv == 0 and ref.m > 1000
    s = seedcg.Solver(dims, u, 0.23, past_factor=2.0, precision="fp64", po_guard=0, m_max=8000)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(_gpu_B(s, eta), X, TOL, 0, 100)
    assert code == seedcg.SEEDCG_OK
    assert info["m_conv"] == 0 and info["m"] > 1000
    a, b, d, m = seedcg.seedcg_get_lanczos(s.h, 10000)
    assert np.allclose(a[:100], ref.alpha[:100], rtol=1e-8, atol=0)
    assert np.allclose(b[:100], ref.beta[:100], rtol=1e-8, atol=0)
    got = host(X).reshape(2, -1)
    assert np.all(np.isfinite(got))
    for j in range(2):
        tr = np.linalg.norm(B[j] - op.M(got[j])) / np.linalg.norm(B[j])
        assert info["true_resid"][j] <= TOL and tr <= TOL * (1 + 1e-6)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_v32"])
def test_original_system_residual_is_binding(precision):
    """resid_mode = 1: B holds eta of D x = eta; the residual Section 3 monitors,
    ||eta - D x|| / ||eta||, recomputed here with the oracle's D, meets tol and
    equals the reported true_resid_D; the solution is D^-1 eta within
    cond(D) * tol."""
    need_gpu()
    dims, u, kappa, op, eta, B, wl = _tiny()
    Dd = op.dense(WilsonOperator.OP_D)
    sv = np.linalg.svd(Dd, compute_uv=False)
    cond_d = sv[0] / sv[-1]
    E = eta.reshape(len(eta), -1)
    Xd = np.linalg.solve(Dd, E.T).T
    s = seedcg.Solver(dims, u, kappa, past_factor=wl.past_factor, precision=precision, resid_mode=1)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(dev(eta), X, TOL, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK
    got = host(X).reshape(len(eta), -1)
    for j in range(len(eta)):
        rd = np.linalg.norm(E[j] - op.D(got[j])) / np.linalg.norm(E[j])
        assert rd <= TOL, (j, rd)
        assert abs(info["true_resid_D"][j] - rd) <= 1e-3 * rd + 1e-15
        assert rel(got[j], Xd[j]) <= cond_d * TOL
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_v32"])
def test_classic_repeated_seeding_matches_oracle(precision):
    """seed_mode = 2, the comparison variant of Section 1, against the oracle's
    classic_seed_cg: every true residual <= tol; in FP64 the per-system iteration
    counts within 2 % and the solutions within 1e-6 of the oracle's."""
    need_gpu()
    dims, u, kappa, op, eta, B, wl = _tiny()
    ref = classic_seed_cg(op.M, B, None, TOL, 4000, wl.reorth_period)
    s = seedcg.Solver(dims, u, kappa, precision=precision, seed_mode=2)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(_gpu_B(s, eta), X, TOL, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK
    got = host(X).reshape(len(eta), -1)
    for j in range(len(eta)):
        tr = np.linalg.norm(B[j] - op.M(got[j])) / np.linalg.norm(B[j])
        assert tr <= TOL and info["true_resid"][j] <= TOL
        if precision == "fp64":
            assert rel(got[j], ref.X[j]) <= 1e-6
            assert _within(info["iters"][j], int(ref.iters[j])), (j, info["iters"], ref.iters)
    # the first round is the seed system's own Lanczos run to convergence
    assert _within(info["m"], int(ref.lanczos_iters[0]))
    s.close()
