"""The even-odd preconditioned operator of Section 3 on the GPU against the
oracle (oracle/evenodd.py): A, A^dag and A^dag A on odd-site vectors (FP64 to
1e-13, FP32 to 1e-5 relative), the source phi and the reconstruction of the full
solution, on a hypercube and on a ragged lattice."""
import numpy as np
import pytest

from oracle.evenodd import EvenOddOperator
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,kappa", [((4, 4, 4, 4), 0.2), ((4, 2, 2, 6), 0.17)])
def test_eo_operator_matches_oracle(dims, kappa):
    need_gpu()
    u = W.gauge_field(dims, 0.5, 61)
    op = WilsonOperator(dims, u, kappa)
    eo = EvenOddOperator(op)
    s = seedcg.Solver(dims, u, kappa)
    vh = W.volume(dims) // 2
    x = W.random_spinors(dims, 2, 62)[:, :vh]
    for code, ref in ((seedcg.EO_A, eo.A), (seedcg.EO_ADAG, eo.Adag), (seedcg.EO_MEO, eo.M)):
        want = np.stack([ref(x[r]) for r in range(2)])
        for prec, tol in ((0, 1e-13), (1, 1e-5)):
            out = dev(np.zeros_like(x))
            seedcg.seedcg_apply_eo(s.h, code, prec, dev(x), out)
            assert rel(host(out), want) <= tol, (code, prec, rel(host(out), want))
    eta = W.random_spinors(dims, 2, 63)
    phi = dev(np.zeros_like(x))
    seedcg.seedcg_eo_source(s.h, dev(eta), phi)
    want_phi = np.stack([eo.source(eta[r]) for r in range(2)])
    assert rel(host(phi), want_phi) <= 1e-13
    full = dev(np.zeros_like(eta))
    seedcg.seedcg_eo_reconstruct(s.h, dev(x), dev(eta), full)
    want_full = np.stack([eo.reconstruct(x[r], eta[r]) for r in range(2)])
    assert rel(host(full), want_full) <= 1e-13
    s.close()


def test_eo_route_solves_the_original_system():
    """Dense solve of the odd-site system on the host, GPU source and
    reconstruction around it: D x = eta to 1e-10."""
    need_gpu()
    dims, kappa = (4, 4, 4, 4), 0.2
    u = W.gauge_field(dims, 0.5, 64)
    op = WilsonOperator(dims, u, kappa)
    eo = EvenOddOperator(op)
    s = seedcg.Solver(dims, u, kappa)
    eta = W.random_spinors(dims, 1, 65)
    vh = W.volume(dims) // 2
    phi = dev(np.zeros((1, vh, 4, 3), dtype=np.complex128))
    seedcg.seedcg_eo_source(s.h, dev(eta), phi)
    Ad = np.empty((eo.n, eo.n), dtype=np.complex128)
    e = np.zeros(eo.n, dtype=np.complex128)
    for k in range(eo.n):
        e[k] = 1.0
        Ad[:, k] = eo.A(e)
        e[k] = 0.0
    x_o = np.linalg.solve(Ad, host(phi).reshape(-1)).reshape(1, vh, 4, 3)
    full = dev(np.zeros_like(eta))
    seedcg.seedcg_eo_reconstruct(s.h, dev(x_o), dev(eta), full)
    r = eta.reshape(-1) - op.D(host(full).reshape(-1))
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(eta)
    s.close()


def test_eo_rejects_host_pointers():
    need_gpu()
    dims = (4, 4, 4, 4)
    s = seedcg.Solver(dims, W.gauge_field(dims, 0.5, 66), 0.1)
    x = np.zeros((1, 128, 4, 3), dtype=np.complex128)
    with pytest.raises(seedcg.SeedCGError) as e:
        seedcg.seedcg_apply_eo(s.h, seedcg.EO_A, 0, x, np.zeros_like(x))
    assert e.value.code == seedcg.SEEDCG_ERR_ARG
    s.close()


def test_eo_seed_cg_matches_oracle():
    """Improved Seed-CG on the even-odd system (Section 3's setup) against the
    oracle's improved_seed_cg on A^dag A (blocked seeds): m_conv, m and the
    per-system iterations within 2 %, the reconstructed full solutions within
    1e-6, and D x = eta solved."""
    need_gpu()
    dims, kappa, tol = (4, 4, 4, 4), 0.21, 1e-10
    u = W.gauge_field(dims, 0.5, 12)
    op = WilsonOperator(dims, u, kappa)
    eo = EvenOddOperator(op)
    from oracle.seedcg import improved_seed_cg
    eta = W.point_sources(dims, 2)
    B = np.stack([eo.Adag(eo.source(e)).reshape(-1) for e in eta])
    ref = improved_seed_cg(eo.M, B, None, tol, 4000, 10, past_factor=1.5, seed_mode="blocked")
    s = seedcg.Solver(dims, u, kappa, precision="fp64", past_factor=1.5, m_max=4000)
    X = dev(np.zeros_like(eta))
    code, info = seedcg.seedcg_solve_eo(s.h, dev(eta), X, tol, 0, 10)
    assert code == seedcg.SEEDCG_OK

    def within(a, b):
        return abs(a - b) <= max(1, int(np.ceil(0.02 * max(a, b))))

    assert within(info["m_conv"], ref.seed.m_conv) and within(info["m"], ref.seed.m), (info, ref.seed.m)
    got = host(X)
    for j in range(2):
        assert within(info["iters"][j], int(ref.iters[j])), (info["iters"], ref.iters)
        assert info["true_resid"][j] <= tol
        want = eo.reconstruct(ref.X[j], eta[j]).reshape(-1)
        assert rel(got[j].reshape(-1), want) <= 1e-6
        rd = np.linalg.norm(eta[j].reshape(-1) - op.D(got[j].reshape(-1))) / np.linalg.norm(eta[j])
        assert rd <= 1e-6, rd
    s.close()
