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


@pytest.mark.parametrize("seed_mode", [0, 1])
def test_eo_seed_cg_matches_oracle(seed_mode):
    """Improved Seed-CG on the even-odd system (Section 3's setup), on the
    device-resident engine, against the oracle's improved_seed_cg on A^dag A
    (literal or blocked seeds): m_conv, m and the per-system iterations within
    2 %, the reconstructed full solutions within 1e-6, and D x = eta solved."""
    need_gpu()
    dims, kappa, tol = (4, 4, 4, 4), 0.21, 1e-10
    u = W.gauge_field(dims, 0.5, 12)
    op = WilsonOperator(dims, u, kappa)
    eo = EvenOddOperator(op)
    from oracle.seedcg import improved_seed_cg
    eta = W.point_sources(dims, 2)
    B = np.stack([eo.Adag(eo.source(e)).reshape(-1) for e in eta])
    ref = improved_seed_cg(eo.M, B, None, tol, 4000, 10, past_factor=1.5,
                           seed_mode="literal" if seed_mode == 0 else "blocked")
    s = seedcg.Solver(dims, u, kappa, precision="fp64", past_factor=1.5, m_max=4000, seed_mode=seed_mode)
    X = dev(np.zeros_like(eta))
    code, info = seedcg.seedcg_solve_eo(s.h, dev(eta), X, tol, 0, 10)
    assert code == seedcg.SEEDCG_OK

    def within(a, b):
        return abs(a - b) <= max(1, int(np.ceil(0.02 * max(a, b))))

    assert within(info["m_conv"], ref.seed.m_conv) and within(info["m"], ref.seed.m), (info, ref.seed.m)
    assert info["po_count"] == ref.seed.po_count
    got = host(X)
    for j in range(2):
        assert within(info["iters"][j], int(ref.iters[j])), (info["iters"], ref.iters)
        assert info["true_resid"][j] <= tol
        want = eo.reconstruct(ref.X[j], eta[j]).reshape(-1)
        assert rel(got[j].reshape(-1), want) <= 1e-6
        rd = np.linalg.norm(eta[j].reshape(-1) - op.D(got[j].reshape(-1))) / np.linalg.norm(eta[j])
        assert rd <= 1e-6, rd
        assert abs(info["true_resid_D"][j] - rd) <= 1e-3 * rd + 1e-15
        # matvecs in applications of the full-lattice D: 2 per A^dag A
        assert info["matvecs"][j] >= 2 * info["iters"][j]
    # the stored basis is the oracle's: odd-site half vectors, orthonormal after PO
    m = info["m"]
    vh = W.volume(dims) // 2
    Vg = dev(np.zeros((m, vh, 4, 3), dtype=np.complex128))
    seedcg.seedcg_get_basis(s.h, 0, m, Vg)
    Vg = host(Vg).reshape(m, -1)
    assert rel(Vg[:20], ref.seed.V[:20]) <= 1e-10
    last = (m // 10) * 10
    G = Vg[:last].conj() @ Vg[:last].T
    assert np.abs(G - np.eye(last)).max() <= 1e-10
    s.close()


@pytest.mark.parametrize("precision,tc", [("mixed_v32", 1), ("mixed_vbf16", 1), ("mixed_vbf16", 0)])
def test_eo_mixed_precision_meets_tol(precision, tc):
    """The even-odd solve in the mixed modes on 4^4: every residual of
    A^dag A x_o = b, recomputed with the oracle, meets tol, the solutions are
    within the distance two residuals <= tol allow of the oracle's (2 cond tol,
    cond of A^dag A from its dense spectrum), and the original system's
    residual is reported."""
    need_gpu()
    from oracle.seedcg import improved_seed_cg
    from tests.gpu_helpers import recompute_slack
    dims, kappa, tol = (4, 4, 4, 4), 0.21, 1e-8
    u = W.gauge_field(dims, 0.5, 12)
    op = WilsonOperator(dims, u, kappa)
    eo = EvenOddOperator(op)
    eta = W.point_sources(dims, 3)
    B = np.stack([eo.Adag(eo.source(e)).reshape(-1) for e in eta])
    n = B.shape[1]
    Md = np.stack([eo.M(e) for e in np.eye(n, dtype=np.complex128)], axis=1)
    ev = np.linalg.eigvalsh(Md)
    cond = ev[-1] / ev[0]
    ref = improved_seed_cg(eo.M, B, None, tol, 4000, 10, past_factor=1.5, seed_mode="blocked")
    s = seedcg.Solver(dims, u, kappa, precision=precision, past_factor=1.5, m_max=4000, use_tensor_cores=tc)
    X = dev(np.zeros_like(eta))
    code, info = seedcg.seedcg_solve_eo(s.h, dev(eta), X, tol, 0, 10)
    assert code == seedcg.SEEDCG_OK
    got = host(X)
    for j in range(3):
        xo = got[j][eo.odd].reshape(-1)
        r = np.linalg.norm(B[j] - eo.M(xo)) / np.linalg.norm(B[j])
        assert r <= tol + recompute_slack(ev[-1], np.linalg.norm(xo), np.linalg.norm(B[j])), (j, r)
        assert rel(xo, ref.X[j]) <= 2 * cond * tol * 1.001
        assert np.isfinite(info["true_resid_D"][j])
    s.close()


def test_eo_8x8x8x16_mixed_bf16_point_sources():
    """The even-odd solve of the 8^3x16 workload (twelve point sources, bf16
    basis with the tcgen05 seed projection): every residual of the even-odd
    system recomputed with the oracle's operator meets tol; the original
    system's residual, recomputed with the oracle's D, equals the reported
    one; fewer Lanczos iterations than the full-lattice system needs."""
    need_gpu()
    from tests.gpu_helpers import recompute_slack
    wl = W.WORKLOADS["small_8x8x8x16_nrhs12"]
    f = wl.fields[0]
    u = f.gauge()
    kappa = W.kappa_for(f.name)
    op = WilsonOperator(f.dims, u, kappa)
    eo = EvenOddOperator(op)
    eta = wl.sources_for(0)
    s = seedcg.Solver(f.dims, u, kappa, precision="mixed_vbf16", past_factor=wl.past_factor, m_max=6000)
    X = dev(np.zeros_like(eta))
    code, info = seedcg.seedcg_solve_eo(s.h, dev(eta), X, wl.tol, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK
    got = host(X)
    lam_max = (1 + 8 * kappa) ** 4      # ||A|| <= 1 + kappa^2 ||H||^2 <= (1 + 8 kappa)^2
    for j in range(len(eta)):
        b = eo.Adag(eo.source(eta[j])).reshape(-1)
        xo = got[j][eo.odd].reshape(-1)
        r = np.linalg.norm(b - eo.M(xo)) / np.linalg.norm(b)
        assert r <= wl.tol + recompute_slack(lam_max, np.linalg.norm(xo), np.linalg.norm(b)), (j, r)
        rd = np.linalg.norm(eta[j].reshape(-1) - op.D(got[j].reshape(-1))) / np.linalg.norm(eta[j])
        assert abs(info["true_resid_D"][j] - rd) <= 1e-3 * rd + 1e-15
    # the full-lattice system needs more iterations: textbook CG on D^dag D for RHS 1 (oracle)
    from oracle.seedcg import cg
    b1 = op.Ddag(eta[0]).reshape(-1)
    full_iters = cg(op.M, b1, None, wl.tol, 20000).iters
    assert info["m_conv"] < full_iters, (info["m_conv"], full_iters)
    print(f"even-odd 8^3x16 bf16: m_conv {info['m_conv']} m {info['m']} iters {info['iters']} "
          f"D residuals max {max(info['true_resid_D']):.2e}")
    s.close()
