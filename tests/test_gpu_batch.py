"""Several gauge fields of uneven size in one seedcg_batch_solve: every seeded
system of every field meets ||b - M x|| <= tol in FP64 (checked with the
oracle's operator), and each field's solutions equal those of a separate
seedcg_solve of that field (the batched CG runs the same arithmetic per
system)."""
import numpy as np
import pytest

from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu

FIELDS = [((4, 4, 4, 4), 0.21, 3, 1), ((6, 4, 4, 6), 0.19, 2, 2), ((8, 4, 4, 8), 0.2, 4, 3)]
TOL = 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed_v32"])
def test_batch_of_uneven_fields(precision):
    need_gpu()
    solvers, Bs, Xs, ops, etas = [], [], [], [], []
    for dims, kappa, nrhs, seed in FIELDS:
        u = W.gauge_field(dims, 0.5, seed)
        op = WilsonOperator(dims, u, kappa)
        eta = W.z2_sources(dims, nrhs, seed)
        s = seedcg.Solver(dims, u, kappa, precision=precision, past_factor=1.5)
        B = dev(np.zeros_like(eta))
        s.apply(seedcg.OP_DDAG, dev(eta), B, prec=0, multi=1)
        solvers.append(s)
        Bs.append(B)
        Xs.append(dev(np.zeros_like(eta)))
        ops.append(op)
        etas.append(eta)
    code, infos = seedcg.seedcg_batch_solve([s.h for s in solvers], Bs, Xs, TOL, 0, 10)
    assert code == seedcg.SEEDCG_OK
    for f, (s, B, X, op, info) in enumerate(zip(solvers, Bs, Xs, ops, infos)):
        Bh, Xh = host(B), host(X)
        assert info["m"] > 0 and info["m_conv"] > 0
        for j in range(Bh.shape[0]):
            assert info["true_resid"][j] <= TOL
            r = Bh[j].reshape(-1) - op.M(Xh[j].reshape(-1))
            assert np.linalg.norm(r) <= TOL * np.linalg.norm(Bh[j])
        # the same field solved alone: the same Lanczos run and seeds; the CG
        # reductions split differently across blocks in the batch, so the two
        # runs agree to rounding amplified by CG (far inside the 1e-6 bar)
        X1 = dev(np.zeros_like(Xh))
        code1, info1 = s.solve(B, X1, TOL, 0, 10)
        assert code1 == 0 and info1["m"] == info["m"] and info1["m_conv"] == info["m_conv"]
        assert rel(host(X1), Xh) <= 1e-6
        for a, b in zip(info1["iters"], info["iters"]):
            assert abs(a - b) <= max(1, 0.02 * a)
    for s in solvers:
        s.close()


def test_batch_rejects_mixed_precision_handles():
    need_gpu()
    dims = (4, 4, 4, 4)
    u = W.gauge_field(dims, 0.5, 1)
    a = seedcg.Solver(dims, u, 0.2, precision="fp64")
    b = seedcg.Solver(dims, u, 0.2, precision="mixed_v32")
    B = dev(W.z2_sources(dims, 2, 1))
    with pytest.raises(seedcg.SeedCGError) as e:
        seedcg.seedcg_batch_solve([a.h, b.h], [B, B], [dev(np.zeros(B.shape, complex)), dev(np.zeros(B.shape, complex))], TOL, 0, 10)
    assert e.value.code == seedcg.SEEDCG_ERR_ARG
    a.close()
    b.close()


def test_uneven_workload_at_full_size_by_the_oracle():
    """The three-field workload the bench's `batch3_uneven` line times
    (8^3x16 / 12^3x24 / 16^3x32, 24 / 12 / 6 Z2 sources, FP32 iteration with a
    complex64 basis and FP64 reliable updates, k = 10) in one seedcg_batch_solve:
    all 42 residuals ||b - M x|| / ||b|| recomputed with the oracle's plain-C
    FP64 operator meet tol, up to the rounding of a recomputation in another
    summation order."""
    need_gpu()
    import torch
    from tests.gpu_helpers import recompute_slack
    wl = W.WORKLOADS["batch3_uneven_nrhs24_12_6"]
    solvers, Bs, Xs, ops, lams = [], [], [], [], []
    for i, f in enumerate(wl.fields):
        u = f.gauge()
        kappa = W.kappa_for(f.name)
        op = WilsonOperator(f.dims, u, kappa)
        eta = wl.sources_for(i)
        B = np.stack([op.Ddag(e) for e in eta])      # the oracle's right-hand sides
        s = seedcg.Solver(f.dims, u, kappa, precision=wl.precision, past_factor=wl.past_factor,
                          m_max=4000)
        solvers.append(s)
        Bs.append(dev(B))
        Xs.append(dev(np.zeros_like(B)))
        ops.append(op)
        lams.append(W.kappa_table().get(f.name, {}).get("lam_max", (1 + 8 * kappa) ** 2))
    code, infos = seedcg.seedcg_batch_solve([s.h for s in solvers], Bs, Xs, wl.tol, 0, wl.reorth_period)
    assert code == seedcg.SEEDCG_OK
    worst = 0.0
    for s, B, X, op, lam, info in zip(solvers, Bs, Xs, ops, lams, infos):
        Bh, Xh = host(B), host(X)
        for j in range(Bh.shape[0]):
            b, x = Bh[j].reshape(-1), Xh[j].reshape(-1)
            r = np.linalg.norm(b - op.M(x)) / np.linalg.norm(b)
            assert r <= wl.tol + recompute_slack(lam, np.linalg.norm(x), np.linalg.norm(b)), (j, r)
            worst = max(worst, r)
        s.close()
    torch.cuda.empty_cache()
    print(f"three uneven fields, 42 systems: worst oracle residual {worst:.3e}; "
          f"m_conv {[i['m_conv'] for i in infos]}, CG max {[i['cg_iters_max'] for i in infos]}")
