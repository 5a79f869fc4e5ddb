"""Parity of the CUDA Wilson dslash with the oracle, element by element:
relative error <= 1e-13 in FP64 and <= 1e-5 in FP32 (the bars the method's
specification sets), for D, D^dag and M = D^dag D, single- and multi-RHS
kernels, on lattices that span several thread blocks and end in a ragged
tile, up to the 16^3x32 production lattice."""
import numpy as np
import pytest

from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu

CASES = [((2, 2, 2, 2), 0.2, 1), ((4, 4, 4, 4), 0.27, 3), ((6, 4, 4, 6), 0.13, 5),
         ((8, 8, 8, 16), 0.2256, 12), ((16, 16, 16, 32), 0.21, 2)]


@pytest.mark.parametrize("dims,kappa,n", CASES)
@pytest.mark.parametrize("multi", [0, 1])
def test_dslash_parity(dims, kappa, n, multi):
    need_gpu()
    u = W.gauge_field(dims, 0.5, 42)
    op = WilsonOperator(dims, u, kappa)
    x = W.random_spinors(dims, n, 7)
    s = seedcg.Solver(dims, u, kappa)
    xd = dev(x)
    out = dev(np.zeros_like(x))
    for code, fn in ((seedcg.OP_D, op.D), (seedcg.OP_DDAG, op.Ddag), (seedcg.OP_M, op.M)):
        want = np.stack([fn(x[r]) for r in range(n)])
        s.apply(code, xd, out, prec=0, multi=multi)
        got = host(out)
        assert rel(got, want) <= 1e-13, (code, rel(got, want))
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
        s.apply(code, xd, out, prec=1, multi=multi)
        got32 = host(out)
        assert rel(got32, want) <= 1e-5, (code, rel(got32, want))
        # element by element: no entry off by more than the FP32 bar of the largest
        assert np.abs(got32 - want).max() <= 1e-5 * np.abs(want).max(), code
    s.close()


def test_dslash_point_source_and_free_field():
    """b = D^dag eta for the point sources at the origin (the headline
    workload's right-hand sides) and the free field (all links 1)."""
    need_gpu()
    dims = (4, 4, 4, 8)
    for u in (W.unit_gauge(dims), W.gauge_field(dims, 0.5, 1)):
        op = WilsonOperator(dims, u, 0.15)
        eta = W.point_sources(dims, 12)
        s = seedcg.Solver(dims, u, 0.15)
        out = dev(np.zeros_like(eta))
        s.apply(seedcg.OP_DDAG, dev(eta), out, prec=0, multi=1)
        want = np.stack([op.Ddag(e) for e in eta])
        assert rel(host(out), want) <= 1e-14
        s.close()


def test_repeated_calls_do_not_leak_device_memory():
    """Per-call device scratch (operator application, solves, projections) is
    released when the call returns: free device memory is unchanged after
    many calls."""
    need_gpu()
    import torch
    dims = (8, 8, 8, 8)
    s = seedcg.Solver(dims, W.gauge_field(dims, 0.5, 41), 0.18, precision="mixed_vbf16", m_max=64)
    x = dev(W.random_spinors(dims, 12, 42))
    y = dev(np.zeros((12,) + x.shape[1:], dtype=np.complex128))
    X = dev(np.zeros((2,) + x.shape[1:], dtype=np.complex128))
    for _ in range(2):   # first calls: autotuning, lazily loaded kernels, handle caches
        s.apply(seedcg.OP_M, x, y, prec=0, multi=1)
        s.apply(seedcg.OP_D, x, y, prec=1, multi=0)
        X.zero_()
        s.solve(x[:2], X, 1e-6, 0, 10, allow_not_converged=True)
        seedcg.seedcg_project_basis(s.h, 16, 3, x[:3], use_tensor_cores=0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        s.apply(seedcg.OP_M, x, y, prec=0, multi=1)
        s.apply(seedcg.OP_D, x, y, prec=1, multi=0)
        X.zero_()
        s.solve(x[:2], X, 1e-6, 0, 10, allow_not_converged=True)
        seedcg.seedcg_project_basis(s.h, 16, 3, x[:3], use_tensor_cores=0)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # 20 leaked operator scratches alone would be ~20 x 28 MB
    assert free1 >= free0 - (32 << 20), (free0, free1)
    s.close()
