"""Failure detection on the GPU without a fault: every mbarrier wait of the
tensor-core kernels is bounded by globaltimer, and on expiry the kernel records
SEEDCG_ERR_TIMEOUT for the host instead of hanging.  The self-check waits on a
barrier that nothing arrives at, with a 20 ms limit."""
import time

import numpy as np
import pytest

from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports_timeout():
    need_gpu()
    t0 = time.perf_counter()
    st = seedcg.seedcg_selftest_bounded_wait(20.0)
    assert st == seedcg.SEEDCG_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # the context stays usable afterwards
    dims = (4, 4, 4, 4)
    s = seedcg.Solver(dims, W.gauge_field(dims, 0.5, 51), 0.2)
    x = dev(W.random_spinors(dims, 1, 52))
    y = dev(np.zeros_like(host(x)))
    s.apply(seedcg.OP_M, x, y, prec=0, multi=0)
    assert np.isfinite(host(y)).all() and np.abs(host(y)).max() > 0
    s.close()


def test_nan_in_one_system_is_reported_and_spares_the_others():
    """Host-side fault injection: one right-hand side (not the first, which
    drives Lanczos) carries a NaN.  The solve returns without a GPU fault,
    reports that system as not converged (its CG residual is not finite), and
    every other system still meets tol; the handle keeps working."""
    need_gpu()
    dims = (4, 4, 4, 4)
    u = W.gauge_field(dims, 0.5, 53)
    s = seedcg.Solver(dims, u, 0.2, precision="mixed_v32")
    eta = W.z2_sources(dims, 3, 54)
    B = dev(np.zeros_like(eta))
    s.apply(seedcg.OP_DDAG, dev(eta), B, prec=0, multi=1)
    Bh = host(B)
    Bh[1, 7, 2, 1] = np.nan
    X = dev(np.zeros_like(Bh))
    code, info = s.solve(dev(Bh), X, 1e-8, 0, 10, allow_not_converged=True)
    assert code == seedcg.SEEDCG_ERR_NOT_CONVERGED
    tr = info["true_resid"]
    assert not np.isfinite(tr[1]) or tr[1] > 1e-8
    assert tr[0] <= 1e-8 and tr[2] <= 1e-8
    # the same handle solves a clean batch afterwards
    X2 = dev(np.zeros_like(Bh))
    code2, info2 = s.solve(B, X2, 1e-8, 0, 10)
    assert code2 == seedcg.SEEDCG_OK and max(info2["true_resid"]) <= 1e-8
    s.close()


def test_nan_in_the_first_system_stops_lanczos_with_a_status():
    """A NaN in the system that drives Lanczos makes its scalars non-finite:
    the run ends with SEEDCG_ERR_NAN (no hang, no fault) and the handle keeps
    working."""
    need_gpu()
    dims = (4, 4, 4, 4)
    u = W.gauge_field(dims, 0.5, 55)
    s = seedcg.Solver(dims, u, 0.2, precision="fp64")
    eta = W.z2_sources(dims, 2, 56)
    B = dev(np.zeros_like(eta))
    s.apply(seedcg.OP_DDAG, dev(eta), B, prec=0, multi=1)
    Bh = host(B)
    Bh[0, 3, 0, 0] = np.inf
    X = dev(np.zeros_like(Bh))
    with pytest.raises(seedcg.SeedCGError) as e:
        s.solve(dev(Bh), X, 1e-8, 0, 10)
    assert e.value.code in (seedcg.SEEDCG_ERR_NAN, seedcg.SEEDCG_ERR_NOT_CONVERGED)
    X2 = dev(np.zeros_like(Bh))
    code2, info2 = s.solve(B, X2, 1e-8, 0, 10)
    assert code2 == seedcg.SEEDCG_OK and max(info2["true_resid"]) <= 1e-8
    s.close()


def test_basis_beyond_device_memory_is_refused_before_allocation():
    """An m_max whose stored basis cannot fit in free device memory is refused
    with SEEDCG_ERR_OOM and a message giving the size, before anything is
    allocated for it; the handle keeps working with a sensible m_max."""
    need_gpu()
    dims = (8, 8, 8, 16)
    u = W.gauge_field(dims, 0.5, 57)
    s = seedcg.Solver(dims, u, 0.2, precision="fp64", m_max=20_000_000)   # ~31 TB of FP64 rows
    eta = W.z2_sources(dims, 2, 58)
    B = dev(np.zeros_like(eta))
    s.apply(seedcg.OP_DDAG, dev(eta), B, prec=0, multi=1)
    X = dev(np.zeros_like(eta))
    with pytest.raises(seedcg.SeedCGError) as e:
        s.solve(B, X, 1e-8, 0, 10)
    assert e.value.code == seedcg.SEEDCG_ERR_OOM
    assert "GB" in str(e.value)
    s.set_options(precision="fp64", m_max=4000)
    code, info = s.solve(B, X, 1e-8, 0, 10)
    assert code == seedcg.SEEDCG_OK and max(info["true_resid"]) <= 1e-8
    s.close()
