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
