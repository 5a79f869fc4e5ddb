"""seedcg_apply_noalloc: the operator application for callers that cannot
allocate device memory (its scratch is a fixed device array).  It must give
the results of seedcg_apply, call after call, and refuse batches too large for
the fixed scratch.  Kept last in collection order so that a failure here
stops a -x run only after every other test has run."""
import numpy as np
import pytest

from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,multi,tol", [(0, 1, 1e-13), (0, 0, 1e-13), (1, 1, 1e-5), (1, 0, 1e-5)])
def test_noalloc_apply_matches_apply(prec, multi, tol):
    """Against seedcg_apply and against the oracle's C operator (D, D^dag and
    M = D^dag D of Section 3), in norm and element by element (max-abs relative to
    the largest entry)."""
    need_gpu()
    from oracle.wilson import WilsonOperator
    dims = (4, 4, 4, 8)
    u = W.gauge_field(dims, 0.5, 31)
    s = seedcg.Solver(dims, u, 0.2)
    op_or = WilsonOperator(dims, u, 0.2)
    apply_or = {seedcg.OP_D: op_or.D, seedcg.OP_DDAG: op_or.Ddag, seedcg.OP_M: op_or.M}
    for call in range(2):  # two calls in a row share the fixed scratch
        x = W.random_spinors(dims, 3, 40 + call)
        xd = dev(x)
        for op in (seedcg.OP_D, seedcg.OP_DDAG, seedcg.OP_M):
            want = dev(np.zeros_like(x))
            got = dev(np.zeros_like(x))
            seedcg.seedcg_apply(s.h, op, prec, multi, 3, xd, want)
            seedcg.seedcg_apply_noalloc(s.h, op, prec, multi, 3, xd, got)
            g = host(got)
            assert rel(g, host(want)) <= tol
            ref = np.stack([apply_or[op](x[j]) for j in range(3)])
            assert rel(g, ref) <= tol
            assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref))
    s.close()


def test_noalloc_rejects_batches_beyond_the_scratch():
    need_gpu()
    dims = (8, 8, 8, 8)
    vol = W.volume(dims)
    s = seedcg.Solver(dims, W.gauge_field(dims, 0.5, 32), 0.2)
    n = seedcg.NOALLOC_SCRATCH_BYTES // (3 * vol * 12 * 16) + 1   # one field more than FP64 fits
    x = dev(np.zeros((n, vol, 4, 3), dtype=np.complex128))
    y = dev(np.zeros((n, vol, 4, 3), dtype=np.complex128))
    with pytest.raises(seedcg.SeedCGError) as e:
        seedcg.seedcg_apply_noalloc(s.h, seedcg.OP_M, 0, 1, n, x, y)
    assert e.value.code == seedcg.SEEDCG_ERR_ARG
    # the largest batch that fits still works
    seedcg.seedcg_apply_noalloc(s.h, seedcg.OP_M, 0, 1, n - 1, x[: n - 1], y[: n - 1])
    s.close()


def test_noalloc_rejects_host_memory():
    """A host array (numpy, or a pinned torch tensor) is refused with
    SEEDCG_ERR_ARG before any kernel could dereference it."""
    need_gpu()
    import torch
    dims = (4, 4, 4, 8)
    s = seedcg.Solver(dims, W.gauge_field(dims, 0.5, 33), 0.2)
    x = W.random_spinors(dims, 2, 50)
    yd = dev(np.zeros_like(x))
    for inp, out in ((np.ascontiguousarray(x), yd), (dev(x), np.zeros_like(x)),
                     (torch.from_numpy(x).pin_memory(), yd)):
        with pytest.raises(seedcg.SeedCGError) as e:
            seedcg.seedcg_apply_noalloc(s.h, seedcg.OP_M, 0, 1, 2, inp, out)
        assert e.value.code == seedcg.SEEDCG_ERR_ARG
    # the device call still works after the refusals
    want = dev(np.zeros_like(x))
    seedcg.seedcg_apply(s.h, seedcg.OP_M, 0, 1, 2, dev(x), want)
    seedcg.seedcg_apply_noalloc(s.h, seedcg.OP_M, 0, 1, 2, dev(x), yd)
    assert rel(host(yd), host(want)) <= 1e-13
    s.close()
