"""The tcgen05 tensor-core projection C = V^dag X against a bf16 basis (the
contraction of Algorithm 1 step 8 and of Eq. 1), against the exact FP64
product of the same stored basis with the same vectors.

Bound: the tensor-core path rounds x_j to bf16 (relative error <= 2^-9 per
entry), so |C_tc - C| <= 2^-9 ||v_a|| ||x_j|| (Cauchy-Schwarz) plus FP32
accumulation; the SIMT path keeps x_j in FP32."""
import numpy as np
import pytest

from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nvec,rows", [((4, 4, 4, 4), 2, 37), ((6, 4, 4, 6), 12, 130),
                                            ((8, 8, 8, 8), 5, 300)])
def test_tc_projection_matches_fp64(dims, nvec, rows):
    need_gpu()
    u = W.gauge_field(dims, 0.5, 3)
    s = seedcg.Solver(dims, u, 0.19, precision="mixed_vbf16", stop_after_seed=1,
                      past_factor=1.0, m_max=rows)
    eta = W.z2_sources(dims, 1, 3)
    X = dev(np.zeros_like(eta))
    # run Lanczos to the full m_max so the basis holds `rows` vectors
    s.solve(dev(eta), X, 1e-14, 0, 10, allow_not_converged=True)
    m = seedcg.seedcg_get_lanczos(s.h, 1)[3]
    # the run may end early when PO against the bf16 basis stops being orthogonal
    assert m >= min(rows, 129)
    rows = min(rows, m)
    V = dev(np.zeros((rows,) + eta.shape[1:], dtype=np.complex128))
    seedcg.seedcg_get_basis(s.h, 0, rows, V)
    Vh = host(V).reshape(rows, -1)
    xs = W.random_spinors(dims, nvec, 11)
    exact = Vh.conj() @ xs.reshape(nvec, -1).T
    scale = np.linalg.norm(Vh, axis=1)[:, None] * np.linalg.norm(xs.reshape(nvec, -1), axis=1)[None, :]
    c_tc = seedcg.seedcg_project_basis(s.h, rows, nvec, dev(xs), use_tensor_cores=1)
    c_simt = seedcg.seedcg_project_basis(s.h, rows, nvec, dev(xs), use_tensor_cores=0)
    assert np.all(np.abs(c_simt - exact) <= 2e-6 * scale)
    assert np.all(np.abs(c_tc - exact) <= (2.0 ** -9 + 2e-6) * scale)
    # and the bf16 rounding of x is really all that separates the two paths
    assert np.abs(c_tc - exact).max() > 0
    s.close()


@pytest.mark.parametrize("shape", ["1,1", "2,1", "4,1", "2,2", "1,2", "1,4"])
def test_tc_projection_every_tile_shape(shape, monkeypatch):
    """Every (row tiles per CTA, K chunks per stage) shape of the tensor-core
    projection gives the FP64 product within the bf16 bound, including CTAs
    whose last row tiles are past the valid rows."""
    need_gpu()
    dims, nvec, rows = (8, 8, 8, 8), 3, 300
    u = W.gauge_field(dims, 0.5, 3)
    s = seedcg.Solver(dims, u, 0.19, precision="mixed_vbf16", stop_after_seed=1,
                      past_factor=1.0, m_max=rows)
    eta = W.z2_sources(dims, 1, 3)
    X = dev(np.zeros_like(eta))
    s.solve(dev(eta), X, 1e-14, 0, 10, allow_not_converged=True)
    m = seedcg.seedcg_get_lanczos(s.h, 1)[3]
    assert m >= 129
    rows = min(rows, m)
    V = dev(np.zeros((rows,) + eta.shape[1:], dtype=np.complex128))
    seedcg.seedcg_get_basis(s.h, 0, rows, V)
    Vh = host(V).reshape(rows, -1)
    xs = W.random_spinors(dims, nvec, 12)
    exact = Vh.conj() @ xs.reshape(nvec, -1).T
    scale = np.linalg.norm(Vh, axis=1)[:, None] * np.linalg.norm(xs.reshape(nvec, -1), axis=1)[None, :]
    monkeypatch.setenv("SEEDCG_TC_SHAPE", shape)
    for r in (rows, 129, 1):   # several tile counts, the last CTA partly or wholly past them
        c_tc = seedcg.seedcg_project_basis(s.h, r, nvec, dev(xs), use_tensor_cores=1)
        assert np.all(np.abs(c_tc - exact[:r]) <= (2.0 ** -9 + 2e-6) * scale[:r]), (shape, r)
    s.close()
