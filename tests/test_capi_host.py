"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/seedcg.h declares, and rejects bad arguments before touching a GPU
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0901_3512_gb300 import build, seedcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "seedcg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(seedcg_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = seedcg.load()
    declared = _declared()
    assert len(declared) >= 9
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in seedcg.h but not exported"
    assert sorted(seedcg.EXPORTS) == sorted(n for n in declared if n in seedcg.EXPORTS)
    assert set(declared) <= set(seedcg.EXPORTS), "binding misses an entry point"


def test_default_options_are_host_only():
    o = seedcg.seedcg_default_options()
    assert o.m_max == 4000 and o.past_factor == 1.0 and o.precision == seedcg.SEEDCG_FP64
    assert o.reliable_delta == pytest.approx(0.1) and o.po_passes == 1 and o.seed_mode == 1
    assert o.use_tensor_cores == 1 and o.use_guess == 0 and o.resid_mode == 0


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 4, 0), (4, 4, 4, 1)])
def test_create_rejects_bad_dims_before_device_work(dims):
    g = np.zeros(max(1, int(np.prod(dims))) * 36, dtype=np.complex128)
    with pytest.raises(seedcg.SeedCGError) as e:
        seedcg.seedcg_create(dims, g, 0.1)
    assert e.value.code == seedcg.SEEDCG_ERR_ARG


def test_create_rejects_bad_options():
    g = np.zeros(16 * 36, dtype=np.complex128)
    for kw in ({"past_factor": 0.5}, {"precision": 7}, {"po_passes": 3},
               {"seed_mode": 0, "precision": "mixed_v32"}, {"m_max": 0}, {"resid_mode": 2},
               {"use_tensor_cores": 3}):
        with pytest.raises(seedcg.SeedCGError) as e:
            seedcg.seedcg_create((2, 2, 2, 2), g, 0.1, seedcg.make_options(**kw))
        assert e.value.code == seedcg.SEEDCG_ERR_ARG


def test_solve_and_apply_reject_null_handle():
    lib = seedcg.load()
    assert lib.seedcg_solve(None, 1, None, None, 1e-8, 0, 10, None, None) == seedcg.SEEDCG_ERR_ARG
    assert lib.seedcg_apply(None, 0, 0, 0, 1, None, None, None) == seedcg.SEEDCG_ERR_ARG
    assert b"NULL" in lib.seedcg_last_error(None)
    lib.seedcg_destroy(None)  # no-op


def test_bounded_wait_selftest_rejects_bad_limits_before_device_work():
    lib = seedcg.load()
    import ctypes
    st = ctypes.c_int(7)
    for bad in (0.0, -1.0, 5000.0):
        assert lib.seedcg_selftest_bounded_wait(bad, ctypes.byref(st)) == seedcg.SEEDCG_ERR_ARG
    assert lib.seedcg_selftest_bounded_wait(1.0, None) == seedcg.SEEDCG_ERR_ARG


def test_tridiag_lowest_matches_scipy():
    """The host Sturm-bisection / inverse-iteration eigensolver the Ritz deflation
    uses, against scipy's tridiagonal eigensolver: a random matrix and the T_m of
    an oracle Lanczos run past convergence."""
    from scipy.linalg import eigh_tridiagonal
    from oracle.seedcg import seed_lanczos
    from oracle.wilson import WilsonOperator
    from paper_0901_3512_gb300 import workloads as W
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(300) + 4.0, rng.standard_normal(299)
    dims = (4, 2, 2, 4)
    op = WilsonOperator(dims, W.gauge_field(dims, 0.5, 7), 0.2)
    B = np.stack([op.Ddag(W.z2_sources(dims, 1, 7).reshape(-1))])
    s = seed_lanczos(op.M, B, None, 1e-10, 4000, 10, 2.0)
    for alpha, beta in ((a, b), (s.alpha, s.beta[:-1])):
        nev = 12
        theta, S = seedcg.seedcg_tridiag_lowest(alpha, beta, nev)
        ref, Sref = eigh_tridiagonal(alpha, beta, select="i", select_range=(0, nev - 1))
        scale = np.abs(ref).max() + np.abs(alpha).max()
        assert np.allclose(theta, ref, rtol=0, atol=1e-12 * scale)
        assert np.allclose(np.linalg.norm(S, axis=0), 1.0, atol=1e-12)
        overlap = np.abs(np.sum(S * Sref, axis=0))
        gaps = np.minimum(np.abs(np.diff(np.r_[-np.inf, ref])), np.abs(np.diff(np.r_[ref, np.inf])))
        for j in range(nev):
            if gaps[j] > 1e-8 * scale:
                assert overlap[j] > 1 - 1e-8, (j, overlap[j], gaps[j])
