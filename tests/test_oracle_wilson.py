"""Pins for the oracle's Wilson operator (CPU only).

Each check compares the oracle with something other than itself: Clifford
algebra identities, the adjoint definition, gauge covariance, and the
closed-form free-field operator in momentum space.
"""
import numpy as np
import pytest

from oracle import freefield
from oracle.wilson import WilsonOperator, gamma, gamma5
from paper_0901_3512_gb300 import workloads as W


def test_gamma_clifford_algebra():
    g = [gamma(mu) for mu in range(4)]
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)  # Hermitian
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    assert np.allclose(gamma5(), np.diag([1, 1, -1, -1]), atol=1e-15)
    assert np.allclose(gamma5(), g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 6), (3, 4, 2, 5)])
def test_adjoint_is_g5_D_g5(dims):
    """<phi, D psi> = <D^dag phi, psi> with D^dag = g5 D g5 (gamma5-hermiticity)."""
    u = W.gauge_field(dims, 0.7, 11)
    op = WilsonOperator(dims, u, 0.137)
    phi, psi = W.random_spinors(dims, 2, 5)
    lhs = np.vdot(phi, op.D(psi))
    rhs = np.vdot(op.Ddag(phi), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # M = D^dag D is Hermitian positive definite
    a = np.vdot(phi, op.M(psi))
    b = np.vdot(op.M(phi), psi)
    assert abs(a - b) <= 1e-13 * abs(a)
    assert np.vdot(psi, op.M(psi)).real > 0


def test_adjoint_dense_tiny():
    dims = (2, 2, 2, 2)
    op = WilsonOperator(dims, W.gauge_field(dims, 0.9, 3), 0.21)
    d = op.dense(WilsonOperator.OP_D)
    dd = op.dense(WilsonOperator.OP_DDAG)
    assert np.abs(dd - d.conj().T).max() < 1e-15
    m = op.dense(WilsonOperator.OP_M)
    assert np.abs(m - d.conj().T @ d).max() < 1e-14


def test_gauge_covariance():
    """D[U^g] (G psi) = G (D[U] psi), U^g_mu(x) = G(x) U_mu(x) G(x+mu)^dag."""
    dims = (4, 2, 3, 4)
    vol = W.volume(dims)
    u = W.gauge_field(dims, 0.6, 9)
    g = W.random_su3(vol, 17)
    idx = np.arange(vol).reshape(dims[::-1])
    ug = np.empty_like(u)
    for mu in range(4):
        fwd = np.roll(idx, -1, axis=3 - mu).reshape(-1)
        ug[:, mu] = g @ u[:, mu] @ np.conj(np.swapaxes(g[fwd], 1, 2))
    psi = W.random_spinors(dims, 1, 2)[0]
    gpsi = np.einsum("sab,sib->sia", g, psi)
    a = WilsonOperator(dims, ug, 0.15).D(gpsi)
    b = np.einsum("sab,sib->sia", g, WilsonOperator(dims, u, 0.15).D(psi))
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_free_field_plane_wave():
    """D e^{ipx} u = e^{ipx} D(p) u, including the (1 - g) forward sign and
    the antiperiodic time momenta."""
    dims = (4, 4, 2, 6)
    op = WilsonOperator(dims, W.unit_gauge(dims), 0.13)
    gam = [gamma(mu) for mu in range(4)]
    rng = np.random.default_rng(1)
    for p in [(2 * np.pi / 4, 0.0, np.pi, 3 * np.pi / 6), (0.0, 3 * np.pi / 2, 0.0, np.pi / 6)]:
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = freefield.plane_wave(dims, p, u)
        got = op.D(psi)
        want = freefield.plane_wave(dims, p, freefield.D_of_p(p, 0.13, gam) @ u)
        assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("dims,kappa", [((2, 2, 2, 2), 0.11), ((4, 4, 4, 4), 0.124)])
def test_free_field_spectrum(dims, kappa):
    """Dense eigenvalues of M on the unit gauge field equal the closed form."""
    op = WilsonOperator(dims, W.unit_gauge(dims), kappa)
    ev = np.linalg.eigvalsh(op.dense(WilsonOperator.OP_M))
    want = freefield.spectrum_M(dims, kappa)
    assert np.abs(ev - want).max() < 1e-12 * want.max()


def test_kappa_zero_is_identity_and_locality():
    dims = (2, 2, 2, 4)
    op = WilsonOperator(dims, W.gauge_field(dims, 0.5, 1), 0.0)
    assert np.allclose(op.dense(), np.eye(op.n), atol=0)
    # nearest-neighbour: block (x, y) nonzero only if y is x or a neighbour
    op = WilsonOperator(dims, W.gauge_field(dims, 0.5, 1), 0.2)
    d = op.dense().reshape(op.vol, 12, op.vol, 12)
    nz = np.abs(d).max(axis=(1, 3)) > 0
    lx, ly, lz, lt = dims
    for s in range(op.vol):
        c = [s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)]
        allowed = {s}
        for mu in range(4):
            for step in (1, -1):
                cc = list(c)
                cc[mu] = (cc[mu] + step) % dims[mu]
                allowed.add(cc[0] + lx * (cc[1] + ly * (cc[2] + lz * cc[3])))
        assert set(np.nonzero(nz[s])[0]) <= allowed
