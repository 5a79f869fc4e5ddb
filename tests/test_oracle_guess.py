"""Pins for the oracle of the learned initial-guess network (CPU only): the
layer reproduces the Wilson operator for the right weights (fixing gather
orientation, U vs U^dag and the boundary sign against the independent C
operator), the linear network is gauge covariant, the gather adjoint is the
adjoint, and the hand-written gradients equal central finite differences."""
import numpy as np
import pytest

from oracle.guess import GuessNet, adam_step, init_weights
from oracle.wilson import WilsonOperator, gamma
from paper_0901_3512_gb300 import workloads as W

DIMS = (2, 2, 2, 4)


def test_one_layer_is_the_wilson_operator():
    dims = (4, 2, 2, 4)
    u = W.gauge_field(dims, 0.6, 4)
    kappa = 0.17
    net = GuessNet(dims, u)
    Wd = np.zeros((9, 1, 1, 4, 4), dtype=np.complex128)
    Wd[0, 0, 0] = np.eye(4)
    for mu in range(4):
        Wd[1 + 2 * mu, 0, 0] = -kappa * (np.eye(4) - gamma(mu))
        Wd[2 + 2 * mu, 0, 0] = -kappa * (np.eye(4) + gamma(mu))
    psi = W.random_spinors(dims, 1, 3)[0]
    got = net.layer(Wd, psi[:, None])[:, 0]
    want = WilsonOperator(dims, u, kappa).D(psi)
    assert np.abs(got - want).max() < 1e-14 * np.abs(want).max()


def test_gather_adjoint():
    u = W.gauge_field(DIMS, 0.7, 2)
    net = GuessNet(DIMS, u)
    rng = np.random.default_rng(0)
    shape = (W.volume(DIMS), 3, 4, 3)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    g = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for d in range(9):
        lhs = np.vdot(g, net.gather(a, d))
        rhs = np.vdot(net.gather_adjoint(g, d), a)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_linear_network_gauge_covariance():
    vol = W.volume(DIMS)
    u = W.gauge_field(DIMS, 0.7, 5)
    G = W.random_su3(vol, 6)
    idx = np.arange(vol).reshape(DIMS[::-1])
    ug = np.empty_like(u)
    for mu in range(4):
        fwd = np.roll(idx, -1, axis=3 - mu).reshape(-1)
        ug[:, mu] = G @ u[:, mu] @ np.conj(np.swapaxes(G[fwd], 1, 2))
    Ws = init_weights(1, scale=1.0)
    b = W.random_spinors(DIMS, 1, 8)[0]
    x0, _ = GuessNet(DIMS, u).forward(Ws, b, linear=True)
    xg, _ = GuessNet(DIMS, ug).forward(Ws, np.einsum("sab,sib->sia", G, b), linear=True)
    assert np.abs(xg - np.einsum("sab,sib->sia", G, x0)).max() < 1e-12 * np.abs(x0).max()


@pytest.mark.parametrize("linear", [True, False])
def test_gradients_match_finite_differences(linear):
    u = W.gauge_field(DIMS, 0.7, 9)
    net = GuessNet(DIMS, u)
    Ws = init_weights(2, scale=1.0)
    B = W.random_spinors(DIMS, 2, 10)
    X = W.random_spinors(DIMS, 2, 11)
    loss, grads = net.loss_and_grad(Ws, B, X, linear)
    rng = np.random.default_rng(3)
    h = 1e-6
    for layer in range(3):
        for _ in range(6):
            i = tuple(rng.integers(0, s) for s in Ws[layer].shape)
            for part, unit in ((0, 1.0), (1, 1j)):
                Wp = [w.copy() for w in Ws]
                Wm = [w.copy() for w in Ws]
                Wp[layer][i] += h * unit
                Wm[layer][i] -= h * unit
                fd = (net.loss_and_grad(Wp, B, X, linear)[0] - net.loss_and_grad(Wm, B, X, linear)[0]) / (2 * h)
                an = grads[layer][i].real if part == 0 else grads[layer][i].imag
                # 1e-7 relative, plus the central difference's own roundoff
                # (about machine epsilon * loss / h)
                bound = 1e-7 * abs(fd) + 8 * np.finfo(float).eps * abs(loss) / h
                assert abs(fd - an) <= bound, (layer, i, part, fd, an)


def test_adam_reduces_the_loss():
    u = W.gauge_field(DIMS, 0.5, 12)
    net = GuessNet(DIMS, u)
    Ws = init_weights(4)
    B = W.random_spinors(DIMS, 4, 13)
    X = 0.3 * B
    state = {}
    l0 = net.loss_and_grad(Ws, B, X)[0]
    for _ in range(30):
        loss, g = net.loss_and_grad(Ws, B, X)
        Ws = adam_step(Ws, g, state, lr=1e-2)
    assert net.loss_and_grad(Ws, B, X)[0] < 0.5 * l0
