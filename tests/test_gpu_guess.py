"""The learned initial guess on the GPU against the FP64 oracle (oracle/guess.py):
forward outputs, loss and hand-written gradients, an Adam step; then a small
training run on pairs the solver itself produced, and what the trained
network gains over x_0 = 0 on held-out sources."""
import numpy as np
import pytest

from oracle.guess import GuessNet, adam_step, init_weights
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


def _setup(seed=3, kappa=0.2):
    u = W.gauge_field(DIMS, 0.5, seed)
    return u, GuessNet(DIMS, u), seedcg.Solver(DIMS, u, kappa)


def test_forward_matches_oracle():
    need_gpu()
    u, net, s = _setup()
    Ws = init_weights(5, scale=1.0)
    seedcg.seedcg_guess_set_weights(s.h, Ws)
    B = W.random_spinors(DIMS, 3, 6)
    X0 = dev(np.zeros_like(B))
    seedcg.seedcg_guess_predict(s.h, dev(B), X0)
    got = host(X0)
    for k in range(3):
        want, _ = net.forward(Ws, B[k])
        assert rel(got[k], want) <= 1e-5
        assert np.abs(got[k] - want).max() <= 1e-5 * np.abs(want).max()
    # weights round-trip
    w = seedcg.seedcg_guess_get_weights(s.h)
    assert np.allclose(w, np.concatenate([x.reshape(-1) for x in Ws]), rtol=1e-6, atol=1e-7)
    s.close()


def test_loss_and_gradient_match_oracle():
    need_gpu()
    u, net, s = _setup(seed=7)
    Ws = init_weights(8, scale=1.0)
    seedcg.seedcg_guess_set_weights(s.h, Ws)
    B = W.random_spinors(DIMS, 2, 9)
    X = W.random_spinors(DIMS, 2, 10)
    loss, g = seedcg.seedcg_guess_loss_grad(s.h, dev(B), dev(X))
    lref, gref = net.loss_and_grad(Ws, B, X)
    assert abs(loss - lref) <= 1e-5 * lref
    gw = seedcg.split_weights(g)
    for layer in range(3):
        assert rel(gw[layer], gref[layer]) <= 1e-4, layer
        assert np.abs(gw[layer] - gref[layer]).max() <= 1e-4 * np.abs(gref[layer]).max(), layer
    s.close()


def test_adam_step_matches_oracle():
    need_gpu()
    u, net, s = _setup(seed=11)
    Ws = init_weights(12)
    seedcg.seedcg_guess_set_weights(s.h, Ws)
    B = W.random_spinors(DIMS, 2, 13)
    X = 0.5 * W.random_spinors(DIMS, 2, 14)
    # Adam's first step is nearly lr * sign(g): compare against the oracle's Adam
    # applied to the GPU's own gradient (the gradient itself is checked above)
    _, g = seedcg.seedcg_guess_loss_grad(s.h, dev(B), dev(X))
    seedcg.seedcg_guess_train(s.h, dev(B), dev(X), epochs=1, batch=2, lr=1e-3)
    Wref = adam_step(Ws, seedcg.split_weights(g), {}, lr=1e-3)
    got = seedcg.split_weights(seedcg.seedcg_guess_get_weights(s.h))
    for layer in range(3):
        assert rel(got[layer], Wref[layer]) <= 1e-5, layer
    s.close()


def test_trained_guess_gain_over_zero_start():
    """Train on (b, x) pairs from the solver, then solve held-out systems from
    the learned x_0 and from 0: the guess must lower the relative error of the
    start and not cost iterations."""
    need_gpu()
    kappa = 0.2
    u, net, s = _setup(seed=21, kappa=kappa)
    op = WilsonOperator(DIMS, u, kappa)
    ntr, nval = 24, 4
    eta = W.z2_sources(DIMS, ntr + nval, 21, stream=5)
    B = dev(np.zeros_like(eta))
    s.apply(seedcg.OP_DDAG, dev(eta), B, prec=0, multi=1)
    X = dev(np.zeros_like(eta))
    code, info = s.solve(B, X, 1e-8, 0, 10)
    assert code == 0
    Bh, Xh = host(B), host(X)
    seedcg.seedcg_guess_set_weights(s.h, init_weights(22))
    untrained, _ = seedcg.seedcg_guess_loss_grad(s.h, dev(Bh[ntr:]), dev(Xh[ntr:]), want_grad=False)
    seedcg.seedcg_guess_train(s.h, dev(Bh[:ntr]), dev(Xh[:ntr]), epochs=40, batch=8, lr=3e-3)
    trained, _ = seedcg.seedcg_guess_loss_grad(s.h, dev(Bh[ntr:]), dev(Xh[ntr:]), want_grad=False)
    assert trained < untrained and trained < 1.0   # better than x_0 = 0 (loss 1)
    Bv = dev(Bh[ntr:])
    s.set_options(past_factor=1.0)
    X0 = dev(np.zeros_like(Bh[ntr:]))
    c0, i0 = s.solve(Bv, X0, 1e-8, 0, 10)
    s.set_options(past_factor=1.0, use_guess=1)
    X1 = dev(np.zeros_like(Bh[ntr:]))
    c1, i1 = s.solve(Bv, X1, 1e-8, 0, 10)
    assert c0 == 0 and c1 == 0
    for j in range(nval):
        r = Bh[ntr + j].reshape(-1) - op.M(host(X1)[j].reshape(-1))
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(Bh[ntr + j])
    assert sum(i1["iters"]) <= sum(i0["iters"])
    print(f"validation loss untrained {untrained:.3f} trained {trained:.3f}; "
          f"iterations from 0: {i0['iters']}, from the learned guess: {i1['iters']}")
    s.close()
