"""The learned initial guess on the GPU against the FP64 oracle (oracle/guess.py):
forward outputs, loss and hand-written gradients, an Adam step; then a small
training run on pairs the solver itself produced, and what the trained
network gains over x_0 = 0 on held-out sources.

The network stores its activations, their gradients and the weights it reads
in bf16 (8 significand bits: a stored value is off by at most u = 2^-9 of
itself) and accumulates in FP32; its middle layer runs on the tensor cores.
Each layer rounds its input and its weights (2u per product term) and its
output (u); with rounding errors of random sign the three layers leave a
relative error of a few u in the output.  The backward pass adds its own
roundings (the output gradient, each layer's data gradient) and evaluates the
ReLU masks on bf16 pre-activations, so entries within a rounding of zero may
switch the mask; the first layer's weight gradient collects all of them.  The
bounds below allow BF16_FWD = 8u (1.6 %) in norm and 16u of the largest entry
element by element for the forward pass, and BF16_GRAD = 32u (6.3 %) in norm
and 64u element by element for the gradients, in place of the FP32 bars 1e-5 /
1e-4.  The Adam step works on FP32 master weights and keeps the FP32 bar."""
import numpy as np
import pytest

from oracle.guess import GuessNet, adam_step, init_weights
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import seedcg, workloads as W
from tests.gpu_helpers import dev, host, need_gpu, rel

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)
U_BF16 = 2.0 ** -9
BF16_FWD = 8 * U_BF16
BF16_GRAD = 32 * U_BF16


def _setup(seed=3, kappa=0.2, dims=DIMS):
    u = W.gauge_field(dims, 0.5, seed)
    return u, GuessNet(dims, u), seedcg.Solver(dims, u, kappa)


@pytest.mark.parametrize("dims", [DIMS, (6, 4, 4, 6)])
def test_forward_matches_oracle(dims):
    """4^4 fills two tensor-core tiles of 128 sites exactly; 6x4x4x6 (576 sites)
    ends in a ragged tile."""
    need_gpu()
    u, net, s = _setup(dims=dims)
    Ws = init_weights(5, scale=1.0)
    seedcg.seedcg_guess_set_weights(s.h, Ws)
    B = W.random_spinors(dims, 3, 6)
    X0 = dev(np.zeros_like(B))
    seedcg.seedcg_guess_predict(s.h, dev(B), X0)
    got = host(X0)
    for k in range(3):
        want, _ = net.forward(Ws, B[k])
        err_n, err_m = rel(got[k], want), np.abs(got[k] - want).max() / np.abs(want).max()
        print(f"forward pair {k}: relative error {err_n:.2e} in norm, {err_m:.2e} max-abs")
        assert err_n <= BF16_FWD
        assert err_m <= 2 * BF16_FWD
    # weights round-trip (the FP32 master copy)
    w = seedcg.seedcg_guess_get_weights(s.h)
    assert np.allclose(w, np.concatenate([x.reshape(-1) for x in Ws]), rtol=1e-6, atol=1e-7)
    s.close()


@pytest.mark.parametrize("dims", [DIMS, (6, 4, 4, 6)])
def test_loss_and_gradient_match_oracle(dims):
    need_gpu()
    u, net, s = _setup(seed=7, dims=dims)
    Ws = init_weights(8, scale=1.0)
    seedcg.seedcg_guess_set_weights(s.h, Ws)
    B = W.random_spinors(dims, 2, 9)
    X = W.random_spinors(dims, 2, 10)
    loss, g = seedcg.seedcg_guess_loss_grad(s.h, dev(B), dev(X))
    lref, gref = net.loss_and_grad(Ws, B, X)
    print(f"loss {loss:.6e} oracle {lref:.6e}")
    assert abs(loss - lref) <= 2 * BF16_FWD * lref
    gw = seedcg.split_weights(g)
    for layer in range(3):
        err_n = rel(gw[layer], gref[layer])
        err_m = np.abs(gw[layer] - gref[layer]).max() / np.abs(gref[layer]).max()
        print(f"layer {layer + 1} gradient: relative error {err_n:.2e} in norm, {err_m:.2e} max-abs")
        assert err_n <= BF16_GRAD, layer
        assert err_m <= 2 * BF16_GRAD, layer
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
