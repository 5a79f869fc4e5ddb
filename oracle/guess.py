"""Oracle: the learned initial-guess network, forward and hand-written backward,
plain FP64 numpy (test infrastructure only).

The network (the project's specification of its learned initial guess; the
paper has no counterpart) maps a right-hand side b to a guess x_0:

  layer:  out_co(x) = sum_ci [ W_0[co,ci] in_ci(x)
                              + sum_{d = +-mu} W_d[co,ci] U(x,d) in_ci(x+d) ]
          U(x,+mu) = U_mu(x),  U(x,-mu) = U_mu(x-mu)^dag, with the same
          antiperiodic-t sign as the Wilson operator on hops that wrap t;
          W_d[co,ci] is a complex 4x4 matrix on spin, U acts on colour.
  net:    1 -> 8 -> 8 -> 1 channels; ReLU on the real and imaginary parts
          separately after layers 1 and 2; input b/||b||, output times ||b||.
  loss:   mean over the batch of ||net(b) - x||^2 / ||x||^2.

Directions d: 0 on-site, then (+x, -x, +y, -y, +z, -z, +t, -t) = 1..8.
Weights of a layer: complex [9][C_out][C_in][4][4].  Activations: complex
[V][C][4][3].  Gradients are dL/dRe(W) + i dL/dIm(W).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (1, 8, 8, 1)


def _geometry(dims):
    lx, ly, lz, lt = dims
    idx = np.arange(lx * ly * lz * lt).reshape(lt, lz, ly, lx)
    fwd, bwd = [], []
    for mu in range(4):
        ax = 3 - mu
        fwd.append(np.roll(idx, -1, axis=ax).reshape(-1))
        bwd.append(np.roll(idx, 1, axis=ax).reshape(-1))
    t = np.broadcast_to(np.arange(lt)[:, None, None, None], (lt, lz, ly, lx)).reshape(-1)
    sf = np.ones((4, idx.size))
    sb = np.ones((4, idx.size))
    sf[3][t == lt - 1] = -1.0   # hop x -> x + t wraps
    sb[3][t == 0] = -1.0        # hop x -> x - t wraps
    return fwd, bwd, sf, sb


class GuessNet:
    def __init__(self, dims, gauge):
        self.dims = tuple(dims)
        self.u = np.asarray(gauge, dtype=np.complex128).reshape(-1, 4, 3, 3)
        self.fwd, self.bwd, self.sf, self.sb = _geometry(self.dims)

    # ---- the gathers g_d(a)(x) = U(x,d) a(x+d) (with the boundary sign) ----
    def gather(self, a, d):
        if d == 0:
            return a
        mu, back = (d - 1) // 2, (d - 1) % 2
        if not back:
            y = self.fwd[mu]
            return self.sf[mu][:, None, None, None] * np.einsum(
                "xab,xisb->xisa", self.u[:, mu], a[y])
        y = self.bwd[mu]
        return self.sb[mu][:, None, None, None] * np.einsum(
            "xba,xisb->xisa", np.conj(self.u[y, mu]), a[y])

    def gather_adjoint(self, g, d):
        """The adjoint map of gather(., d): returns a with <a', g> = <gather(a'), ...>."""
        if d == 0:
            return g
        mu, back = (d - 1) // 2, (d - 1) % 2
        out = np.zeros_like(g)
        if not back:
            # g(x) = s(x) U_mu(x) a(x+mu)  =>  a(y) += s(y-mu) U_mu(y-mu)^dag g(y-mu)
            y = self.fwd[mu]
            contrib = self.sf[mu][:, None, None, None] * np.einsum(
                "xba,xisb->xisa", np.conj(self.u[:, mu]), g)
            np.add.at(out, y, contrib)
        else:
            # g(x) = s(x) U_mu(x-mu)^dag a(x-mu)  =>  a(y) += s(y+mu) U_mu(y) g(y+mu)
            y = self.bwd[mu]
            contrib = self.sb[mu][:, None, None, None] * np.einsum(
                "xab,xisb->xisa", self.u[y, mu], g)
            np.add.at(out, y, contrib)
        return out

    # ---- one layer ----
    def layer(self, W, a):
        out = 0
        for d in range(9):
            out = out + np.einsum("oist,xitc->xosc", W[d], self.gather(a, d))
        return out

    @staticmethod
    def relu(z):
        return np.maximum(z.real, 0.0) + 1j * np.maximum(z.imag, 0.0)

    @staticmethod
    def relu_back(pre, dpost):
        return dpost.real * (pre.real > 0) + 1j * dpost.imag * (pre.imag > 0)

    def forward(self, Ws, b, linear=False):
        """b: [V][4][3] complex.  Returns (x0, cache)."""
        nb = np.linalg.norm(b)
        a0 = (b / nb)[:, None]                      # [V][1][4][3]
        z1 = self.layer(Ws[0], a0)
        h1 = z1 if linear else self.relu(z1)
        z2 = self.layer(Ws[1], h1)
        h2 = z2 if linear else self.relu(z2)
        z3 = self.layer(Ws[2], h2)
        x0 = nb * z3[:, 0]
        return x0, (nb, a0, z1, h1, z2, h2)

    def layer_backward(self, W, a, dout):
        """dout = dL/dRe(out) + i dL/dIm(out).  Returns (dW, da)."""
        dW = np.zeros_like(W)
        da = np.zeros_like(a)
        for d in range(9):
            g = self.gather(a, d)
            dW[d] = np.einsum("xosc,xitc->oist", dout, np.conj(g))
            dg = np.einsum("oist,xosc->xitc", np.conj(W[d]), dout)
            da = da + self.gather_adjoint(dg, d)
        return dW, da

    def loss_and_grad(self, Ws, B, X, linear=False):
        """Mean relative L2 loss over pairs (B[k], X[k]) and its gradient."""
        n = len(B)
        grads = [np.zeros_like(W) for W in Ws]
        loss = 0.0
        for b, x in zip(B, X):
            x0, (nb, a0, z1, h1, z2, h2) = self.forward(Ws, b, linear)
            xn2 = np.vdot(x, x).real
            loss += np.vdot(x0 - x, x0 - x).real / xn2 / n
            dx0 = 2.0 * (x0 - x) / xn2 / n
            dz3 = (nb * dx0)[:, None]
            g3, dh2 = self.layer_backward(Ws[2], h2, dz3)
            dz2 = dh2 if linear else self.relu_back(z2, dh2)
            g2, dh1 = self.layer_backward(Ws[1], h1, dz2)
            dz1 = dh1 if linear else self.relu_back(z1, dh1)
            g1, _ = self.layer_backward(Ws[0], a0, dz1)
            grads[0] += g1
            grads[1] += g2
            grads[2] += g3
        return loss, grads


def init_weights(seed: int, scale: float = 0.1):
    """Seeded complex Gaussian weights for the 1 -> 8 -> 8 -> 1 network."""
    rng = np.random.default_rng(seed)
    Ws = []
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        shape = (9, co, ci, 4, 4)
        s = scale / np.sqrt(9 * ci * 4)
        Ws.append(s * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)))
    return Ws


def adam_step(Ws, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam on the real and imaginary parts as independent parameters."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = []
    for k, (W, g) in enumerate(zip(Ws, grads)):
        m = state.setdefault(("m", k), np.zeros(W.shape + (2,)))
        v = state.setdefault(("v", k), np.zeros(W.shape + (2,)))
        gg = np.stack([g.real, g.imag], axis=-1)
        m[:] = b1 * m + (1 - b1) * gg
        v[:] = b2 * v + (1 - b2) * gg * gg
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        step = lr * mh / (np.sqrt(vh) + eps)
        out.append(W - (step[..., 0] + 1j * step[..., 1]))
    return out
