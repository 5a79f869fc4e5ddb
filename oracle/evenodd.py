"""Even-odd (red-black) preconditioned Wilson system, the paper's own setup
(Section 3): test infrastructure, like the rest of oracle/.

Sites of even parity (x + y + z + t even) and odd parity are coupled only by
the hopping term H, so with the sites ordered (even, odd)

    D = [[1, -kappa H_eo], [-kappa H_oe, 1]].

Eliminating the even sites leaves the Schur complement on the odd sites,

    A = 1 - kappa^2 H_oe H_eo,   A x_o = phi,   phi = eta_o + kappa H_oe eta_e,

after which x_e = eta_e + kappa H_eo x_o.  A is not Hermitian; the seed method
runs on A^dag A x_o = A^dag phi (Section 3), and because gamma5 H gamma5 = H^dag
with gamma5 acting site by site, A^dag = gamma5 A gamma5.  Half-lattice vectors
here are the odd sites of a full-lattice vector, in lexicographic site order
(any order of the odd sites would do; the GPU path may pack them differently).
"""
import numpy as np

from .wilson import WilsonOperator

GAMMA5_DIAG = np.array([1.0, 1.0, -1.0, -1.0])   # chiral basis, spin index 0..3


def parity(dims) -> np.ndarray:
    """(x + y + z + t) mod 2 per site, sites lexicographic with x fastest."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1)


class EvenOddOperator:
    def __init__(self, op: WilsonOperator):
        self.op = op
        self.kappa = op.kappa
        par = parity(op.dims)
        self.odd = np.flatnonzero(par == 1)
        self.even = np.flatnonzero(par == 0)
        self.n = 12 * len(self.odd)

    # full-lattice helpers: vectors [V][4][3]
    def _full(self, x):
        return np.asarray(x, dtype=np.complex128).reshape(self.op.vol, 4, 3)

    def hop(self, psi):
        """H psi = (psi - D psi) / kappa on the full lattice."""
        psi = self._full(psi)
        return (psi - self.op.D(psi)) / self.kappa

    def embed_odd(self, x_o):
        full = np.zeros((self.op.vol, 4, 3), dtype=np.complex128)
        full[self.odd] = np.asarray(x_o, dtype=np.complex128).reshape(len(self.odd), 4, 3)
        return full

    def embed_even(self, x_e):
        full = np.zeros((self.op.vol, 4, 3), dtype=np.complex128)
        full[self.even] = np.asarray(x_e, dtype=np.complex128).reshape(len(self.even), 4, 3)
        return full

    # the odd-site system
    def A(self, x_o):
        """A x_o = x_o - kappa^2 H_oe H_eo x_o."""
        x_o = np.asarray(x_o, dtype=np.complex128)
        he = self.hop(self.embed_odd(x_o))[self.even]                 # H_eo x_o
        ho = self.hop(self.embed_even(he))[self.odd]                  # H_oe H_eo x_o
        return (x_o.reshape(len(self.odd), 4, 3) - self.kappa ** 2 * ho).reshape(np.shape(x_o))

    def gamma5(self, x):
        x = np.asarray(x, dtype=np.complex128)
        return (x.reshape(-1, 4, 3) * GAMMA5_DIAG[None, :, None]).reshape(np.shape(x))

    def Adag(self, x_o):
        return self.gamma5(self.A(self.gamma5(x_o)))

    def M(self, x_o):
        """A^dag A, Hermitian positive definite on the odd sites."""
        return self.Adag(self.A(x_o))

    def source(self, eta):
        """phi = eta_o + kappa H_oe eta_e."""
        eta = self._full(eta)
        return eta[self.odd] + self.kappa * self.hop(self.embed_even(eta[self.even]))[self.odd]

    def reconstruct(self, x_o, eta):
        """The full solution of D x = eta: x_o and x_e = eta_e + kappa H_eo x_o."""
        eta = self._full(eta)
        x = self.embed_odd(x_o)
        x[self.even] = eta[self.even] + self.kappa * self.hop(x)[self.even]
        return x
