"""Oracle: Improved Seed-CG in plain FP64 numpy (test infrastructure only).

Every function follows the paper (Abdel-Rehim, Morgan, Wilcox, "Seed methods
for linear equations in lattice QCD problems with multiple right-hand sides",
Lattice 2008) in its own order and notation.  `M` is any callable applying the
Hermitian positive-definite matrix to a flat complex128 vector.

Readings taken where the paper is silent (all listed in the design notes):
  * alpha_i = Re(v_i^dag f): the imaginary part is roundoff (T is real).
  * v_2 = f / beta_1 after the first Lanczos iteration (Algorithm 1, step 2
    never names v_2; step 9 does the same for later i).
  * Steps 6-7 use v_i before step 8 re-orthogonalises it; the re-orthogonalised
    v_i is what is stored in V and what step 5 of iteration i+1 uses.  T is
    not changed by the re-orthogonalisation.
  * Re-orthogonalisation is classical Gram-Schmidt in the paper's order:
    v_i against v_1..v_{i-1} then renormalised; f against v_1..v_i.  `po_passes`
    = 2 repeats each projection once (CGS2).
  * m_conv is the first i with beta_i |zeta_i / delta_i| <= tol ||b^1||
    (the D-Lanczos residual norm); the run stops at
    m = min(m_max, max(m_conv + extra_iters, ceil(past_factor * m_conv))).
  * Lanczos stops early (m = i) if beta_i <= BREAKDOWN * |alpha_i| (invariant
    subspace: x^1 is then exact in exact arithmetic).
  * CG for j >= 2 is textbook Hestenes-Stiefel; convergence is the true
    residual ||b - M x|| <= tol ||b|| recomputed in FP64.  When the recursive
    residual says "converged" but the true one does not, CG restarts from the
    true residual.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

BREAKDOWN = 1e-14


def _norm(a: np.ndarray) -> float:
    return math.sqrt(np.vdot(a, a).real)


# ---------------------------------------------------------------------------
# Algorithm 1 (Section 2): Seed-CG(m, k), literal
# ---------------------------------------------------------------------------

@dataclass
class LanczosSeedResult:
    X: np.ndarray                 # [nrhs][N]: x^1 and the seeded guesses x^j (j >= 2)
    R0: np.ndarray                # [nrhs][N]: r_0^j = b^j - M x_0^j
    V: np.ndarray                 # [m][N]: stored basis v_1..v_m (after any re-orthogonalisation)
    alpha: np.ndarray             # [m]
    beta: np.ndarray              # [m]: beta_1..beta_m
    beta0: float
    delta: np.ndarray             # [m]
    gamma: np.ndarray             # [m-1]: gamma_1..gamma_{m-1}
    zeta: np.ndarray              # [m]
    eta: np.ndarray               # [nrhs-1][m]: eta^j after each iteration i
    resid_est: np.ndarray         # [m]: beta_i |zeta_i / delta_i|
    m_conv: int
    m: int
    po_count: int
    breakdown: bool = False
    x1_history: Optional[List[np.ndarray]] = None


def seed_lanczos(M: Callable[[np.ndarray], np.ndarray], B: np.ndarray, X0: Optional[np.ndarray],
                 tol: float, m_max: int, reorth_period: int, past_factor: float = 1.0,
                 extra_iters: int = 0, po_passes: int = 1,
                 keep_x1_history: bool = False, po_guard: bool = True) -> LanczosSeedResult:
    """Algorithm 1, steps 1-9, for the first right-hand side, seeding the others.

    B: [nrhs][N] right-hand sides; X0: initial guesses (None = zero).
    reorth_period = k (0 = never).  po_guard = False runs step 8 as printed,
    ending the run only if v_i vanishes.  Returns the seeded X and all scalars.
    """
    B = np.asarray(B, dtype=np.complex128)
    nrhs, n = B.shape
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.complex128)
    # Step 1: initial residuals
    R0 = np.empty_like(B)
    for j in range(nrhs):
        R0[j] = B[j] - M(X[j]) if X0 is not None else B[j].copy()
    bnorm1 = _norm(B[0])

    V = np.empty((max(m_max, 1), n), dtype=np.complex128)
    alpha = np.zeros(m_max)
    beta = np.zeros(m_max)
    delta = np.zeros(m_max)
    gamma = np.zeros(max(m_max - 1, 0))
    zeta = np.zeros(m_max)
    eta_hist = np.zeros((max(nrhs - 1, 0), m_max), dtype=np.complex128)
    resid = np.zeros(m_max)
    hist = [] if keep_x1_history else None

    beta0 = _norm(R0[0])
    if beta0 == 0.0 or m_max < 1:
        return LanczosSeedResult(X, R0, V[:0], alpha[:0], beta[:0], beta0, delta[:0], gamma[:0],
                                 zeta[:0], eta_hist[:, :0], resid[:0], 0, 0, 0, False, hist)

    # Step 2: first Lanczos iteration
    v = R0[0] / beta0
    f = M(v)
    alpha[0] = np.vdot(v, f).real
    f = f - alpha[0] * v
    beta[0] = _norm(f)
    V[0] = v
    # Step 3: linear equations for the first iteration
    delta[0] = alpha[0]
    w = v / delta[0]
    zeta[0] = beta0
    X[0] = X[0] + zeta[0] * w
    # Step 4: other right-hand sides
    eta = np.zeros(max(nrhs - 1, 0), dtype=np.complex128)
    for j in range(1, nrhs):
        eta[j - 1] = np.vdot(v, R0[j])
        X[j] = X[j] + eta[j - 1] * w
    eta_hist[:, 0] = eta
    resid[0] = beta[0] * abs(zeta[0] / delta[0])
    if hist is not None:
        hist.append(X[0].copy())

    m = m_max
    m_conv = 0
    po_count = 0
    breakdown = False

    def set_m(i_conv: int) -> int:
        return min(m_max, max(i_conv + extra_iters, int(math.ceil(past_factor * i_conv))))

    if resid[0] <= tol * bnorm1:
        m_conv = 1
        m = set_m(1)
    if beta[0] <= BREAKDOWN * abs(alpha[0]):
        breakdown = True
        m = 1
    i = 1  # 1-based iteration index of the last completed iteration
    v_prev = v
    if m > 1:
        v = f / beta[0]  # reading: v_2 = f / beta_1
    while i < m:
        i += 1
        k0 = i - 1  # 0-based slot of iteration i
        # Step 5: Lanczos iteration
        f = M(v) - beta[k0 - 1] * v_prev
        alpha[k0] = np.vdot(v, f).real
        f = f - alpha[k0] * v
        # Step 6: linear equations
        g = beta[k0 - 1] / delta[k0 - 1]
        gamma[k0 - 1] = g
        delta[k0] = alpha[k0] - g * beta[k0 - 1]
        w = (v - beta[k0 - 1] * w) / delta[k0]
        zeta[k0] = -g * zeta[k0 - 1]
        X[0] = X[0] + zeta[k0] * w
        # Step 7: other right-hand sides (uses r_0^j, and v_i before step 8)
        for j in range(1, nrhs):
            eta[j - 1] = np.vdot(v, R0[j]) - g * eta[j - 1]
            X[j] = X[j] + eta[j - 1] * w
        eta_hist[:, k0] = eta
        # Step 8: periodic re-orthogonalisation.  The paper is silent on a PO
        # step that finds v_i mostly inside span(v_1..v_{i-1}) (the basis lost
        # orthogonality beyond repair between two PO steps, or the Krylov space
        # is exhausted).  Reading: the run ends at i - 1 when a projection
        # pass leaves ||v_i|| < 1/2, or when re-orthogonalising lengthens f
        # by more than 1 %; the systems then go to CG.  Both follow from
        # ||v - V c||^2 = ||v||^2 - ||c||^2 + c^dag (V^dag V - I) c, c = V^dag v:
        # with an orthonormal V a pass never lengthens a vector (growth beyond
        # rounding means V^dag V has an eigenvalue above 2, a direction stored
        # more than once), and ||v'|| < 1/2 means v_i lies within 30 degrees
        # of the stored space, an order-one loss of orthogonality.
        if reorth_period > 0 and i % reorth_period == 0:
            beta_pre = _norm(f)
            if po_guard:
                v_po, f_po, ok = periodic_reorth(V, i, v, f, po_passes, guard=True)
                broken = not ok or not (_norm(f_po) <= 1.01 * beta_pre)
            else:
                with np.errstate(all="ignore"):
                    v_po, f_po = periodic_reorth(V, i, v, f, po_passes)
                broken = not (np.all(np.isfinite(v_po)) and np.isfinite(_norm(f_po)))
            if broken:
                breakdown = True
                i -= 1
                break
            po_count += 1
            v, f = v_po, f_po
        V[k0] = v
        # Step 9: finish the iteration
        beta[k0] = _norm(f)
        resid[k0] = beta[k0] * abs(zeta[k0] / delta[k0])
        if hist is not None:
            hist.append(X[0].copy())
        if m_conv == 0 and resid[k0] <= tol * bnorm1:
            m_conv = i
            m = set_m(i)
        if beta[k0] <= BREAKDOWN * abs(alpha[k0]):
            breakdown = True
            m = i
            break
        v_prev = v
        v = f / beta[k0]

    m = i
    return LanczosSeedResult(X, R0, V[:m].copy(), alpha[:m].copy(), beta[:m].copy(), beta0,
                             delta[:m].copy(), gamma[:m - 1].copy(), zeta[:m].copy(),
                             eta_hist[:, :m].copy(), resid[:m].copy(), m_conv, m, po_count,
                             breakdown, hist)


def periodic_reorth(V: np.ndarray, i: int, v: np.ndarray, f: np.ndarray, passes: int = 1,
                    guard: bool = False):
    """Step 8 of Algorithm 1 at iteration i (1-based), classical Gram-Schmidt.

    V holds v_1..v_{i-1} in rows 0..i-2.  Re-orthonormalise v_i against
    v_1..v_{i-1}; then re-orthogonalise f (the un-normalised v_{i+1}) against
    v_1..v_i, v_i being the new one.  Row i-1 of V receives the new v_i.
    With guard=True the result is (v, f, ok): ok is False, and V is left
    untouched, when a pass leaves ||v|| below 1/2 (v_i was a unit vector).
    """
    prev = V[:i - 1]
    for _ in range(passes):
        v = v - (prev.conj() @ v) @ prev
        if guard and not (_norm(v) >= 0.5):
            return v, f, False
    v = v / _norm(v)
    V[i - 1] = v
    upto = V[:i]
    for _ in range(passes):
        f = f - (upto.conj() @ f) @ upto
    return (v, f, True) if guard else (v, f)


# ---------------------------------------------------------------------------
# Eq. (1): the Galerkin seed from the stored basis and T
# ---------------------------------------------------------------------------

def tridiag(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Dense Lanczos T (Eq. 2, left side) of order m from alpha_1..m, beta_1..m-1."""
    m = len(alpha)
    t = np.diag(np.asarray(alpha, dtype=np.float64))
    if m > 1:
        t += np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    return t


def galerkin_seed(V: np.ndarray, alpha: np.ndarray, beta: np.ndarray, R0: np.ndarray,
                  X0: Optional[np.ndarray] = None) -> np.ndarray:
    """Eq. (1): x^j = x_0^j + V y^j, y^j = T^{-1} (V^dag r_0^j), all j at once."""
    import scipy.linalg as sla
    m = V.shape[0]
    if m == 0:
        return np.zeros_like(R0) if X0 is None else np.array(X0)
    rhs = V.conj() @ R0.T                       # [m][nrhs] = V^dag R0
    ab = np.zeros((3, m), dtype=np.complex128)  # banded storage of T
    ab[1] = alpha
    if m > 1:
        ab[0, 1:] = beta[:m - 1]
        ab[2, :-1] = beta[:m - 1]
    Y = sla.solve_banded((1, 1), ab, rhs)
    X = (V.T @ Y).T
    return X if X0 is None else X0 + X


def lu_factors(alpha: np.ndarray, beta: np.ndarray):
    """Eq. (2): T = L U with L unit lower bidiagonal (gamma below the
    diagonal) and U upper bidiagonal (delta on, beta above the diagonal)."""
    m = len(alpha)
    delta = np.zeros(m)
    gamma = np.zeros(max(m - 1, 0))
    delta[0] = alpha[0]
    for i in range(1, m):
        gamma[i - 1] = beta[i - 1] / delta[i - 1]
        delta[i] = alpha[i] - gamma[i - 1] * beta[i - 1]
    L = np.eye(m) + np.diag(gamma, -1)
    U = np.diag(delta) + (np.diag(beta[:m - 1], 1) if m > 1 else 0)
    return L, U, gamma, delta


# ---------------------------------------------------------------------------
# Standard CG for the seeded systems (Section 2: "a standard CG solver")
# ---------------------------------------------------------------------------

@dataclass
class CGResult:
    x: np.ndarray
    iters: int
    true_resid: float      # ||b - M x|| / ||b||
    converged: bool
    resid_history: List[float] = field(default_factory=list)


def cg(M: Callable[[np.ndarray], np.ndarray], b: np.ndarray, x0: Optional[np.ndarray], tol: float,
       maxiter: int, keep_history: bool = False, max_restarts: int = 5) -> CGResult:
    """Hestenes-Stiefel CG; stops on the FP64 true relative residual <= tol."""
    b = np.asarray(b, dtype=np.complex128)
    bnorm = _norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    if bnorm == 0.0:
        return CGResult(np.zeros_like(b), 0, 0.0, True, [])
    hist: List[float] = []
    it = 0
    restarts = 0
    r = b - M(x)
    while True:
        rr = np.vdot(r, r).real
        p = r.copy()
        if keep_history:
            hist.append(math.sqrt(rr) / bnorm)
        while math.sqrt(rr) > tol * bnorm and it < maxiter:
            q = M(p)
            a = rr / np.vdot(p, q).real
            x = x + a * p
            r = r - a * q
            rr_new = np.vdot(r, r).real
            p = r + (rr_new / rr) * p
            rr = rr_new
            it += 1
            if keep_history:
                hist.append(math.sqrt(rr) / bnorm)
        r = b - M(x)
        tr = _norm(r) / bnorm
        if tr <= tol or it >= maxiter or restarts >= max_restarts:
            return CGResult(x, it, tr, tr <= tol, hist)
        restarts += 1


# ---------------------------------------------------------------------------
# The whole method: Algorithm 1 for RHS 1, then CG for the seeded systems
# ---------------------------------------------------------------------------

@dataclass
class SolveResult:
    X: np.ndarray
    iters: np.ndarray          # per RHS: Lanczos iterations (j=1) + CG iterations
    true_resid: np.ndarray     # ||b - M x|| / ||b|| per RHS
    seed: LanczosSeedResult
    cg_iters: np.ndarray       # CG iterations per RHS (0 for j = 1 unless it needed CG)


def improved_seed_cg(M, B, X0, tol, m_max, reorth_period, past_factor=1.0, extra_iters=0,
                     po_passes=1, seed_mode="literal", cg_maxiter=100000, po_guard=True) -> SolveResult:
    """Seed once with RHS 1 past convergence (Section 2, improvements 1-3),
    then standard CG for every system whose true residual exceeds tol."""
    B = np.asarray(B, dtype=np.complex128)
    nrhs = B.shape[0]
    res = seed_lanczos(M, B, X0, tol, m_max, reorth_period, past_factor, extra_iters, po_passes,
                       po_guard=po_guard)
    if seed_mode == "blocked":
        # Eq. (1) is the closed form of steps 4 and 7 for the systems j >= 2; the
        # first system's x^1 is the one steps 3 and 6 build by the LU recurrence
        X = galerkin_seed(res.V, res.alpha, res.beta, res.R0,
                          None if X0 is None else np.asarray(X0, dtype=np.complex128))
        X[0] = res.X[0]
    else:
        X = res.X.copy()
    iters = np.zeros(nrhs, dtype=np.int64)
    cg_iters = np.zeros(nrhs, dtype=np.int64)
    tr = np.zeros(nrhs)
    iters[0] = res.m
    for j in range(nrhs):
        bn = _norm(B[j])
        t = _norm(B[j] - M(X[j])) / bn if bn > 0 else 0.0
        if j == 0 and t <= tol:
            tr[0] = t
            continue
        out = cg(M, B[j], X[j], tol, cg_maxiter)
        X[j] = out.x
        cg_iters[j] = out.iters
        iters[j] += out.iters
        tr[j] = out.true_resid
    return SolveResult(X, iters, tr, res, cg_iters)


# ---------------------------------------------------------------------------
# Lanczos estimate of the extreme eigenvalues of M (kappa tuning; set-up only)
# ---------------------------------------------------------------------------

@dataclass
class ClassicResult:
    X: np.ndarray
    iters: np.ndarray          # per RHS: Lanczos iterations of its own round + final CG iterations
    lanczos_iters: np.ndarray  # per RHS: iterations of the round in which it was the seed system
    cg_iters: np.ndarray       # per RHS: CG iterations after the rounds (0 when already at tol)
    true_resid: np.ndarray


def classic_seed_cg(M, B, X0, tol, m_max, reorth_period=0, po_passes=1, seed_mode="blocked",
                    cg_maxiter=100000) -> ClassicResult:
    """Repeated ("traditional") seeding, the comparison variant of Section 1: each
    unsolved system in turn is the seed system.  Its Lanczos run (Algorithm 1 steps
    1-9, from its current guess, stopped at convergence: no past-convergence) seeds
    every later system by the Galerkin projection onto the new Krylov subspace
    (Eq. 1, or the literal per-iteration updates), then the next system, starting
    from its seeded guess, becomes the seed.  A system whose true residual is still
    above tol after the rounds finishes by CG."""
    B = np.asarray(B, dtype=np.complex128)
    nrhs = B.shape[0]
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.complex128)
    have_x0 = X0 is not None
    lz = np.zeros(nrhs, dtype=np.int64)
    for j in range(nrhs):
        start = X[j:] if (have_x0 or j > 0) else None
        res = seed_lanczos(M, B[j:], start, tol, m_max, reorth_period, 1.0, 0, po_passes)
        if seed_mode == "blocked":
            X[j:] = galerkin_seed(res.V, res.alpha, res.beta, res.R0, start)
            X[j] = res.X[0]      # the seed system's own x by steps 3 and 6
        else:
            X[j:] = res.X
        lz[j] = res.m
    cg_iters = np.zeros(nrhs, dtype=np.int64)
    tr = np.zeros(nrhs)
    for j in range(nrhs):
        bn = _norm(B[j])
        t = _norm(B[j] - M(X[j])) / bn if bn > 0 else 0.0
        if t <= tol:
            tr[j] = t
            continue
        out = cg(M, B[j], X[j], tol, cg_maxiter)
        X[j] = out.x
        cg_iters[j] = out.iters
        tr[j] = out.true_resid
    return ClassicResult(X, lz + cg_iters, lz, cg_iters, tr)


def lanczos_extremes(M, n: int, seed: int = 12345, max_iters: int = 4000, rtol: float = 2e-3,
                     check_every: int = 25):
    """Plain Lanczos from a seeded random start; returns (lam_min, lam_max, iters).

    The extreme Ritz values of T_i converge first and are unaffected by the
    ghost copies that loss of orthogonality produces; iteration stops when
    both extremes changed by less than rtol over the last two checks.
    """
    import scipy.linalg as sla
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v /= _norm(v)
    v_prev = np.zeros_like(v)
    b_prev = 0.0
    al, be = [], []
    hist = []
    for it in range(1, max_iters + 1):
        f = M(v) - b_prev * v_prev
        a = np.vdot(v, f).real
        f -= a * v
        b = _norm(f)
        al.append(a)
        be.append(b)
        if it % check_every == 0 or b == 0.0 or it == max_iters:
            ev = sla.eigvalsh_tridiagonal(np.array(al), np.array(be[:-1]))
            hist.append((ev[0], ev[-1]))
            if len(hist) >= 3:
                (l0, h0), (l2, h2) = hist[-3], hist[-1]
                if abs(l2 - l0) <= rtol * abs(l2) and abs(h2 - h0) <= rtol * abs(h2):
                    return ev[0], ev[-1], it
        if b == 0.0:
            ev = sla.eigvalsh_tridiagonal(np.array(al), np.array(be[:-1]))
            return ev[0], ev[-1], it
        v_prev, v = v, f / b
        b_prev = b
    return hist[-1][0], hist[-1][1], max_iters
