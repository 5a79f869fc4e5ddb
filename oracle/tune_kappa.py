"""Tune kappa per gauge field so that cond(M) reaches its target (set-up only).

Run as a script:  python -m oracle.tune_kappa [field-name ...]
It calls nothing but the oracle and the seeded input generators, and writes
`paper_0901_3512_gb300/kappa.json` (kappa, the cond it reached, and how).

Reading of "kappa tuned by the oracle's Lanczos so that cond(M) ~ target":
kappa* is the smallest kappa > 0 at which cond(M(kappa)) first reaches the
target.  cond is not monotone in kappa, so the search scans upward from 0.05
in steps of 0.005 and then bisects the bracketing step until
|log10 cond - log10 target| <= 0.02.  cond comes from a dense eigensolve on
lattices of at most 4^4 sites, from the extreme Ritz values of plain Lanczos
on M otherwise.
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np

from oracle.seedcg import lanczos_extremes
from oracle.wilson import WilsonOperator
from paper_0901_3512_gb300 import workloads as W

KAPPA0, KSTEP, LOG_TOL = 0.05, 0.005, 0.02


def cond_of(op: WilsonOperator):
    if op.n <= 3072:
        ev = np.linalg.eigvalsh(op.dense(WilsonOperator.OP_M))
        return ev[-1] / ev[0], ev[0], ev[-1], 0
    lo, hi, it = lanczos_extremes(op.M, op.n, max_iters=6000)
    return hi / lo, lo, hi, it


def tune(dims, gauge, target, log=print):
    def c_at(k):
        op = WilsonOperator(dims, gauge, k)
        t0 = time.time()
        c = cond_of(op)
        log(f"  kappa={k:.6f} cond={c[0]:.4g} iters={c[3]} ({time.time() - t0:.1f}s)")
        return c

    lt = math.log10(target)
    k_lo, c_lo = None, None
    k = KAPPA0
    while True:
        c = c_at(k)
        if abs(math.log10(c[0]) - lt) <= LOG_TOL:
            return k, c
        if c[0] >= target:
            break
        k_lo, c_lo = k, c
        k = round(k + KSTEP, 10)
        if k > 1.0:
            raise RuntimeError("target cond not reached for kappa <= 1")
    k_hi = k
    if k_lo is None:
        raise RuntimeError("target already exceeded at the first kappa")
    for _ in range(60):
        km = 0.5 * (k_lo + k_hi)
        c = c_at(km)
        d = math.log10(c[0]) - lt
        if abs(d) <= LOG_TOL:
            return km, c
        if d < 0:
            k_lo = km
        else:
            k_hi = km
    return km, c


def main(argv):
    names = argv or list(W.FIELDS)
    path = W._KAPPA_FILE
    for name in names:
        f = W.FIELDS[name]
        print(f"tuning {name} dims={f.dims} eps={f.eps} seed={f.seed} target={f.cond_target:g}",
              flush=True)
        g = f.gauge()
        t0 = time.time()
        k, c = tune(f.dims, g, f.cond_target, log=lambda s: print(s, flush=True))
        table = W.kappa_table()  # merge with entries other runs wrote meanwhile
        table[name] = {"kappa": k, "cond": c[0], "lam_min": c[1], "lam_max": c[2],
                       "lanczos_iters": c[3], "target": f.cond_target,
                       "method": "dense eigvalsh" if c[3] == 0 else "Lanczos extreme Ritz values",
                       "seconds": round(time.time() - t0, 1)}
        with open(path + f".tmp{os.getpid()}", "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        os.replace(path + f".tmp{os.getpid()}", path)
        print(f"  -> kappa={k:.6f} cond={c[0]:.4g}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
