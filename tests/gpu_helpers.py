"""Shared helpers for the GPU parity tests (inputs from the seeded
generators, oracle on the CPU, CUDA path through the C-ABI binding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.cpu().numpy()


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def recompute_slack(lam_max, xnorm, bnorm):
    """How far two FP64 evaluations of ||b - M x|| / ||b|| in different
    summation orders may differ: a small multiple of eps ||M|| ||x|| / ||b||
    (100 covers the two stencil passes and the reductions with room)."""
    return 100 * 2.0 ** -53 * lam_max * xnorm / bnorm
