"""The autotuners' shared SEEDCG_TUNE_CACHE file: a first process tunes the
brick dslash and the batched CG and appends both kinds of lines; a second
process reading the same file finds every entry it needs and appends nothing."""
import os
import subprocess
import sys

import pytest

from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
from paper_0901_3512_gb300 import seedcg, workloads as W
dims = (8, 8, 8, 8)
s = seedcg.Solver(dims, W.gauge_field(dims, 0.5, 71), 0.18, precision="mixed_v32")
x = torch.from_numpy(W.random_spinors(dims, 12, 72)).cuda()
y = torch.zeros_like(x)
s.apply(seedcg.OP_D, x, y, prec=1, multi=1)
b = torch.from_numpy(W.z2_sources(dims, 3, 71)).cuda()
X = torch.zeros_like(b)
code, info = s.solve(b, X, 1e-8, 0, 10)
assert code == 0
s.close()
print("done")
'''


def test_shared_tune_cache_round_trip(tmp_path):
    need_gpu()
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, SEEDCG_TUNE_CACHE=str(cache))
    for run in range(2):
        r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, env=env,
                           timeout=600)
        assert r.returncode == 0 and "done" in r.stdout, r.stderr[-2000:]
        lines = cache.read_text().splitlines()
        if run == 0:
            first = lines
            assert any(l.startswith("brick_") and len(l.split()) == 4 for l in lines), lines
            assert any(l.startswith("mf_dslash") and len(l.split()) == 2 for l in lines), lines
    assert lines == first
