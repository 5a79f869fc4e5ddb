"""The N > 1 path of the bench on CPU: two gloo ranks run the replica
bookkeeping of paper_0901_3512_gb300/replicas.py (barrier, the slowest rank's
time by a MAX all-reduce, whole-job seconds per solve), and the reference arm
prints only on rank 0.  No GPU is used."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    from paper_0901_3512_gb300 import replicas
    w, r, _ = replicas.init("gloo")
    replicas.barrier()
    local_s = 1.5 + 2.0 * rank          # rank 1 is the slow one
    slowest = replicas.max_over_ranks(local_s)
    q.put((r, w, slowest, replicas.job_seconds_per_solve(slowest, w)))
    replicas.finish()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, slowest, per_solve in out:
        assert w == 2 and slowest == pytest.approx(3.5) and per_solve == pytest.approx(1.75)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    from paper_0901_3512_gb300 import replicas
    assert replicas.max_over_ranks(2.25) == 2.25
    assert replicas.job_seconds_per_solve(2.25, 1) == 2.25


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_on_rank_zero_only(rank):
    env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-sample-iters", "2",
                        "--workload", "tiny_4x4x4x4_nrhs4"],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if rank == 0:
        assert len(lines) == 1 and json.loads(lines[0])["impl"] == "reference"
    else:
        assert lines == []


def test_reference_arm_line_contract():
    """The reference arm (the oracle timed on the host cores) prints one JSON line
    with the bench contract's keys, on the same config as the GPU arm."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--cpu-sample-iters", "4"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["config"]["workload"] == "large_16x16x16x32_nrhs12"
    assert d["config"]["lattice"] == [16, 16, 16, 32] and d["config"]["nrhs"] == 12
