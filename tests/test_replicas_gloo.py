"""The N-GPU path of the benchmark, exercised on host cores with world size 2.

The time step has no exchange between devices, so an N-GPU run is N
independent replicas: the ranks meet at barriers around the timed region and
report the slowest rank's time.  These tests run that host logic over the
gloo backend, and the reference arm under the launcher the driver uses.
"""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    r, lr, w = bench.dist_env()
    reps = bench.Replicas(w, "gloo")
    reps.barrier()
    slow = reps.max(1.5 + 2.0 * rank)      # rank 1 is the slow replica
    fast = reps.max(10.0 - rank)           # rank 0 is the slow replica
    reps.barrier()
    reps.close()
    q.put((r, lr, w, slow, fast))


def test_replicas_two_gloo_ranks_agree_on_slowest():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[:3] for g in got] == [(0, 0, 2), (1, 1, 2)]
    for g in got:
        assert g[3] == 3.5 and g[4] == 10.0


def test_replicas_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas(1, "gloo")
    reps.barrier()
    assert reps.max(2.25) == 2.25
    reps.close()


def test_config_names_replicas_for_two_ranks():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1408_4675_gb300 import inputs
    cfg = inputs.make_config(3, n=32, n_steps=1)
    assert bench.bench_config(cfg, 2)["parallelism"] == "replicas"
    assert bench.bench_config(cfg, 1)["parallelism"] == "single_gpu"


def test_reference_arm_under_two_rank_launcher():
    """Rank 0 alone times the oracle and prints one line; rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--grid", "32"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["config"]["parallelism"] == "replicas"
    assert out["value"] > 0 and out["e2e"]["value"] == out["value"]
    assert out["steps"] == 1 and "32^3" in out["cpu_baseline"]["sample"]


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
