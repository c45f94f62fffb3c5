"""The host paths of bench.py on CPU: world-size-2 gloo ranks, each an
independent replica, aggregated as (sum of units) / (max of seconds); and the
reference arm (the oracle on a bounded sample), alone and under torchrun."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    units, secs = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank, ws)
    assert bench.dist_env() == (ws, rank, rank)
    dist.destroy_process_group()
    q.put((rank, units, secs))


def test_replica_aggregation_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, units, secs in res:
        assert units == 3000.0 and secs == 1.5


def _json_lines(out):
    import json
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check_reference_line(r, n_gpus):
    assert r["impl"] == "reference" and r["n_gpus"] == n_gpus and r["steps"] == 1 and r["warmup"] == 3
    assert r["value"] > 0 and r["unit"] == "DOF*steps/s" and r["higher_is_better"] is True
    assert r["dtype"] == "f64" and r["data"] == "synthetic" and "1024x1024" in r["config"]["workload"]
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == r["value"] and cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_one_process():
    # bench.py --impl reference: the oracle on a bounded sample, one JSON line
    import subprocess
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _json_lines(p.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 1)


def test_reference_arm_two_ranks_gloo():
    # under torchrun with two ranks only rank 0 runs the oracle and prints;
    # the other rank exits 0 without work
    import subprocess
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _json_lines(p.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 2)
