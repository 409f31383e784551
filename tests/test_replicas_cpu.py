"""The multi-process path of bench.py on CPU (gloo, world size 2): independent
replicas with no data-path collective, whole-job rate = the units of all ranks over
the slowest rank's timed region; the reference arm prints one line from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, units, seconds, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.replica_rate(units[rank], seconds[rank], "cpu")
    finally:
        dist.destroy_process_group()


def test_replica_rate_sums_units_over_the_slowest_rank():
    import torch.multiprocessing as mp
    units, seconds = [3.0e9, 5.0e9], [2.0, 4.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), units, seconds, out), nprocs=2, start_method="spawn")
        res = dict(out)
    for r in (0, 1):
        rate, total, sec = res[r]
        assert total == sum(units) and sec == max(seconds)
        assert rate == pytest.approx(sum(units) / max(seconds))


def test_replica_rate_of_one_process_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_rate(6.0, 3.0) == (2.0, 6.0, 3.0)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    env = dict(os.environ, PYTHONPATH=ROOT, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny", "--gpus", "2",
           "--steps", "5", "--warmup", "3"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
