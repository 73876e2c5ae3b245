"""The multi-rank path of bench.py (replicas, max-over-ranks timing) on CPU
with two gloo ranks: every rank reports its own time, the job rate uses the
slowest rank and counts every rank's gradients."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_own = 0.5 + rank  # rank 1 is the slow one
    value, t_max = bench.job_throughput(t_own, 10, dist, torch.device("cpu"))
    dist.barrier()
    q.put((rank, value, t_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max in got:
        assert t_max == pytest.approx(1.5)
        assert value == pytest.approx(2 * 10 / 1.5)


def test_single_rank_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(2.0, 8, None, torch.device("cpu")) == (4.0, 2.0)


def test_bench_starts_its_own_ranks():
    """`bench.py --gpus 2` outside torchrun starts two ranks itself (under
    torch.distributed.run on 127.0.0.1); the reference arm runs on rank 0
    alone, which prints one line reporting the true world size."""
    import json
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--workload", "mcvqe8", "--cpu-seconds", "0.3",
                        "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_relaunch_command():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    cmd = bench.relaunch_cmd(["--gpus", "4", "--steps", "3"], 4, 29500)
    assert cmd[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"]
    assert "--nproc-per-node=4" in cmd and cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[-3:] == ["--gpus", "4", "--steps", "3"][-3:]
