"""The multi-GPU form of bench.py: one replica per rank, no collective on the data path,
and a MAX over ranks of the timings, so that the job throughput is
world x (units per rank) / (slowest rank's time). Run here as two gloo ranks on CPU
processes (the host logic of the N>1 path; no GPU)."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    # each replica timed its own steps; rank 1 is the slower one on the first value
    mine = [1.0 + r, 5.0 - r, 0.25]
    got = bench.max_over_ranks(mine, dist, device="cpu")
    value = bench.job_throughput(1000.0, w, got[0])
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, w, local, got, value))


def test_two_gloo_ranks_reduce_timings_by_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, local, got, value) in enumerate(res):
        assert (rank, w, local) == (r, world, r)
        assert got == [2.0, 5.0, 0.25]  # the slowest rank's time for each entry
        assert value == pytest.approx(world * 1000.0 / 2.0)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([3, 1.5]) == [3.0, 1.5]
    assert bench.job_throughput(10.0, 1, 2.0) == 5.0


def test_gpus_flag_spawns_its_own_ranks():
    """bench.py --gpus 2 started as a plain process runs itself under torchrun as two
    ranks: the reference arm (CPU only) prints one line, from rank 0, with n_gpus 2."""
    import json
    import subprocess

    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.05"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_launch_command_names_torchrun_on_localhost():
    sys.path.insert(0, ROOT)
    import bench

    cmd = bench.launch_command(["--gpus", "4", "--steps", "3"], 4, 29555)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "--master-addr=127.0.0.1" in cmd and "--master-port=29555" in cmd
    assert cmd[-4:] == ["--gpus", "4", "--steps", "3"]
