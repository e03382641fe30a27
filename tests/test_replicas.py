"""The N > 1 path of bench.py (replicas only: each rank runs an independent
simulation, no data-path collective) with world_size-2 gloo process groups
on the CPU: max-over-ranks timing and the whole-job throughput, and the
reference arm printing on rank 0 only."""

import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = (100.0 + 50.0 * rank, 200.0 - 30.0 * rank)         # rank 1 slower in the first timing only
    t, v = bench.replica_throughput(dist, world, work=1000, steps=4, times_ms=times)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == [150.0, 200.0]                               # max over ranks, per timing
        assert v == pytest.approx([2 * 1000 * 4 / 0.150, 2 * 1000 * 4 / 0.200])


def _reference_rank(rank, world, port):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", str(world),
                           "--steps", "1", "--warmup", "0", "--workload", "pm32_mesh64"],
                          env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_on_rank_zero_only():
    port = _free_port()
    r1 = _reference_rank(1, 2, port)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _reference_rank(0, 2, port)
    assert r0.returncode == 0
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
