"""The N > 1 path of the benchmark on the CPU: two gloo ranks on 127.0.0.1.

Each rank is a replica of the same single-GPU job (the path has no exchange step), so the only
cross-rank logic is the timing: the job waits for its slowest rank, and the whole-job rate counts
every rank's atoms in that time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench._env_rank()
        ms = bench.slowest_rank_ms(1.0 + 0.5 * r, dist, "cpu")
        out[rank] = (r, w, ms, bench.job_rate(w, 12288, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, ms, rate) in res.items():
        assert (r, w) == (rank, world)
        assert ms == 1.5  # rank 1's 1.5 ms is the job's step time on both ranks
        assert rate == pytest.approx(2 * 12288 / 1.5e-3)


def test_single_rank_is_its_own_time():
    import bench
    assert bench.slowest_rank_ms(2.0, None, "cpu") == 2.0
    assert bench.job_rate(1, 12288, 2.0) == pytest.approx(12288 / 2e-3)


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched as the driver launches it for N > 1: rank 0 alone runs the
    oracle and prints one JSON line; the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout[-2000:]
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
