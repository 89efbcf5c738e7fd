"""The N > 1 path of bench.py: independent replicas, one per rank, no data-path collective; the job's
time is the slowest rank's and its throughput counts every rank's units.  Checked with world size 2
on the gloo backend (CPU); the CUDA path of each replica is the single-GPU path."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        sys.path.insert(0, ROOT)
        import bench
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")   # rank 1 is the slow replica
        rate = bench.whole_job_rate(1_000_000, ws, ms)
        out[rank] = (ms, rate)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_world_size_2():
    ws = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]                       # every rank reports the same job time
    ms, rate = res[0]
    assert ms == 15.0                             # the slowest replica
    assert rate == pytest.approx(2 * 1_000_000 / 15.0 * 1e-6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(90_518_849, 1, 12.0) == pytest.approx(90_518_849 / 12.0 * 1e-6)


def test_reference_arm_other_ranks_exit_silently():
    # under torchrun only rank 0 runs the CPU reference arm; the other ranks exit 0 without output
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
