"""The multi-rank path of bench.py on CPU: world size 2 over gloo.  Each rank is an
independent replica; the job's time is the slowest rank's, and the whole-job value
counts the units of all ranks.  (On GPUs the same helpers run over NCCL.)"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]      # rank 1 is the slow replica
        m = bench.max_over_ranks(ms)
        v = bench.whole_job_value(1000, m, world)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{m} {v}\n")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        m, v = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        assert m == 150.0                       # every rank sees the slowest replica's time
        assert abs(v - 2 * 1000 / 0.150) < 1e-9  # units of both ranks per second of the slowest


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.5) == 42.5
    assert bench.whole_job_value(500, 250.0, 1) == 2000.0
