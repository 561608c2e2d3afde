"""The bench's multi-rank (replicas) logic on CPU with gloo, world size 2:
max-over-ranks timing, whole-job throughput, and the reference arm printing
on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    # rank r took (r + 1) * 100 ms for 4 steps of 1000 units
    value, tmax = bench.whole_job((rank + 1) * 100.0, 1000, 4, dist)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{value} {tmax}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp

    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    for r in range(ws):
        value, tmax = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert tmax == 200.0  # max over ranks, seen by every rank
        assert value == pytest.approx(1000 * 4 * ws / 0.2)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    value, tmax = bench.whole_job(50.0, 10, 5)
    assert tmax == 50.0 and value == pytest.approx(10 * 5 / 0.05)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(steps=1, warmup=3, workload=bench.WORKLOAD)
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""
