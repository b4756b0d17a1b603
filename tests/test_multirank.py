"""The multi-process path of bench.py on the CPU (gloo, world size 2).

The cascade is run as independent replicas, one per GPU, with no exchange
on the data path; the only collectives are the barrier and the max over
ranks of the timed region.  Here two gloo ranks stand in for two GPUs: they
report different times, and both must see the slowest one and the same
whole-job rate.  The reference arm must print on rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    tdist.barrier()
    my_ms = 100.0 + 50.0 * rank                    # rank 1 is the slow replica
    slowest = bench.reduce_max(my_ms, world)
    rate = bench.replica_rate(2.0e9, world, slowest)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_replicas_agree_on_the_slowest_time(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert got[0] == got[1]
    assert got[0]["slowest"] == 150.0
    assert got[0]["rate"] == pytest.approx(2 * 2.0e9 / 0.150)


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(12.5, 1) == 12.5
    assert bench.replica_rate(1.0e9, 1, 1000.0) == pytest.approx(1.0e9)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 3})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, bench.WORKLOADS["256"])
    assert buf.getvalue() == ""
