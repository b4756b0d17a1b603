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


def test_reference_arm_line_has_the_contract_keys(monkeypatch):
    """Rank 0 (or a single process) prints one JSON line with the keys of
    the bench contract, for the oracle timed on the host cores."""
    sys.path.insert(0, ROOT)
    import bench
    for var in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(var, raising=False)
    args = type("A", (), {"steps": 1, "warmup": 3})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, bench.WORKLOADS["256"])
    lines = buf.getvalue().strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
