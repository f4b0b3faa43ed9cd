"""Host-side logic of bench.py: replica aggregation over ranks (gloo, two
processes on CPU), the clock-record parser and the traffic digest."""

import json
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    d = bench.init_dist(world, "gloo")
    secs = 2.0 if rank == 1 else 1.0  # rank 1 is the slow one
    bench.barrier(d)
    slowest = bench.reduce_max(d, secs)
    value = bench.aggregate(4e6, world, slowest)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"slowest": slowest, "value": value}, fh)
    d.destroy_process_group()


def test_two_rank_replica_aggregation_uses_the_slowest_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        res = json.load(open(tmp_path / f"r{r}.json"))
        assert res["slowest"] == 2.0
        assert res["value"] == pytest.approx(4e6 * 2 / 2.0 / 1e6)


def test_single_process_needs_no_process_group():
    assert bench.init_dist(1, "gloo") is None
    assert bench.reduce_max(None, 3.5) == 3.5


def test_clock_parser_flags_throttle_reasons(tmp_path):
    s = bench.ClockSampler(0)
    s.proc = object()
    s.path = str(tmp_path / "c.csv")
    with open(s.path, "w") as fh:
        fh.write("0, 1900, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        fh.write("0, 1950, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        fh.write("0, 300, 2070, 100.0, 0x1, Not Active, Not Active, Not Active, Not Active\n")
    out = s.summary()
    assert out["sm_max_mhz"] == 2070
    assert out["sm_mhz"] == pytest.approx(1925)
    assert out["reasons"] == ["sw_power_cap"]


def test_traffic_is_dropped_when_the_kernel_changed(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    for rel in bench.STEP_KERNEL_SOURCES:
        p = tmp_path / rel
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_text("kernel v1")
    (tmp_path / "profiles").mkdir()
    rec = {"source_digest": bench.step_kernel_digest(), "dram_bytes_per_launch": 123,
           "storage": "f32", "wall": 2}
    (tmp_path / "profiles" / "step_kernel_traffic.json").write_text(json.dumps(rec))
    assert bench.profiled_traffic() == 123
    assert bench.profiled_traffic("bf16", 2) is None
    (tmp_path / bench.STEP_KERNEL_SOURCES[0]).write_text("kernel v2")
    assert bench.profiled_traffic() is None


def test_warmup_below_three_is_rejected():
    with pytest.raises(SystemExit):
        bench.main(["--warmup", "2"])
