"""The multi-rank path of bench.py on CPU (gloo, world size 2): max-over-ranks
timing, barriers, the aggregate throughput formula, and the reference arm
running on rank 0 only."""
import multiprocessing as mp
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.barrier_max(10.0 * (rank + 1), world)
    bench.barrier(world)
    q.put((rank, v))
    dist.destroy_process_group()


def test_barrier_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 20.0, 1: 20.0}


def test_aggregate_throughput_is_weak_scaling():
    m, iters, steps = 1 << 26, 20, 10
    one = bench.aggregate_gteps(m, iters, steps, 1, 100.0)
    assert bench.aggregate_gteps(m, iters, steps, 4, 100.0) == pytest.approx(4 * one)
    # the slowest rank sets the time
    assert bench.aggregate_gteps(m, iters, steps, 2, 200.0) == pytest.approx(one)


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, workload = 1, 0, "rmat16"

    assert bench.run_reference(Args(), bench.WORKLOADS["rmat16"]) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_reports_our_config(capsys):
    # both arms name the same workload, metric and config (the reference runs
    # the oracle's iteration loop only; its CSR is built before the steps)
    import json

    class Args:
        steps, warmup, workload = 2, 1, "rmat16"

    w = bench.WORKLOADS["rmat16"]
    assert bench.run_reference(Args(), w) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench.config_for(w, "rmat16")
    assert line["metric"] == bench.METRIC and line["unit"] == "GTEPS"
    assert line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_default_workload_is_the_scale_26_graph():
    w = bench.WORKLOADS["rmat26"]
    cfg = bench.config_for(w, "rmat26")
    assert cfg["m"] == 1_476_395_008 and cfg["n"] == 1 << 26 and cfg["P"] == 64
    assert cfg["iters_per_step"] == 10
    import argparse  # noqa: F401  (the parser's default is checked by name below)
    src = open(bench.__file__).read()
    assert 'ap.add_argument("--workload", default="rmat26"' in src


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    # the committed DRAM-traffic record applies only while the sweep kernel's
    # sources hash to what was captured; any edit turns it into null
    import hashlib
    import json

    root = tmp_path
    (root / "profiles").mkdir()
    src = root / "k.cu"
    src.write_text("kernel v1")
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    (root / "profiles" / "traffic.json").write_text(json.dumps(
        {"rmatX": {"bytes_per_launch": 123, "sources_sha256": {"k.cu": h}}}))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_record("rmatX") == 123
    assert bench.traffic_record("other") is None
    src.write_text("kernel v2")
    assert bench.traffic_record("rmatX") is None


def test_committed_traffic_record_matches_the_current_sweep_kernel():
    import hashlib
    import json
    import os

    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for wl in ("rmat25", "rmat26"):
        ent = rec[wl]
        assert ent["bytes_per_launch"] > 0
        for f, h in ent["sources_sha256"].items():
            assert hashlib.sha256(open(os.path.join(bench.ROOT, f), "rb").read()).hexdigest() == h, f


def test_compact_extras_keep_scalars_and_errors():
    out = bench.compact({"rmat22": {"gteps": 1.0, "roofline_frac": 0.2, "D": 5},
                         "scc": {"error": "x" * 500}, "unknown": {"a": 1}, "bad": 3})
    assert out["rmat22"] == {"gteps": 1.0, "roofline_frac": 0.2}
    assert len(out["scc"]["error"]) == 120
    assert out["unknown"] == {} and "bad" not in out


def test_link_roofline_only_for_runs_that_stream():
    resident = {"h2d_bytes": 0, "d2h_bytes": 4096, "ms": 10.0}  # activity flags only
    assert bench.link_roofline(resident, 50.0) is None
    streamed = {"h2d_bytes": 500_000_000, "d2h_bytes": 0, "ms": 20.0}
    r = bench.link_roofline(streamed, 50.0)
    assert abs(r["link_gbs"] - 25.0) < 1e-9 and abs(r["link_frac"] - 0.5) < 1e-12


def test_compact_keeps_the_named_scalars_and_errors():
    extras = {"rmat26_programs": {"spu_bfs_ms": 1.0, "mpu6gb_wcc_link_frac": 0.9, "spu_bfs": {"ms": 1.0}},
              "scc": {"error": "x" * 500}, "unknown": {"a": 1}, "not_a_dict": 3}
    out = bench.compact(extras)
    assert out["rmat26_programs"] == {"spu_bfs_ms": 1.0, "mpu6gb_wcc_link_frac": 0.9}
    assert out["scc"] == {"error": "x" * 120}
    assert out["unknown"] == {} and "not_a_dict" not in out
