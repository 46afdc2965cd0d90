"""Host logic of bench.py's multi-process runs, on CPU with the gloo backend (world size 2):
each GPU runs an independent replica, the job's time is the slowest rank's, and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        local_ms = 100.0 + 25.0 * rank          # rank 1 is the slower replica
        total = bench.max_over_ranks(local_ms, ws, torch.device("cpu"))
        fps = bench.replica_fps(total, steps=20, ws=ws, channels=3)
        out.put((rank, total, fps))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_replica():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, total, fps in res:
        assert total == 125.0
        # 2 replicas x 20 frames in the slowest rank's 125 ms
        assert fps == pytest.approx(40 / 0.125)


def test_single_process_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    # a 1-channel profiling variant counts thirds of an RGB frame
    assert bench.replica_fps(100.0, steps=30, ws=1, channels=1) == pytest.approx(100.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        gpus, steps, warmup = 2, 1, 0

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_headline_line_has_the_contract_keys():
    # the JSON line's keys and their meaning, from synthetic measurements (no GPU)
    import json
    prof = {"row_first": (0.9, 20), "row": (2.6, 60), "column": (2.4, 80), "row_inverse": (0.45, 20)}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    line = bench.headline_line(ws=1, steps=20, warmup=5, ch=3, hh=1080, ww=1920, fps=3900.0, total_ms=20 / 3.9,
                               pct=[0.25, 0.256, 0.26], prof=prof, e2e_fps=2290.0, frame_nbytes=24883200,
                               clocks=clocks)
    json.dumps(line)   # serializable
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["unit"] == "fps" and line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["config"]["workload"].startswith("ILS 1920x1080 RGB")
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["kernel"] == "row" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    # the row pass moves 12 B per pixel and channel: 74.6 MB per 1080p RGB launch
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(12 * 1920 * 1080 * 3, rel=1e-3)
    assert r["achieved"] == pytest.approx(r["algorithmic_bytes_per_launch"] / (2.6 / 60 / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    e = line["e2e"]
    assert e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 24883200 and e["unit"] == "fps"
    assert line["gpu_launches"] == 180
