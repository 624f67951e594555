"""The benchmark's multi-replica logic on the CPU: two gloo ranks, as
torchrun launches them for --gpus 2 (one process per GPU, replicas only).
Whole-job throughput counts every rank's frames over the slowest rank's
time; replicas decode distinct frames; the reference arm runs on rank 0
alone."""
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) seconds for its 10 frames
        rate, tmax = bench.job_rate(10, float(rank + 1), world, torch.device("cpu"))
        dist.barrier()
        q.put((rank, rate, tmax))
    finally:
        dist.destroy_process_group()


def test_job_rate_is_max_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    # both ranks: 2 x 10 frames over the slowest rank's 2 s
    assert got == [(0, 10.0, 2.0), (1, 10.0, 2.0)]


def test_job_rate_single_process():
    assert bench.job_rate(128, 0.5, 1, torch.device("cpu")) == (256.0, 0.5)


def test_replicas_decode_distinct_frames():
    seeds = {bench.replica_seed(r, 128, b) for r in range(8) for b in range(128)}
    assert len(seeds) == 8 * 128


def test_reference_arm_runs_on_rank_zero_only():
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert bench.run_reference(args, rank=1) == 0          # no work, no output


def test_reference_arm_line_on_rank_zero(capsys):
    """Rank 0 times the FP64 oracle on a one-row crop and prints one JSON
    line with the reference arm's keys: the same metric and unit as ours,
    its own cpu_baseline (the oracle, the threads used, the sample) and an
    e2e object with no host-device bytes."""
    import json
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-rows", "1"])
    assert bench.run_reference(args, rank=0) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "frames/s"
    assert d["higher_is_better"] is True and d["value"] > 0 and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "1 rows" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same config object as our arm's for the same flags
    assert d["config"] == bench.arm_config(args, 1, 1)


def test_clock_samples_summary():
    """nvidia-smi rows (index, SM MHz, max MHz, power, active mask, then the
    four reasons): the median SM clock, the maximum, every reason seen
    active once, unparsable rows skipped."""
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1200.5, 0x0, Not Active, Active, Not Active, Not Active",
        "garbage",
    ]
    s = bench.Clocks.summarise("\n".join(rows))
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    s = bench.Clocks.summarise("0, 1500, 2070, 1000, 0x8, Active, Not Active, Not Active, Not Active")
    assert s["reasons"] == ["hw_slowdown"] and s["sm_mhz"] == 1500.0
    assert bench.Clocks.summarise("")["sm_mhz"] is None


def test_traffic_figure_is_dropped_once_its_kernel_source_changes(tmp_path, monkeypatch):
    """The committed DRAM-traffic figure is reported only while the hash of
    the kernel source it was taken on still matches."""
    import hashlib
    import json
    src = tmp_path / "k.cu"
    src.write_text("// kernel\n")
    (tmp_path / "profiles").mkdir()
    entry = {"source": "k.cu", "sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
             "dram_bytes_per_launch": 123.0}
    (tmp_path / "profiles" / "traffic.txt").write_text(json.dumps({"k": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("k") == 123.0
    assert bench.traffic_for("other") is None
    src.write_text("// kernel, changed\n")
    assert bench.traffic_for("k") is None
