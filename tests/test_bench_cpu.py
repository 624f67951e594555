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
