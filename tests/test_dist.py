"""Host logic of the multi-process (replica) path, on CPU with gloo and two
ranks: the max-over-ranks time, the whole-job throughput, and the reference
arm doing its work on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(1.0 + rank * 2.5)           # rank 1 is the slowest
        value = bench.whole_job_mpix_s(1_000_000, world, ms)
        ref = bench.run_reference(type("A", (), {})(), rank, world) if rank != 0 else "skipped"
        out[rank] = (ms, value, ref)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_rank_timing_reduction_and_reference_rank_gating():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        ms, value, _ = res[r]
        assert ms == pytest.approx(3.5)
        assert value == pytest.approx(2 * 1_000_000 / 3.5e-3 / 1e6)
    assert res[1][2] is None          # non-zero ranks of the reference arm do no work


def test_single_process_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(4.25) == 4.25
    assert bench.whole_job_mpix_s(1_016_814, 1, 2.0) == pytest.approx(508.407)


def test_reference_arm_prints_the_contract_line():
    """The reference arm (the FP64 oracle on the host cores) on a reduced
    scene: one JSON line with the contract's keys, the oracle named as the
    CPU baseline, and no host<->device bytes."""
    import bench
    args = type("A", (), dict(steps=2, warmup=1, n=20_000, ref_fraction=1.0 / 64.0))()
    out = bench.run_reference(args, 0, 1)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["impl"] == "reference" and out["dtype"] == "f64" and out["steps"] == 2
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
    assert out["cpu_baseline"]["value"] == out["value"] and out["e2e"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    assert out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
