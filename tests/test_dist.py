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
