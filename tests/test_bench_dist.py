"""The multi-GPU contract of bench.py on CPU: two gloo ranks take the maximum of their timings
(the slowest replica sets the job time) and the whole-job throughput counts every replica's DoFs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r: step time 10 + r ms, apply time 2 - r/2 ms
        ms_total, apply_ms = bench.max_over_ranks([10.0 + rank, 2.0 - 0.5 * rank], ws, "cpu")
        out[rank] = (ms_total, apply_ms, bench.job_gdofs(ws, 1_000_000, apply_ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_with_two_gloo_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms_total, apply_ms, val = res[r]
        assert ms_total == 11.0 and apply_ms == 2.0
        assert val == pytest.approx(2 * 1_000_000 / 2e-3 / 1e9)


def test_single_rank_passes_values_through():
    assert bench.max_over_ranks([3.0, 4.5], 1) == [3.0, 4.5]
    assert bench.job_gdofs(1, 8_586_756, 0.66) == pytest.approx(13.01, rel=1e-3)
