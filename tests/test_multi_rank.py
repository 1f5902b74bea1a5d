"""The multi-rank host logic of bench.py on CPU with two gloo ranks:
max-over-ranks timing, the whole-job value, independent per-rank channels
(replicas), and the sharding rule for one long stream (contiguous ranges
with their absolute start index; the exact integer bins add up)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        fs, fc, fo = 64_000, 1000, 10
        L = oracle.plan(fs, fc, fo)["L"]
        # replicas: each rank its own channel (stream id = rank)
        own = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=1e-6, seed=9, stream=rank).bits2(0, 4 * 5000)
        mine = oracle.counts_2bit(own, 0, L)
        gathered = [torch.zeros_like(torch.from_numpy(mine)) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(mine))
        # max over ranks and the aggregate value
        t_ms = 10.0 * (rank + 1)
        mx = bench.reduce_max(t_ms, dist, "cpu")
        value = bench.aggregate_value(world, 1000, 5, mx)
        # one stream sharded into contiguous ranges, bins summed exactly
        n_total = 4 * 7777 + 4
        start, count = bench.shard_range(n_total, world, rank)
        s = synth.Stream(fs=fs, fc=fc, fo=fo, amp=0.05, td=1e-6, seed=3)
        part = torch.from_numpy(oracle.counts_2bit(s.bits2(start, count), start, L))
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        whole = oracle.counts_2bit(s.bits2(0, n_total), 0, L)
        out[rank] = {
            "max": mx, "value": value,
            "replicas_differ": not np.array_equal(gathered[0].numpy(), gathered[1].numpy()),
            "own_matches_gathered": np.array_equal(gathered[rank].numpy(), mine),
            "shard_sum_exact": np.array_equal(part.numpy(), whole),
            "range": (start, count),
        }
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        assert res[r]["max"] == 20.0
        assert res[r]["value"] == pytest.approx(world * 1000 * 5 / 0.020 / 1e9)
        assert res[r]["replicas_differ"] and res[r]["own_matches_gathered"]
        assert res[r]["shard_sum_exact"]
    (s0, c0), (s1, c1) = res[0]["range"], res[1]["range"]
    assert s0 == 0 and s1 == c0 and c0 + c1 == 4 * 7777 + 4 and c0 % 4 == 0


def test_shard_range_covers_stream():
    import bench

    for n in (0, 4, 4 * 1001 + 3, 512_000_000):
        for world in (1, 2, 3, 8):
            spans = [bench.shard_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (a, ca), (b, _) in zip(spans, spans[1:]):
                assert a + ca == b and a % 4 == 0
            assert sum(c for _, c in spans) == n
