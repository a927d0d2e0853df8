"""Batch sharding across ranks, tested with two gloo processes on CPU (no GPU).

Each rank takes its contiguous graph range, coarsens it (the CPU oracle stands in for the GPU
worker here, since this test covers only the host-side sharding and the final all-gather), and
the gathered per-graph super-node counts must equal a single-process run.
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2204_11757_gb300 import inputs as I
from paper_2204_11757_gb300 import shard as S


def test_shard_ranges_partition_and_balance():
    rng = np.random.default_rng(0)
    ec = rng.integers(100, 10000, size=997)
    for ws in (1, 2, 3, 8):
        rs = S.shard_ranges(ec, ws)
        assert rs[0][0] == 0 and rs[-1][1] == len(ec)
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        loads = [ec[a:b].sum() for a, b in rs]
        assert max(loads) - min(loads) <= 2 * ec.max()
    assert S.shard_ranges(np.array([5, 5]), 4)[-1] == (2, 2)


def _worker(rank, ws, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from oracle import oracle as O
    b, cfg = I.config_graph("s5_batch40_f32")
    sub, (g0, g1) = S.local_batch(b, rank, ws)
    res = O.coarsen_batch(sub, cfg["ratio"], cfg["mode"])
    counts = np.array([lv[0][-1].n_c for lv in res], dtype=np.int64)
    ranges = S.shard_ranges(S.batch_edge_counts(b), ws)
    off = S.global_offsets(counts, ranges, ws, all_gather=dist.all_gather)
    if rank == 0:
        np.save(out_path, off)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_batch_sharding(tmp_path):
    port = 29500 + (os.getpid() % 1000)
    out = str(tmp_path / "off.npy")
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    off = np.load(out)
    from oracle import oracle as O
    b, cfg = I.config_graph("s5_batch40_f32")
    res = O.coarsen_batch(b, cfg["ratio"], cfg["mode"])
    ref = np.concatenate([[0], np.cumsum([lv[0][-1].n_c for lv in res])])
    assert np.array_equal(off, ref)
