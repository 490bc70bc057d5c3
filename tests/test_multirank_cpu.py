"""Multi-process path on the CPU (gloo, world size 2).

Root edges are independent units and counts are additive over roots, so
ranks shard the roots with no collective on the data path; the benchmark
only reduces its timing (MAX over ranks).  This test runs two gloo ranks:
each counts its share of the roots with the oracle, and the SUM of the
shares must equal the count over all roots; the MAX reduction of per-rank
times must be the largest of them.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2507_14813_b300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    src, dst, t = synth.make_graph(synth.TINY)
    roots = np.arange(len(src), dtype=np.int32)
    mine = roots[rank::world]
    part = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA, roots=mine)
    tot = torch.from_numpy(part.copy())
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms = torch.tensor([10.0 + 7.0 * rank])
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.save(out, np.concatenate([tot.numpy().astype(np.float64), ms.numpy().astype(np.float64)]))
    dist.destroy_process_group()


def test_two_rank_root_shards_sum_to_full_count(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_2507_14813_b300 import synth
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = np.load(out)
    src, dst, t = synth.make_graph(synth.TINY)
    full = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    assert res[:4].astype(np.int64).tolist() == full.tolist()
    assert res[4] == 17.0


def test_bench_rank_environment(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "4")
    assert bench.env_rank() == (3, 1, 4)
    # every rank mines its own seeded root sample
    a = bench.load_workload("tiny", 500, 0)[-1]
    b = bench.load_workload("tiny", 500, 1)[-1]
    assert len(a) == len(b) == 500 and not np.array_equal(a, b)
