"""The library under several ranks: each gloo rank counts its shard of the
root edges with the CUDA path on the one GPU (the ranks' kernels never wait
on each other: counts are additive over roots, so no device collective is
needed), and the SUM of the shards over the host collective must equal the
oracle's count over all roots, per motif, bit-exact.  Multi-GPU runs place
one rank per GPU the same way."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from paper_2507_14813_b300 import synth, tmotif
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    roots = np.arange(len(src), dtype=np.int32)[rank::world]          # this rank's shard
    part = tmotif.count(g, tr, roots=roots, mode=tmotif.TM_SCHED_DYNAMIC)
    tot = torch.from_numpy(part.copy())
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)                          # host collective
    if rank == 0:
        q.put(tot.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_roots_and_sum_counts():
    import torch.multiprocessing as mp

    import oracle
    from paper_2507_14813_b300 import build, synth
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    src, dst, t = synth.make_graph(synth.TINY)
    want = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    assert got == want.tolist()
