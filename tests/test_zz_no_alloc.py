"""The allocation-free entry point against the regular one.

tm_count_noalloc serves callers that must not allocate device memory while
they count; its scratch is a static array inside the library that every
call reuses.  This file runs last (pytest collects it after the others), and
passes both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2507_14813_b300 import build, synth, tmotif

pytestmark = pytest.mark.gpu


def _pool_high_water():
    """Used-memory high-water mark of the device's default memory pool (the
    pool cudaMallocAsync draws from), reset to the current use first; None
    when the CUDA driver API bindings are missing."""
    try:
        from cuda.bindings import driver as cu
    except ImportError:
        return None
    import torch
    cu.cuInit(0)
    err, dev = cu.cuDeviceGet(torch.cuda.current_device())
    err, pool = cu.cuDeviceGetDefaultMemPool(dev)
    if err != cu.CUresult.CUDA_SUCCESS:
        return None
    attr = cu.CUmemPool_attribute.CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def read():
        e, v = cu.cuMemPoolGetAttribute(pool, attr)
        assert e == cu.CUresult.CUDA_SUCCESS
        return int(v)

    def reset():
        (e,) = cu.cuMemPoolSetAttribute(pool, attr, cu.cuuint64_t(0))
        assert e == cu.CUresult.CUDA_SUCCESS

    return read, reset


def test_noalloc_matches_tm_count_twice_in_a_row():
    import torch
    build.build()
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    tr1 = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    tr2 = tmotif.Tree([((0, 1), (1, 2), (2, 0)), ((0, 1), (0, 2), (0, 3)), ((0, 1), (1, 0))], [3000, 8000, 500])
    roots = torch.from_numpy(synth.root_sample(5, len(src), 20000)).cuda()
    # first call: tree 1 over a root list; second call: tree 2 over a range,
    # so stale counters from the first call would show up in the second
    want1 = tmotif.tm_count(g.h, tr1.h, roots=roots)
    want2 = tmotif.tm_count(g.h, tr2.h, root_lo=1000, root_hi=45000)
    out1 = torch.full((4,), -7, dtype=torch.int64, device="cuda")
    out2 = torch.full((3,), -7, dtype=torch.int64, device="cuda")
    # the set-up call (address of the static array) before the measured ones
    tmotif.tm_count_noalloc(g.h, tr1.h, out1, roots=roots)
    torch.cuda.synchronize()
    pool = _pool_high_water()
    if pool is not None:
        read, reset = pool
        reset()
        high0 = read()
    torch_before = torch.cuda.memory_allocated()
    tmotif.tm_count_noalloc(g.h, tr1.h, out1, roots=roots)
    torch.cuda.synchronize()
    tmotif.tm_count_noalloc(g.h, tr2.h, out2, root_lo=1000, root_hi=45000)
    torch.cuda.synchronize()
    # nothing was drawn from the stream-ordered pool, nothing through torch
    if pool is not None:
        assert read() == high0
    assert torch.cuda.memory_allocated() == torch_before
    assert out1.cpu().tolist() == want1.tolist()
    assert out2.cpu().tolist() == want2.tolist()
    # and the first again, after the second has used the scratch
    tmotif.tm_count_noalloc(g.h, tr1.h, out1, roots=roots)
    torch.cuda.synchronize()
    assert out1.cpu().tolist() == want1.tolist()


def test_noalloc_rejects_oversize_and_bad_range():
    import torch
    build.build()
    src, dst, t = synth.tiny_graph(77, 10, 200, 1000)
    g = tmotif.Graph(src, dst, t, 10)
    big = tmotif.Tree([((0, 1), (1, 2))] * 1025, 10)
    out = torch.zeros(1025, dtype=torch.int64, device="cuda")
    with pytest.raises(tmotif.TMError) as e:
        tmotif.tm_count_noalloc(g.h, big.h, out)
    assert e.value.code == tmotif.TM_EUNSUPPORTED
    small = tmotif.Tree([((0, 1), (1, 2))], 10)
    with pytest.raises(tmotif.TMError) as e:
        tmotif.tm_count_noalloc(g.h, small.h, out[:1], root_lo=0, root_hi=201)
    assert e.value.code == tmotif.TM_EINVAL


def test_noalloc_rejects_short_counts_before_any_launch():
    import torch
    build.build()
    src, dst, t = synth.tiny_graph(78, 10, 200, 1000)
    g = tmotif.Graph(src, dst, t, 10)
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, 10)
    out = torch.full((4,), -7, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        tmotif.tm_count_noalloc(g.h, tr.h, out[:3])
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [-7] * 4
