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
    tmotif.tm_count_noalloc(g.h, tr1.h, out1, roots=roots)
    torch.cuda.synchronize()
    tmotif.tm_count_noalloc(g.h, tr2.h, out2, root_lo=1000, root_hi=45000)
    torch.cuda.synchronize()
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
