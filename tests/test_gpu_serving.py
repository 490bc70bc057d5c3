"""Serving: continuous batching over a resident graph.  Every request's
counts must equal what tm_count gives for that request alone (integers,
tolerance 0), admission must respect the memory budget, and requests that
arrive while batches run must be admitted and overlap."""
import time

import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import build, synth, tmotif

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


@pytest.fixture(scope="module")
def tiny():
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    return src, dst, t, g


def _queries(n, E, seed0=700):
    qs = []
    for i in range(n):
        ms = synth.query_motifs(seed0 + i, hi_edges=4)
        rng = np.random.default_rng(seed0 + i)
        deltas = [int(d) for d in np.exp(rng.uniform(np.log(60), np.log(20000), len(ms)))]
        roots = synth.root_sample(seed0 + i, E, int(rng.integers(1, 400)))
        qs.append((ms, deltas, roots))
    return qs


@pytest.mark.parametrize("mode", [tmotif.TM_SCHED_DYNAMIC, 0])
def test_each_result_equals_alone(tiny, mode):
    src, dst, t, g = tiny
    qs = _queries(40, len(src))
    srv = tmotif.Server(g, streams=3, max_batch=16, mode=mode)
    tickets = [srv.submit(ms, d, r) for ms, d, r in qs]
    results = [srv.poll(tk, wait=True) for tk in tickets]
    info = srv.info()
    srv.close()
    assert info["requests_done"] == len(qs)
    assert info["batches"] < len(qs)            # requests were merged
    assert max(st["batch_size"] for _, st in results) > 1
    for (ms, d, r), (counts, st) in zip(qs, results):
        alone = tmotif.count(g, tmotif.Tree(ms, d), roots=r)
        assert counts.tolist() == alone.tolist()
        assert st["latency_ms"] >= st["queue_ms"] >= 0


@pytest.mark.parametrize("mode", [tmotif.TM_SCHED_DYNAMIC, tmotif.TM_LEAF_SCAN])
def test_served_counts_equal_oracle(tiny, mode):
    """Each served request's counts against the oracle (Algorithm 1 per motif
    with the request's own window and roots, Section 2), while the requests
    share merged trees and launches."""
    src, dst, t, g = tiny
    qs = _queries(24, len(src), seed0=1500)
    srv = tmotif.Server(g, streams=3, max_batch=8, mode=mode)
    tickets = [srv.submit(ms, d, r) for ms, d, r in qs]
    results = [srv.poll(tk, wait=True) for tk in tickets]
    srv.close()
    assert max(st["batch_size"] for _, st in results) > 1
    for (ms, d, r), (counts, _) in zip(qs, results):
        want = [oracle.count_motif(src, dst, t, m, dm, roots=r, n_nodes=synth.TINY.n_nodes) for m, dm in zip(ms, d)]
        assert counts.tolist() == want


def test_arrivals_overlap_running_batches(tiny):
    src, dst, t, g = tiny
    qs = _queries(60, len(src), seed0=900)
    srv = tmotif.Server(g, streams=2, max_batch=8)
    tickets = []
    for i, (ms, d, r) in enumerate(qs):      # staggered arrivals
        tickets.append(srv.submit(ms, d, r))
        if i % 10 == 9:
            time.sleep(0.002)
    res = [srv.poll(tk, wait=True) for tk in tickets]
    srv.close()
    for (ms, d, r), (counts, _) in zip(qs, res):
        assert counts.tolist() == tmotif.count(g, tmotif.Tree(ms, d), roots=r).tolist()


def test_budget_is_respected_and_oversize_rejected(tiny):
    src, dst, t, g = tiny
    # room for one batch's scratch plus a few small requests at a time
    probe = tmotif.Server(g, streams=4, max_batch=64)
    probe.close()
    budget = 80 << 20
    srv = tmotif.Server(g, streams=4, max_batch=64, mem_budget=budget)
    qs = _queries(30, len(src), seed0=1200)
    tickets = [srv.submit(ms, d, r) for ms, d, r in qs]
    res = [srv.poll(tk, wait=True) for tk in tickets]
    info = srv.info()
    assert info["peak_admitted_bytes"] <= budget
    for (ms, d, r), (counts, _) in zip(qs, res):
        assert counts.tolist() == tmotif.count(g, tmotif.Tree(ms, d), roots=r).tolist()
    # a request whose roots alone need more than the budget
    big = np.arange(len(src), dtype=np.int32)
    big = np.concatenate([big] * 200)
    tk = srv.submit([((0, 1), (1, 2))], 100, big)
    with pytest.raises(tmotif.TMError) as e:
        srv.poll(tk, wait=True)
    assert e.value.code == tmotif.TM_ENOMEM
    srv.close()


def test_mid_graph_requests(request):
    src, dst, t = synth.make_graph(synth.MID)
    g = tmotif.Graph(src, dst, t, synth.MID.n_nodes, presorted=True)
    srv = tmotif.Server(g, streams=2, max_batch=16)
    qs = []
    for i in range(12):
        ms = synth.query_motifs(3000 + i, hi_edges=3)
        qs.append((ms, [600 + 300 * (j % 4) for j in range(len(ms))], synth.root_sample(3000 + i, len(src), 8)))
    tickets = [srv.submit(*q) for q in qs]
    res = [srv.poll(tk, wait=True) for tk in tickets]
    srv.close()
    for (ms, d, r), (counts, _) in zip(qs, res):
        assert counts.tolist() == tmotif.count(g, tmotif.Tree(ms, d), roots=r, mode=tmotif.TM_SCHED_DYNAMIC).tolist()
