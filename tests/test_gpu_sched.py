"""Learned scheduling on the GPU: features, the FP16/FP32 cost model and its
hand-written forward/backward kernels against the float64 reference, and the
plan it drives (counts unchanged, time against static scheduling)."""
import time

import numpy as np
import pytest

from oracle import mlp
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
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    return src, dst, t, g, tr


def _features_ref(src, dst, t, roots, delta, V, depth, fanout):
    E = len(src)
    eid = np.arange(E)
    hi = np.searchsorted(t, t[roots] + delta, side="right") - 1
    outdeg = np.bincount(src, minlength=V)
    indeg = np.bincount(dst, minlength=V)
    o = np.lexsort((eid, src))
    i = np.lexsort((eid, dst))

    def win(keys_sorted, eids_sorted, key, lo, h):
        a = np.searchsorted(keys_sorted, key, side="left")
        b = np.searchsorted(keys_sorted, key, side="right")
        out = np.zeros(len(key))
        for j in range(len(key)):
            seg = eids_sorted[a[j]:b[j]]
            out[j] = np.searchsorted(seg, h[j], side="right") - np.searchsorted(seg, lo[j], side="right")
        return out
    a, b = src[roots], dst[roots]
    F = np.stack([outdeg[b], indeg[b], outdeg[a],
                  win(src[o], o, b, roots, hi), win(dst[i], i, b, roots, hi), win(src[o], o, a, roots, hi),
                  np.full(len(roots), depth), np.full(len(roots), fanout)], axis=1).astype(np.float64)
    return np.log1p(F)


def test_features_match_reference(tiny):
    import torch
    src, dst, t, g, tr = tiny
    roots = synth.root_sample(31, len(src), 3000)
    d_roots = torch.from_numpy(roots).cuda()
    feats = torch.zeros((len(roots), tmotif.TM_FEATURES), dtype=torch.float32, device="cuda")
    tmotif.tm_features(g.h, tr.h, d_roots, feats)
    want = _features_ref(src, dst, t, roots, synth.TINY_DELTA, synth.TINY.n_nodes, 3, 2)
    assert np.allclose(feats.cpu().numpy(), want, rtol=1e-5, atol=1e-5)


def _half_theta(model):
    w, norm = model.params()
    return w.astype(np.float16).astype(np.float64), norm.astype(np.float64)


def _std(X, norm):
    return (X - norm[:8]) * norm[8:]


def test_forward_and_gradient_match_float64_reference():
    import torch
    rng = np.random.default_rng(7)
    n = 300
    X = rng.normal(2, 1.5, (n, 8)).astype(np.float32)
    T = rng.normal(5, 2, n).astype(np.float32)
    m = tmotif.Model(seed=11)
    dX = torch.from_numpy(X).cuda()
    dT = torch.from_numpy(T).cuda()
    m.fit_norm(dX)
    torch.cuda.synchronize()
    theta, norm = _half_theta(m)
    # the standardisation itself
    assert np.allclose(norm[:8], X.mean(0), rtol=1e-4, atol=1e-4)
    assert np.allclose(norm[8:], 1 / X.std(0), rtol=1e-3)
    Xs = _std(X.astype(np.float64), norm)
    y_ref, _ = mlp.forward(theta, Xs)
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    m.predict(dX, y)
    torch.cuda.synchronize()
    assert np.allclose(y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-4)
    loss, g = m.loss_grad(dX, dT)
    loss_ref, g_ref = mlp.loss_grad(theta, Xs, T.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-4 * abs(loss_ref) + 1e-5
    scale = np.abs(g_ref).max()
    assert np.max(np.abs(g - g_ref)) <= 2e-4 * scale


def test_gradient_over_many_tiles_and_reproducible_training():
    """More 64-sample tiles than gradient blocks (each block takes several,
    the last one ragged) against the float64 reference; and the sums have no
    floating-point atomics, so two trainings from one seed on the same data
    end with the same parameters and losses, bit for bit."""
    import torch
    rng = np.random.default_rng(9)
    n = 64 * 64 * 2 + 37                 # 129 tiles over 64 blocks
    X = rng.normal(1, 2, (n, 8)).astype(np.float32)
    T = (X[:, 0] * X[:, 1] + rng.normal(3, 1, n)).astype(np.float32)
    dX, dT = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m = tmotif.Model(seed=5)
    m.fit_norm(dX)
    torch.cuda.synchronize()
    theta, norm = _half_theta(m)
    assert np.allclose(norm[:8], X.mean(0), rtol=1e-4, atol=1e-4)
    assert np.allclose(norm[8:], 1 / X.std(0), rtol=1e-3)
    loss, g = m.loss_grad(dX, dT)
    loss_ref, g_ref = mlp.loss_grad(theta, _std(X.astype(np.float64), norm), T.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-4 * abs(loss_ref) + 1e-5
    assert np.max(np.abs(g - g_ref)) <= 2e-4 * np.abs(g_ref).max()
    runs = []
    for _ in range(2):
        mm = tmotif.Model(seed=5)
        mm.fit_norm(dX)
        hist = mm.train(dX, dT, epochs=6, batch=5000, lr=3e-3)
        w, nrm = mm.params()
        runs.append((w, nrm, np.asarray(hist), mm.loss_grad(dX, dT)[0]))
        mm.close()
    (w0, n0, h0, l0), (w1, n1, h1, l1) = runs
    assert np.array_equal(w0, w1) and np.array_equal(n0, n1) and np.array_equal(h0, h1) and l0 == l1
    assert h0[-1] < h0[0]


def test_training_reduces_error():
    import torch
    rng = np.random.default_rng(8)
    n = 4096
    X = rng.normal(0, 1, (n, 8)).astype(np.float32)
    T = (np.sin(X[:, 0]) * 2 + X[:, 1] * X[:, 2] + 0.5 * X[:, 3] ** 2).astype(np.float32)
    dX, dT = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m = tmotif.Model(seed=3)
    m.fit_norm(dX)
    l0, _ = m.loss_grad(dX, dT)
    hist = m.train(dX, dT, epochs=60, batch=256, lr=3e-3)
    l1, _ = m.loss_grad(dX, dT)
    assert l1 < 0.1 * l0 and l1 < 0.2 * float(np.var(T))
    assert hist[-1] < hist[0]


def test_plan_is_sorted_permutation(tiny):
    import torch
    src, dst, t, g, tr = tiny
    roots = torch.from_numpy(synth.root_sample(32, len(src), 5000)).cuda()
    feats = torch.zeros((len(roots), 8), dtype=torch.float32, device="cuda")
    tmotif.tm_features(g.h, tr.h, roots, feats)
    m = tmotif.Model(seed=5)
    m.fit_norm(feats)
    pred = torch.zeros(len(roots), dtype=torch.float32, device="cuda")
    m.predict(feats, pred)
    ro = torch.zeros_like(roots)
    sp = torch.zeros_like(roots)
    m.plan(feats, roots, ro, sp, unit_work=2.0, max_split=16)
    torch.cuda.synchronize()
    assert sorted(ro.cpu().tolist()) == sorted(roots.cpu().tolist())
    p = dict(zip(roots.cpu().tolist(), pred.cpu().tolist()))
    ordered = [p[r] for r in ro.cpu().tolist()]
    assert all(ordered[i] >= ordered[i + 1] for i in range(len(ordered) - 1))
    s = sp.cpu().numpy()
    assert s.min() >= 1 and s.max() <= 16


def _labels(work):
    return np.log1p(work[:, 0] + work[:, 2]).astype(np.float32)


@pytest.mark.parametrize("mode", [0, tmotif.TM_LEAF_SCAN])
def test_planned_counts_equal_static(tiny, mode):
    import torch
    src, dst, t, g, tr = tiny
    roots = torch.from_numpy(synth.root_sample(33, len(src), 8000)).cuda()
    want = tmotif.tm_count(g.h, tr.h, roots=roots, mode=mode)
    split = torch.full((len(roots),), 7, dtype=torch.int32, device="cuda")
    got, st = tmotif.tm_count(g.h, tr.h, roots=roots, mode=mode | tmotif.TM_SCHED_PLANNED, root_split=split,
                              stats=True)
    assert got.tolist() == want.tolist()
    assert st["tasks_split"] > 0
    both = tmotif.tm_count(g.h, tr.h, roots=roots, root_split=split,
                           mode=mode | tmotif.TM_SCHED_PLANNED | tmotif.TM_SCHED_DYNAMIC)
    assert both.tolist() == want.tolist()


@pytest.fixture(scope="module")
def mid():
    src, dst, t = synth.make_graph(synth.MID)
    g = tmotif.Graph(src, dst, t, synth.MID.n_nodes, presorted=True)
    return src, dst, t, g


def test_learned_plan_beats_static_on_mid_graph(mid):
    """The mid graph with its 3-edge motifs: train the cost model on measured
    per-root work of 2048 roots, then schedule 256 held-out roots by it.
    Counts stay exact; the planned launch is faster than static scheduling
    (one warp per root, sample order), which waits on its heaviest roots."""
    import torch
    src, dst, t, g = mid
    ms = [m for m in synth.CONFIG2_MOTIFS if len(m) == 3]
    tr = tmotif.Tree(ms, synth.MID_DELTA)
    allr = synth.root_sample(41, len(src), 2048 + 256)
    train_r = torch.from_numpy(allr[:2048]).cuda()
    test_r = torch.from_numpy(allr[2048:]).cuda()
    work = torch.zeros((2048, tmotif.TM_WORK_FIELDS), dtype=torch.int64, device="cuda")
    tmotif.tm_count(g.h, tr.h, roots=train_r, per_root_work=work, mode=tmotif.TM_SCHED_DYNAMIC, stats=True)
    y = torch.from_numpy(_labels(work.cpu().numpy())).cuda()
    X = torch.zeros((2048, 8), dtype=torch.float32, device="cuda")
    tmotif.tm_features(g.h, tr.h, train_r, X)
    model = tmotif.Model(seed=1)
    model.fit_norm(X)
    model.train(X, y, epochs=80, batch=256, lr=3e-3)
    # error of the prediction against measured work on held-out roots
    wt = torch.zeros((256, tmotif.TM_WORK_FIELDS), dtype=torch.int64, device="cuda")
    static = tmotif.tm_count(g.h, tr.h, roots=test_r, per_root_work=wt, mode=tmotif.TM_SCHED_DYNAMIC, stats=True)[0]
    Xt = torch.zeros((256, 8), dtype=torch.float32, device="cuda")
    tmotif.tm_features(g.h, tr.h, test_r, Xt)
    pred = torch.zeros(256, dtype=torch.float32, device="cuda")
    model.predict(Xt, pred)
    yt = _labels(wt.cpu().numpy())
    p = pred.cpu().numpy()
    resid = np.mean((p - yt) ** 2)
    assert resid < 0.5 * np.var(yt), (resid, np.var(yt))
    # plan and time
    ro = torch.zeros_like(test_r)
    sp = torch.zeros_like(test_r)
    model.plan(Xt, test_r, ro, sp, unit_work=2e5, max_split=256)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = fn()
        torch.cuda.synchronize()
        return c, time.perf_counter() - t0
    c_static, t_static = timed(lambda: tmotif.tm_count(g.h, tr.h, roots=test_r))
    c_plan, t_plan = timed(lambda: tmotif.tm_count(g.h, tr.h, roots=ro, root_split=sp,
                                                   mode=tmotif.TM_SCHED_PLANNED))
    assert c_plan.tolist() == c_static.tolist() == static.tolist()
    assert t_plan < t_static, (t_plan, t_static)
