"""Pins for the per-root closed forms (tests/refimpl.py) on tiny graphs.

The closed forms restate the definition of Section 2 for particular motif
shapes with range counts over time-sorted lists (no search tree).  They are
pinned here against brute force over all edge tuples and against the
oracle's per-root counts on tie-heavy graphs with self-loops and parallel
edges, so that the GPU tests may use them at sizes no enumeration reaches.
"""
import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import synth
from tests import refimpl

CLOSED = [
    ((0, 1), (1, 2)), ((0, 1), (1, 0)), ((0, 1), (0, 2)), ((0, 1), (2, 1)),
    ((0, 1), (0, 1)), ((0, 1), (0, 1), (0, 1)),
    ((0, 1), (0, 2), (0, 3)), ((0, 1), (0, 2), (0, 3), (0, 4)),
    ((0, 1), (2, 1), (3, 1)), ((0, 1), (2, 1), (3, 1), (4, 1)),
    ((0, 1), (1, 2), (2, 0)), ((0, 1), (1, 2), (2, 3)), ((0, 1), (0, 2), (1, 2)),
    ((0, 1), (2, 1), (1, 3)), ((0, 1), (1, 0), (0, 1)), ((0, 1), (1, 0), (0, 2)),
    ((0, 1), (1, 0), (0, 1), (1, 0)),
]


@pytest.mark.parametrize("seed", range(6))
def test_closed_forms_equal_brute_force(seed):
    src, dst, t = synth.tiny_graph(4000 + seed, 5 + seed % 3, 18, 10 + seed, zipf_s=0.7,
                                   self_loops=seed % 2 == 0)
    roots = np.arange(len(src))
    for m in CLOSED:
        for delta in (0, 4, 50):
            got = refimpl.closed_form_per_root(src, dst, t, m, delta, roots).sum()
            assert got == refimpl.brute_force(src, dst, t, m, delta), (m, delta)


@pytest.mark.parametrize("seed", range(5))
def test_closed_forms_equal_oracle_per_root(seed):
    # larger tie-heavy graphs: hubs with long windows, many parallel edges
    src, dst, t = synth.tiny_graph(4100 + seed, 12 + 4 * seed, 1500, 3000, zipf_s=1.4,
                                   self_loops=seed != 1)
    idx = refimpl.ListIndex(src, dst)
    roots = synth.root_sample(seed, len(src), 300)
    for m in CLOSED:
        for delta in (0, 37, 400):
            got = refimpl.closed_form_per_root(src, dst, t, m, delta, roots, idx=idx)
            _, want = oracle.count_motif(src, dst, t, m, delta, roots=roots, per_root=True)
            assert np.array_equal(got, want), (m, delta)


def test_closed_forms_relabelled_motif_and_saturated_window():
    src, dst, t = synth.tiny_graph(4200, 9, 400, 50, zipf_s=1.0, self_loops=True)
    t = t + (2**62)
    roots = np.arange(len(src))
    # any labelling of a shape is canonicalised first
    a = refimpl.closed_form_per_root(src, dst, t, ((5, 3), (3, 7), (7, 5)), 2**63 - 1, roots)
    b = refimpl.closed_form_per_root(src, dst, t, ((0, 1), (1, 2), (2, 0)), 2**63 - 1, roots)
    assert np.array_equal(a, b)
    _, want = oracle.count_motif(src, dst, t, ((0, 1), (1, 2), (2, 0)), 2**63 - 1, roots=roots, per_root=True)
    assert np.array_equal(a, want)
    with pytest.raises(KeyError):
        refimpl.closed_form_per_root(src, dst, t, ((0, 1), (1, 2), (2, 3), (3, 0)), 5, roots)


def test_elementary_symmetric_polynomials():
    # e_k of multiplicities counts k-subsets of pairwise distinct far ends
    import itertools
    mult = [3, 1, 4, 1, 5]
    items = [i for i, m in enumerate(mult) for _ in range(m)]
    for k in range(1, 5):
        brute = sum(1 for c in itertools.combinations(range(len(items)), k)
                    if len({items[j] for j in c}) == k)
        assert refimpl._esym(np.array(mult), k) == brute
