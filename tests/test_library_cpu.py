"""Host-side checks of the CUDA library: it loads, exports every symbol the
header declares, rejects bad input, and builds MG-Trees (host code) that
agree with the oracle's Algorithm 2 construction.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2507_14813_b300 import build, synth, tmotif
from oracle import mgtree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tmotif.lib()


def test_exports_every_declared_symbol(lib):
    decl = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            decl |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tm_[a-z_0-9]+)\s*\(", txt, re.M))
    assert decl, "no declarations found"
    for name in decl:
        assert hasattr(lib, name), name
    assert set(tmotif.EXPORTS) == decl
    assert "sm_103a" in tmotif.tm_version()


def _shape(tree: tmotif.Tree):
    nodes = tree.nodes()
    kids = {i: [] for i in range(len(nodes))}
    for i, n in enumerate(nodes):
        if n["parent"] >= 0:
            kids[n["parent"]].append(i)

    def rec(i):
        return (nodes[i]["C"], nodes[i]["n_refs"] > 0, [rec(c) for c in kids[i]])
    return rec(0)


def test_tree_matches_oracle_tiny_and_mid(lib):
    for motifs in (synth.CONFIG1_MOTIFS, synth.CONFIG2_MOTIFS):
        t = tmotif.Tree(motifs, 100)
        o = mgtree.construct_mg_tree(motifs)
        assert _shape(t) == o.shape()
        assert abs(t.info()["similarity"] - o.similarity()) < 1e-12


@pytest.mark.parametrize("seed", range(25))
def test_tree_matches_oracle_random(lib, seed):
    motifs = synth.random_motif_tree(700 + seed, max_edges=6, max_motifs=24)
    motifs = motifs + [tuple((u + 2, v + 2) for u, v in motifs[-1])]   # a relabelled duplicate
    t = tmotif.Tree(motifs, 50)
    o = mgtree.construct_mg_tree(motifs)
    assert _shape(t) == o.shape()
    info = t.info()
    assert info["n_motifs"] == len(motifs)
    assert abs(info["similarity"] - o.similarity()) < 1e-12


def test_tree_walkthrough(lib):
    M3 = ((0, 1), (1, 2), (2, 0))
    M4 = ((0, 1), (1, 2), (2, 3), (3, 0))
    M5 = ((0, 1), (1, 2), (2, 3), (3, 1))
    t = tmotif.Tree([M3, M4, M5], 30)
    assert abs(t.info()["similarity"] - 5 / 11) < 1e-12
    assert t.info()["n_nodes"] == 5 and t.info()["n_leaves"] == 3


def test_tree_rejects_bad_motifs(lib):
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Tree([((0, 0),)], 10)
    assert e.value.code == tmotif.TM_EINVAL
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Tree([((0, 1), (1, 2))], -1)
    assert e.value.code == tmotif.TM_EINVAL
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Tree([tuple((i, i + 1) for i in range(9))], 10)
    assert e.value.code == tmotif.TM_EUNSUPPORTED
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Tree([((0, 1), (2, 3), (4, 5), (6, 7), (8, 9))], 10)   # 10 vertices
    assert e.value.code == tmotif.TM_EUNSUPPORTED
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Tree([((0, 1), (1, 2))] * 65, list(range(65)))         # 65 windows
    assert e.value.code == tmotif.TM_EUNSUPPORTED
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Tree([()], 10)
    assert e.value.code == tmotif.TM_EINVAL


def test_graph_load_rejects_bad_sizes(lib):
    # argument checks happen before any device call
    z = np.zeros(1, np.int32)
    with pytest.raises(tmotif.TMError) as e:
        tmotif.tm_graph_load(z, z, np.zeros(1, np.int64), 0)
    assert e.value.code == tmotif.TM_EINVAL


def test_header_cites_the_paper():
    txt = open(os.path.join(ROOT, "include", "tmotif.h")).read()
    for s in ("Section 2", "Algorithm 2", "Algorithm 3", "Algorithm 1", "Section 4.2"):
        assert s in txt


def test_new_entry_points_check_arguments_on_the_host(lib):
    """Argument checks that run before any device work: a NULL handle or output."""
    import ctypes
    tr = tmotif.Tree([((0, 1), (1, 2))], 10)
    args = tmotif.tm_count_args()
    n = ctypes.c_int64(0)
    out = ctypes.c_int32(0)
    assert lib.tm_enumerate(None, tr.h, ctypes.byref(args), None, 0, ctypes.byref(n), None, None) == tmotif.TM_EINVAL
    assert lib.tm_enumerate(None, tr.h, None, None, 0, ctypes.byref(n), None, None) == tmotif.TM_EINVAL
    assert lib.tm_graph_bipartite(None, ctypes.byref(out), None) == tmotif.TM_EINVAL
    assert lib.tm_comine_advice(None, tr.h, ctypes.byref(out), None) == tmotif.TM_EINVAL
    assert "NULL" in lib.tm_last_error().decode()
    tr.close()


def test_auto_mode_and_threshold_are_declared():
    txt = open(os.path.join(ROOT, "include", "tmotif.h")).read()
    assert "#define TM_AUTO 0x2u" in txt and tmotif.TM_AUTO == 0x2
    assert "#define TM_COMINE_MIN_SM 0.44" in txt and tmotif.TM_COMINE_MIN_SM == 0.44
    # one match record: motif, n_edges, TM_MAX_EDGES edge ids, all int32
    assert tmotif.MATCH_FIELDS == 2 + tmotif.TM_MAX_EDGES


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the size and field offsets the C
    header gives it (compiled with the host compiler)."""
    import subprocess
    structs = [tmotif.tm_graph_info, tmotif.tm_tree_info, tmotif.tm_tree_node, tmotif.tm_count_args,
               tmotif.tm_server_config, tmotif.tm_request_stats, tmotif.tm_server_info, tmotif.tm_tune,
               tmotif.tm_run_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tmotif.h"', "int main(void) {"]
    for st in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (st.__name__, st.__name__))
        for name, _ in st._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st.__name__, name, st.__name__, name))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for st in structs:
        assert int(got[st.__name__]) == ctypes.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert int(got["%s.%s" % (st.__name__, name)]) == getattr(st, name).offset, (st.__name__, name)
