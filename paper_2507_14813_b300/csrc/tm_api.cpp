// C-ABI entry points (include/tmotif.h): argument checks, handle lifetime,
// error reporting.  The work itself is in tm_graph.cu, tm_tree.cpp,
// tm_mine.cu, tm_heur.cu and tm_enum.cu.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "tm_codegen.h"
#include "tm_internal.h"

namespace tmo {
namespace {
thread_local std::string g_last_error;
}
void set_error(const std::string &msg) { g_last_error = msg; }
}  // namespace tmo

using namespace tmo;

extern "C" {

const char *tm_last_error(void) { return g_last_error.c_str(); }

const char *tm_version(void) { return "tmotif 0.1 (sm_103a)"; }

int tm_graph_load(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t n_edges, int32_t n_nodes,
                  uint32_t flags, void *stream, tm_graph **out) {
    g_last_error.clear();
    if (!out) { set_error("tm_graph_load: out is NULL"); return TM_EINVAL; }
    *out = nullptr;
    if (n_edges < 0 || n_edges >= (int64_t)1 << 31) {
        set_error("tm_graph_load: n_edges must be in [0, 2^31)");
        return TM_EINVAL;
    }
    if (n_nodes < 1) { set_error("tm_graph_load: n_nodes must be >= 1"); return TM_EINVAL; }
    if (n_edges > 0 && (!src || !dst || !t)) { set_error("tm_graph_load: NULL edge array"); return TM_EINVAL; }
    if (flags & ~(TM_INPUT_DEVICE | TM_PRESORTED)) { set_error("tm_graph_load: unknown flag"); return TM_EINVAL; }
    return graph_build(src, dst, t, n_edges, n_nodes, flags, (cudaStream_t)stream, out);
}

int tm_graph_get_info(const tm_graph *g, tm_graph_info *info) {
    if (!g || !info) { set_error("tm_graph_get_info: NULL argument"); return TM_EINVAL; }
    memset(info, 0, sizeof(*info));
    info->n_edges = g->d.E;
    info->n_nodes = g->d.V;
    info->n_pairs = g->n_pairs;
    info->max_out_degree = g->max_out;
    info->max_in_degree = g->max_in;
    info->device_bytes = g->bytes;
    return TM_OK;
}

int tm_graph_edges(const tm_graph *g, int32_t *src, int32_t *dst, int64_t *t) {
    if (!g) { set_error("tm_graph_edges: NULL graph"); return TM_EINVAL; }
    int64_t E = g->d.E;
    if (E == 0) return TM_OK;
    if (src) TM_CUDA_TRY(cudaMemcpy(src, g->d.src, sizeof(int32_t) * E, cudaMemcpyDeviceToHost));
    if (dst) TM_CUDA_TRY(cudaMemcpy(dst, g->d.dst, sizeof(int32_t) * E, cudaMemcpyDeviceToHost));
    if (t) TM_CUDA_TRY(cudaMemcpy(t, g->d.t, sizeof(int64_t) * E, cudaMemcpyDeviceToHost));
    return TM_OK;
}

int tm_graph_free(tm_graph *g) {
    if (!g) return TM_OK;
    graph_release(g);
    delete g;
    return TM_OK;
}

int tm_tree_build(const int8_t *motif_uv, const int32_t *motif_off, int32_t n_motifs, const int64_t *delta,
                  tm_tree **out) {
    g_last_error.clear();
    if (!out) { set_error("tm_tree_build: out is NULL"); return TM_EINVAL; }
    *out = nullptr;
    return tree_build(motif_uv, motif_off, n_motifs, delta, out);
}

int tm_tree_get_info(const tm_tree *tr, tm_tree_info *info) {
    if (!tr || !info) { set_error("tm_tree_get_info: NULL argument"); return TM_EINVAL; }
    memset(info, 0, sizeof(*info));
    info->n_motifs = tr->h.n_motifs;
    info->n_nodes = (int32_t)tr->h.nodes.size();
    info->n_leaves = tr->h.n_leaves;
    info->depth = tr->h.depth;
    info->n_deltas = tr->h.n_deltas;
    info->max_vertices = tr->h.max_vertices;
    info->similarity = tr->h.similarity;
    info->specialized = (spec_kernel(tr, 0) ? 1 : 0);
    for (int i = 0; i < (int)tr->chains.size(); i++) info->specialized += spec_kernel(tr, 1 + i) ? 1 : 0;
    return TM_OK;
}

int tm_tree_get_node(const tm_tree *tr, int32_t index, tm_tree_node *node) {
    if (!tr || !node) { set_error("tm_tree_get_node: NULL argument"); return TM_EINVAL; }
    if (index < 0 || index >= (int32_t)tr->h.nodes.size()) { set_error("tm_tree_get_node: index out of range"); return TM_EINVAL; }
    const HostNode &n = tr->h.nodes[index];
    memset(node, 0, sizeof(*node));
    node->parent = n.parent;
    node->n_edges = (int32_t)n.C.size();
    node->n_children = (int32_t)n.children.size();
    node->n_refs = (int32_t)n.refs.size();
    for (size_t k = 0; k < n.C.size() && k < TM_MAX_EDGES; k++) {
        node->u[k] = n.C[k].first;
        node->v[k] = n.C[k].second;
    }
    return TM_OK;
}

int tm_tree_free(tm_tree *tr) {
    if (!tr) return TM_OK;
    tree_release(tr);
    delete tr;
    return TM_OK;
}

int tm_tree_compile(tm_tree *tr, uint32_t flags, tm_compile_info *info) {
    g_last_error.clear();
    if (!tr) { set_error("tm_tree_compile: NULL tree"); return TM_EINVAL; }
    if (flags & ~(TM_COMPILE_CHAINS | TM_COMPILE_CHECK)) { set_error("tm_tree_compile: unknown flag"); return TM_EINVAL; }
    return tree_compile(tr, flags, info);
}

int tm_count(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, int64_t *counts, tm_run_stats *stats,
             void *stream) {
    g_last_error.clear();
    if (!g || !tr || !args || !counts) { set_error("tm_count: NULL argument"); return TM_EINVAL; }
    if (args->mode & ~(TM_PERMOTIF | TM_AUTO | TM_LEAF_SCAN | TM_SCHED_DYNAMIC | TM_SCHED_PLANNED | TM_SCHED_SIBLINGS |
                       TM_SCHED_TIERS | TM_GENERIC)) {
        set_error("tm_count: unknown mode bit");
        return TM_EINVAL;
    }
    if ((args->mode & TM_AUTO) && (args->mode & TM_PERMOTIF)) {
        set_error("tm_count: TM_AUTO and TM_PERMOTIF together");
        return TM_EINVAL;
    }
    if (args->flags & ~(TM_ROOTS_DEVICE | TM_COUNTS_DEVICE)) { set_error("tm_count: unknown flag"); return TM_EINVAL; }
    if (args->roots && args->n_roots < 0) { set_error("tm_count: n_roots < 0"); return TM_EINVAL; }
    if (args->mode & TM_AUTO) {
        int32_t co = 1;
        TM_TRY(comine_advice(g, tr, (cudaStream_t)stream, &co));
        tm_count_args a = *args;
        a.mode = (a.mode & ~TM_AUTO) | (co ? TM_COMINE : TM_PERMOTIF);
        return mine(g, tr, &a, counts, stats, (cudaStream_t)stream);
    }
    return mine(g, tr, args, counts, stats, (cudaStream_t)stream);
}

int tm_enumerate(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, tm_match *out, int64_t cap,
                 int64_t *n_found, int64_t *counts, void *stream) {
    g_last_error.clear();
    if (!g || !tr || !args || !n_found) { set_error("tm_enumerate: NULL argument"); return TM_EINVAL; }
    if (cap < 0 || (cap > 0 && !out)) { set_error("tm_enumerate: out must hold cap >= 0 records"); return TM_EINVAL; }
    if (args->mode & (TM_PERMOTIF | TM_AUTO | TM_LEAF_SCAN)) {
        set_error("tm_enumerate: enumeration walks the MG-Tree (no TM_PERMOTIF, TM_AUTO, TM_LEAF_SCAN)");
        return TM_EINVAL;
    }
    if (args->mode & ~(TM_SCHED_DYNAMIC | TM_SCHED_PLANNED)) { set_error("tm_enumerate: unknown mode bit"); return TM_EINVAL; }
    if (args->flags & ~(TM_ROOTS_DEVICE | TM_COUNTS_DEVICE)) { set_error("tm_enumerate: unknown flag"); return TM_EINVAL; }
    if (args->roots && args->n_roots < 0) { set_error("tm_enumerate: n_roots < 0"); return TM_EINVAL; }
    *n_found = 0;
    return enumerate(g, tr, args, out, cap, n_found, counts, (cudaStream_t)stream);
}

int tm_graph_bipartite(const tm_graph *g, int32_t *out, void *stream) {
    g_last_error.clear();
    if (!g || !out) { set_error("tm_graph_bipartite: NULL argument"); return TM_EINVAL; }
    return graph_bipartite(g, (cudaStream_t)stream, out);
}

int tm_comine_advice(const tm_graph *g, const tm_tree *tr, int32_t *out, void *stream) {
    g_last_error.clear();
    if (!g || !tr || !out) { set_error("tm_comine_advice: NULL argument"); return TM_EINVAL; }
    return comine_advice(g, tr, (cudaStream_t)stream, out);
}

}  // extern "C"
