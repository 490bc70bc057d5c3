// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/tmotif.h"
#include "tm_device.h"

namespace tmo {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);

#define TM_CUDA_TRY(expr)                                                            \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess) {                                                     \
            ::tmo::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));     \
            return _e == cudaErrorMemoryAllocation ? TM_ENOMEM : TM_ECUDA;           \
        }                                                                            \
    } while (0)

#define TM_TRY(expr)                \
    do {                            \
        int _rc = (expr);           \
        if (_rc != TM_OK) return _rc; \
    } while (0)

}  // namespace tmo

struct tm_graph {
    tmo::DevGraph d;
    std::vector<void *> allocs;
    int64_t n_pairs = 0;
    int64_t max_out = 0, max_in = 0;
    int64_t bytes = 0;
    int device = 0;
    mutable std::mutex heur_mutex;    // guards the cached analysis below
    mutable int32_t bipartite = -1;   // undirected view bipartite (1), not (0), unknown (-1)
};

namespace tmo {

// The MG-Tree on the host: nodes in preorder, root first.
struct HostNode {
    std::vector<std::pair<int8_t, int8_t>> C;  // C_N, canonical labels
    std::vector<int32_t> children;             // preorder indices, lexicographic by next edge
    std::vector<int32_t> refs;                 // caller motif positions with canonical form == C_N
    int32_t parent = -1;
};

struct HostTree {
    std::vector<HostNode> nodes;
    std::vector<int64_t> motif_delta;          // window of each caller motif
    std::vector<int32_t> motif_query;          // query of each caller motif (empty: all 0)
    int32_t n_motifs = 0;
    int32_t n_leaves = 0;
    int32_t depth = 0;
    int32_t max_vertices = 0;
    int32_t n_deltas = 0;
    double similarity = 0;
};

}  // namespace tmo

namespace tmo {
// The device node table of a tree as one host byte image: nodes, then refs
// at o_refs, then the window table at o_deltas (offsets 256-byte aligned).
struct TreeImage {
    std::vector<char> bytes;
    size_t o_refs = 0, o_deltas = 0, o_qdmax = 0;
    int32_t n_nodes = 0, n_refs = 0, n_deltas = 0, n_counters = 0;
};
DevTree image_tree(const TreeImage &img, const void *dev);
void tree_image(const HostTree &h, bool par_leaves, TreeImage *img);

// A tree uploaded to the device once, on first use, per leaf mode.
struct DevTreeCache {
    bool ready = false;
    DevTree d{};
    void *mem = nullptr;
};
}  // namespace tmo

namespace tmo { struct SpecKernel; }

struct tm_tree {
    tmo::HostTree h;                      // the MG-Tree
    std::vector<tmo::HostTree> chains;    // one single-node tree per distinct motif (TM_PERMOTIF)
    // device copies: [leaf mode][0 = MG-Tree, 1 + i = chain i]
    std::vector<tmo::DevTreeCache> dev[2];
    void *mutex = nullptr;               // std::mutex guarding the lazy upload
    tmo::TreeImage image;                // MG-Tree node table (window-arithmetic leaves), built once
    // kernels specialised to this tree (tm_tree_compile), or null: owned by the process cache
    const tmo::SpecKernel *spec_tree = nullptr;
    std::vector<const tmo::SpecKernel *> spec_chains;
};

namespace tmo {

// graph build (tm_graph.cu)
int graph_build(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t E, int32_t V,
                uint32_t flags, cudaStream_t s, tm_graph **out);
void graph_release(tm_graph *g);

// tree build (tm_tree.cpp)
int tree_build(const int8_t *uv, const int32_t *off, int32_t n, const int64_t *delta, tm_tree **out);
// the same, with the query (0..63) of every motif for masked counting
int tree_build_q(const int8_t *uv, const int32_t *off, int32_t n, const int64_t *delta, const int32_t *query,
                 tm_tree **out);
void tree_release(tm_tree *tr);
// device copy of tree `which` (0 = MG-Tree, 1 + i = chain i), uploaded on first use
int tree_device(const tm_tree *tr, int which, bool par_leaves, cudaStream_t s, DevTree *out);

// tm_heur.cu: bipartiteness of the undirected view (cached in the handle) and
// the co-mining decision built on it
int graph_bipartite(const tm_graph *g, cudaStream_t s, int32_t *out);
int comine_advice(const tm_graph *g, const tm_tree *tr, cudaStream_t s, int32_t *out);

// tm_enum.cu: every match written to a bounded device buffer
int enumerate(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, tm_match *out, int64_t cap,
              int64_t *n_found, int64_t *counts, cudaStream_t s);

// mining (tm_mine.cu)
int mine(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, int64_t *counts,
         tm_run_stats *stats, cudaStream_t s);
// a serving batch: MG-Tree already on the device (dt), roots with query masks;
// no allocation, no synchronisation
size_t batch_scratch_bytes(const tm_graph *g, const tm_tree *tr, uint32_t mode);
int batch_enqueue(const tm_graph *g, const tm_tree *tr, uint32_t mode, const DevTree &dt, const int32_t *d_roots,
                  const uint64_t *d_qmask, int64_t n_roots, char *scratch, int64_t *d_counts, int32_t *d_status,
                  cudaStream_t s);

}  // namespace tmo
