// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/tmotif.h"

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

// ---------------------------------------------------------------- device graph
// One adjacency entry: the other endpoint and the edge id.  Lists are in
// ascending edge id, which is also ascending (t, input index).
struct DevGraph {
    int64_t E;
    int32_t V;
    const int32_t *src;       // by eid
    const int32_t *dst;
    const int64_t *t;
    const int64_t *out_off;   // V + 1
    const int2 *out_adj;      // (dst, eid) grouped by src
    const int64_t *in_off;    // V + 1
    const int2 *in_adj;       // (src, eid) grouped by dst
    const int32_t *pair_eid;  // eids ordered by (src, dst, eid)
    const int32_t *pr_pos;    // by eid: position of the edge in pair_eid
    const int32_t *pr_end;    // by eid: end of its (src, dst) run in pair_eid
    // by eid e: position in a list of the first entry after e (absolute index)
    const int32_t *after_os;  // in out(src e)
    const int32_t *after_od;  // in out(dst e)
    const int32_t *after_is;  // in in(src e)
    const int32_t *after_id;  // in in(dst e)
    const ulonglong2 *pair_tab; // open-addressing table: x = key (src<<32|dst), y = start | len<<32
    uint64_t pair_mask;       // table capacity - 1 (power of two)
};

static constexpr unsigned long long kEmptyKey = ~0ull;

__host__ __device__ inline uint64_t pair_hash(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

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

// ---------------------------------------------------------------- device tree
static constexpr int kMaxE = TM_MAX_EDGES;
static constexpr int kMaxV = TM_MAX_VERTICES;

// Node flags
static constexpr uint8_t kNodeParLeaf = 1;   // last level counted from the previous level's survivors
static constexpr uint8_t kNodeStarLeaf = 2;  // ... and that last edge extends the same list as the level
                                             //     before it (a star: same mapped centre, new other end)
static constexpr uint8_t kNodeStarKids = 4;  // some single-edge leaf child has kNodeStarLeaf

struct DevNode {
    uint64_t qmask;          // queries (bit q) with a ref in this node's subtree
    int8_t k_begin;          // first level owned by this node (= |C_parent|)
    int8_t k_end;            // |C_N|
    int8_t flags;
    int8_t dmax;             // index of the largest window among the subtree's refs
    int16_t child_begin;     // children are contiguous: [child_begin, child_begin + n_seq + n_par)
    int8_t n_seq;            // children descended one candidate at a time
    int8_t n_par;            // single-edge leaf children counted in parallel
    int16_t ref_begin;
    int16_t n_ref;
    int16_t parent;
    int16_t pad;
    uint8_t eu[kMaxE];       // C_N, canonical labels
    uint8_t ev[kMaxE];
    uint8_t nvb[kMaxE];      // motif vertices mapped before level k
};

struct DevRef {
    int32_t counter;         // index into the caller's motif list
    int16_t delta;           // index into the window table
    int16_t query;           // query the motif belongs to (0..63; 0 outside serving batches)
};

struct DevTree {
    const DevNode *nodes;
    const DevRef *refs;
    const int64_t *deltas;   // distinct windows, ascending
    const int8_t *qdmax;     // per query 0..63: largest window index of its refs (-1: none)
    int32_t n_nodes;
    int32_t n_refs;
    int32_t n_deltas;
    int32_t n_counters;
};

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

struct tm_tree {
    tmo::HostTree h;                      // the MG-Tree
    std::vector<tmo::HostTree> chains;    // one single-node tree per distinct motif (TM_PERMOTIF)
    // device copies: [leaf mode][0 = MG-Tree, 1 + i = chain i]
    std::vector<tmo::DevTreeCache> dev[2];
    void *mutex = nullptr;               // std::mutex guarding the lazy upload
    tmo::TreeImage image;                // MG-Tree node table (window-arithmetic leaves), built once
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
