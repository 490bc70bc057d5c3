/*
 * tmotif: exact co-mining of delta-temporal motifs on a B300 (sm_103a).
 *
 * The library loads a temporal graph onto the GPU, builds a Motif-Group Tree
 * (MG-Tree) from a motif set, and returns one exact 64-bit count per motif.
 *
 * Problem statement (Section 2, "A Temporal Graph", "A delta-Temporal
 * Motif", "Temporal Motif Mining"): edges are ordered by (t, input index),
 * which fixes the edge id (eid).  A match of motif ((u_1,v_1),...,(u_m,v_m))
 * with window delta is a tuple of eids e_1 < ... < e_m with
 * t(e_m) - t(e_1) <= delta and one injective map f from motif vertices to
 * graph vertices with f(u_i) = src(e_i), f(v_i) = dst(e_i).  A motif's count
 * is its number of matches (no division by automorphisms).
 *
 * Conventions for every call:
 *   - return value 0 (TM_OK) on success, a negative TM_E* code otherwise;
 *     tm_last_error() then gives a message for the calling thread;
 *   - inputs are copied; the caller keeps ownership of every pointer passed;
 *   - handles (tm_graph, tm_tree) are immutable after creation and may be
 *     used from several streams at once; free them once, after all work that
 *     uses them has finished;
 *   - "stream" is a cudaStream_t (NULL = legacy default stream).
 */
#ifndef TMOTIF_H
#define TMOTIF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define TM_OK 0
#define TM_EINVAL (-1)        /* invalid argument or input data */
#define TM_ENOMEM (-2)        /* device or host allocation failed */
#define TM_ECUDA (-3)         /* a CUDA call failed */
#define TM_ETIMEOUT (-4)      /* a bounded device-side wait ran out */
#define TM_EUNSUPPORTED (-5)  /* motif beyond TM_MAX_EDGES / TM_MAX_VERTICES */
#define TM_ECHECK (-6)        /* the checking build (TM_CHECK) found an index outside its range:
                                 an internal error of the library; counts are incomplete */

/* ------------------------------------------------------------ limits */
#define TM_MAX_EDGES 8        /* edges per motif */
#define TM_MAX_VERTICES 8     /* vertices per motif */
#define TM_MAX_DELTAS 64      /* distinct windows in one tree */
#define TM_MAX_NODES 4096     /* nodes in one tree */

typedef struct tm_graph tm_graph;   /* opaque, library-owned */
typedef struct tm_tree tm_tree;     /* opaque, library-owned */

/* ------------------------------------------------------------ graph */
#define TM_INPUT_DEVICE 0x1u  /* src/dst/t point to device memory */
#define TM_PRESORTED 0x2u     /* input is already in (t, index) order; checked */

/*
 * Load a temporal graph (Section 2; the time-sorted adjacency of Section 4.1,
 * step 2 of the workflow).
 *   src, dst: n_edges int32 vertex ids in [0, n_nodes)
 *   t:        n_edges int64 timestamps (any order unless TM_PRESORTED)
 *   flags:    TM_INPUT_DEVICE, TM_PRESORTED
 * The library orders the edges by (t, input index), then builds on the device
 * the per-vertex out- and in-lists in edge-id order and a (src, dst) pair
 * index.  Self-loops are accepted (no motif can match them).  Errors:
 * TM_EINVAL for n_edges < 0 or >= 2^31, n_nodes < 1, an id out of range,
 * TM_PRESORTED input that is not sorted; TM_ENOMEM; TM_ECUDA.
 * The call synchronises `stream` before returning.
 */
int tm_graph_load(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t n_edges,
                  int32_t n_nodes, uint32_t flags, void *stream, tm_graph **out);

typedef struct {
    int64_t n_edges;
    int32_t n_nodes;
    int32_t reserved;
    int64_t n_pairs;          /* distinct (src, dst) pairs */
    int64_t max_out_degree;
    int64_t max_in_degree;
    int64_t device_bytes;     /* device memory held by the handle */
} tm_graph_info;

int tm_graph_get_info(const tm_graph *g, tm_graph_info *info);

/* Copy the edge list in edge-id order to host arrays (n_edges each; any may be NULL). */
int tm_graph_edges(const tm_graph *g, int32_t *src, int32_t *dst, int64_t *t);

int tm_graph_free(tm_graph *g);

/* ------------------------------------------------------------ MG-Tree */
/*
 * Build the Motif-Group Tree of a motif set (Section 4.2, Algorithm 2;
 * node composition <C_N, Children(N), Q_N> of Appendix A).
 *   motif_uv:  2 * sum(m_i) int8 vertex labels, edge j of motif i at
 *              motif_uv[2*(motif_off[i]+j)] (source), [.. + 1] (destination)
 *   motif_off: n_motifs + 1 offsets (in edges) into motif_uv
 *   delta:     n_motifs int64 windows (>= 0); motifs may carry different
 *              windows, each counted with its own
 * Labels are canonicalised (order of first appearance); motifs equal after
 * that share one node and keep separate counts.  The tree is the radix trie
 * of canonical edge sequences: one node per branch point or motif end, the
 * root at the longest common prefix.  Errors: TM_EINVAL for an empty motif,
 * a self-loop edge (u == v), a negative label or delta; TM_EUNSUPPORTED for
 * more than TM_MAX_EDGES edges or TM_MAX_VERTICES vertices in a motif, more
 * than TM_MAX_DELTAS distinct windows or TM_MAX_NODES nodes.
 */
int tm_tree_build(const int8_t *motif_uv, const int32_t *motif_off, int32_t n_motifs,
                  const int64_t *delta, tm_tree **out);

typedef struct {
    int32_t n_motifs;
    int32_t n_nodes;
    int32_t n_leaves;
    int32_t depth;            /* edges of the longest motif */
    int32_t n_deltas;         /* distinct windows */
    int32_t max_vertices;
    double similarity;        /* SM of Section 6: 1 - sum(|E_N|-|E_parent|) / sum |E_M| */
    int32_t specialized;      /* kernels compiled for this tree (tm_tree_compile): 0, 1 + chains */
    int32_t reserved;
} tm_tree_info;

int tm_tree_get_info(const tm_tree *tr, tm_tree_info *info);

/* One node of the tree in preorder (root = 0), for inspection. */
typedef struct {
    int32_t parent;           /* -1 for the root */
    int32_t n_edges;          /* |C_N| */
    int32_t n_children;
    int32_t n_refs;           /* motifs whose canonical form equals C_N */
    int8_t u[TM_MAX_EDGES];   /* C_N, canonical labels */
    int8_t v[TM_MAX_EDGES];
} tm_tree_node;

int tm_tree_get_node(const tm_tree *tr, int32_t index, tm_tree_node *node);

int tm_tree_free(tm_tree *tr);

/* ------------------------------------------------------------ code generation */
/*
 * Compile mining kernels specialised to this tree (Section 5.1, "GPU
 * Code-generation": the paper generates a kernel per motif group so that the
 * matching order, the mapped-vertex checks and the counters of each node are
 * fixed in the code).  The library compiles its own kernel source at run time
 * (NVRTC, sm_103a) behind a generated prelude: the node, ref and window
 * tables become constant data of the kernel, the tree's depth and vertex
 * count size every per-level array and mapped-label loop (and so the
 * registers and shared memory), and the window and counter counts are
 * compile-time constants.  Afterwards tm_count uses the specialised kernel
 * for this tree whenever mode has neither TM_LEAF_SCAN nor TM_GENERIC; the
 * counts are those of the table-driven kernel.
 *   flags: TM_COMPILE_CHAINS also compiles one kernel per distinct motif, used
 *          by TM_PERMOTIF
 *   info:  optional, filled on success
 * Kernels are cached for the life of the process by their generated program,
 * so trees of the same shape and windows compile once.  Compilation takes
 * seconds; call it before timing or capturing counts, not inside a stream
 * capture.  Not thread-safe against tm_count on the same tree.  Errors:
 * TM_EINVAL (NULL tree, unknown flag), TM_EUNSUPPORTED (more than
 * TM_SPEC_MAX_NODES nodes: such trees keep the table-driven kernel), TM_ECUDA
 * (the runtime compiler or loader failed; tm_last_error has its log).
 */
#define TM_COMPILE_CHAINS 0x1u
#define TM_COMPILE_CHECK 0x2u   /* compile only (no device needed): the tree keeps its kernels */
#define TM_SPEC_MAX_NODES 256

typedef struct {
    int32_t kernels;          /* programs the tree now has */
    int32_t compiled;         /* of them compiled by this call; the rest came from the cache */
    double wall_ms;           /* wall time of the call */
    int32_t registers;        /* per thread, MG-Tree kernel (counting launch) */
    int32_t local_bytes;      /* local memory per thread (register spills), same kernel */
    int32_t static_smem;      /* static shared memory per CTA, same kernel */
    int32_t reserved;
    uint64_t source_hash;     /* FNV-1a of that kernel's generated program */
} tm_compile_info;

int tm_tree_compile(tm_tree *tr, uint32_t flags, tm_compile_info *info);

/* ------------------------------------------------------------ counting */
/* mode bits */
#define TM_COMINE 0x0u        /* walk the MG-Tree (Algorithm 3) */
#define TM_PERMOTIF 0x1u      /* one chain per distinct motif, one launch each (Algorithm 1) */
#define TM_AUTO 0x2u          /* TM_COMINE or TM_PERMOTIF, as tm_comine_advice decides */
#define TM_LEAF_SCAN 0x10u    /* count a leaf's last edge by scanning its window only */
#define TM_SCHED_DYNAMIC 0x100u /* persistent launch, heavy subtrees split across warps */
#define TM_SCHED_PLANNED 0x200u /* persistent launch; cut root i's first-level lists into root_split[i] slices */
#define TM_GENERIC 0x1000u    /* the table-driven kernel even when the tree has a specialised one */
#define TM_SCHED_TIERS 0x800u /* with TM_SCHED_PLANNED: the roots at the tail of the order whose
                                 root_split is 0 (tm_plan_tiers marks those predicted light) run one
                                 per lane (thread tier); the others one per warp (warp tier), those
                                 with root_split > 1 cut into slices for many warps.  Ignored for
                                 trees of more than 8 windows */
#define TM_SCHED_SIBLINGS 0x400u /* TM_SCHED_DYNAMIC with the paper's sibling splitting (a warp about to
                                    descend into several children hands all but the first to idle
                                    warps as separate tasks) and multi-offload (a donation hands
                                    over up to one piece per idle warp, at most offload_max) */

/* flags */
#define TM_ROOTS_DEVICE 0x1u  /* roots points to device memory */
#define TM_COUNTS_DEVICE 0x2u /* counts points to device memory (no sync) */

/* per-root work counters, TM_WORK_FIELDS int64 per root */
#define TM_WORK_CANDIDATES 0  /* adjacency entries scanned in windows */
#define TM_WORK_EXPANSIONS 1  /* candidate lists opened */
#define TM_WORK_PROBES 2      /* binary-search and hash probes */
#define TM_WORK_LEAF_EVALS 3  /* leaf edges counted by range arithmetic */
#define TM_WORK_FIELDS 4

typedef struct {
    uint32_t mode;            /* TM_COMINE, TM_PERMOTIF or TM_AUTO, | TM_LEAF_SCAN, | TM_SCHED_* */
    uint32_t flags;           /* TM_ROOTS_DEVICE, TM_COUNTS_DEVICE */
    const int32_t *roots;     /* root edge ids (any order, may repeat); NULL: range below */
    int64_t n_roots;
    int64_t root_lo;          /* with roots == NULL: roots are eids [root_lo, root_hi) */
    int64_t root_hi;          /*   root_hi <= 0 means n_edges */
    int64_t *per_root_counts; /* device, [n_roots][n_motifs], or NULL; overwritten */
    int64_t *per_root_work;   /* device, [n_roots][TM_WORK_FIELDS], or NULL; overwritten */
    int32_t ctas_per_sm;      /* 0: library default */
    int32_t offload_max;      /* TM_SCHED_SIBLINGS: most pieces one donation hands over (0: default 8) */
    const int32_t *root_split; /* device, per root: slices for TM_SCHED_PLANNED (<= 1: none), or NULL */
    int32_t poll_every;       /* TM_SCHED_DYNAMIC: chunk loads between looks for idle warps (0: default 4) */
    int32_t donate_seq;       /* min unscanned entries to split a level that descends (0: default 64) */
    int32_t donate_leaf;      /* ... a level whose survivors are only counted (0: default 1024) */
    int32_t sibling_always;   /* TM_SCHED_SIBLINGS: split siblings even when no warp is idle (tests) */
} tm_count_args;

typedef struct {
    int64_t n_roots;
    int64_t candidates;       /* totals of the work counters above */
    int64_t expansions;
    int64_t probes;
    int64_t leaf_evals;
    int64_t algo_bytes;       /* bytes the method reads: 16 per root + 8 per candidate
                                 + 8 per list probe + 16 per hash probe + 4 per pair probe */
    int64_t tasks_split;      /* subtrees handed to other warps (TM_SCHED_DYNAMIC) */
    int64_t launches;         /* kernel launches issued by the call */
    double kernel_ms;         /* device time of the mining launches */
    double warp_imbalance;    /* max / mean over warps of busy cycles (time not spent waiting
                                 for work) in the stats launch: 1 is perfect balance */
    int64_t algo_bytes_lists; /* bytes by list accounting: 16 per root + 8 per candidate scanned
                                 + 12 * ceil(log2(len + 1)) per candidate list opened (an edge-id
                                 and a time probe per binary-search step) */
    int64_t idle_expired;     /* warps of the persistent launch whose bounded idle wait ran out
                                 while other warps still held work (they left the launch early;
                                 counts are unaffected) */
    int64_t roots_thread_tier; /* tier histogram: roots counted one per lane (TM_SCHED_TIERS) */
    int64_t roots_split;      /* ... roots whose first-level lists were cut into planned slices;
                                 the rest (n_roots - both) ran one per warp */
} tm_run_stats;

/*
 * Count every motif of `tr` in `g` (Algorithm 3 when mode has TM_COMINE,
 * Algorithm 1 per motif with TM_PERMOTIF); both give the same counts.
 *   counts: n_motifs int64, caller-owned, host memory (the call then
 *           synchronises `stream`) or device memory with TM_COUNTS_DEVICE;
 *           overwritten with the counts of the selected roots
 *   stats:  optional; when non-NULL the call collects work counters and
 *           synchronises `stream`
 * Roots: every edge is a candidate for the first motif edge (Algorithm 1,
 * first call); counts are additive over roots, so a root list or range
 * yields the counts of matches whose first edge is in it.  A host root list
 * is range-checked before launch; a device list (TM_ROOTS_DEVICE) is checked
 * by the kernel, which skips a root outside [0, n_edges) and reports
 * TM_EINVAL when the call synchronises (host counts, stats or a
 * TM_SCHED_* mode); with device counts and static scheduling such a root
 * only counts nothing.  per_root_counts, per_root_work and root_split must
 * hold n_roots rows (the library cannot check their lengths).  Errors:
 * TM_EINVAL (NULL handle, root out of range, n_roots < 0); TM_ETIMEOUT if a
 * bounded device wait of TM_SCHED_DYNAMIC ran out (counts are then invalid);
 * TM_ECUDA; TM_ENOMEM.
 */
int tm_count(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, int64_t *counts,
             tm_run_stats *stats, void *stream);

/* ------------------------------------------------------------ enumeration */
/* One match: the motif (index into the caller's motif list) and the ids of the
 * edges matched to its edges, in the motif's edge order (so ascending). */
typedef struct {
    int32_t motif;
    int32_t n_edges;          /* edges of that motif */
    int32_t eid[TM_MAX_EDGES]; /* -1 past n_edges */
} tm_match;

/*
 * Enumerate the matches that tm_count counts.  Algorithm 1 records each match
 * it completes; the paper's experiments only count (reading 13).  Every match
 * of every motif of `tr` whose first edge is a selected root (args->roots /
 * n_roots or root_lo / root_hi, as tm_count; args->mode must not hold
 * TM_PERMOTIF, TM_AUTO or TM_LEAF_SCAN, scheduling bits are ignored) is
 * written to `out`, in no particular order, until `cap` records are written.
 *   out:     device memory, cap records, caller-owned (may be NULL if cap == 0)
 *   n_found: host; the number of matches, which exceeds cap when records were
 *            dropped (then which cap matches were written is unspecified)
 *   counts:  optional host int64[n_motifs]: matches per motif (= tm_count)
 * Synchronises `stream`.  Errors: TM_EINVAL (NULL handle, out NULL with
 * cap > 0, cap < 0, bad mode, root out of range), TM_ENOMEM, TM_ECUDA.
 */
int tm_enumerate(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, tm_match *out, int64_t cap,
                 int64_t *n_found, int64_t *counts, void *stream);

/* ------------------------------------------------------------ co-mining decision */
/*
 * Whether the undirected view of the graph is bipartite.  Section 6 found
 * co-mining faster on bipartite data graphs in every experiment: matches
 * cannot join two vertices of one side, so shared prefixes are pruned early.
 * Computed on the device once per graph and cached in the handle (connected
 * components of the bipartite double cover by label hooking and pointer
 * jumping; bipartite iff no vertex is in the component of its own copy).
 * A graph with a self-loop is not bipartite; a graph without edges is.
 *   out: 1 bipartite, 0 not.  Synchronises `stream` on first use.
 * Errors: TM_EINVAL (NULL argument), TM_ENOMEM (2 x n_nodes int32 labels),
 * TM_EUNSUPPORTED (n_nodes >= 2^30), TM_ECUDA.
 */
int tm_graph_bipartite(const tm_graph *g, int32_t *out, void *stream);

/* Below this similarity metric (SM, tm_tree_info.similarity) per-motif
 * mining beat co-mining on the GPU in Section 6. */
#define TM_COMINE_MIN_SM 0.44

/*
 * The co-mining decision of Section 6 ("Heuristic for Co-Mining"): co-mine on
 * a bipartite graph; otherwise co-mine iff the tree's SM >= TM_COMINE_MIN_SM.
 * (The paper's remaining advice, to prefer a smaller window, is the caller's
 * choice of delta.)  tm_count with TM_AUTO applies it.
 *   out: 1 co-mine (TM_COMINE), 0 mine each motif alone (TM_PERMOTIF).
 * Errors: as tm_graph_bipartite.
 */
int tm_comine_advice(const tm_graph *g, const tm_tree *tr, int32_t *out, void *stream);

/* ------------------------------------------------------------ serving */
/*
 * A request loop over a resident graph with continuous batching.  The paper
 * answers one query per run (Section 4.1); serving is an addition of this
 * library.  A worker thread keeps up to `streams` batches on the device.
 * When a stream is free it admits the oldest pending requests (at most
 * `max_batch` <= 64, within `mem_budget` device bytes), merges their motifs
 * into one MG-Tree (each motif keeps its own window and its request), runs
 * one count over the union of their roots (each root counted only for the
 * requests that listed it) and scatters the counts back.  Requests that
 * arrive while batches run are admitted as streams and memory free up, so
 * their work overlaps on the device.  Each request gets exactly the counts
 * that tm_count gives for its motifs, windows and roots alone.
 */
typedef struct tm_server tm_server;

typedef struct {
    int32_t streams;          /* batches in flight (default 2, at most 16) */
    int32_t max_batch;        /* requests merged into one batch (default 32, at most 64) */
    int64_t mem_budget;       /* device bytes for admitted batches (default 4 GiB); a
                                 request that alone exceeds it fails with TM_ENOMEM */
    uint32_t mode;            /* count mode of every batch: 0, TM_SCHED_DYNAMIC (default
                                 when cfg is NULL), | TM_LEAF_SCAN */
    uint32_t reserved;
} tm_server_config;

typedef struct {
    double queue_ms;          /* submit -> batch launch */
    double latency_ms;        /* submit -> counts ready on the host */
    int32_t batch;            /* batch id */
    int32_t batch_size;       /* requests in that batch */
} tm_request_stats;

typedef struct {
    int64_t batches;
    int64_t requests_done;
    int64_t pending;
    int64_t in_flight;        /* batches on the device */
    int64_t admitted_bytes;   /* bytes counted against the budget now */
    int64_t peak_admitted_bytes;
} tm_server_info;

/* The graph must outlive the server.  cfg may be NULL for the defaults. */
int tm_server_open(const tm_graph *g, const tm_server_config *cfg, tm_server **out);
/* Copy a request (motifs as for tm_tree_build, host root list) into the
 * queue; *ticket identifies it.  Motifs are validated here (TM_EINVAL /
 * TM_EUNSUPPORTED as tm_tree_build); a root outside [0, n_edges) is TM_EINVAL. */
int tm_server_submit(tm_server *s, const int8_t *motif_uv, const int32_t *motif_off, int32_t n_motifs,
                     const int64_t *delta, const int32_t *roots, int64_t n_roots, int64_t *ticket);
/* 1 when done (counts, n_motifs int64, and stats filled; the ticket is then
 * released), 0 while pending (wait = 0), or the request's error code.  With
 * wait != 0 the call blocks until the request finishes. */
int tm_server_poll(tm_server *s, int64_t ticket, int32_t wait, int64_t *counts, tm_request_stats *stats);
int tm_server_get_info(tm_server *s, tm_server_info *info);
/* Finishes every admitted and pending request, then stops the worker. */
int tm_server_close(tm_server *s);

/* ------------------------------------------------------------ replay and tuning */
/*
 * A count captured once as a CUDA graph and replayed: scratch is allocated
 * at creation, each replay resets it, runs the mining launches and writes
 * the counts to `counts` (device, n_motifs int64).  `args` must name device
 * roots (TM_ROOTS_DEVICE) or a range; per-root outputs and stats are not
 * available.  Used for batches of many motif sets (one tree built from all
 * of them, each motif with its own window) launched repeatedly.
 * tm_exec_status synchronises `stream` and returns TM_ETIMEOUT when a bounded
 * device wait expired in the last replay.
 */
typedef struct tm_exec tm_exec;
int tm_exec_create(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, int64_t *counts, void *stream,
                   tm_exec **out);
int tm_exec_launch(tm_exec *x, void *stream);
int tm_exec_status(tm_exec *x, void *stream);
int tm_exec_free(tm_exec *x);

/* Launch shape and split thresholds picked by tm_autotune (times a grid on the
 * caller's roots, best of two runs each; the counts are not returned). */
typedef struct {
    int32_t ctas_per_sm;
    int32_t donate_seq;
    int32_t donate_leaf;
    int32_t poll_every;
    float ms;                 /* time of the chosen configuration */
} tm_tune;
int tm_autotune(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, tm_tune *best, void *stream);

/*
 * Allocation-free counting.  The paper has no counterpart: this is a
 * service of the library.
 *
 * Some callers must not allocate device memory while they count: a
 * long-running service that fixed its memory budget at start-up, code under
 * an external allocator that rejects stray cudaMalloc calls, or a loop with
 * a latency limit that an allocation could break.  tm_count allocates its
 * scratch (counters, root cursor, task queue) on every call; this variant
 * allocates nothing.  Its scratch is one static device array of 256 KiB in
 * the library, which every GPU that loads the library holds until the
 * process exits.
 *
 * It counts like tm_count with mode TM_COMINE (MG-Tree, window-arithmetic
 * leaves) and static scheduling (one warp per root edge), same counts.
 *   roots:  device array of n_roots root edge ids, or NULL for the eids
 *           [root_lo, root_hi) (root_hi <= 0 means n_edges)
 *   counts: device array of n_motifs int64, overwritten; the call does not
 *           synchronise `stream`
 *   Each device root must lie in [0, n_edges); the list is not read on the
 *   host, and the kernel skips a root outside that range (it counts nothing
 *   and no error is returned, as the call does not synchronise).
 * Limits: at most 1024 motifs; any tree within TM_MAX_NODES nodes fits.
 * Beyond 1024 motifs the call returns TM_EUNSUPPORTED.
 * Set-up: the first call on a device (made with that device current)
 * looks up the address of the static array there and caches it for the
 * life of the process, which assumes the device is not reset
 * (cudaDeviceReset) in between; make that first call before any stream
 * capture.  All calls share the one array, which keeps the
 * last call's contents; each call clears its counters itself, but calls
 * whose work overlaps on the GPU (several streams or threads at once) race
 * on the array and give wrong counts, so serialise them.
 * Errors: TM_EINVAL (NULL handle or counts, bad root range, n_roots < 0),
 * TM_EUNSUPPORTED (limits above), TM_ECUDA.
 */
int tm_count_noalloc(const tm_graph *g, const tm_tree *tr, const int32_t *roots, int64_t n_roots,
                     int64_t root_lo, int64_t root_hi, int64_t *counts, void *stream);

/* ------------------------------------------------------------ learned scheduling */
/*
 * A small cost model predicts each root edge's search cost so the launch can
 * start the heaviest roots first and cut them into slices for other warps.
 * The paper has no learned part (its GPU runtime rebalances reactively,
 * Section 4.5); this follows the scheduling scheme the library adds on top.
 *
 * Features (tm_features), TM_FEATURES float32 per root, each log1p-scaled:
 * out- and in-degree of the root's destination, out-degree of its source,
 * the number of entries of those three lists inside the root's window (the
 * tree's largest delta), the tree's depth and the root node's fan-out.
 * Model: TM_FEATURES -> 64 -> 64 -> 1, ReLU, standardised inputs, FP16
 * weights and FP32 accumulation on the device, FP32 master weights for
 * training (Adam, mean squared error).  Parameters in one float32 vector:
 * W1 (64 x 8, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1).
 * Labels are log1p of measured work (tm_count's per-root work counters:
 * candidates + probes).  All pointers to features, labels, predictions and
 * plans are device pointers; the calls that do not say otherwise do not
 * synchronise `stream`.
 */
#define TM_FEATURES 8
#define TM_MODEL_PARAMS 4801

typedef struct tm_model tm_model;   /* opaque, library-owned, device resident */

int tm_features(const tm_graph *g, const tm_tree *tr, const int32_t *roots, int64_t n_roots, float *feats,
                void *stream);
/* He-initialised weights from `seed`; synchronises the device. */
int tm_model_create(uint64_t seed, tm_model **out);
int tm_model_free(tm_model *m);
/* Host copies of the FP32 parameters (TM_MODEL_PARAMS) and of the input
 * standardisation (mean[8] then inverse std[8]); either pointer may be NULL. */
int tm_model_get_params(const tm_model *m, float *params, float *norm);
int tm_model_set_params(tm_model *m, const float *params, const float *norm);
/* Input standardisation from n feature rows. */
int tm_model_fit_norm(tm_model *m, const float *feats, int64_t n, void *stream);
/* Predicted log1p(work) of n rows into out. */
int tm_model_predict(const tm_model *m, const float *feats, int64_t n, float *out, void *stream);
/* Mean squared error and its gradient over n rows at the current weights
 * (host outputs, TM_MODEL_PARAMS gradients; either may be NULL); synchronises. */
int tm_model_loss_grad(const tm_model *m, const float *feats, const float *labels, int64_t n, float *loss,
                       float *grad, void *stream);
/* Adam over contiguous minibatches for `epochs` passes; loss_history
 * (host, epochs floats, may be NULL) gets each pass's mean loss; synchronises. */
int tm_model_train(tm_model *m, const float *feats, const float *labels, int64_t n, int32_t epochs, int32_t batch,
                   float lr, float *loss_history, void *stream);
/* Plan: roots_out = roots ordered by decreasing predicted work; split_out[i] =
 * number of slices (1..max_split) for root roots_out[i], about one slice per
 * unit_work of predicted work.  Pass both to tm_count with TM_SCHED_PLANNED. */
int tm_plan(const tm_model *m, const float *feats, const int32_t *roots, int64_t n, double unit_work,
            int32_t max_split, int32_t *roots_out, int32_t *split_out, void *stream);
/* The same with tiers: roots whose predicted work is below thread_work get
 * split_out 0, which TM_SCHED_TIERS runs one per lane; being the least
 * predicted, they form the tail of roots_out. */
int tm_plan_tiers(const tm_model *m, const float *feats, const int32_t *roots, int64_t n, double unit_work,
                  int32_t max_split, double thread_work, int32_t *roots_out, int32_t *split_out, void *stream);

/* Message describing the last error on the calling thread ("" if none). */
const char *tm_last_error(void);

/* Library version string. */
const char *tm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TMOTIF_H */
