/*
 * CPU oracle for exact delta-temporal motif counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only tests/, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA library.
 *
 * What it computes (Section 2, "A delta-Temporal Motif" / "Temporal Motif
 * Mining"): for a motif M = ((u_1,v_1),...,(u_m,v_m)) and window delta, the
 * number of edge tuples e_1 < e_2 < ... < e_m (edge ids of the time-ordered
 * edge list) with t(e_m) - t(e_1) <= delta for which one injective map f from
 * motif vertices to graph vertices has f(u_i) = src(e_i), f(v_i) = dst(e_i).
 *
 * Two procedures, each a plain recursion:
 *   - oracle_count_motif: Algorithm 1 (TemporalMining / MatchEdge /
 *     RollOnEdge / RollBackEdge), one motif at a time (oracle_enumerate_motif
 *     runs the same recursion and also records each match it completes);
 *   - oracle_comine: Algorithm 3 (TemporalCoMining / CoMatchEdge) guided by
 *     a Motif-Group Tree given as a node table.
 *
 * Readings where the paper is silent or garbled (each is listed again in the
 * design notes):
 *   R1 ties: edges are totally ordered by (t, input index); a match needs
 *      strictly increasing edge ids (with unique timestamps this is the
 *      paper's t_1 < ... < t_m);
 *   R2 the window is inclusive (t_m - t_1 <= delta) and measured from the
 *      first edge of the whole motif;
 *   R3 injectivity is checked for both endpoints: a newly mapped motif vertex
 *      may not land on a graph vertex that is already an image;
 *   R4 when u_M is unmapped but v_M is mapped, the candidates are the
 *      in-edges of m2g[v_M]; when both are unmapped, all edges;
 *   R5 RollBackEdge releases (u, v) of the popped edge (the listing passes
 *      u twice);
 *   R14 t_1 + delta saturates at INT64_MAX.
 *
 * Candidate lists are walked in edge-id order starting at the first edge id
 * greater than the previous match (located by binary search) and stop at the
 * first edge outside the window.  Every edge skipped that way fails the
 * temporal test of MatchEdge anyway, because time is non-decreasing in edge
 * id; every edge visited still goes through that test.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define OR_MAXE 16
#define OR_MAXV 32

typedef struct {
    int64_t E;
    int32_t V;
    const int32_t *src, *dst;
    const int64_t *t;
    int64_t *out_off; int32_t *out_e;   /* out-edges of each vertex, ascending eid */
    int64_t *in_off;  int32_t *in_e;    /* in-edges of each vertex, ascending eid */
} og_graph;

/* per-search book-keeping context (Algorithm 1, book-keeping line) */
typedef struct {
    const og_graph *g;
    int32_t m2g[OR_MAXV];
    int32_t *g2m;       /* size V, -1 = not an image */
    int32_t *incnt;     /* size V */
    int32_t e_stack[OR_MAXE];
    int64_t t_first;
    int64_t t_limit;    /* t_first + delta, saturated */
    int64_t work;       /* candidates examined */
    int64_t max_work;   /* abort when exceeded (<= 0: unlimited) */
    double deadline;    /* CLOCK_MONOTONIC seconds; abort after it (<= 0: none) */
    int aborted;
    /* motif (Algorithm 1) */
    int m;
    const int8_t *mu, *mv;
    int64_t count;
    int32_t *rec;       /* enumeration: completed matches, m edge ids each (NULL: count only) */
    int64_t rec_cap;    /* ... room for this many */
    /* tree (Algorithm 3) */
    int n_nodes;
    const int32_t *node_len;      /* |C_N| */
    const int8_t *node_u, *node_v;/* C_N edges, node n at [n*OR_MAXE, ...) */
    const int32_t *child_off, *child_idx;
    const int32_t *ref_off, *ref_idx; /* Q_N: query indices counted at N */
    int64_t *counts;              /* per query */
} og_ctx;

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static int64_t sat_add(int64_t a, int64_t b) {
    if (b > 0 && a > INT64_MAX - b) return INT64_MAX;
    return a + b;
}

static void build_adj(og_graph *g) {
    int64_t E = g->E; int32_t V = g->V;
    g->out_off = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
    g->in_off = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
    g->out_e = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    g->in_e = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    for (int64_t e = 0; e < E; e++) { g->out_off[g->src[e] + 1]++; g->in_off[g->dst[e] + 1]++; }
    for (int32_t v = 0; v < V; v++) { g->out_off[v + 1] += g->out_off[v]; g->in_off[v + 1] += g->in_off[v]; }
    int64_t *po = (int64_t *)malloc(sizeof(int64_t) * ((size_t)V + 1));
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * ((size_t)V + 1));
    memcpy(po, g->out_off, sizeof(int64_t) * ((size_t)V + 1));
    memcpy(pi, g->in_off, sizeof(int64_t) * ((size_t)V + 1));
    for (int64_t e = 0; e < E; e++) {      /* ascending e keeps each list in eid order */
        g->out_e[po[g->src[e]]++] = (int32_t)e;
        g->in_e[pi[g->dst[e]]++] = (int32_t)e;
    }
    free(po); free(pi);
}

static void free_adj(og_graph *g) {
    free(g->out_off); free(g->in_off); free(g->out_e); free(g->in_e);
}

/* first position p in list[lo,hi) with list[p] > key */
static int64_t first_after(const int32_t *list, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (list[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* RollOnEdge */
static void roll_on(og_ctx *c, int uM, int vM, int32_t uG, int32_t vG) {
    c->m2g[uM] = uG; c->g2m[uG] = uM;
    c->m2g[vM] = vG; c->g2m[vG] = vM;
    c->incnt[uG]++; c->incnt[vG]++;
}

/* RollBackEdge, releasing both endpoints of the popped edge (reading R5) */
static void roll_back(og_ctx *c, int32_t uG, int32_t vG) {
    c->incnt[uG]--; c->incnt[vG]--;
    if (c->incnt[uG] == 0) { int uM = c->g2m[uG]; c->g2m[uG] = -1; c->m2g[uM] = -1; }
    if (c->incnt[vG] == 0) { int vM = c->g2m[vG]; c->g2m[vG] = -1; c->m2g[vM] = -1; }
}

typedef void (*descend_fn)(og_ctx *, int, int);

/*
 * The body shared by MatchEdge and CoMatchEdge: match motif edge (uM, vM) at
 * position em, with `next(ctx, node, em + 1)` as the recursive call.
 */
static void match_one_edge(og_ctx *c, int node, int em, int uM, int vM, descend_fn next) {
    const og_graph *g = c->g;
    int32_t uG = c->m2g[uM], vG = c->m2g[vM];
    const int32_t *list; int64_t lo, hi;
    int all_edges = 0;
    if (uG != -1) { list = g->out_e; lo = g->out_off[uG]; hi = g->out_off[uG + 1]; }
    else if (vG != -1) { list = g->in_e; lo = g->in_off[vG]; hi = g->in_off[vG + 1]; }   /* R4 */
    else { list = NULL; lo = 0; hi = g->E; all_edges = 1; }
    int32_t last = c->e_stack[em - 1];
    if (all_edges) lo = (int64_t)last + 1;
    else lo = first_after(list, lo, hi, last);
    for (int64_t p = lo; p < hi; p++) {
        if (c->aborted) return;
        int32_t e = all_edges ? (int32_t)p : list[p];
        int64_t te = g->t[e];
        if (te > c->t_limit) break;                       /* every later edge fails too */
        c->work++;
        if (c->max_work > 0 && c->work > c->max_work) { c->aborted = 1; return; }
        if (c->deadline > 0 && (c->work & 0xFFFFF) == 0 && now_s() > c->deadline) { c->aborted = 1; return; }
        /* temporal constraints (order: strictly later edge id, R1; window, R2) */
        if (e <= last || te > c->t_limit) continue;
        int32_t eu = g->src[e], ev = g->dst[e];
        /* structural constraints with full injectivity (R3) */
        if (uG != -1 && eu != uG) continue;
        if (vG != -1 && ev != vG) continue;
        if (uG == -1 && c->g2m[eu] != -1) continue;
        if (vG == -1 && c->g2m[ev] != -1) continue;
        if (uG == -1 && vG == -1 && eu == ev) continue;
        c->e_stack[em] = e;
        roll_on(c, uM, vM, eu, ev);
        next(c, node, em + 1);
        roll_back(c, eu, ev);
    }
}

/* ---------------------------------------------------------------- Algorithm 1 */

static void match_edge(og_ctx *c, int unused_node, int em) {
    (void)unused_node;
    if (em == c->m) {                          /* match found: record it, count it */
        if (c->rec && c->count < c->rec_cap)
            memcpy(c->rec + c->count * c->m, c->e_stack, sizeof(int32_t) * (size_t)c->m);
        c->count++;
        return;
    }
    match_one_edge(c, 0, em, c->mu[em], c->mv[em], match_edge);
}

/* first motif edge fixed to the root edge r */
static int start_root(og_ctx *c, int32_t r, int uM, int vM, int64_t delta) {
    const og_graph *g = c->g;
    int32_t eu = g->src[r], ev = g->dst[r];
    if (eu == ev) return 0;                    /* both unmapped: injective needs eu != ev */
    c->e_stack[0] = r;
    c->t_first = g->t[r];
    c->t_limit = sat_add(c->t_first, delta);  /* R14 */
    roll_on(c, uM, vM, eu, ev);
    return 1;
}

static og_ctx *new_ctx(const og_graph *g) {
    og_ctx *c = (og_ctx *)calloc(1, sizeof(og_ctx));
    c->g = g;
    c->g2m = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->V > 0 ? g->V : 1));
    c->incnt = (int32_t *)calloc((size_t)(g->V > 0 ? g->V : 1), sizeof(int32_t));
    for (int32_t v = 0; v < g->V; v++) c->g2m[v] = -1;
    for (int i = 0; i < OR_MAXV; i++) c->m2g[i] = -1;
    return c;
}

static void free_ctx(og_ctx *c) { free(c->g2m); free(c->incnt); free(c); }

/*
 * Count one motif (Algorithm 1).
 *   mu, mv: motif edges (m of them, labels < OR_MAXV, mu[i] != mv[i])
 *   roots:  edge ids allowed as the first motif edge (NULL: all edges)
 *   per_root: optional output, count for each root
 *   work_out: optional, candidates examined per root
 *   root_budget: when non-zero, max_work applies to each root separately and
 *     a root that exceeds it gets per_root = -1 (excluded from *total)
 * Returns 0, or 1 when max_work was exceeded (outputs then incomplete),
 * or -1 for invalid input.
 */
int oracle_count_motif(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t E, int32_t V,
                       const int8_t *mu, const int8_t *mv, int m, int64_t delta,
                       const int32_t *roots, int64_t n_roots, int64_t max_work, int root_budget,
                       int64_t *total, int64_t *per_root, int64_t *work_out) {
    if (m < 1 || m > OR_MAXE || delta < 0) return -1;
    for (int i = 0; i < m; i++)
        if (mu[i] < 0 || mv[i] < 0 || mu[i] >= OR_MAXV || mv[i] >= OR_MAXV || mu[i] == mv[i]) return -1;
    og_graph g = {E, V, src, dst, t, 0, 0, 0, 0};
    build_adj(&g);
    og_ctx *c = new_ctx(&g);
    c->m = m; c->mu = mu; c->mv = mv; c->max_work = max_work;
    int64_t nr = roots ? n_roots : E;
    int64_t sum = 0;
    int rc = 0;
    for (int64_t i = 0; i < nr; i++) {
        int32_t r = roots ? roots[i] : (int32_t)i;
        int64_t before = c->count, w0 = c->work;
        if (start_root(c, r, mu[0], mv[0], delta)) {
            match_edge(c, 0, 1);
            roll_back(c, src[r], dst[r]);
        }
        if (per_root) per_root[i] = c->count - before;
        if (work_out) work_out[i] = c->work - w0;
        if (c->aborted && root_budget) {
            /* this root alone ran past the budget: mark it and go on */
            if (per_root) per_root[i] = -1;
            c->count = before;
            c->aborted = 0;
            c->work = 0;
            /* undo the mappings left by the interrupted recursion */
            for (int32_t v = 0; v < g.V; v++) { c->g2m[v] = -1; c->incnt[v] = 0; }
            for (int q = 0; q < OR_MAXV; q++) c->m2g[q] = -1;
            continue;
        }
        if (c->aborted) { rc = 1; break; }
        if (root_budget) c->work = 0;
    }
    sum = c->count;
    if (total) *total = sum;
    free_ctx(c);
    free_adj(&g);
    return rc;
}

/*
 * The matches themselves (Algorithm 1 records each match it completes):
 * every tuple counted by oracle_count_motif over `roots` (NULL: all edges),
 * written as m edge ids in motif edge order to out[0 .. min(total, cap) * m)
 * in search order; *n_found gets the total.  Returns 0, or -1 for invalid
 * input.
 */
int oracle_enumerate_motif(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t E, int32_t V,
                           const int8_t *mu, const int8_t *mv, int m, int64_t delta,
                           const int32_t *roots, int64_t n_roots, int32_t *out, int64_t cap, int64_t *n_found) {
    if (m < 1 || m > OR_MAXE || delta < 0 || cap < 0) return -1;
    for (int i = 0; i < m; i++)
        if (mu[i] < 0 || mv[i] < 0 || mu[i] >= OR_MAXV || mv[i] >= OR_MAXV || mu[i] == mv[i]) return -1;
    og_graph g = {E, V, src, dst, t, 0, 0, 0, 0};
    build_adj(&g);
    og_ctx *c = new_ctx(&g);
    c->m = m; c->mu = mu; c->mv = mv;
    c->rec = out; c->rec_cap = out ? cap : 0;
    int64_t nr = roots ? n_roots : E;
    for (int64_t i = 0; i < nr; i++) {
        int32_t r = roots ? roots[i] : (int32_t)i;
        if (start_root(c, r, mu[0], mv[0], delta)) {
            match_edge(c, 0, 1);
            roll_back(c, src[r], dst[r]);
        }
    }
    *n_found = c->count;
    free_ctx(c);
    free_adj(&g);
    return 0;
}

/* ---------------------------------------------------------------- Algorithm 3 */

static void co_match_edge(og_ctx *c, int node, int em) {
    int len = c->node_len[node];
    if (em == len) {                                  /* C_N fully matched */
        for (int q = c->ref_off[node]; q < c->ref_off[node + 1]; q++)
            c->counts[c->ref_idx[q]]++;               /* Q_N != empty: count */
        for (int k = c->child_off[node]; k < c->child_off[node + 1]; k++)
            co_match_edge(c, c->child_idx[k], em);    /* children from this partial match */
        return;
    }
    const int8_t *u = c->node_u + (size_t)node * OR_MAXE, *v = c->node_v + (size_t)node * OR_MAXE;
    match_one_edge(c, node, em, u[em], v[em], co_match_edge);
}

/*
 * Co-mine a Motif-Group Tree (Algorithm 3) with one window delta.
 *   node_len[n], node_u/node_v[n*16 + i]: C_N of node n (full edge list)
 *   child_off/child_idx: Children(N) in CSR form; node 0 is the root
 *   ref_off/ref_idx: query indices whose motif equals C_N (Q_N)
 *   counts: n_queries outputs; per_root: optional [n_roots][n_queries]
 */
int oracle_comine(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t E, int32_t V,
                  int n_nodes, const int32_t *node_len, const int8_t *node_u, const int8_t *node_v,
                  const int32_t *child_off, const int32_t *child_idx,
                  const int32_t *ref_off, const int32_t *ref_idx, int n_queries, int64_t delta,
                  const int32_t *roots, int64_t n_roots, int64_t max_work,
                  int64_t *counts, int64_t *per_root, int64_t *work_out) {
    if (n_nodes < 1 || delta < 0 || node_len[0] < 1) return -1;
    og_graph g = {E, V, src, dst, t, 0, 0, 0, 0};
    build_adj(&g);
    og_ctx *c = new_ctx(&g);
    c->n_nodes = n_nodes; c->node_len = node_len; c->node_u = node_u; c->node_v = node_v;
    c->child_off = child_off; c->child_idx = child_idx; c->ref_off = ref_off; c->ref_idx = ref_idx;
    c->max_work = max_work;
    int64_t *acc = (int64_t *)calloc((size_t)n_queries, sizeof(int64_t));
    c->counts = acc;
    int64_t nr = roots ? n_roots : E;
    int rc = 0;
    int64_t *prev = (int64_t *)calloc((size_t)n_queries, sizeof(int64_t));
    for (int64_t i = 0; i < nr; i++) {
        int32_t r = roots ? roots[i] : (int32_t)i;
        int64_t w0 = c->work;
        if (per_root) memcpy(prev, acc, sizeof(int64_t) * (size_t)n_queries);
        if (start_root(c, r, node_u[0], node_v[0], delta)) {
            co_match_edge(c, 0, 1);
            roll_back(c, src[r], dst[r]);
        }
        if (per_root)
            for (int q = 0; q < n_queries; q++) per_root[i * n_queries + q] = acc[q] - prev[q];
        if (work_out) work_out[i] = c->work - w0;
        if (c->aborted) { rc = 1; break; }
    }
    memcpy(counts, acc, sizeof(int64_t) * (size_t)n_queries);
    free(prev); free(acc);
    free_ctx(c);
    free_adj(&g);
    return rc;
}

/*
 * Algorithm 1 over roots spread across threads with dynamic scheduling (the
 * paper's CPU task manager, Section 4.5), for the timed CPU baseline only.
 * Each thread owns a private context.  Stops once time_limit seconds (> 0)
 * have passed, also inside a root; *n_done roots were finished, and
 * per_root is -1 for every other root.  Returns 0, 1 when the limit was
 * reached, -1 for invalid input.
 */
int oracle_count_motif_mt(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t E, int32_t V,
                          const int8_t *mu, const int8_t *mv, int m, int64_t delta,
                          const int32_t *roots, int64_t n_roots, int n_threads, double time_limit,
                          int64_t *per_root, int64_t *n_done) {
    if (m < 1 || m > OR_MAXE || delta < 0) return -1;
    og_graph g = {E, V, src, dst, t, 0, 0, 0, 0};
    build_adj(&g);
    double t0 = now_s();
    int64_t done = 0;
    volatile int timed_out = 0;
    for (int64_t i = 0; i < n_roots; i++) per_root[i] = -1;
#pragma omp parallel num_threads(n_threads) reduction(+:done)
    {
        og_ctx *c = new_ctx(&g);
        c->m = m; c->mu = mu; c->mv = mv;
        c->deadline = time_limit > 0 ? t0 + time_limit : 0;
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < n_roots; i++) {
            if (timed_out || c->aborted) continue;
            if (time_limit > 0 && now_s() > t0 + time_limit) { timed_out = 1; continue; }
            int32_t r = roots[i];
            int64_t before = c->count;
            if (start_root(c, r, mu[0], mv[0], delta)) {
                match_edge(c, 0, 1);
                roll_back(c, src[r], dst[r]);
            }
            if (c->aborted) { timed_out = 1; continue; }   /* interrupted inside this root */
            per_root[i] = c->count - before;
            done++;
        }
        free_ctx(c);
    }
    *n_done = done;
    free_adj(&g);
    return timed_out ? 1 : 0;
}
