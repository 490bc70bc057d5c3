// Co-mining decision (Section 6, "Heuristic for Co-Mining"): co-mine on a
// bipartite data graph, otherwise only when the MG-Tree's similarity metric
// reaches the threshold below which per-motif mining was faster on the GPU.
//
// Bipartiteness of the undirected view, on the device.  The bipartite double
// cover has vertices v and v' = v + V and, for every edge {a, b}, the edges
// {a, b'} and {a', b}.  A connected component of the graph is bipartite iff v
// and v' fall into different components of the cover (an odd cycle through v
// is exactly a path from v to v' in the cover; a self-loop {a, a} joins a and
// a' directly).  Components are found by label hooking and pointer jumping:
// every label is the id of a vertex in the same component and only
// decreases, so the loop ends, and at its fixpoint every edge joins equal
// labels.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "tm_internal.h"

namespace tmo {
namespace {

__global__ void k_cc_init(int32_t *L, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) L[i] = (int32_t)i;
}

// Hook: for both cover edges of graph edge e, lower the larger label's own
// label to the smaller one.
__global__ void k_cc_hook(const int32_t *src, const int32_t *dst, int64_t E, int32_t V, int32_t *L, int *changed) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int32_t a = src[e], b = dst[e];
    const int32_t ends[2][2] = {{a, b + V}, {a + V, b}};
    bool ch = false;
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const int32_t la = L[ends[j][0]], lb = L[ends[j][1]];
        if (la == lb) continue;
        const int32_t lo = min(la, lb), hi = max(la, lb);
        if (atomicMin(&L[hi], lo) > lo) ch = true;
    }
    if (ch) *changed = 1;
}

// Jump: replace each label by its label's label, a few times per launch.
__global__ void k_cc_jump(int32_t *L, int64_t n, int *changed) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t l = L[i];
    bool ch = false;
#pragma unroll 1
    for (int it = 0; it < 8; it++) {
        const int32_t ll = L[l];
        if (ll == l) break;
        l = ll;
        ch = true;
    }
    if (ch) {
        L[i] = l;
        *changed = 1;
    }
}

__global__ void k_cc_odd(const int32_t *L, int32_t V, int *odd) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V && L[v] == L[v + V]) *odd = 1;
}

inline unsigned grid(int64_t n) { return (unsigned)((n + 255) / 256); }

// Rounds of hook + jump: each round at least halves the depth of every label
// chain or merges components; 2^16 rounds are far beyond any graph that fits.
constexpr int kMaxRounds = 1 << 16;

}  // namespace

int graph_bipartite(const tm_graph *g, cudaStream_t s, int32_t *out) {
    std::lock_guard<std::mutex> lock(g->heur_mutex);
    if (g->bipartite >= 0) {
        *out = g->bipartite;
        return TM_OK;
    }
    const int64_t E = g->d.E;
    const int32_t V = g->d.V;
    const int64_t n = 2 * (int64_t)V;
    if (n > INT32_MAX) {
        set_error("tm_graph_bipartite: more than 2^30 vertices");
        return TM_EUNSUPPORTED;
    }
    if (E == 0) {
        g->bipartite = 1;
        *out = 1;
        return TM_OK;
    }
    int32_t *L = nullptr;
    int *flags = nullptr;        // [0] changed, [1] odd
    if (cudaMalloc(&L, sizeof(int32_t) * n) != cudaSuccess) {
        cudaGetLastError();
        set_error("tm_graph_bipartite: out of device memory");
        return TM_ENOMEM;
    }
    if (cudaMalloc(&flags, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(L);
        set_error("tm_graph_bipartite: out of device memory");
        return TM_ENOMEM;
    }
    int rc = TM_OK;
    int h[2] = {0, 0};
    auto fail = [&](cudaError_t e) {
        set_error(std::string("tm_graph_bipartite: ") + cudaGetErrorString(e));
        rc = TM_ECUDA;
    };
    k_cc_init<<<grid(n), 256, 0, s>>>(L, n);
    int round = 0;
    for (; round < kMaxRounds && rc == TM_OK; round++) {
        cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int), s);
        if (e != cudaSuccess) { fail(e); break; }
        k_cc_hook<<<grid(E), 256, 0, s>>>(g->d.src, g->d.dst, E, V, L, flags);
        // jump until every label is a root; any change means another hook round
        bool again = false;
        for (int j = 0; j < kMaxRounds; j++) {
            e = cudaMemsetAsync(flags + 1, 0, sizeof(int), s);
            if (e != cudaSuccess) { fail(e); break; }
            k_cc_jump<<<grid(n), 256, 0, s>>>(L, n, flags + 1);
            e = cudaMemcpyAsync(h, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { fail(e); break; }
            again = again || h[0] || h[1];
            if (!h[1]) break;
        }
        if (rc != TM_OK || !again) break;
    }
    if (rc == TM_OK && round >= kMaxRounds) {
        set_error("tm_graph_bipartite: labelling did not converge");
        rc = TM_ECUDA;
    }
    if (rc == TM_OK) {
        cudaError_t e = cudaMemsetAsync(flags + 1, 0, sizeof(int), s);
        if (e == cudaSuccess) {
            k_cc_odd<<<grid(V), 256, 0, s>>>(L, V, flags + 1);
            e = cudaMemcpyAsync(h, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) fail(e);
    }
    cudaFree(flags);
    cudaFree(L);
    if (rc != TM_OK) return rc;
    g->bipartite = h[1] ? 0 : 1;
    *out = g->bipartite;
    return TM_OK;
}

int comine_advice(const tm_graph *g, const tm_tree *tr, cudaStream_t s, int32_t *out) {
    int32_t bip = 0;
    TM_TRY(graph_bipartite(g, s, &bip));
    *out = (bip || tr->h.similarity >= TM_COMINE_MIN_SM) ? 1 : 0;
    return TM_OK;
}

}  // namespace tmo
