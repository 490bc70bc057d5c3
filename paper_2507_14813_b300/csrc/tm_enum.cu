// Match enumeration: Algorithm 1 records each match it completes (the
// "output" of the recursion); the paper's experiments only count.  This
// kernel walks the MG-Tree like Algorithm 3 and writes every completed match
// of every motif to a bounded device buffer.
//
// One warp per root edge, depth first.  Every motif edge is its own level
// (the scan form of the tree, no leaf arithmetic), so a match is complete
// exactly where its node's refs are counted: for each ref, the surviving
// lanes of the chunk whose edge lies in the ref's window each own one match
// and write it.  Slots are reserved with one atomic per warp and chunk; a
// match whose slot is at or past the capacity is counted but not written, so
// the total found is exact whatever the capacity.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tm_internal.h"

namespace tmo {
namespace {

constexpr int kEnumWarps = 8;
constexpr int kEnumThreads = kEnumWarps * 32;

enum : int8_t { kOut = 0, kIn = 1, kAll = 2 };

struct EnumWarp {
    int2 cand[kMaxE][32];     // the chunk held at each level: (other endpoint, edge id)
    int64_t pos[kMaxE];       // next chunk start
    int64_t end[kMaxE];       // end of the level's slice
    uint32_t mask[kMaxE];     // survivors of the held chunk not yet descended
    int32_t lvert[kMaxE];     // list vertex
    int32_t eid[kMaxE];       // matched edge per level
    int16_t node[kMaxE];
    int16_t sib_end[kMaxE];
    int8_t ltype[kMaxE];
    int32_t m2g[kMaxV];       // motif label -> graph vertex
    int32_t ehi[TM_MAX_DELTAS]; // last edge id inside each window of the current root
};

struct EnumParams {
    DevGraph g;
    DevTree tr;
    const int32_t *roots;     // or null: the range root_lo + [0, n_roots)
    int64_t n_roots;
    int64_t root_lo;
    tm_match *out;
    int64_t cap;
    unsigned long long *found;   // [0] matches found, [1] root cursor, [2] bad root
    unsigned long long *counts;  // per caller motif
};

// first position in adj[lo, hi) whose edge id exceeds key
__device__ int64_t upper_eid(const int2 *adj, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&adj[mid].y) <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// last edge id e >= r with t[e] <= limit
__device__ int32_t last_in_window(const int64_t *t, int64_t E, int32_t r, int64_t limit) {
    int64_t lo = r, hi = E;            // t[lo] <= limit; answer in [lo, hi)
    while (hi - lo > 1) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(t + mid) <= limit) lo = mid; else hi = mid;
    }
    return (int32_t)lo;
}

struct Enumerator {
    const EnumParams &p;
    EnumWarp &w;
    int lane;

    // Write the matches completed by the lanes of S at level k of node N.
    __device__ void emit(const DevNode &N, int k, uint32_t S, int2 c) {
        for (int i = 0; i < N.n_ref; i++) {
            const DevRef ref = p.tr.refs[N.ref_begin + i];
            const uint32_t in = __ballot_sync(0xffffffffu, c.y <= w.ehi[ref.delta]) & S;
            if (!in) continue;
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(&p.found[0], (unsigned long long)__popc(in));
                atomicAdd(&p.counts[ref.counter], (unsigned long long)__popc(in));
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((in >> lane) & 1u) {
                const unsigned long long slot = base + __popc(in & ((1u << lane) - 1u));
                if (slot < (unsigned long long)p.cap) {
                    tm_match m;
                    m.motif = ref.counter;
                    m.n_edges = k + 1;
#pragma unroll
                    for (int j = 0; j < kMaxE; j++) m.eid[j] = j < k ? w.eid[j] : (j == k ? c.y : -1);
                    p.out[slot] = m;
                }
            }
        }
    }

    // A chunk of level k of node N filtered to S: write completed matches,
    // keep the survivors that descend.
    __device__ void take(int k, const DevNode &N, uint32_t S, int2 c) {
        w.cand[k][lane] = c;
        const bool complete = k == N.k_end - 1;
        if (complete && N.n_ref > 0) emit(N, k, S, c);
        const bool descend = complete ? N.n_seq > 0 : true;
        __syncwarp();
        if (lane == 0) w.mask[k] = descend ? S : 0u;
        __syncwarp();
    }

    // Open level k for `node` (siblings up to sib_end): the slice of its
    // candidate list with edge ids in (eid[k-1], last edge of the node's window].
    __device__ void open(int k, int node, int sib_end) {
        const DevNode &N = p.tr.nodes[node];
        const int u = N.eu[k], v = N.ev[k], nv = N.nvb[k];
        const bool um = u < nv, vm = v < nv;
        const int32_t last = w.eid[k - 1], hi = w.ehi[N.dmax];
        int8_t lt;
        int32_t x = 0;
        if (um && vm) {
            const int32_t xu = w.m2g[u], xv = w.m2g[v];
            const int64_t du = __ldg(p.g.out_off + xu + 1) - __ldg(p.g.out_off + xu);
            const int64_t dv = __ldg(p.g.in_off + xv + 1) - __ldg(p.g.in_off + xv);
            if (du <= dv) { lt = kOut; x = xu; } else { lt = kIn; x = xv; }
        } else if (um) { lt = kOut; x = w.m2g[u]; }
        else if (vm) { lt = kIn; x = w.m2g[v]; }
        else lt = kAll;
        int64_t a = 0, b = 0;
        if (lane == 0) {
            if (lt == kAll) {
                a = (int64_t)last + 1;
                b = (int64_t)hi + 1;
            } else {
                const int64_t *off = lt == kOut ? p.g.out_off : p.g.in_off;
                const int2 *adj = lt == kOut ? p.g.out_adj : p.g.in_adj;
                const int64_t b0 = __ldg(off + x), b1 = __ldg(off + x + 1);
                a = upper_eid(adj, b0, b1, last);
                b = upper_eid(adj, a, b1, hi);
            }
            if (b < a) b = a;
            w.node[k] = (int16_t)node;
            w.sib_end[k] = (int16_t)sib_end;
            w.ltype[k] = lt;
            w.lvert[k] = x;
            w.pos[k] = a;
            w.end[k] = b;
            w.mask[k] = 0;
        }
        __syncwarp();
    }

    // Load and filter the next chunk of level k.
    __device__ void load(int k) {
        const DevNode &N = p.tr.nodes[w.node[k]];
        const int8_t lt = w.ltype[k];
        const int64_t i = w.pos[k] + lane, end = w.end[k];
        const int32_t last = w.eid[k - 1], hi = w.ehi[N.dmax];
        const int u = N.eu[k], v = N.ev[k], nv = N.nvb[k];
        const bool um = u < nv, vm = v < nv;
        bool ok = i < end;
        int2 c = make_int2(0, 0);
        if (ok) {
            if (lt == kOut) c = __ldg(&p.g.out_adj[i]);
            else if (lt == kIn) c = __ldg(&p.g.in_adj[i]);
            else c = make_int2(0, (int32_t)i);
            ok = c.y > last && c.y <= hi;
        }
        if (ok) {
            // injective map (reading 3): a new endpoint is no mapped vertex,
            // a mapped one is the vertex it is mapped to
            if (lt == kAll) {
                const int32_t s = __ldg(p.g.src + c.y), d = __ldg(p.g.dst + c.y);
                ok = s != d;
                for (int l = 0; l < nv; l++) ok = ok && s != w.m2g[l] && d != w.m2g[l];
            } else if (um && vm) {
                ok = c.x == (lt == kOut ? w.m2g[v] : w.m2g[u]);
            } else {
                for (int l = 0; l < nv; l++) ok = ok && c.x != w.m2g[l];
            }
        }
        const uint32_t S = __ballot_sync(0xffffffffu, ok);
        __syncwarp();
        if (lane == 0) w.pos[k] += 32;
        __syncwarp();
        take(k, N, S, c);
    }

    __device__ void root(int32_t r) {
        const int32_t a = __ldg(p.g.src + r), b = __ldg(p.g.dst + r);
        if (a == b) return;
        const int64_t t0 = __ldg(p.g.t + r);
        for (int j = lane; j < p.tr.n_deltas; j += 32) {
            const int64_t d = __ldg(p.tr.deltas + j);
            const int64_t lim = (d > 0 && t0 > INT64_MAX - d) ? INT64_MAX : t0 + d;
            w.ehi[j] = last_in_window(p.g.t, p.g.E, r, lim);
        }
        if (lane == 0) {
            w.node[0] = 0;
            w.sib_end[0] = 1;
            w.ltype[0] = kAll;
            w.pos[0] = 0;
            w.end[0] = 0;
        }
        __syncwarp();
        // level 0: the root edge, a one-candidate chunk on lane 0
        take(0, p.tr.nodes[0], 1u, make_int2(lane == 0 ? b : 0, lane == 0 ? r : 0));
        int k = 0;
        while (k >= 0) {
            const uint32_t m = w.mask[k];
            if (m) {
                const int j = __ffs(m) - 1;
                const int2 cj = w.cand[k][j];
                const DevNode &N = p.tr.nodes[w.node[k]];
                int32_t cs, cd;
                if (k == 0) { cs = a; cd = b; }
                else if (w.ltype[k] == kOut) { cs = w.lvert[k]; cd = cj.x; }
                else if (w.ltype[k] == kIn) { cs = cj.x; cd = w.lvert[k]; }
                else { cs = __ldg(p.g.src + cj.y); cd = __ldg(p.g.dst + cj.y); }
                __syncwarp();
                if (lane == 0) {
                    w.mask[k] = m & (m - 1);
                    w.eid[k] = cj.y;
                    w.m2g[N.eu[k]] = cs;
                    w.m2g[N.ev[k]] = cd;
                }
                __syncwarp();
                if (k == N.k_end - 1) open(k + 1, N.child_begin, N.child_begin + N.n_seq);
                else open(k + 1, w.node[k], w.node[k] + 1);
                k++;
                continue;
            }
            if (w.pos[k] < w.end[k]) {
                load(k);
                continue;
            }
            if (w.node[k] + 1 < w.sib_end[k]) {
                open(k, w.node[k] + 1, w.sib_end[k]);
                continue;
            }
            k--;
        }
    }
};

__global__ void __launch_bounds__(kEnumThreads) k_enum(EnumParams p) {
    __shared__ EnumWarp s_w[kEnumWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Enumerator M{p, s_w[warp], lane};
    while (true) {
        unsigned long long ri = 0;
        if (lane == 0) ri = atomicAdd(&p.found[1], 1ull);
        ri = __shfl_sync(0xffffffffu, ri, 0);
        if (ri >= (unsigned long long)p.n_roots) break;
        const int64_t r = p.roots ? (int64_t)__ldg(p.roots + ri) : p.root_lo + (int64_t)ri;
        if (r < 0 || r >= p.g.E) {
            if (lane == 0) atomicOr(&p.found[2], 1ull);
            continue;
        }
        M.root((int32_t)r);
    }
}

}  // namespace

int enumerate(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, tm_match *out, int64_t cap,
              int64_t *n_found, int64_t *counts, cudaStream_t s) {
    const int n_m = tr->h.n_motifs;
    int64_t n_roots = 0, root_lo = 0;
    const int32_t *roots = nullptr;
    if (args->roots) {
        n_roots = args->n_roots;
        roots = args->roots;
        if (!(args->flags & TM_ROOTS_DEVICE))
            for (int64_t i = 0; i < n_roots; i++)
                if (roots[i] < 0 || roots[i] >= g->d.E) {
                    set_error("tm_enumerate: root out of range");
                    return TM_EINVAL;
                }
    } else {
        root_lo = args->root_lo;
        const int64_t hi = (args->root_hi > 0 || args->root_lo > 0) ? args->root_hi : g->d.E;
        if (root_lo < 0 || hi > g->d.E || hi < root_lo) {
            set_error("tm_enumerate: root range outside [0, n_edges]");
            return TM_EINVAL;
        }
        n_roots = hi - root_lo;
    }
    DevTree dt;
    TM_TRY(tree_device(tr, 0, false, s, &dt));
    // scratch: found / cursor / bad-root flag, per-motif counts, host roots
    const size_t b_hdr = 256, b_cnt = sizeof(unsigned long long) * std::max(n_m, 1);
    const size_t b_roots = (args->roots && !(args->flags & TM_ROOTS_DEVICE)) ? sizeof(int32_t) * n_roots : 0;
    char *scr = nullptr;
    if (cudaMalloc(&scr, b_hdr + b_cnt + b_roots) != cudaSuccess) {
        cudaGetLastError();
        set_error("tm_enumerate: out of device memory");
        return TM_ENOMEM;
    }
    int rc = TM_OK;
    auto cuda = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TM_OK) {
            set_error(std::string("tm_enumerate: ") + cudaGetErrorString(e));
            rc = TM_ECUDA;
        }
    };
    unsigned long long *hdr = (unsigned long long *)scr;
    unsigned long long *d_cnt = (unsigned long long *)(scr + b_hdr);
    cuda(cudaMemsetAsync(scr, 0, b_hdr + b_cnt, s));
    if (b_roots) {
        int32_t *d_roots = (int32_t *)(scr + b_hdr + b_cnt);
        cuda(cudaMemcpyAsync(d_roots, roots, b_roots, cudaMemcpyHostToDevice, s));
        roots = d_roots;
    }
    if (rc == TM_OK && n_roots > 0) {
        int dev = 0, n_sm = 0, per_sm = 0;
        cuda(cudaGetDevice(&dev));
        cuda(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
        cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enum, kEnumThreads, 0));
        if (rc == TM_OK) {
            EnumParams prm{};
            prm.g = g->d;
            prm.tr = dt;
            prm.roots = roots;
            prm.n_roots = n_roots;
            prm.root_lo = root_lo;
            prm.out = out;
            prm.cap = cap;
            prm.found = hdr;
            prm.counts = d_cnt;
            const int64_t want = (n_roots + kEnumWarps - 1) / kEnumWarps;   // one warp per root at most
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)n_sm * std::max(per_sm, 1), want));
            k_enum<<<blocks, kEnumThreads, 0, s>>>(prm);
            cuda(cudaGetLastError());
        }
    }
    unsigned long long h[3] = {0, 0, 0};
    std::vector<unsigned long long> hc(std::max(n_m, 1));
    cuda(cudaMemcpyAsync(h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
    cuda(cudaMemcpyAsync(hc.data(), d_cnt, b_cnt, cudaMemcpyDeviceToHost, s));
    cuda(cudaStreamSynchronize(s));
    cudaFree(scr);
    if (rc != TM_OK) return rc;
    if (h[2]) {
        set_error("tm_enumerate: root out of range");
        return TM_EINVAL;
    }
    *n_found = (int64_t)h[0];
    if (counts)
        for (int i = 0; i < n_m; i++) counts[i] = (int64_t)hc[i];
    return TM_OK;
}

}  // namespace tmo
