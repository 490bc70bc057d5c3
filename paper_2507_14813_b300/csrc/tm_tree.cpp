// Motif-Group Tree (Section 4.2; Appendix A) on the host, and its flattened
// device node table.
//
// A node is <C_N, Children(N), Q_N>: C_N is a prefix shared by every motif
// below N, each child extends C_N by the longest common continuation of its
// group, and Q_N names the motifs equal to C_N.  Grouping motifs by their
// edge at position T, reusing the node of an unsplit group and opening a new
// node per split group (Algorithm 2) yields the path-compressed trie of the
// motifs' canonical edge sequences; this file builds that trie directly:
// insert every canonical motif into an uncompressed trie, then keep only the
// root (the longest common prefix), motif ends and branch points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "tm_internal.h"

namespace tmo {
namespace {

using Edge = std::pair<int8_t, int8_t>;

struct TrieNode {
    std::map<Edge, int> next;      // ordered: lexicographic sibling order
    std::vector<int32_t> refs;
};

// Vertices relabelled in order of first appearance (edge order, source first).
std::vector<Edge> canonical(const int8_t *uv, int m, int *n_vertices) {
    std::map<int, int> lab;
    std::vector<Edge> out;
    for (int j = 0; j < m; j++) {
        int u = uv[2 * j], v = uv[2 * j + 1];
        if (!lab.count(u)) { int k = (int)lab.size(); lab[u] = k; }
        if (!lab.count(v)) { int k = (int)lab.size(); lab[v] = k; }
        out.push_back({(int8_t)lab[u], (int8_t)lab[v]});
    }
    *n_vertices = (int)lab.size();
    return out;
}

void build_chain(const std::vector<Edge> &m, const std::vector<int32_t> &refs,
                 const std::vector<int64_t> &deltas, const std::vector<int32_t> &queries, int32_t n_motifs,
                 HostTree *out) {
    HostNode n;
    n.C = m;
    n.refs = refs;
    out->nodes = {n};
    out->motif_delta = deltas;
    out->motif_query = queries;
    out->n_motifs = n_motifs;
    out->n_leaves = 1;
    out->depth = (int32_t)m.size();
    int nv = 0;
    for (auto &e : m) nv = std::max(nv, 1 + std::max<int>(e.first, e.second));
    out->max_vertices = nv;
    std::set<int64_t> ds;
    for (int32_t r : refs) ds.insert(deltas[r]);
    out->n_deltas = (int32_t)ds.size();
    out->similarity = 0.0;
}

}  // namespace

int tree_build(const int8_t *uv, const int32_t *off, int32_t n, const int64_t *delta, tm_tree **out) {
    return tree_build_q(uv, off, n, delta, nullptr, out);
}

int tree_build_q(const int8_t *uv, const int32_t *off, int32_t n, const int64_t *delta, const int32_t *query,
                 tm_tree **out) {
    if (n < 1 || !uv || !off || !delta || !out) {
        set_error("tm_tree_build: need at least one motif and non-NULL arrays");
        return TM_EINVAL;
    }
    std::vector<std::vector<Edge>> canon(n);
    int max_v = 0, depth = 0;
    std::set<int64_t> distinct;
    for (int i = 0; i < n; i++) {
        int m = off[i + 1] - off[i];
        if (m < 1) { set_error("tm_tree_build: motif " + std::to_string(i) + " is empty"); return TM_EINVAL; }
        if (m > kMaxE) {
            set_error("tm_tree_build: motif " + std::to_string(i) + " has more than TM_MAX_EDGES edges");
            return TM_EUNSUPPORTED;
        }
        const int8_t *p = uv + 2 * (int64_t)off[i];
        for (int j = 0; j < m; j++) {
            if (p[2 * j] < 0 || p[2 * j + 1] < 0) {
                set_error("tm_tree_build: negative vertex label in motif " + std::to_string(i));
                return TM_EINVAL;
            }
            if (p[2 * j] == p[2 * j + 1]) {
                set_error("tm_tree_build: self-loop edge in motif " + std::to_string(i));
                return TM_EINVAL;
            }
        }
        if (delta[i] < 0) { set_error("tm_tree_build: negative delta for motif " + std::to_string(i)); return TM_EINVAL; }
        int nv = 0;
        canon[i] = canonical(p, m, &nv);
        if (nv > kMaxV) {
            set_error("tm_tree_build: motif " + std::to_string(i) + " has more than TM_MAX_VERTICES vertices");
            return TM_EUNSUPPORTED;
        }
        max_v = std::max(max_v, nv);
        depth = std::max(depth, m);
        distinct.insert(delta[i]);
    }
    if ((int)distinct.size() > TM_MAX_DELTAS) {
        set_error("tm_tree_build: more than TM_MAX_DELTAS distinct windows");
        return TM_EUNSUPPORTED;
    }

    // uncompressed trie of canonical edge sequences
    std::vector<TrieNode> trie(1);
    for (int i = 0; i < n; i++) {
        int cur = 0;
        for (const Edge &e : canon[i]) {
            auto it = trie[cur].next.find(e);
            if (it == trie[cur].next.end()) {
                trie.push_back(TrieNode());
                int nx = (int)trie.size() - 1;
                trie[cur].next[e] = nx;
                cur = nx;
            } else {
                cur = it->second;
            }
        }
        trie[cur].refs.push_back(i);
    }

    // compress: root at the longest common prefix, then keep motif ends and branch points
    std::unique_ptr<tm_tree> tr(new tm_tree());
    HostTree &h = tr->h;
    h.n_motifs = n;
    h.depth = depth;
    h.max_vertices = max_v;
    h.n_deltas = (int32_t)distinct.size();
    h.motif_delta.assign(delta, delta + n);
    if (query) {
        for (int i = 0; i < n; i++)
            if (query[i] < 0 || query[i] > 63) { set_error("tree: query index outside 0..63"); return TM_EINVAL; }
        h.motif_query.assign(query, query + n);
    }
    std::vector<Edge> path;
    int cur = 0;
    while (trie[cur].refs.empty() && trie[cur].next.size() == 1) {
        path.push_back(trie[cur].next.begin()->first);
        cur = trie[cur].next.begin()->second;
    }
    struct Item { int trie_node; std::vector<Edge> C; int parent; };
    // preorder via explicit stack (children pushed in reverse to pop in order)
    std::vector<Item> stack;
    stack.push_back({cur, path, -1});
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        int idx = (int)h.nodes.size();
        HostNode hn;
        hn.C = it.C;
        hn.refs = trie[it.trie_node].refs;
        hn.parent = it.parent;
        h.nodes.push_back(hn);
        if ((int)h.nodes.size() > TM_MAX_NODES) {
            set_error("tm_tree_build: more than TM_MAX_NODES tree nodes");
            return TM_EUNSUPPORTED;
        }
        if (it.parent >= 0) h.nodes[it.parent].children.push_back(idx);
        std::vector<Item> kids;
        for (auto &kv : trie[it.trie_node].next) {
            std::vector<Edge> C = it.C;
            C.push_back(kv.first);
            int c = kv.second;
            while (trie[c].refs.empty() && trie[c].next.size() == 1) {
                C.push_back(trie[c].next.begin()->first);
                c = trie[c].next.begin()->second;
            }
            kids.push_back({c, C, idx});
        }
        for (auto r = kids.rbegin(); r != kids.rend(); ++r) stack.push_back(*r);
    }
    // children were appended in pop order, which is lexicographic
    int64_t num = 0, den = 0;
    for (auto &nd : h.nodes) {
        num += (int64_t)nd.C.size() - (nd.parent >= 0 ? (int64_t)h.nodes[nd.parent].C.size() : 0);
        if (nd.children.empty()) h.n_leaves++;
        if (!nd.refs.empty()) den += (int64_t)nd.C.size();
    }
    h.similarity = 1.0 - (double)num / (double)den;

    // per-motif chains: one node per distinct canonical motif
    for (size_t i = 0; i < h.nodes.size(); i++) {
        const HostNode &nd = h.nodes[i];
        if (nd.refs.empty()) continue;
        HostTree c;
        build_chain(nd.C, nd.refs, h.motif_delta, h.motif_query, n, &c);
        tr->chains.push_back(c);
    }
    tr->dev[0].resize(1 + tr->chains.size());
    tr->dev[1].resize(1 + tr->chains.size());
    tr->mutex = new std::mutex();
    tree_image(h, true, &tr->image);
    *out = tr.release();
    return TM_OK;
}

namespace {

// Flatten a host tree into the device table.  Nodes are renumbered
// breadth-first so that each node's children are contiguous; among them the
// children descended one candidate at a time come first and the single-edge
// leaves counted in parallel last.
void flatten(const HostTree &h, bool par_leaves, TreeImage *img) {
    const int nn = (int)h.nodes.size();
    // distinct windows and per-motif delta index
    std::vector<int64_t> ds;
    for (auto &nd : h.nodes)
        for (int32_t r : nd.refs) ds.push_back(h.motif_delta[r]);
    std::sort(ds.begin(), ds.end());
    ds.erase(std::unique(ds.begin(), ds.end()), ds.end());
    auto didx = [&](int64_t x) { return (int)(std::lower_bound(ds.begin(), ds.end(), x) - ds.begin()); };

    // subtree max window and subtree queries
    auto qof = [&](int32_t r) { return h.motif_query.empty() ? 0 : h.motif_query[r]; };
    std::vector<int> dmax(nn, -1);
    std::vector<uint64_t> qmask(nn, 0);
    for (int i = nn - 1; i >= 0; i--) {  // preorder: children after parents
        for (int32_t r : h.nodes[i].refs) {
            dmax[i] = std::max(dmax[i], didx(h.motif_delta[r]));
            qmask[i] |= 1ull << qof(r);
        }
        for (int32_t c : h.nodes[i].children) {
            dmax[i] = std::max(dmax[i], dmax[c]);
            qmask[i] |= qmask[c];
        }
    }
    auto nvb_of = [&](const std::vector<Edge> &C, int k) {
        int nv = 0;
        for (int j = 0; j < k; j++) nv = std::max(nv, 1 + std::max<int>(C[j].first, C[j].second));
        return nv;
    };
    auto is_par = [&](int i) {
        const HostNode &nd = h.nodes[i];
        int m = (int)nd.C.size();
        if (!par_leaves || !nd.children.empty() || m < 2) return false;
        int nvb = nvb_of(nd.C, m - 1);
        const Edge &e = nd.C[m - 1];
        return e.first < nvb || e.second < nvb;   // connected last edge
    };
    // The last edge extends the same candidate list as the edge before it
    // (same mapped centre, new far end), so its candidates are the later
    // entries of that list minus the new vertex's own repeats.
    auto is_star = [&](int i) {
        const HostNode &nd = h.nodes[i];
        int m = (int)nd.C.size();
        if (m < 2) return false;
        const Edge &e2 = nd.C[m - 2], &e1 = nd.C[m - 1];
        int nv2 = nvb_of(nd.C, m - 2), nv1 = nvb_of(nd.C, m - 1);
        bool out = e2.first < nv2 && e2.second >= nv2 && e1.first == e2.first && e1.second >= nv1;
        bool in = e2.second < nv2 && e2.first >= nv2 && e1.second == e2.second && e1.first >= nv1;
        return out || in;
    };
    // BFS order with seq children before par children
    std::vector<int> order;
    std::vector<int> newid(nn, -1);
    order.push_back(0);
    newid[0] = 0;
    for (size_t q = 0; q < order.size(); q++) {
        int i = order[q];
        const HostNode &nd = h.nodes[i];
        for (int pass = 0; pass < 2; pass++)
            for (int32_t c : nd.children) {
                bool par1 = is_par(c) && h.nodes[c].C.size() == nd.C.size() + 1;
                if ((pass == 0) == !par1) {
                    newid[c] = (int)order.size();
                    order.push_back(c);
                }
            }
    }
    std::vector<DevNode> nodes(nn);
    std::vector<DevRef> refs;
    for (int q = 0; q < nn; q++) {
        int i = order[q];
        const HostNode &nd = h.nodes[i];
        DevNode &dn = nodes[q];
        memset(&dn, 0, sizeof(dn));
        int m = (int)nd.C.size();
        dn.k_begin = (int8_t)(nd.parent >= 0 ? h.nodes[nd.parent].C.size() : 0);
        dn.k_end = (int8_t)m;
        dn.flags = is_par(i) ? kNodeParLeaf : 0;
        if (is_par(i) && is_star(i)) dn.flags |= kNodeStarLeaf;
        for (int32_t c : nd.children)
            if (is_par(c) && is_star(c) && h.nodes[c].C.size() == nd.C.size() + 1) dn.flags |= kNodeStarKids;
        dn.dmax = (int8_t)std::max(dmax[i], 0);
        dn.qmask = qmask[i];
        dn.parent = (int16_t)(nd.parent >= 0 ? newid[nd.parent] : -1);
        int n_par = 0, n_seq = 0;
        for (int32_t c : nd.children) {
            bool par1 = is_par(c) && h.nodes[c].C.size() == nd.C.size() + 1;
            if (par1) n_par++; else n_seq++;
        }
        dn.n_seq = (int8_t)n_seq;
        dn.n_par = (int8_t)n_par;
        dn.child_begin = (int16_t)(nd.children.empty() ? 0 : newid[nd.children[0]]);
        if (!nd.children.empty()) {
            int lo = nn;
            for (int32_t c : nd.children) lo = std::min(lo, newid[c]);
            dn.child_begin = (int16_t)lo;
        }
        for (int k = 0; k < m; k++) {
            dn.eu[k] = (uint8_t)nd.C[k].first;
            dn.ev[k] = (uint8_t)nd.C[k].second;
            dn.nvb[k] = (uint8_t)nvb_of(nd.C, k);
        }
        dn.ref_begin = (int16_t)refs.size();
        dn.n_ref = (int16_t)nd.refs.size();
        for (int32_t r : nd.refs) refs.push_back(DevRef{r, (int16_t)didx(h.motif_delta[r]), (int16_t)qof(r)});
    }
    std::vector<int8_t> qd(64, -1);
    for (const DevRef &r : refs) qd[r.query] = (int8_t)std::max<int>(qd[r.query], r.delta);
    size_t b_nodes = sizeof(DevNode) * nodes.size();
    size_t b_refs = sizeof(DevRef) * std::max<size_t>(refs.size(), 1);
    size_t b_ds = sizeof(int64_t) * std::max<size_t>(ds.size(), 1);
    img->o_refs = (b_nodes + 255) / 256 * 256;
    img->o_deltas = img->o_refs + (b_refs + 255) / 256 * 256;
    img->o_qdmax = img->o_deltas + (b_ds + 255) / 256 * 256;
    img->bytes.assign(img->o_qdmax + 64, 0);
    memcpy(img->bytes.data() + img->o_qdmax, qd.data(), 64);
    memcpy(img->bytes.data(), nodes.data(), b_nodes);
    if (!refs.empty()) memcpy(img->bytes.data() + img->o_refs, refs.data(), sizeof(DevRef) * refs.size());
    if (!ds.empty()) memcpy(img->bytes.data() + img->o_deltas, ds.data(), sizeof(int64_t) * ds.size());
    img->n_nodes = nn;
    img->n_refs = (int32_t)refs.size();
    img->n_deltas = (int32_t)ds.size();
    img->n_counters = h.n_motifs;
}

int upload(const HostTree &h, bool par_leaves, DevTree *d, void **mem) {
    TreeImage img;
    flatten(h, par_leaves, &img);
    const size_t total = img.bytes.size();
    char *dev = nullptr;
    TM_CUDA_TRY(cudaMalloc(&dev, total));
    cudaError_t e = cudaMemcpy(dev, img.bytes.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        set_error(std::string("tree upload: ") + cudaGetErrorString(e));
        return TM_ECUDA;
    }
    *d = image_tree(img, dev);
    *mem = dev;
    return TM_OK;
}

}  // namespace

void tree_image(const HostTree &h, bool par_leaves, TreeImage *img) { flatten(h, par_leaves, img); }

DevTree image_tree(const TreeImage &img, const void *dev) {
    DevTree d;
    const char *b = (const char *)dev;
    d.nodes = (const DevNode *)b;
    d.refs = (const DevRef *)(b + img.o_refs);
    d.deltas = (const int64_t *)(b + img.o_deltas);
    d.qdmax = (const int8_t *)(b + img.o_qdmax);
    d.n_nodes = img.n_nodes;
    d.n_refs = img.n_refs;
    d.n_deltas = img.n_deltas;
    d.n_counters = img.n_counters;
    return d;
}

int tree_device(const tm_tree *trc, int which, bool par_leaves, cudaStream_t s, DevTree *out) {
    (void)s;
    tm_tree *tr = const_cast<tm_tree *>(trc);
    std::lock_guard<std::mutex> lk(*(std::mutex *)tr->mutex);
    DevTreeCache &c = tr->dev[par_leaves ? 1 : 0][which];
    if (!c.ready) {
        const HostTree &h = which == 0 ? tr->h : tr->chains[which - 1];
        TM_TRY(upload(h, par_leaves, &c.d, &c.mem));
        c.ready = true;
    }
    *out = c.d;
    return TM_OK;
}

void tree_release(tm_tree *tr) {
    if (!tr) return;
    for (int m = 0; m < 2; m++)
        for (auto &c : tr->dev[m])
            if (c.mem) cudaFree(c.mem);
    delete (std::mutex *)tr->mutex;
}

}  // namespace tmo
