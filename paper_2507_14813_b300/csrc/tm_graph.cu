// Graph ingest on the device: order the edge list, build the time-sorted
// out- and in-lists and the (src, dst) pair index.
//
// The temporal graph of Section 2 is an edge list in chronological order;
// the workflow's preprocessing step (Section 4.1) turns it into per-vertex
// adjacency whose entries are in ascending time, so that every candidate
// list of MatchEdge (Algorithm 1) is a contiguous range.  Here the order is
// (t, input index) and an adjacency entry is (other endpoint, edge id).
//
// All ordering is done by one primitive: a stable LSD radix sort of
// (key, int32 value) pairs, 8-bit digits, written here.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tm_internal.h"

namespace tmo {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------ exclusive scan (int32)

__global__ void k_scan_tile(const int32_t *in, int32_t *out, int64_t n, int32_t *tile_sums) {
    __shared__ int32_t warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        v[j] = (base + j < n) ? in[base + j] : 0;
        s += v[j];
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1 && tile_sums) tile_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    int32_t run = warp_tot[warp] + incl - s;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *tile_off) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / kScanTile];
}

// exclusive scan of n int32 values (in may equal out); returns via out
int scan_exclusive(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return TM_OK;
    int64_t tiles = cdiv(n, kScanTile);
    if (tiles == 1) {
        k_scan_tile<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        TM_CUDA_TRY(cudaGetLastError());
        return TM_OK;
    }
    int32_t *sums = nullptr;
    TM_CUDA_TRY(cudaMallocAsync(&sums, sizeof(int32_t) * tiles, s));
    k_scan_tile<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums);
    TM_CUDA_TRY(cudaGetLastError());
    int rc = scan_exclusive(sums, sums, tiles, s);
    if (rc == TM_OK) {
        k_scan_add<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(out, n, sums);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = TM_ECUDA; }
    }
    cudaFreeAsync(sums, s);
    return rc;
}

// ------------------------------------------------------------ stable LSD radix sort

template <typename K>
__global__ void k_rs_hist(const K *keys, int64_t n, int shift, int32_t *hist, int64_t tiles) {
    __shared__ int32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int j = 0; j < kRsItems; j++) {
        int64_t i = base + (int64_t)j * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & 255)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * tiles + blockIdx.x] = h[d];
}

// Each warp owns a contiguous run of 32*kRsItems items and walks it in order
// in rounds of 32, so ranks within a digit follow input order (stability).
template <typename K>
__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(const K *keys, const int32_t *vals, int64_t n, int shift, const int32_t *offs,
             int64_t tiles, K *keys_out, int32_t *vals_out) {
    __shared__ int32_t wcnt[kRsWarps][256];
    __shared__ int32_t boff[256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) boff[d] = offs[(int64_t)d * tiles + blockIdx.x];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)warp * (32 * kRsItems);
    const unsigned lt = (1u << lane) - 1u;
    K k[kRsItems];
    int32_t v[kRsItems];
    int32_t rank[kRsItems];
    int16_t dig[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; r++) {
        int64_t i = base + r * 32 + lane;
        int d = 256;
        if (i < n) {
            k[r] = keys[i];
            v[r] = vals[i];
            d = (int)((k[r] >> shift) & 255);
        }
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = d < 256 ? wcnt[warp][d] : 0;
        __syncwarp();
        if (d < 256 && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
        dig[r] = (int16_t)d;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int acc = 0;
        for (int w = 0; w < kRsWarps; w++) {
            int c = wcnt[w][d];
            wcnt[w][d] = acc;
            acc += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsItems; r++) {
        int d = dig[r];
        if (d < 256) {
            int64_t pos = (int64_t)boff[d] + wcnt[warp][d] + rank[r];
            keys_out[pos] = k[r];
            vals_out[pos] = v[r];
        }
    }
}

// Sort (keys, vals) by the low `bits` bits of the key, stably.  Result ends
// in (*keys, *vals); the other pair of buffers is scratch.
template <typename K>
int radix_sort(K **keys, int32_t **vals, K **keys_alt, int32_t **vals_alt, int64_t n, int bits,
               cudaStream_t s) {
    if (n <= 1 || bits <= 0) return TM_OK;
    int64_t tiles = cdiv(n, kRsTile);
    int32_t *hist = nullptr;
    TM_CUDA_TRY(cudaMallocAsync(&hist, sizeof(int32_t) * 256 * tiles, s));
    int rc = TM_OK;
    for (int shift = 0; shift < bits && rc == TM_OK; shift += 8) {
        k_rs_hist<K><<<(unsigned)tiles, kRsThreads, 0, s>>>(*keys, n, shift, hist, tiles);
        rc = scan_exclusive(hist, hist, 256 * tiles, s);
        if (rc != TM_OK) break;
        k_rs_scatter<K><<<(unsigned)tiles, kRsThreads, 0, s>>>(*keys, *vals, n, shift, hist, tiles,
                                                              *keys_alt, *vals_alt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); rc = TM_ECUDA; }
        std::swap(*keys, *keys_alt);
        std::swap(*vals, *vals_alt);
    }
    cudaFreeAsync(hist, s);
    return rc;
}

int bit_width(uint64_t x) {
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}

// ------------------------------------------------------------ helper kernels

__global__ void k_iota(int32_t *v, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

__global__ void k_validate(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t n,
                           int32_t V, int check_sorted, unsigned long long *tmin,
                           unsigned long long *tmax, int *bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = src[i], b = dst[i];
    if (a < 0 || a >= V || b < 0 || b >= V) atomicOr(bad, 1);
    if (check_sorted && i > 0 && t[i - 1] > t[i]) atomicOr(bad, 2);
    // order-preserving map of int64 to uint64
    unsigned long long u = (unsigned long long)t[i] ^ 0x8000000000000000ull;
    atomicMin(tmin, u);
    atomicMax(tmax, u);
}

__global__ void k_time_keys(const int64_t *t, int64_t n, const unsigned long long *tmin, uint64_t *key) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) key[i] = ((unsigned long long)t[i] ^ 0x8000000000000000ull) - *tmin;
}

__global__ void k_gather_edges(const int32_t *order, int64_t n, const int32_t *src, const int32_t *dst,
                               const int64_t *t, int32_t *src_o, int32_t *dst_o, int64_t *t_o) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t j = order[i];
    src_o[i] = src[j];
    dst_o[i] = dst[j];
    t_o[i] = t[j];
}

__global__ void k_gather_u32(const int32_t *idx, const int32_t *from, int64_t n, uint32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)from[idx[i]];
}

__global__ void k_copy_u32(const int32_t *from, int64_t n, uint32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)from[i];
}

// off[v] = first position whose key >= v, for v in [0, V]
__global__ void k_offsets(const uint32_t *key, int64_t n, int32_t V, int64_t *off) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    int64_t prev = i == 0 ? -1 : (int64_t)key[i - 1];
    int64_t cur = i == n ? (int64_t)V : (int64_t)key[i];
    for (int64_t v = prev + 1; v <= cur; v++) off[v] = i;
}

__global__ void k_adj(const int32_t *eids, const int32_t *other, int64_t n, int2 *adj) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int32_t e = eids[i];
        adj[i] = make_int2(other[e], e);
    }
}

// after[e] = first position in the list of vertex key[e] whose edge id exceeds e
__global__ void k_after(const int32_t *key, int64_t n, const int64_t *off, const int2 *adj, int32_t *after) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int32_t x = key[e];
    int64_t lo = off[x], hi = off[x + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (adj[mid].y <= (int32_t)e) lo = mid + 1; else hi = mid;
    }
    after[e] = (int32_t)lo;
}

__global__ void k_pair_starts(const int32_t *pe, int64_t n, const int32_t *src, const int32_t *dst,
                              int32_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t e = pe[i];
    int f = 1;
    if (i > 0) {
        int32_t q = pe[i - 1];
        f = (src[q] != src[e]) || (dst[q] != dst[e]);
    }
    flag[i] = f;
}

__global__ void k_pair_compact(const int32_t *flag, const int32_t *pos, int64_t n, int32_t *starts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) starts[pos[i]] = (int32_t)i;
}

__global__ void k_pair_insert(const int32_t *starts, int64_t n_pairs, int64_t n, const int32_t *pe,
                              const int32_t *src, const int32_t *dst, ulonglong2 *tab, uint64_t mask,
                              int *bad) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pairs) return;
    int64_t st = starts[j];
    int64_t en = j + 1 < n_pairs ? starts[j + 1] : n;
    int32_t e = pe[st];
    unsigned long long key = ((unsigned long long)(uint32_t)src[e] << 32) | (uint32_t)dst[e];
    uint64_t h = pair_hash(key) & mask;
    for (uint64_t probe = 0; probe <= mask; probe++) {
        unsigned long long prev = atomicCAS(&tab[h].x, kEmptyKey, key);
        if (prev == kEmptyKey) {
            tab[h].y = (unsigned long long)st | ((unsigned long long)(en - st) << 32);
            return;
        }
        h = (h + 1) & mask;
    }
    atomicOr(bad, 4);
}

// pr_pos[e] = position of e in pair order; pr_end[e] = end of its run
__global__ void k_pair_pos(const int32_t *pe, int64_t n, const int32_t *starts, int64_t n_pairs,
                           int32_t *pr_pos, int32_t *pr_end) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t lo = 0, hi = n_pairs;      // last run start <= i
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (starts[mid] <= i) lo = mid; else hi = mid;
    }
    int32_t e = pe[i];
    pr_pos[e] = (int32_t)i;
    pr_end[e] = (int32_t)(lo + 1 < n_pairs ? starts[lo + 1] : n);
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_max_degree(const int64_t *off, int32_t V, unsigned long long *mx) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V) atomicMax(mx, (unsigned long long)(off[v + 1] - off[v]));
}

struct Scratch {
    std::vector<void *> ptrs;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename T>
    int get(T **p, int64_t n) {
        void *q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, sizeof(T) * (size_t)std::max<int64_t>(n, 1), s);
        if (e != cudaSuccess) {
            set_error(std::string("scratch allocation: ") + cudaGetErrorString(e));
            return TM_ENOMEM;
        }
        ptrs.push_back(q);
        *p = (T *)q;
        return TM_OK;
    }
};

template <typename T>
int keep(tm_graph *g, T **p, int64_t n) {
    void *q = nullptr;
    size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(n, 1);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_error(std::string("graph allocation: ") + cudaGetErrorString(e));
        return TM_ENOMEM;
    }
    g->allocs.push_back(q);
    g->bytes += (int64_t)bytes;
    *p = (T *)q;
    return TM_OK;
}

unsigned grid(int64_t n, int b = 256) { return (unsigned)std::max<int64_t>(1, cdiv(n, b)); }

}  // namespace

// Stable sort of (uint32 key, int32 value) pairs by the low `bits` bits of the
// key; the result is left in (keys, vals).
int sort_u32_pairs(uint32_t *keys, int32_t *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1) return TM_OK;
    uint32_t *k2 = nullptr;
    int32_t *v2 = nullptr;
    TM_CUDA_TRY(cudaMallocAsync((void **)&k2, sizeof(uint32_t) * n, s));
    cudaError_t e = cudaMallocAsync((void **)&v2, sizeof(int32_t) * n, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(k2, s);
        set_error("sort: allocation");
        return TM_ENOMEM;
    }
    uint32_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    int rc = radix_sort<uint32_t>(&ka, &va, &kb, &vb, n, bits, s);
    if (rc == TM_OK && ka != keys) {
        cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
    cudaFreeAsync(k2, s);
    cudaFreeAsync(v2, s);
    return rc;
}

void graph_release(tm_graph *g) {
    if (!g) return;
    for (void *p : g->allocs) cudaFree(p);
    g->allocs.clear();
}

static int graph_build_impl(const int32_t *src_in, const int32_t *dst_in, const int64_t *t_in, int64_t E,
                            int32_t V, uint32_t flags, cudaStream_t s, tm_graph *g) {
    Scratch sc(s);
    DevGraph &d = g->d;
    d.E = E;
    d.V = V;
    int32_t *src, *dst;
    int64_t *t;
    TM_TRY(keep(g, &src, E));
    TM_TRY(keep(g, &dst, E));
    TM_TRY(keep(g, &t, E));

    // stage the input on the device
    const int32_t *s0 = src_in, *d0 = dst_in;
    const int64_t *t0 = t_in;
    cudaMemcpyKind kind = (flags & TM_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    bool presorted = (flags & TM_PRESORTED) != 0;
    int32_t *ss = src, *dd = dst;
    int64_t *tt = t;
    if (!presorted) {  // unsorted input lands in scratch, then is gathered in order
        TM_TRY(sc.get(&ss, E));
        TM_TRY(sc.get(&dd, E));
        TM_TRY(sc.get(&tt, E));
    }
    if (E > 0) {
        TM_CUDA_TRY(cudaMemcpyAsync(ss, s0, sizeof(int32_t) * E, kind, s));
        TM_CUDA_TRY(cudaMemcpyAsync(dd, d0, sizeof(int32_t) * E, kind, s));
        TM_CUDA_TRY(cudaMemcpyAsync(tt, t0, sizeof(int64_t) * E, kind, s));
    }
    unsigned long long *tminmax;
    int *bad;
    TM_TRY(sc.get(&tminmax, 2));
    TM_TRY(sc.get(&bad, 1));
    unsigned long long init[2] = {~0ull, 0ull};
    TM_CUDA_TRY(cudaMemcpyAsync(tminmax, init, sizeof(init), cudaMemcpyHostToDevice, s));
    TM_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (E > 0) {
        k_validate<<<grid(E), 256, 0, s>>>(ss, dd, tt, E, V, presorted ? 1 : 0, tminmax, tminmax + 1, bad);
        TM_CUDA_TRY(cudaGetLastError());
    }
    int hbad = 0;
    unsigned long long hmm[2];
    TM_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    TM_CUDA_TRY(cudaMemcpyAsync(hmm, tminmax, sizeof(hmm), cudaMemcpyDeviceToHost, s));
    TM_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad & 1) { set_error("tm_graph_load: vertex id outside [0, n_nodes)"); return TM_EINVAL; }
    if (hbad & 2) { set_error("tm_graph_load: TM_PRESORTED given but timestamps decrease"); return TM_EINVAL; }

    int32_t *ia, *ib;  // value buffers
    TM_TRY(sc.get(&ia, E));
    TM_TRY(sc.get(&ib, E));
    if (!presorted && E > 1) {
        uint64_t *ka, *kb;
        TM_TRY(sc.get(&ka, E));
        TM_TRY(sc.get(&kb, E));
        k_time_keys<<<grid(E), 256, 0, s>>>(tt, E, tminmax, ka);
        k_iota<<<grid(E), 256, 0, s>>>(ia, E);
        TM_CUDA_TRY(cudaGetLastError());
        int bits = bit_width(hmm[1] - hmm[0]);
        TM_TRY(radix_sort<uint64_t>(&ka, &ia, &kb, &ib, E, bits, s));
        k_gather_edges<<<grid(E), 256, 0, s>>>(ia, E, ss, dd, tt, src, dst, t);
        TM_CUDA_TRY(cudaGetLastError());
    } else if (!presorted && E == 1) {
        TM_CUDA_TRY(cudaMemcpyAsync(src, ss, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        TM_CUDA_TRY(cudaMemcpyAsync(dst, dd, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        TM_CUDA_TRY(cudaMemcpyAsync(t, tt, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    }
    d.src = src;
    d.dst = dst;
    d.t = t;

    // adjacency: stable sort of eids by src (out) and by dst (in)
    int vbits = bit_width((uint64_t)(V > 1 ? V - 1 : 1));
    uint32_t *ka, *kb;
    TM_TRY(sc.get(&ka, E));
    TM_TRY(sc.get(&kb, E));
    int64_t *out_off, *in_off;
    int2 *out_adj, *in_adj;
    TM_TRY(keep(g, &out_off, (int64_t)V + 1));
    TM_TRY(keep(g, &in_off, (int64_t)V + 1));
    TM_TRY(keep(g, &out_adj, E));
    TM_TRY(keep(g, &in_adj, E));

    // out-lists
    k_copy_u32<<<grid(E), 256, 0, s>>>(src, E, ka);
    k_iota<<<grid(E), 256, 0, s>>>(ia, E);
    TM_CUDA_TRY(cudaGetLastError());
    TM_TRY(radix_sort<uint32_t>(&ka, &ia, &kb, &ib, E, vbits, s));
    k_offsets<<<grid(E + 1), 256, 0, s>>>(ka, E, V, out_off);
    k_adj<<<grid(E), 256, 0, s>>>(ia, dst, E, out_adj);
    TM_CUDA_TRY(cudaGetLastError());

    // in-lists
    k_copy_u32<<<grid(E), 256, 0, s>>>(dst, E, ka);
    k_iota<<<grid(E), 256, 0, s>>>(ia, E);
    TM_CUDA_TRY(cudaGetLastError());
    TM_TRY(radix_sort<uint32_t>(&ka, &ia, &kb, &ib, E, vbits, s));
    k_offsets<<<grid(E + 1), 256, 0, s>>>(ka, E, V, in_off);
    k_adj<<<grid(E), 256, 0, s>>>(ia, src, E, in_adj);
    TM_CUDA_TRY(cudaGetLastError());

    // pair order: the in-order (dst, eid) re-sorted stably by src gives (src, dst, eid)
    k_gather_u32<<<grid(E), 256, 0, s>>>(ia, src, E, ka);
    TM_CUDA_TRY(cudaGetLastError());
    TM_TRY(radix_sort<uint32_t>(&ka, &ia, &kb, &ib, E, vbits, s));
    int32_t *pair_eid;
    TM_TRY(keep(g, &pair_eid, E));
    if (E > 0) TM_CUDA_TRY(cudaMemcpyAsync(pair_eid, ia, sizeof(int32_t) * E, cudaMemcpyDeviceToDevice, s));

    // runs of equal (src, dst) -> hash table
    int32_t *flag, *pos;
    TM_TRY(sc.get(&flag, E));
    TM_TRY(sc.get(&pos, E));
    int64_t n_pairs = 0;
    if (E > 0) {
        k_pair_starts<<<grid(E), 256, 0, s>>>(pair_eid, E, src, dst, flag);
        TM_CUDA_TRY(cudaGetLastError());
        TM_TRY(scan_exclusive(flag, pos, E, s));
        int32_t last_pos = 0, last_flag = 0;
        TM_CUDA_TRY(cudaMemcpyAsync(&last_pos, pos + E - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TM_CUDA_TRY(cudaMemcpyAsync(&last_flag, flag + E - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TM_CUDA_TRY(cudaStreamSynchronize(s));
        n_pairs = (int64_t)last_pos + last_flag;
    }
    uint64_t cap = 16;
    while (cap < (uint64_t)(2 * n_pairs)) cap <<= 1;
    ulonglong2 *tab;
    TM_TRY(keep(g, &tab, (int64_t)cap));
    k_fill_u64<<<grid(2 * (int64_t)cap), 256, 0, s>>>((unsigned long long *)tab, 2 * (int64_t)cap, kEmptyKey);
    TM_CUDA_TRY(cudaGetLastError());
    int32_t *pr_pos, *pr_end;
    TM_TRY(keep(g, &pr_pos, E));
    TM_TRY(keep(g, &pr_end, E));
    if (n_pairs > 0) {
        int32_t *starts;
        TM_TRY(sc.get(&starts, n_pairs));
        k_pair_compact<<<grid(E), 256, 0, s>>>(flag, pos, E, starts);
        k_pair_insert<<<grid(n_pairs), 256, 0, s>>>(starts, n_pairs, E, pair_eid, src, dst, tab, cap - 1, bad);
        k_pair_pos<<<grid(E), 256, 0, s>>>(pair_eid, E, starts, n_pairs, pr_pos, pr_end);
        TM_CUDA_TRY(cudaGetLastError());
    }
    int32_t *a_os, *a_od, *a_is, *a_id;
    TM_TRY(keep(g, &a_os, E));
    TM_TRY(keep(g, &a_od, E));
    TM_TRY(keep(g, &a_is, E));
    TM_TRY(keep(g, &a_id, E));
    if (E > 0) {
        k_after<<<grid(E), 256, 0, s>>>(src, E, out_off, out_adj, a_os);
        k_after<<<grid(E), 256, 0, s>>>(dst, E, out_off, out_adj, a_od);
        k_after<<<grid(E), 256, 0, s>>>(src, E, in_off, in_adj, a_is);
        k_after<<<grid(E), 256, 0, s>>>(dst, E, in_off, in_adj, a_id);
        TM_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long *mx;
    TM_TRY(sc.get(&mx, 2));
    TM_CUDA_TRY(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), s));
    k_max_degree<<<grid(V), 256, 0, s>>>(out_off, V, mx);
    k_max_degree<<<grid(V), 256, 0, s>>>(in_off, V, mx + 1);
    TM_CUDA_TRY(cudaGetLastError());
    unsigned long long hmx[2];
    TM_CUDA_TRY(cudaMemcpyAsync(hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
    TM_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    TM_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad & 4) { set_error("tm_graph_load: pair table overflow"); return TM_ECUDA; }

    d.out_off = out_off;
    d.in_off = in_off;
    d.out_adj = out_adj;
    d.in_adj = in_adj;
    d.pair_eid = pair_eid;
    d.pr_pos = pr_pos;
    d.pr_end = pr_end;
    d.after_os = a_os;
    d.after_od = a_od;
    d.after_is = a_is;
    d.after_id = a_id;
    d.pair_tab = tab;
    d.pair_mask = cap - 1;
    g->n_pairs = n_pairs;
    g->max_out = (int64_t)hmx[0];
    g->max_in = (int64_t)hmx[1];
    return TM_OK;
}

int graph_build(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t E, int32_t V,
                uint32_t flags, cudaStream_t s, tm_graph **out) {
    tm_graph *g = new tm_graph();
    TM_CUDA_TRY(cudaGetDevice(&g->device));
    int rc = graph_build_impl(src, dst, t, E, V, flags, s, g);
    cudaError_t e = cudaStreamSynchronize(s);
    if (rc == TM_OK && e != cudaSuccess) {
        set_error(std::string("tm_graph_load: ") + cudaGetErrorString(e));
        rc = TM_ECUDA;
    }
    if (rc != TM_OK) {
        graph_release(g);
        delete g;
        return rc;
    }
    *out = g;
    return TM_OK;
}

}  // namespace tmo
