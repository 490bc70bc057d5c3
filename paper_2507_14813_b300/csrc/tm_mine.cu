// Host side of counting: launch planning, scratch, the table-driven kernel
// and its entry points (tm_count, replay, autotuning, allocation-free
// counting).  The kernel itself is tm_kernel.cuh; its four instantiations
// are compiled in tm_kmine_*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tm_codegen.h"
#include "tm_internal.h"
#include "tm_instances.h"

namespace tmo {
using namespace dev;

namespace {

// The thread tier's first root: the tail of a planned order whose slice
// count is 0 (the plan marks roots predicted light so; counts are
// non-increasing along the order, found by binary search).
__global__ void k_tier_bound(const int32_t *split, int64_t n, QueueHdr *q) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (split[mid] > 0) lo = mid + 1; else hi = mid;
    }
    q->lane_from = lo;
}

__global__ void k_to_i64(const unsigned long long *a, int64_t *b, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int64_t)a[i];
}

__global__ void k_status(const QueueHdr *q, int n_launch, int32_t *status) {
    int e = 0;
    for (int i = 0; i < n_launch; i++) e |= q[i].error;
    *status = e;
}

// Static shared memory plus up to kSmemCounters per-CTA counters exceeds the
// default 48 KiB per block; allow the larger dynamic part once per device.
int allow_counter_smem() {
    static int done[64] = {0};
    int dev = 0;
    TM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && done[dev]) return TM_OK;
    const int bytes = (int)(sizeof(unsigned long long) * kSmemCounters);
    TM_CUDA_TRY(cudaFuncSetAttribute(mine_kernel<false, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    TM_CUDA_TRY(cudaFuncSetAttribute(mine_kernel<true, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    TM_CUDA_TRY(cudaFuncSetAttribute(mine_kernel<false, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    TM_CUDA_TRY(cudaFuncSetAttribute(mine_kernel<true, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    if (dev >= 0 && dev < 64) done[dev] = 1;
    return TM_OK;
}

// Everything a count needs besides its inputs: where the scratch lives and
// how the launches are shaped.
struct Plan {
    int n_motifs = 0, n_launch = 0;
    bool comine = true, par = true, react = false, planned = false, dynamic = false, stats = false;
    bool spec = false;                  // counting launches may use the tree's specialised kernels
    bool siblings = false;              // sibling splitting and multi-offload
    bool tiers = false;                 // the planned order's light tail runs one root per lane
    int64_t n_roots = 0, root_lo = 0;
    const int32_t *roots = nullptr;     // device
    const uint64_t *root_qmask = nullptr; // device, serving batches only
    int blocks = 0, dyn_smem = 0, n_sm = 0, ctas_cap = 0;
    bool smem_cnt = true, warp_cnt = true;
    int32_t chunk = 1;
    int poll_every = kPollEvery, donate_seq = kDonateSeq, donate_leaf = kDonateLeaf;
    size_t o_q = 0, o_tasks = 0, o_ready = 0, bytes = 0, b_ready = 0;
};

// The table-driven kernel for a launch: stats or not, extended schedules or not.
MineKernel kernel_of(bool stats, bool ext) {
    if (ext) return stats ? mine_kernel<true, true>() : mine_kernel<false, true>();
    return stats ? mine_kernel<true, false>() : mine_kernel<false, false>();
}

// roots a warp claims at a time: 1, or up to 16 when there are many roots per warp
int32_t chunk_for(int64_t n_roots, int blocks) {
    const int64_t warps_total = (int64_t)blocks * kWarps;
    return (int32_t)std::max<int64_t>(1, std::min<int64_t>(16, n_roots / (warps_total * 64)));
}

int make_plan(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, bool stats, Plan *P) {
    P->n_motifs = tr->h.n_motifs;
    P->comine = (args->mode & TM_PERMOTIF) == 0;
    P->par = (args->mode & TM_LEAF_SCAN) == 0;
    P->siblings = (args->mode & TM_SCHED_SIBLINGS) != 0;
    // the thread tier keeps a window end per window in each lane: at most kLaneDeltas
    P->tiers = (args->mode & TM_SCHED_TIERS) && (args->mode & TM_SCHED_PLANNED) && tr->h.n_deltas <= kLaneDeltas;
    P->react = (args->mode & (TM_SCHED_DYNAMIC | TM_SCHED_SIBLINGS)) != 0;
    P->planned = (args->mode & TM_SCHED_PLANNED) != 0;
    P->dynamic = P->react || P->planned;
    P->stats = stats;
    // the runtime-compiled kernels are the default schedules' (no extended ones)
    P->spec = !(args->mode & TM_GENERIC) && P->par && !stats && !(args->mode & (TM_SCHED_TIERS | TM_SCHED_SIBLINGS));
    if (P->planned && !args->root_split) {
        set_error("tm_count: TM_SCHED_PLANNED needs root_split");
        return TM_EINVAL;
    }
    if (args->roots) {
        P->n_roots = args->n_roots;
        P->root_lo = 0;
    } else {
        int64_t hi = args->root_hi > 0 ? args->root_hi : g->d.E;
        if (args->root_lo < 0 || hi > g->d.E || args->root_lo > hi) {
            set_error("tm_count: root range outside [0, n_edges]");
            return TM_EINVAL;
        }
        P->n_roots = hi - args->root_lo;
        P->root_lo = args->root_lo;
    }
    if (P->n_roots < 0) { set_error("tm_count: n_roots < 0"); return TM_EINVAL; }
    if (args->poll_every > 0) P->poll_every = args->poll_every;
    if (args->donate_seq > 0) P->donate_seq = args->donate_seq;
    if (args->donate_leaf > 0) P->donate_leaf = args->donate_leaf;
    P->n_launch = P->comine ? 1 : (int)tr->chains.size();
    const size_t b_cnt = sizeof(unsigned long long) * (size_t)(P->n_motifs + kStatFields + kBusyFields);
    P->o_q = (b_cnt + 255) / 256 * 256;
    const size_t b_q = sizeof(QueueHdr) * (size_t)P->n_launch;
    P->o_tasks = (P->o_q + b_q + 255) / 256 * 256;
    const size_t b_tasks = P->dynamic ? sizeof(Task) * kQueueCap : 0;
    P->o_ready = P->o_tasks + b_tasks;
    P->b_ready = P->dynamic ? sizeof(int) * kQueueCap : 0;
    P->bytes = P->o_ready + P->b_ready;

    int dev = 0, n_sm = 0;
    TM_CUDA_TRY(cudaGetDevice(&dev));
    TM_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    P->smem_cnt = P->n_motifs <= kSmemCounters;
    P->warp_cnt = P->n_motifs <= kWarpCounters;
    P->dyn_smem = (int)(sizeof(unsigned long long) * P->n_motifs) * (P->warp_cnt ? kWarps : P->smem_cnt ? 1 : 0);
    TM_TRY(allow_counter_smem());
    int per_sm = 0;
    TM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_of(stats, P->tiers || P->siblings),
                                                              kThreads, P->dyn_smem));
    P->ctas_cap = args->ctas_per_sm;
    P->n_sm = n_sm;
    if (args->ctas_per_sm > 0) per_sm = std::min(per_sm, (int)args->ctas_per_sm);
    per_sm = std::max(per_sm, 1);
    P->blocks = n_sm * per_sm;
    P->chunk = chunk_for(P->n_roots, P->blocks);
    return TM_OK;
}

// Launch shape of a tree-specialised kernel: its own occupancy (registers
// and shared memory are sized to the tree), capped like the table-driven one.
int spec_shape(const SpecKernel *sk, const Plan &P, int *blocks, int32_t *chunk) {
    const void *f = (const void *)sk->kern;
    TM_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(unsigned long long) * kSmemCounters)));
    int per_sm = 0;
    TM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kThreads, P.dyn_smem));
    if (P.ctas_cap > 0) per_sm = std::min(per_sm, P.ctas_cap);
    per_sm = std::max(per_sm, 1);
    *blocks = P.n_sm * per_sm;
    *chunk = chunk_for(P.n_roots, *blocks);
    return TM_OK;
}

// Enqueue a count on `s`: scratch reset, mining launches, counts (int64) to
// `counts_dev` when non-null, error bits to `status_dev` when non-null.  No
// allocation and no synchronisation, so it can be captured in a CUDA graph
// (the tree must already be on the device).
int enqueue(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, const Plan &P, char *scratch,
            int64_t *counts_dev, int32_t *status_dev, cudaStream_t s, int64_t *launches,
            const DevTree *given = nullptr) {
    unsigned long long *d_cnt = (unsigned long long *)scratch;
    unsigned long long *d_st = d_cnt + P.n_motifs;
    QueueHdr *d_q = (QueueHdr *)(scratch + P.o_q);
    Task *d_tasks = P.dynamic ? (Task *)(scratch + P.o_tasks) : nullptr;
    int *d_ready = P.dynamic ? (int *)(scratch + P.o_ready) : nullptr;
    TM_CUDA_TRY(cudaMemsetAsync(scratch, 0, P.o_tasks, s));
    if (args->per_root_counts && P.n_roots > 0)
        TM_CUDA_TRY(cudaMemsetAsync(args->per_root_counts, 0, sizeof(int64_t) * P.n_roots * P.n_motifs, s));
    if (args->per_root_work && P.n_roots > 0)
        TM_CUDA_TRY(cudaMemsetAsync(args->per_root_work, 0, sizeof(int64_t) * P.n_roots * TM_WORK_FIELDS, s));
    auto kern = kernel_of(P.stats, P.tiers || P.siblings);
    int64_t n = 0;
    for (int L = 0; L < P.n_launch && P.n_roots > 0; L++) {
        DevTree dt;
        if (given) dt = *given;
        else TM_TRY(tree_device(tr, P.comine ? 0 : 1 + L, P.par, s, &dt));
        if (P.dynamic) TM_CUDA_TRY(cudaMemsetAsync(d_ready, 0, P.b_ready, s));
        Params prm{};                 // every field not set below is zero
        prm.g = g->d;
        prm.tr = dt;
        prm.roots = P.roots;
        prm.n_roots = P.n_roots;
        prm.root_lo = P.root_lo;
        prm.counts = d_cnt;
        prm.per_root_counts = args->per_root_counts;
        prm.per_root_work = args->per_root_work;
        prm.q = d_q + L;
        prm.tasks = d_tasks;
        prm.ready = d_ready;
        prm.stats = d_st;
        prm.chunk = P.chunk;
        prm.smem_counters = P.warp_cnt ? 2 : P.smem_cnt ? 1 : 0;
        prm.dynamic = P.dynamic ? 1 : 0;
        prm.react = P.react ? 1 : 0;
        prm.split = P.planned ? args->root_split : nullptr;
        prm.poll_every = P.poll_every;
        prm.donate_seq = P.donate_seq;
        prm.donate_leaf = P.donate_leaf;
        prm.siblings = P.siblings ? 1 : 0;
        prm.sib_always = args->sibling_always ? 1 : 0;
        prm.offload_max = args->offload_max > 0 ? args->offload_max : kOffloadMax;
        prm.tiers = (P.tiers && !P.root_qmask) ? 1 : 0;
        prm.root_qmask = P.root_qmask;
        if (prm.tiers) {                         // where the thread tier starts
            k_tier_bound<<<1, 32, 0, s>>>(args->root_split, P.n_roots, d_q + L);
            TM_CUDA_TRY(cudaGetLastError());
        }
        const SpecKernel *sk = (P.spec && !P.root_qmask) ? spec_kernel(tr, P.comine ? 0 : 1 + L) : nullptr;
        cudaError_t e;
        if (sk) {                                // the kernel compiled for this tree
            int blocks = 0;
            TM_TRY(spec_shape(sk, P, &blocks, &prm.chunk));
            void *kargs[] = {&prm};
            e = cudaLaunchKernel((const void *)sk->kern, dim3(blocks), dim3(kThreads), kargs, (size_t)P.dyn_smem, s);
        } else {
            kern<<<P.blocks, kThreads, P.dyn_smem, s>>>(prm);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            set_error(std::string("tm_count: launch: ") + cudaGetErrorString(e));
            return TM_ECUDA;
        }
        n++;
    }
    if (counts_dev) {
        k_to_i64<<<(P.n_motifs + 255) / 256, 256, 0, s>>>(d_cnt, counts_dev, P.n_motifs);
        TM_CUDA_TRY(cudaGetLastError());
    }
    if (status_dev) {
        k_status<<<1, 1, 0, s>>>(d_q, P.n_launch, status_dev);
        TM_CUDA_TRY(cudaGetLastError());
    }
    if (launches) *launches = n;
    return TM_OK;
}

int check_roots(const tm_graph *g, const tm_count_args *args, int64_t n_roots) {
    if (args->roots && !(args->flags & TM_ROOTS_DEVICE)) {
        for (int64_t i = 0; i < n_roots; i++)
            if (args->roots[i] < 0 || args->roots[i] >= g->d.E) {
                set_error("tm_count: root edge id out of range");
                return TM_EINVAL;
            }
    }
    return TM_OK;
}

}  // namespace

size_t batch_scratch_bytes(const tm_graph *g, const tm_tree *tr, uint32_t mode) {
    tm_count_args a;
    memset(&a, 0, sizeof(a));
    a.mode = mode & ~(uint32_t)(TM_PERMOTIF | TM_SCHED_PLANNED);
    a.root_lo = 0;
    a.root_hi = 0;
    Plan P;
    if (make_plan(g, tr, &a, false, &P) != TM_OK) return 0;
    return P.bytes;
}

int batch_enqueue(const tm_graph *g, const tm_tree *tr, uint32_t mode, const DevTree &dt, const int32_t *d_roots,
                  const uint64_t *d_qmask, int64_t n_roots, char *scratch, int64_t *d_counts, int32_t *d_status,
                  cudaStream_t s) {
    tm_count_args a;
    memset(&a, 0, sizeof(a));
    a.mode = mode & ~(uint32_t)(TM_PERMOTIF | TM_SCHED_PLANNED);
    a.flags = TM_ROOTS_DEVICE;
    a.roots = d_roots;
    a.n_roots = n_roots;
    Plan P;
    TM_TRY(make_plan(g, tr, &a, false, &P));
    P.roots = d_roots;
    P.root_qmask = d_qmask;
    return enqueue(g, tr, &a, P, scratch, d_counts, d_status, s, nullptr, &dt);
}

int mine(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, int64_t *counts,
         tm_run_stats *stats, cudaStream_t s) {
    Plan P;
    TM_TRY(make_plan(g, tr, args, stats != nullptr, &P));
    TM_TRY(check_roots(g, args, P.n_roots));
    char *scratch = nullptr;
    TM_CUDA_TRY(cudaMallocAsync((void **)&scratch, P.bytes, s));
    void *roots_copy = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto finish = [&](int code) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (roots_copy) cudaFreeAsync(roots_copy, s);
        cudaFreeAsync(scratch, s);
        return code;
    };
    P.roots = args->roots;
    if (args->roots && !(args->flags & TM_ROOTS_DEVICE) && P.n_roots > 0) {
        if (cudaMallocAsync(&roots_copy, sizeof(int32_t) * P.n_roots, s) != cudaSuccess) {
            set_error("tm_count: root list allocation");
            return finish(TM_ENOMEM);
        }
        cudaMemcpyAsync(roots_copy, args->roots, sizeof(int32_t) * P.n_roots, cudaMemcpyHostToDevice, s);
        P.roots = (const int32_t *)roots_copy;
    }
    const bool dev_counts = (args->flags & TM_COUNTS_DEVICE) != 0;
    if (stats) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
    }
    int64_t launches = 0;
    int rc = enqueue(g, tr, args, P, scratch, nullptr, nullptr, s, &launches);
    if (rc != TM_OK) return finish(rc);
    if (stats) cudaEventRecord(e1, s);

    // error bits (expired waits, skipped device roots) come back with the
    // queue headers whenever the call synchronises anyway; the dynamic mode
    // always synchronises for them
    int64_t idle_expired = 0;
    if (P.dynamic || !dev_counts || stats) {
        std::vector<QueueHdr> hq(P.n_launch);
        cudaMemcpyAsync(hq.data(), scratch + P.o_q, sizeof(QueueHdr) * P.n_launch, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error(std::string("tm_count: ") + cudaGetErrorString(e));
            return finish(TM_ECUDA);
        }
        for (auto &q : hq) {
            idle_expired += q.idle_expired;
            if (q.error & kErrTimeout) {
                set_error("tm_count: a bounded device wait expired; counts are incomplete");
                return finish(TM_ETIMEOUT);
            }
            if (q.error & kErrBadRoot) {
                set_error("tm_count: a device root edge id is outside [0, n_edges)");
                return finish(TM_EINVAL);
            }
            if (q.error & kErrCheck) {
                set_error("tm_count: the checking build found an index outside its range; counts are incomplete");
                return finish(TM_ECHECK);
            }
        }
    }
    const unsigned long long *d_cnt = (const unsigned long long *)scratch;
    if (dev_counts) {
        k_to_i64<<<(P.n_motifs + 255) / 256, 256, 0, s>>>(d_cnt, counts, P.n_motifs);
    } else {
        std::vector<unsigned long long> h(P.n_motifs);
        cudaMemcpyAsync(h.data(), d_cnt, sizeof(unsigned long long) * P.n_motifs, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error(std::string("tm_count: ") + cudaGetErrorString(e));
            return finish(TM_ECUDA);
        }
        for (int i = 0; i < P.n_motifs; i++) counts[i] = (int64_t)h[i];
    }
    if (stats) {
        unsigned long long hs[kStatFields + kBusyFields];
        cudaMemcpyAsync(hs, d_cnt + P.n_motifs, sizeof(hs), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error(std::string("tm_count: ") + cudaGetErrorString(e));
            return finish(TM_ECUDA);
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        memset(stats, 0, sizeof(*stats));
        stats->n_roots = (int64_t)hs[kStRoots];
        stats->candidates = (int64_t)hs[kStCand];
        stats->expansions = (int64_t)hs[kStExp];
        stats->probes = (int64_t)(hs[kStListProbe] + hs[kStHashProbe] + hs[kStPairProbe]);
        stats->leaf_evals = (int64_t)hs[kStLeaf];
        stats->algo_bytes = (int64_t)(16 * hs[kStRoots] + 8 * hs[kStCand] + 8 * hs[kStListProbe] +
                                      16 * hs[kStHashProbe] + 4 * hs[kStPairProbe]);
        stats->tasks_split = (int64_t)hs[kStSplit];
        stats->algo_bytes_lists = (int64_t)(16 * hs[kStRoots] + 8 * hs[kStCand] + 12 * hs[kStLogDeg]);
        stats->roots_thread_tier = (int64_t)hs[kStLaneRoots];
        stats->roots_split = (int64_t)hs[kStSplitRoots];
        stats->idle_expired = idle_expired;
        const unsigned long long *hb = hs + kStatFields;
        stats->warp_imbalance = hb[kBusySum] ? (double)hb[kBusyMax] * (double)hb[kBusyWarps] / (double)hb[kBusySum] : 0.0;
        stats->launches = launches;
        stats->kernel_ms = ms;
    }
    return finish(TM_OK);
}

}  // namespace tmo

// ---------------------------------------------------------------------------
// Replayable counts: one tm_count configuration captured once in a CUDA graph.

struct tm_exec {
    cudaGraphExec_t exec = nullptr;
    char *scratch = nullptr;
    int32_t *status = nullptr;     // device, error bits of the last replay
};

extern "C" int tm_exec_create(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, int64_t *counts,
                              void *stream, tm_exec **out) {
    using namespace tmo;
    if (!g || !tr || !args || !counts || !out) { set_error("tm_exec_create: NULL argument"); return TM_EINVAL; }
    *out = nullptr;
    if (args->roots && !(args->flags & TM_ROOTS_DEVICE)) {
        set_error("tm_exec_create: roots must be device memory (TM_ROOTS_DEVICE)");
        return TM_EINVAL;
    }
    Plan P;
    TM_TRY(make_plan(g, tr, args, false, &P));
    P.roots = args->roots;
    cudaStream_t s = (cudaStream_t)stream;
    // trees go to the device before capture
    for (int L = 0; L < P.n_launch; L++) {
        DevTree dt;
        TM_TRY(tree_device(tr, P.comine ? 0 : 1 + L, P.par, s, &dt));
    }
    tm_exec *x = new tm_exec();
    auto fail = [&](int code) {
        if (x->exec) cudaGraphExecDestroy(x->exec);
        if (x->scratch) cudaFree(x->scratch);
        if (x->status) cudaFree(x->status);
        delete x;
        return code;
    };
    if (cudaMalloc((void **)&x->scratch, P.bytes) != cudaSuccess || cudaMalloc((void **)&x->status, 4) != cudaSuccess) {
        set_error("tm_exec_create: scratch allocation");
        return fail(TM_ENOMEM);
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("tm_exec_create: stream");
        return fail(TM_ECUDA);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = TM_OK;
    if (e == cudaSuccess) {
        rc = enqueue(g, tr, args, P, x->scratch, counts, x->status, cs, nullptr);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (rc == TM_OK && e2 != cudaSuccess) { set_error(std::string("capture: ") + cudaGetErrorString(e2)); rc = TM_ECUDA; }
    } else {
        set_error(std::string("capture: ") + cudaGetErrorString(e));
        rc = TM_ECUDA;
    }
    if (rc == TM_OK && cudaGraphInstantiate(&x->exec, graph, 0) != cudaSuccess) {
        set_error("tm_exec_create: graph instantiation");
        rc = TM_ECUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc != TM_OK) return fail(rc);
    *out = x;
    return TM_OK;
}

extern "C" int tm_exec_launch(tm_exec *x, void *stream) {
    using namespace tmo;
    if (!x) { set_error("tm_exec_launch: NULL"); return TM_EINVAL; }
    TM_CUDA_TRY(cudaGraphLaunch(x->exec, (cudaStream_t)stream));
    return TM_OK;
}

extern "C" int tm_exec_status(tm_exec *x, void *stream) {
    using namespace tmo;
    if (!x) { set_error("tm_exec_status: NULL"); return TM_EINVAL; }
    int32_t st = 0;
    TM_CUDA_TRY(cudaMemcpyAsync(&st, x->status, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (st & kErrTimeout) {
        set_error("tm_exec: a bounded device wait expired in the last replay; its counts are incomplete");
        return TM_ETIMEOUT;
    }
    if (st & kErrBadRoot) {
        set_error("tm_exec: a device root edge id is outside [0, n_edges)");
        return TM_EINVAL;
    }
    if (st & kErrCheck) {
        set_error("tm_exec: the checking build found an index outside its range");
        return TM_ECHECK;
    }
    return TM_OK;
}

extern "C" int tm_exec_free(tm_exec *x) {
    if (!x) return TM_OK;
    if (x->exec) cudaGraphExecDestroy(x->exec);
    cudaFree(x->scratch);
    cudaFree(x->status);
    delete x;
    return TM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times a small grid of launch shapes and split thresholds on the
// caller's roots and keeps the fastest (coordinate descent, best of 2 runs).

extern "C" int tm_autotune(const tm_graph *g, const tm_tree *tr, const tm_count_args *args, tm_tune *best,
                           void *stream) {
    using namespace tmo;
    if (!g || !tr || !args || !best) { set_error("tm_autotune: NULL argument"); return TM_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> counts(tr->h.n_motifs);
    tm_count_args a = *args;
    a.flags &= ~TM_COUNTS_DEVICE;
    auto timed = [&](const tm_count_args &c, float *ms) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float bestms = 1e30f;
        int rc = TM_OK;
        for (int rep = 0; rep < 2 && rc == TM_OK; rep++) {
            cudaEventRecord(e0, s);
            rc = mine(g, tr, &c, counts.data(), nullptr, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            bestms = std::min(bestms, t);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *ms = bestms;
        return rc;
    };
    tm_tune cur{0, kDonateSeq, kDonateLeaf, kPollEvery, 0.f};
    auto apply = [&](const tm_tune &t) {
        tm_count_args c = a;
        c.ctas_per_sm = t.ctas_per_sm;
        c.donate_seq = t.donate_seq;
        c.donate_leaf = t.donate_leaf;
        c.poll_every = t.poll_every;
        return c;
    };
    float cur_ms = 0;
    TM_TRY(timed(apply(cur), &cur_ms));
    const int ctas[] = {2, 3, 4};
    const int seqs[] = {32, 64, 256, 1024};
    const int leaves[] = {256, 1024, 4096};
    const int polls[] = {1, 4, 16};
    for (int pass = 0; pass < 2; pass++) {
        for (int c : ctas) { tm_tune t = cur; t.ctas_per_sm = c; float ms; TM_TRY(timed(apply(t), &ms)); if (ms < cur_ms) { cur = t; cur_ms = ms; } }
        if (!(a.mode & (TM_SCHED_DYNAMIC | TM_SCHED_SIBLINGS))) break;
        for (int v : seqs) { tm_tune t = cur; t.donate_seq = v; float ms; TM_TRY(timed(apply(t), &ms)); if (ms < cur_ms) { cur = t; cur_ms = ms; } }
        for (int v : leaves) { tm_tune t = cur; t.donate_leaf = v; float ms; TM_TRY(timed(apply(t), &ms)); if (ms < cur_ms) { cur = t; cur_ms = ms; } }
        for (int v : polls) { tm_tune t = cur; t.poll_every = v; float ms; TM_TRY(timed(apply(t), &ms)); if (ms < cur_ms) { cur = t; cur_ms = ms; } }
    }
    cur.ms = cur_ms;
    *best = cur;
    return TM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free counting.
//
// For callers that may not allocate device memory while they count: code
// that runs between the set-up and tear-down of a long-lived service with a
// fixed memory budget, under an external allocator that forbids stray
// cudaMalloc calls, or with a latency limit that an allocation could break.
// The graph and tree handles are built beforehand (that does allocate); the
// counting call below then uses only the static array that follows, which
// every GPU that loads this library holds until the process exits.
#include <mutex>

namespace tmo {
namespace {

constexpr size_t kNoAllocBytes = 256u << 10;          // 256 KiB in total
constexpr int kNoAllocMaxMotifs = 1024;               // counters: 8 KiB
constexpr size_t kNoAllocHdr = 8u << 10;              // queue header at 8 KiB
constexpr size_t kNoAllocTree = 16u << 10;            // tree image from 16 KiB to the end
constexpr size_t kNoAllocMaxTree = kNoAllocBytes - kNoAllocTree;
constexpr int kNoAllocMaxDevices = 64;

// the largest tree image: TM_MAX_NODES nodes, one ref per motif, the window
// and query tables, each section 256-byte aligned
static_assert(sizeof(DevNode) * TM_MAX_NODES + 256 + sizeof(DevRef) * kNoAllocMaxMotifs + 256 +
                      sizeof(int64_t) * TM_MAX_DELTAS + 256 + 64 + 256 <= kNoAllocMaxTree,
              "every tree within the limits fits the static scratch");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices];

// Device address of the static array on the current device, looked up once
// per device and cached: the cache assumes the device's primary context is
// not reset (cudaDeviceReset) while the library is loaded.
int noalloc_scratch(int dev, void **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error(std::string("tm_count_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return TM_ECUDA;
        }
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return TM_OK;
}

}  // namespace
}  // namespace tmo

extern "C" int tm_count_noalloc(const tm_graph *g, const tm_tree *tr, const int32_t *roots, int64_t n_roots,
                                int64_t root_lo, int64_t root_hi, int64_t *counts, void *stream) {
    using namespace tmo;
    if (!g || !tr || !counts) { set_error("tm_count_noalloc: NULL argument"); return TM_EINVAL; }
    const int n_motifs = tr->h.n_motifs;
    if (n_motifs > kNoAllocMaxMotifs) {
        set_error("tm_count_noalloc: more than 1024 motifs do not fit its static scratch");
        return TM_EUNSUPPORTED;
    }
    const TreeImage &img = tr->image;
    if (img.bytes.size() > kNoAllocMaxTree) {   // cannot happen within the limits (static_assert above)
        set_error("tm_count_noalloc: tree node table larger than its static scratch");
        return TM_EUNSUPPORTED;
    }
    if (roots) {
        if (n_roots < 0) { set_error("tm_count_noalloc: n_roots < 0"); return TM_EINVAL; }
    } else {
        int64_t hi = root_hi > 0 ? root_hi : g->d.E;
        if (root_lo < 0 || hi > g->d.E || root_lo > hi) {
            set_error("tm_count_noalloc: root range outside [0, n_edges]");
            return TM_EINVAL;
        }
        n_roots = hi - root_lo;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    TM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) { set_error("tm_count_noalloc: device index too large"); return TM_EUNSUPPORTED; }
    void *base = nullptr;
    TM_TRY(noalloc_scratch(dev, &base));
    char *b = (char *)base;
    unsigned long long *d_cnt = (unsigned long long *)b;
    QueueHdr *d_q = (QueueHdr *)(b + kNoAllocHdr);
    // counters and the root cursor start at zero on every call
    TM_CUDA_TRY(cudaMemsetAsync(b, 0, kNoAllocTree, s));
    TM_CUDA_TRY(cudaMemcpyAsync(b + kNoAllocTree, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, s));
    if (n_roots > 0) {
        int n_sm = 0, per_sm = 0;
        TM_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
        const int dyn_smem = (int)(sizeof(unsigned long long) * n_motifs);
        TM_TRY(allow_counter_smem());
        TM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mine_kernel<false, false>(), kThreads, dyn_smem));
        per_sm = std::max(per_sm, 1);
        const int blocks = n_sm * per_sm;
        Params prm{};                 // every field not set below is zero
        prm.g = g->d;
        prm.tr = image_tree(img, b + kNoAllocTree);
        prm.roots = roots;
        prm.n_roots = n_roots;
        prm.root_lo = roots ? 0 : root_lo;
        prm.counts = d_cnt;
        prm.per_root_counts = nullptr;
        prm.per_root_work = nullptr;
        prm.q = d_q;
        prm.tasks = nullptr;
        prm.ready = nullptr;
        prm.stats = nullptr;
        prm.chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(16, n_roots / ((int64_t)blocks * kWarps * 64)));
        prm.smem_counters = 1;
        prm.dynamic = 0;
        prm.react = 0;
        prm.split = nullptr;
        prm.poll_every = kPollEvery;
        prm.donate_seq = kDonateSeq;
        prm.donate_leaf = kDonateLeaf;
        prm.siblings = 0;
        prm.sib_always = 0;
        prm.offload_max = kOffloadMax;
        prm.tiers = 0;
        prm.root_qmask = nullptr;
        mine_kernel<false, false>()<<<blocks, kThreads, dyn_smem, s>>>(prm);
        TM_CUDA_TRY(cudaGetLastError());
    }
    k_to_i64<<<(n_motifs + 255) / 256, 256, 0, s>>>(d_cnt, counts, n_motifs);
    TM_CUDA_TRY(cudaGetLastError());
    return TM_OK;
}
