// Serving: a request loop over a resident graph with continuous batching.
//
// Requests (a motif set, a window per motif, a set of root edges) arrive at
// any time through tm_server_submit.  A worker thread keeps up to `streams`
// batches on the device at once.  Whenever a stream is free it admits the
// oldest pending requests -- up to `max_batch` of them and within the device
// memory budget -- merges their motifs into one MG-Tree (each motif keeps
// its own window and the index of its request), takes the union of their
// roots with a per-root bit mask of the requests that asked for that root,
// and launches one count.  The kernel counts a motif at a root only when the
// root's mask has the motif's request bit, and skips subtrees with no such
// motif, so every request gets exactly the counts it would get alone.
// Finished batches are retired by polling their events; their counts are
// scattered back per request with submit, start and finish times.
//
// The paper answers one query (a motif group, one window) per run (Section
// 4.1); serving is an addition of this library.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tm_internal.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket = 0;
    std::vector<int8_t> uv;
    std::vector<int32_t> off;
    std::vector<int64_t> delta;
    std::vector<int32_t> roots;
    int32_t n_motifs = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    std::vector<int64_t> counts;
    int state = 0;            // 0 pending, 1 running, 2 done, < 0 error code
    int32_t batch = -1, batch_size = 0;
    std::string error;
};

struct Batch {
    std::vector<Request *> reqs;
    std::vector<int32_t> motif_base;   // first counter of each request
    tm_tree *tree = nullptr;
    char *dmem = nullptr;
    size_t bytes = 0;                  // device bytes used
    size_t budgeted = 0;               // bytes counted against the budget (an upper bound of `bytes`)
    int64_t *h_counts = nullptr;       // pinned
    int32_t *h_status = nullptr;       // pinned
    int32_t n_motifs = 0;
    cudaEvent_t done = nullptr;
    int stream = -1;
    int32_t id = 0;
};

}  // namespace

struct tm_server {
    const tm_graph *g = nullptr;
    tm_server_config cfg{};
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_busy;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;
    std::unordered_map<int64_t, std::unique_ptr<Request>> all;
    std::vector<Batch *> inflight;
    size_t admitted = 0, peak = 0;
    size_t fixed = 0;                  // per-batch scratch (task queue, headers) and slack
    int64_t next_ticket = 1;
    int32_t next_batch = 0;
    int64_t batches = 0, requests_done = 0;
    bool stop = false;
    std::thread worker;
    std::string fatal;
};

namespace tmo {
namespace {

// Upper bound of the device bytes one request adds to a batch: tree nodes
// (at most one per motif edge, 56 B each), refs, windows and counters (32 B
// per motif), roots and masks (12 B per root), alignment slack.
size_t request_bytes(const Request &r) {
    return 56 * (size_t)r.off[r.n_motifs] + 32 * (size_t)r.n_motifs + 12 * r.roots.size() + 2048;
}

void finish_batch(tm_server *S, Batch *b) {
    const double t = now_ms();
    const bool bad = *b->h_status != 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t i = 0; i < b->reqs.size(); i++) {
            Request *r = b->reqs[i];
            r->counts.assign(b->h_counts + b->motif_base[i], b->h_counts + b->motif_base[i] + r->n_motifs);
            r->t_done = t;
            r->state = bad ? TM_ETIMEOUT : 2;
            if (bad) r->error = "a bounded device wait expired in this request's batch";
        }
        S->admitted -= b->budgeted;
        S->stream_busy[b->stream] = 0;
        S->requests_done += (int64_t)b->reqs.size();
    }
    S->cv.notify_all();
    cudaFreeAsync(b->dmem, S->streams[b->stream]);
    cudaFreeHost(b->h_counts);
    cudaEventDestroy(b->done);
    tm_tree_free(b->tree);
    delete b;
}

// Build and launch one batch on stream `si`; requests are already marked running.
int launch_batch(tm_server *S, Batch *b, int si) {
    cudaStream_t st = S->streams[si];
    // merged motif list with per-motif request index
    std::vector<int8_t> uv;
    std::vector<int32_t> off{0}, query;
    std::vector<int64_t> delta;
    for (size_t q = 0; q < b->reqs.size(); q++) {
        Request *r = b->reqs[q];
        b->motif_base.push_back((int32_t)delta.size());
        for (int i = 0; i < r->n_motifs; i++) {
            for (int j = r->off[i]; j < r->off[i + 1]; j++) {
                uv.push_back(r->uv[2 * j]);
                uv.push_back(r->uv[2 * j + 1]);
            }
            off.push_back(off.back() + (r->off[i + 1] - r->off[i]));
            delta.push_back(r->delta[i]);
            query.push_back((int32_t)q);
        }
    }
    b->n_motifs = (int32_t)delta.size();
    TM_TRY(tree_build_q(uv.data(), off.data(), b->n_motifs, delta.data(), query.data(), &b->tree));
    // union of roots, each with the requests that asked for it
    std::map<int32_t, uint64_t> um;
    for (size_t q = 0; q < b->reqs.size(); q++)
        for (int32_t r : b->reqs[q]->roots) um[r] |= 1ull << q;
    std::vector<int32_t> roots;
    std::vector<uint64_t> masks;
    roots.reserve(um.size());
    masks.reserve(um.size());
    for (auto &kv : um) {
        roots.push_back(kv.first);
        masks.push_back(kv.second);
    }
    const int64_t n = (int64_t)roots.size();
    TreeImage scan_img;
    if (S->cfg.mode & TM_LEAF_SCAN) tree_image(b->tree->h, false, &scan_img);
    const TreeImage &img = (S->cfg.mode & TM_LEAF_SCAN) ? scan_img : b->tree->image;
    const size_t scratch = batch_scratch_bytes(S->g, b->tree, S->cfg.mode);
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_tree = 0, o_roots = al(img.bytes.size()), o_masks = o_roots + al(4 * (size_t)n);
    const size_t o_counts = o_masks + al(8 * (size_t)n), o_status = o_counts + al(8 * (size_t)b->n_motifs);
    const size_t o_scr = o_status + 256;
    b->bytes = o_scr + scratch;
    TM_CUDA_TRY(cudaMallocAsync((void **)&b->dmem, b->bytes, st));
    TM_CUDA_TRY(cudaMallocHost((void **)&b->h_counts, 8 * (size_t)b->n_motifs + 64));
    b->h_status = (int32_t *)(b->h_counts + b->n_motifs);
    TM_CUDA_TRY(cudaMemcpyAsync(b->dmem + o_tree, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, st));
    if (n > 0) {
        TM_CUDA_TRY(cudaMemcpyAsync(b->dmem + o_roots, roots.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st));
        TM_CUDA_TRY(cudaMemcpyAsync(b->dmem + o_masks, masks.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, st));
    }
    const DevTree dt = image_tree(img, b->dmem + o_tree);
    int64_t *d_counts = (int64_t *)(b->dmem + o_counts);
    int32_t *d_status = (int32_t *)(b->dmem + o_status);
    TM_CUDA_TRY(cudaMemsetAsync(d_counts, 0, 8 * (size_t)b->n_motifs, st));
    TM_CUDA_TRY(cudaMemsetAsync(d_status, 0, 4, st));
    TM_TRY(batch_enqueue(S->g, b->tree, S->cfg.mode, dt, (const int32_t *)(b->dmem + o_roots),
                         (const uint64_t *)(b->dmem + o_masks), n, b->dmem + o_scr, d_counts, d_status, st));
    TM_CUDA_TRY(cudaMemcpyAsync(b->h_counts, d_counts, 8 * (size_t)b->n_motifs, cudaMemcpyDeviceToHost, st));
    TM_CUDA_TRY(cudaMemcpyAsync(b->h_status, d_status, 4, cudaMemcpyDeviceToHost, st));
    TM_CUDA_TRY(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
    TM_CUDA_TRY(cudaEventRecord(b->done, st));
    return TM_OK;
}

void worker_loop(tm_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // retire finished batches
        bool progressed = false;
        for (size_t i = 0; i < S->inflight.size();) {
            Batch *b = S->inflight[i];
            if (cudaEventQuery(b->done) == cudaSuccess) {
                S->inflight.erase(S->inflight.begin() + i);
                lk.unlock();
                finish_batch(S, b);
                lk.lock();
                progressed = true;
            } else {
                i++;
            }
        }
        if (S->stop && S->pending.empty() && S->inflight.empty()) break;
        // admit a batch while a stream is free
        int si = -1;
        for (size_t k = 0; k < S->streams.size(); k++)
            if (!S->stream_busy[k]) { si = (int)k; break; }
        if (si >= 0 && !S->pending.empty()) {
            Batch *b = new Batch();
            size_t need = 0;
            const size_t fixed = S->fixed;
            std::set<int64_t> windows;        // the merged tree's limits: distinct windows and nodes
            int64_t edges = 0;
            while (!S->pending.empty() && (int)b->reqs.size() < S->cfg.max_batch) {
                Request *r = S->pending.front();
                const size_t rb = request_bytes(*r);
                std::set<int64_t> w2 = windows;
                w2.insert(r->delta.begin(), r->delta.end());
                if (!b->reqs.empty() && ((int)w2.size() > TM_MAX_DELTAS || edges + r->off[r->n_motifs] + 1 > TM_MAX_NODES))
                    break;
                if (fixed + rb > (size_t)S->cfg.mem_budget) {   // can never be admitted
                    S->pending.pop_front();
                    r->state = TM_ENOMEM;
                    r->error = "request needs more device memory than the server's budget";
                    r->t_done = now_ms();
                    S->cv.notify_all();
                    continue;
                }
                if (S->admitted + fixed + need + rb > (size_t)S->cfg.mem_budget) break;   // wait for memory
                S->pending.pop_front();
                windows.swap(w2);
                edges += r->off[r->n_motifs];
                r->state = 1;
                r->t_start = now_ms();
                r->batch = S->next_batch;
                b->reqs.push_back(r);
                need += rb;
            }
            if (b->reqs.empty()) {
                delete b;
            } else {
                b->id = S->next_batch++;
                for (Request *r : b->reqs) r->batch_size = (int32_t)b->reqs.size();
                S->stream_busy[si] = 1;
                b->stream = si;
                lk.unlock();
                int rc = launch_batch(S, b, si);
                lk.lock();
                if (rc != TM_OK) {
                    std::string msg = tm_last_error();
                    for (Request *r : b->reqs) {
                        r->state = rc;
                        r->error = msg;
                        r->t_done = now_ms();
                    }
                    S->stream_busy[si] = 0;
                    if (b->dmem) cudaFreeAsync(b->dmem, S->streams[si]);
                    if (b->h_counts) cudaFreeHost(b->h_counts);
                    if (b->tree) tm_tree_free(b->tree);
                    delete b;
                    S->cv.notify_all();
                } else {
                    b->budgeted = fixed + need;
                    S->admitted += b->budgeted;
                    S->peak = std::max(S->peak, S->admitted);
                    S->inflight.push_back(b);
                    S->batches++;
                }
                progressed = true;
            }
        }
        if (!progressed) S->cv.wait_for(lk, std::chrono::microseconds(100));
    }
}

}  // namespace
}  // namespace tmo

using namespace tmo;

extern "C" {

int tm_server_open(const tm_graph *g, const tm_server_config *cfg, tm_server **out) {
    if (!g || !out) { set_error("tm_server_open: NULL argument"); return TM_EINVAL; }
    *out = nullptr;
    std::unique_ptr<tm_server> S(new tm_server());
    S->g = g;
    S->cfg.streams = 2;
    S->cfg.max_batch = 32;
    S->cfg.mem_budget = (int64_t)4 << 30;
    S->cfg.mode = TM_SCHED_DYNAMIC;
    if (cfg) {
        if (cfg->streams > 0) S->cfg.streams = cfg->streams;
        if (cfg->max_batch > 0) S->cfg.max_batch = cfg->max_batch;
        if (cfg->mem_budget > 0) S->cfg.mem_budget = cfg->mem_budget;
        S->cfg.mode = cfg->mode;
    }
    if (S->cfg.max_batch > 64) { set_error("tm_server_open: max_batch above 64"); return TM_EINVAL; }
    if (S->cfg.streams > 16) { set_error("tm_server_open: more than 16 streams"); return TM_EINVAL; }
    if (S->cfg.mode & ~(uint32_t)(TM_LEAF_SCAN | TM_SCHED_DYNAMIC)) {
        set_error("tm_server_open: mode may hold TM_LEAF_SCAN and TM_SCHED_DYNAMIC only");
        return TM_EINVAL;
    }
    TM_CUDA_TRY(cudaGetDevice(&S->device));
    {   // per-batch scratch of a one-motif tree; counters are in the per-request bound
        const int8_t uv[2] = {0, 1};
        const int32_t off[2] = {0, 1};
        const int64_t d = 0;
        tm_tree *t1 = nullptr;
        TM_TRY(tree_build(uv, off, 1, &d, &t1));
        S->fixed = batch_scratch_bytes(g, t1, S->cfg.mode) + (8u << 10);
        tm_tree_free(t1);
        if (S->fixed > (size_t)S->cfg.mem_budget) { set_error("tm_server_open: budget below one batch's scratch"); return TM_EINVAL; }
    }
    for (int i = 0; i < S->cfg.streams; i++) {
        cudaStream_t st;
        TM_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        S->streams.push_back(st);
        S->stream_busy.push_back(0);
    }
    tm_server *raw = S.get();
    S->worker = std::thread(worker_loop, raw);
    *out = S.release();
    return TM_OK;
}

int tm_server_submit(tm_server *S, const int8_t *motif_uv, const int32_t *motif_off, int32_t n_motifs,
                     const int64_t *delta, const int32_t *roots, int64_t n_roots, int64_t *ticket) {
    if (!S || !motif_uv || !motif_off || !delta || !ticket || n_motifs < 1 || n_roots < 0 || (n_roots > 0 && !roots)) {
        set_error("tm_server_submit: bad argument");
        return TM_EINVAL;
    }
    // validate the motifs the way tm_tree_build does
    tm_tree *probe = nullptr;
    TM_TRY(tree_build(motif_uv, motif_off, n_motifs, delta, &probe));
    tm_tree_free(probe);
    for (int64_t i = 0; i < n_roots; i++)
        if (roots[i] < 0 || roots[i] >= S->g->d.E) { set_error("tm_server_submit: root out of range"); return TM_EINVAL; }
    std::unique_ptr<Request> r(new Request());
    r->n_motifs = n_motifs;
    r->off.assign(motif_off, motif_off + n_motifs + 1);
    r->uv.assign(motif_uv, motif_uv + 2 * (size_t)motif_off[n_motifs]);
    r->delta.assign(delta, delta + n_motifs);
    r->roots.assign(roots, roots + n_roots);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->ticket = S->next_ticket++;
        r->t_submit = now_ms();
        *ticket = r->ticket;
        S->pending.push_back(r.get());
        S->all[r->ticket] = std::move(r);
    }
    S->cv.notify_all();
    return TM_OK;
}

int tm_server_poll(tm_server *S, int64_t ticket, int32_t wait, int64_t *counts, tm_request_stats *st) {
    if (!S) { set_error("tm_server_poll: NULL server"); return TM_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { set_error("tm_server_poll: unknown ticket"); return TM_EINVAL; }
    Request *r = it->second.get();
    if (wait)
        S->cv.wait(lk, [&] { return r->state == 2 || r->state < 0; });
    if (r->state == 0 || r->state == 1) return 0;
    if (st) {
        st->queue_ms = r->t_start - r->t_submit;
        st->latency_ms = r->t_done - r->t_submit;
        st->batch = r->batch;
        st->batch_size = r->batch_size;
    }
    if (r->state < 0) {
        set_error("tm_server_poll: " + r->error);
        int rc = r->state;
        S->all.erase(it);
        return rc;
    }
    if (counts) std::copy(r->counts.begin(), r->counts.end(), counts);
    S->all.erase(it);
    return 1;
}

int tm_server_get_info(tm_server *S, tm_server_info *info) {
    if (!S || !info) { set_error("tm_server_get_info: NULL argument"); return TM_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    info->batches = S->batches;
    info->requests_done = S->requests_done;
    info->pending = (int64_t)S->pending.size();
    info->in_flight = (int64_t)S->inflight.size();
    info->admitted_bytes = (int64_t)S->admitted;
    info->peak_admitted_bytes = (int64_t)S->peak;
    return TM_OK;
}

int tm_server_close(tm_server *S) {
    if (!S) return TM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete S;
    return TM_OK;
}

}  // extern "C"
