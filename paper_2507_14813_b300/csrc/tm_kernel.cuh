// Co-mining kernel: exact counts of every motif of an MG-Tree.
//
// Algorithm 3 (CoMatchEdge) walked by one warp per root edge.  Every edge is
// a candidate for the first motif edge (Algorithm 1, first call); each later
// motif edge draws candidates from the out-list of the mapped source or the
// in-list of the mapped destination (reading 4), restricted to edge ids in
// (previous match, last edge within the window] (temporal constraints,
// readings 1-2) and filtered for structure with full injectivity (reading 3).
// When C_N of a node is complete the node's queries are counted and its
// children are mined from the same partial match, in table order.
//
// Per level the warp loads 32 adjacency entries (one coalesced 8-byte load
// per lane), evaluates the predicate branch-free, and takes the ballot.
// Surviving candidates are kept in a per-warp shared-memory stack and
// descended one at a time, depth first.
//
// Leaf edges.  The last edge of a leaf node is never descended.  In scan
// mode the warp counts its survivors with popc per chunk (the paper's scan).
// Otherwise every survivor of the level above counts its own leaf edge in
// parallel (one lane per survivor) by exact window arithmetic:
//     |candidates| = |list in (last, hi]| - sum over mapped w of |pair (x,w) in (last, hi]|
// using binary searches on the time-sorted list and the (src, dst) pair
// index; lanes with a short window scan it instead.  Both give the count the
// scan gives.
//
// Scheduling.  In the static mode each warp claims root edges from a counter
// and mines them alone.  In the dynamic mode (TM_SCHED_DYNAMIC) the launch is
// persistent: a warp that sees idle warps hands the unscanned half of its
// shallowest long candidate slice to a global task queue, and idle warps take
// tasks before new roots.  A task owns its slice exclusively (the donor
// stops before it, and the task never moves on to the node's siblings), so
// no match is counted twice -- the ownership rule of the paper's inter-warp
// balancing (Section 4.5), applied to any level.  Every wait is bounded; an
// expired wait sets an error flag that the host turns into TM_ETIMEOUT.
//
// This file is the kernel alone.  The library compiles it once as the
// table-driven kernel (tm_kmine_*.cu, launched from tm_mine.cu): the
// MG-Tree is read from a node table in device memory and every array is
// sized to the library's limits.  For one tree the library can also
// compile it at run time (NVRTC, tm_codegen.cpp) behind a generated
// prelude that defines TM_K_SPEC: the node, ref and window tables are then
// constant data of the kernel, the tree's counts and properties are
// compile-time constants, and arrays and label loops are sized to the
// tree's depth and vertex count (the code generation of Section 5.1, "GPU
// Code-generation").
#pragma once

#include "tm_device.h"

namespace tmo {
namespace dev {

#ifdef TM_K_SPEC
// the tree's tables and constants come from the generated prelude:
//   tmk_nodes[], tmk_refs[], tmk_deltas[], tmk_qdmax[] (__constant__ data),
//   TM_K_NDELTAS, TM_K_NCOUNTERS, TM_K_HAS_GLOBAL
#define TM_NODE(i) (tmk_nodes[(i)])
#define TM_REF(i) (tmk_refs[(i)])
#define TM_DELTA(j) (tmk_deltas[(j)])
#define TM_QDMAX(q) (tmk_qdmax[(q)])
#define TM_NDELTAS TM_K_NDELTAS
#define TM_NCOUNTERS TM_K_NCOUNTERS
#define TM_NNODES TM_K_NNODES
constexpr bool kHasGlobal = TM_K_HAS_GLOBAL != 0;
#else
#define TM_NODE(i) (p.tr.nodes[(i)])
#define TM_REF(i) (p.tr.refs[(i)])
#define TM_DELTA(j) (__ldg(p.tr.deltas + (j)))
#define TM_QDMAX(q) (p.tr.qdmax[(q)])
#define TM_NDELTAS (p.tr.n_deltas)
#define TM_NCOUNTERS (p.tr.n_counters)
#define TM_NNODES (p.tr.n_nodes)
constexpr bool kHasGlobal = true;
#endif

// The checking build (TM_CHECK): every index into a per-warp shared-memory
// array, the counters, the window table and the tree that the kernel takes
// from data is checked where it is used; one outside its range sets an error
// bit (returned as TM_ECHECK), and the access is skipped instead of made.
#ifdef TM_CHECK
constexpr bool kCheck = true;
#else
constexpr bool kCheck = false;
#endif

// Test builds only: a shorter bound on waiting for a claimed task's payload,
// and a pause of donors before they publish one, so that a test can make the
// bounded wait run out (off by default: TM_TEST_READY_SPINS unset, no pause).
#ifndef TM_TEST_PUBLISH_PAUSE
#define TM_TEST_PUBLISH_PAUSE 0                // iterations of __nanosleep(1000) before publishing
#endif

constexpr int kWarps = 8;                 // warps per CTA
constexpr int kThreads = kWarps * 32;
constexpr int kSmemCounters = 2048;       // per-CTA counters kept in shared memory up to this many
constexpr int kWarpCounters = kSmemCounters / kWarps;  // up to this many: one private slice per warp
constexpr int kLaneScanMax = 24;          // leaf windows up to this size are scanned by the lane
constexpr int kLaneDeltas = 8;            // thread tier: trees with at most this many windows
constexpr uint32_t kCacheEmpty = 0xffffffffu;
constexpr unsigned long long kSlotEmpty = (unsigned long long)kCacheEmpty << 32;
constexpr int kSlots = 256;               // occurrence-table slots per warp
constexpr int kSlotShift = 24;            // 32 - log2(kSlots)
// star frames: later entries with the same far end come from ...
enum : int8_t { kSameGallop = 0,          // ... the pair run (galloping search)
                kSameTable = 1,           // ... the frame's occurrence table (pair run when the slot is taken)
                kSameChunk = 2 };         // ... the chunk itself (the whole window is one chunk)

constexpr int kQueueCap = 1 << 20;        // tasks per launch (slots are not reused)
constexpr int kPollEvery = 4;             // default: chunk loads between looks at the idle counter
constexpr int kDonateSeq = 64;            // default: min unscanned entries to split a level that descends
constexpr int kDonateLeaf = 1024;         // default: ... a level whose survivors are only counted
constexpr int kOffloadMax = 8;            // default: most pieces one multi-offload hands over
#ifdef TM_TEST_READY_SPINS
constexpr long long kReadySpins = TM_TEST_READY_SPINS;
#else
constexpr long long kReadySpins = 1 << 22;  // bound on waiting for a claimed task's payload
#endif
constexpr long long kIdleSpins = 1 << 20;   // bound on an idle warp's wait for work

// candidate lists: out-list of a mapped source, in-list of a mapped
// destination, the global edge window (neither mapped), or -- both mapped --
// the run of edges between the two in the (src, dst) pair order
enum : int8_t { kListOut = 0, kListIn = 1, kListGlobal = 2, kListPair = 3 };

// A unit of work: the slice [lo, hi) of level k's candidate list of `node`,
// under the partial match eid[0..k-1] (eid[0] is the root edge).  lo < 0
// marks a sibling task: open `node` at level k afresh (its whole list) and
// mine that node's subtree only.
struct __align__(16) Task {
    int32_t ri;               // root index, for per-root outputs
    int16_t node;
    int8_t k;
    int8_t pad0;
    int64_t wend;             // end of the level's whole window (beyond the slice)
    int32_t eid[TM_MAX_EDGES];  // the partial match (kMaxE used)
    int64_t lo, hi;
};
static_assert(sizeof(Task) == 64, "task layout");

enum : int { kErrTimeout = 1,          // a bounded wait expired
             kErrBadRoot = 2,          // a root edge id outside [0, E) was skipped
             kErrCheck = 4 };          // the checking build found an index outside its range

struct QueueHdr {
    unsigned long long root_cursor;
    unsigned long long lane_cursor;   // thread tier: roots handed out, 32 per warp
    long long lane_from;              // thread tier: first root index (the tail of a planned order)
    unsigned int head;        // next task to claim
    unsigned int tail;        // tasks reserved by donors
    int idle;                 // warps waiting for work
    int busy;                 // warps holding work
    int error;                // kErr* bits
    int idle_expired;         // warps that left after their bounded idle wait ran out with work still held
};

struct Params {
    DevGraph g;
    DevTree tr;
    const int32_t *roots;
    int64_t n_roots;
    int64_t root_lo;
    unsigned long long *counts;       // n_counters
    int64_t *per_root_counts;         // [n_roots][n_counters] or null
    int64_t *per_root_work;           // [n_roots][TM_WORK_FIELDS] or null
    QueueHdr *q;                      // zeroed before launch
    Task *tasks;                      // kQueueCap (dynamic mode)
    int *ready;                       // kQueueCap publish flags, zeroed (dynamic mode)
    unsigned long long *stats;        // kStatFields totals, then kBusyFields, or null
    int32_t chunk;                    // roots claimed per cursor step
    int32_t smem_counters;            // 1: per-CTA counters in shared memory, 2: one slice per warp
    int32_t dynamic;                  // 1: persistent launch with a task queue
    int32_t react;                    // 1: warps donate slices when others are idle
    const int32_t *split;             // per root index: slices for its first-level lists, or null
    int32_t poll_every;               // chunk loads between looks at the idle counter
    int32_t donate_seq;               // min unscanned entries to split a level that descends
    int32_t donate_leaf;              // ... a level whose survivors are only counted
    int32_t siblings;                 // 1: sibling splitting and multi-offload (TM_SCHED_SIBLINGS)
    int32_t sib_always;               // 1: split siblings even when no warp is idle
    int32_t offload_max;              // most pieces one donation hands over (multi-offload)
    int32_t tiers;                    // 1: roots from q->lane_from on run one per lane (thread tier)
    const uint64_t *root_qmask;       // per root index: queries it serves (bit q), or null = all
};

// kStLogDeg: sum over opened lists of ceil(log2(list length + 1)), the
// probes a binary search of each list costs
// kStLaneRoots: roots counted by the thread tier; kStSplitRoots: roots whose
// first-level lists were cut into planned slices
enum { kStCand = 0, kStExp, kStListProbe, kStHashProbe, kStPairProbe, kStLeaf, kStRoots, kStSplit, kStLogDeg,
       kStLaneRoots, kStSplitRoots, kStatFields };
// after the kStatFields totals: busy cycles of the busiest warp, their sum, and the warps
enum { kBusyMax = 0, kBusySum, kBusyWarps, kBusyFields };

struct WarpState {
    int2 cand[kMaxE][32];
    int64_t pos[kMaxE];       // next chunk start (absolute index into the list array)
    int64_t end[kMaxE];       // end of the candidate slice
    int64_t cbase[kMaxE];     // start of the chunk held in cand[k]
    uint32_t mask[kMaxE];     // survivors of the held chunk not yet descended
    int32_t lvert[kMaxE];     // list vertex (out/in lists; the source of a pair list)
    int32_t lfar[kMaxE];      // pair lists: the mapped destination
    int32_t eid[kMaxE];       // matched edge id per level
    int64_t mpos[kMaxE];      // list position of the matched candidate
    int16_t node[kMaxE];
    int16_t sib_end[kMaxE];
    int8_t ltype[kMaxE];
    int8_t seq[kMaxE];        // survivors of level k are descended (not only counted)
    int8_t star[kMaxE];       // star leaves are counted from level k: scanned top-down, suf[k] kept
    int64_t wend[kMaxE];      // end of level k's window (a donated slice may end earlier)
    int64_t suf[kMaxE];       // star frames: survivors of level k above the scan cursor, up to wend
    int8_t same_mode[kMaxE];  // star frames: how later same-endpoint entries are found (kSame*)
    // later-occurrence counts per candidate endpoint, for one star frame:
    // (endpoint << 32) | survivors with that endpoint scanned so far
    unsigned long long cslot[kSlots];
    int32_t cache_owner;      // level whose star frame owns cslot, or -1
    // the last uniform pair window (leaf_batch): key (source, destination),
    // (window end, frame start); the run's start and the window [wlo, whi) in it
    unsigned long long pc_k1, pc_k2;
    int64_t pc_st;
    int32_t pc_wlo, pc_whi;
    int32_t m2g[kMaxV];
    int32_t ehi[TM_MAX_DELTAS];
};

struct Work {
    unsigned long long v[kStatFields];
};

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
    // 32 values below 2^27 sum below 2^32: one reduction instruction
    if (__all_sync(0xffffffffu, x < (1ull << 27))) return __reduce_add_sync(0xffffffffu, (unsigned)x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ int64_t sat_add(int64_t a, int64_t b) {
    return (b > 0 && a > INT64_MAX - b) ? INT64_MAX : a + b;
}

// last edge id e >= r with t[e] <= limit (t[r] <= limit holds); serial, per lane
static __device__ int32_t window_end(const int64_t *__restrict__ t, int64_t E, int32_t r, int64_t limit, unsigned long long &probes) {
    int64_t lo = r, step = 1;          // t[lo] <= limit
    int64_t hi = E;                    // t[hi] > limit or hi == E
    while (true) {                     // gallop
        int64_t q = lo + step;
        if (q >= E) break;
        probes++;
        if (__ldg(t + q) <= limit) { lo = q; step <<= 1; } else { hi = q; break; }
    }
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        probes++;
        if (__ldg(t + mid) <= limit) lo = mid; else hi = mid;
    }
    return (int32_t)lo;
}

// first position in adj[lo, hi) whose edge id exceeds key (hi if none); per lane
__device__ __forceinline__ int64_t lane_upper(const int2 *__restrict__ adj, int64_t lo, int64_t hi, int32_t key,
                                              unsigned long long &probes) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        probes++;
        if (__ldg(&adj[mid].y) <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t lane_upper_e(const int32_t *__restrict__ a, int64_t lo, int64_t hi, int32_t key,
                                                unsigned long long &probes) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        probes++;
        if (__ldg(a + mid) <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// first position in adj[lo, hi) whose edge id exceeds key, galloping from lo; per lane
__device__ __forceinline__ int64_t lane_gallop(const int2 *__restrict__ adj, int64_t lo, int64_t hi, int32_t key,
                                               unsigned long long &probes) {
    if (lo >= hi) return lo;
    probes++;
    if (__ldg(&adj[lo].y) > key) return lo;
    int64_t a = lo, step = 1, b = hi;          // adj[a].y <= key; answer in (a, b]
    while (true) {
        int64_t q = a + step;
        if (q >= hi) break;
        probes++;
        if (__ldg(&adj[q].y) <= key) { a = q; step <<= 1; } else { b = q; break; }
    }
    while (b - a > 1) {
        int64_t mid = a + ((b - a) >> 1);
        probes++;
        if (__ldg(&adj[mid].y) <= key) a = mid; else b = mid;
    }
    return b;
}

// First position in the list of x after edge `last`, when x is an endpoint of
// `last` (per-edge index), else -1.
__device__ __forceinline__ int64_t after_pos(const DevGraph &g, bool out, int32_t x, int32_t last, int32_t s,
                                             int32_t d) {
    if (out) {
        if (x == s) return __ldg(g.after_os + last);
        if (x == d) return __ldg(g.after_od + last);
    } else {
        if (x == d) return __ldg(g.after_id + last);
        if (x == s) return __ldg(g.after_is + last);
    }
    return -1;
}

// first position in adj[lo, hi) whose edge id exceeds key; warp-cooperative
static __device__ int64_t warp_upper(const int2 *__restrict__ adj, int64_t lo, int64_t hi, int32_t key, int lane,
                              unsigned long long &probes);

// the same, galloping from lo: one round of probes at lo + 2^lane - 1 brackets
// the answer, then the 32-ary search narrows it
static __device__ int64_t warp_gallop(const int2 *__restrict__ adj, int64_t lo, int64_t hi, int32_t key, int lane,
                               unsigned long long &probes) {
    if (hi - lo <= 32) return warp_upper(adj, lo, hi, key, lane, probes);
    int64_t q = lane == 31 ? hi - 1 : lo + ((int64_t)1 << lane) - 1;
    if (q > hi - 1) q = hi - 1;
    const bool gt = __ldg(&adj[q].y) > key;
    probes += 1;
    const uint32_t b = __ballot_sync(0xffffffffu, gt);
    if (b == 0) return hi;
    const int f = __ffs(b) - 1;
    const int64_t qf = __shfl_sync(0xffffffffu, q, f);
    const int64_t qp = __shfl_sync(0xffffffffu, q, f > 0 ? f - 1 : 0);
    return warp_upper(adj, f > 0 ? qp + 1 : lo, qf, key, lane, probes) ;
}

static __device__ int64_t warp_upper(const int2 *__restrict__ adj, int64_t lo, int64_t hi, int32_t key, int lane,
                              unsigned long long &probes) {
    while (hi - lo > 32) {
        int64_t step = (hi - lo + 31) >> 5;
        int64_t q = lo + (int64_t)(lane + 1) * step - 1;
        if (q > hi - 1) q = hi - 1;
        bool gt = __ldg(&adj[q].y) > key;
        probes += 1;
        uint32_t b = __ballot_sync(0xffffffffu, gt);
        if (b == 0) return hi;
        int f = __ffs(b) - 1;
        int64_t qf = __shfl_sync(0xffffffffu, q, f);
        int64_t qp = __shfl_sync(0xffffffffu, q, f > 0 ? f - 1 : 0);
        lo = f > 0 ? qp + 1 : lo;
        hi = qf;                        // answer <= qf; hi is returned if nothing in [lo, qf) qualifies
    }
    int64_t q = lo + lane;
    bool gt = q < hi && __ldg(&adj[q].y) > key;
    probes += q < hi;
    uint32_t b = __ballot_sync(0xffffffffu, gt);
    return b ? lo + (__ffs(b) - 1) : hi;
}

// The run of edges x -> w in the pair order: pair_eid[*st, *st + *len),
// ascending edge ids (*len = 0 when there is none).
__device__ __forceinline__ void pair_run(const DevGraph &g, int32_t x, int32_t w, int64_t *st, int64_t *len,
                                         unsigned long long &hprobes) {
    const unsigned long long key = ((unsigned long long)(uint32_t)x << 32) | (uint32_t)w;
    uint64_t h = pair_hash(key) & g.pair_mask;
    *st = 0;
    *len = 0;
    while (true) {
        hprobes++;
        const ulonglong2 e = __ldg(&g.pair_tab[h]);
        if (e.x == key) {
            *st = (int64_t)(e.y & 0xffffffffull);
            *len = (int64_t)(e.y >> 32);
            return;
        }
        if (e.x == kEmptyKey) return;
        h = (h + 1) & g.pair_mask;
    }
}

// first position in a[lo, hi) whose value exceeds key, galloping from lo; per lane
__device__ __forceinline__ int64_t lane_gallop_e(const int32_t *__restrict__ a, int64_t lo, int64_t hi, int32_t key,
                                                 unsigned long long &probes) {
    if (lo >= hi) return lo;
    probes++;
    if (__ldg(a + lo) > key) return lo;
    int64_t x = lo, step = 1, y = hi;          // a[x] <= key; answer in (x, y]
    while (true) {
        const int64_t q = x + step;
        if (q >= hi) break;
        probes++;
        if (__ldg(a + q) <= key) { x = q; step <<= 1; } else { y = q; break; }
    }
    while (y - x > 1) {
        const int64_t mid = x + ((y - x) >> 1);
        probes++;
        if (__ldg(a + mid) <= key) x = mid; else y = mid;
    }
    return y;
}

// first position in a[lo, hi) whose value exceeds key; warp-cooperative (int32 arrays)
static __device__ int64_t warp_upper_e(const int32_t *__restrict__ a, int64_t lo, int64_t hi, int32_t key, int lane,
                                unsigned long long &probes) {
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) >> 5;
        int64_t q = lo + (int64_t)(lane + 1) * step - 1;
        if (q > hi - 1) q = hi - 1;
        const bool gt = __ldg(a + q) > key;
        probes += 1;
        const uint32_t b = __ballot_sync(0xffffffffu, gt);
        if (b == 0) return hi;
        const int f = __ffs(b) - 1;
        const int64_t qf = __shfl_sync(0xffffffffu, q, f);
        const int64_t qp = __shfl_sync(0xffffffffu, q, f > 0 ? f - 1 : 0);
        lo = f > 0 ? qp + 1 : lo;
        hi = qf;
    }
    const int64_t q = lo + lane;
    const bool gt = q < hi && __ldg(a + q) > key;
    probes += q < hi;
    const uint32_t b = __ballot_sync(0xffffffffu, gt);
    return b ? lo + (__ffs(b) - 1) : hi;
}

// |edges x -> w with lo < eid <= hi|
static __device__ int64_t pair_count(const DevGraph &g, int32_t x, int32_t w, int32_t lo, int32_t hi,
                              unsigned long long &hprobes, unsigned long long &pprobes) {
    if (hi <= lo) return 0;
    int64_t st, len;
    pair_run(g, x, w, &st, &len, hprobes);
    if (len == 0) return 0;
    const int32_t *run = g.pair_eid + st;
    if (len <= 16) {
        int64_t c = 0;
        for (int64_t i = 0; i < len; i++) {
            int32_t v = __ldg(run + i);
            c += (v > lo) & (v <= hi);
        }
        pprobes += len;
        return c;
    }
    // the window (lo, hi] is short against a run over the whole time span:
    // binary search for its start, gallop from there for its end
    const int64_t a = lane_upper_e(run, 0, len, lo, pprobes);
    const int64_t b = lane_gallop_e(run, a, len, hi, pprobes);
    return b - a;
}

__device__ __forceinline__ int vload(const int *p) { return *(volatile const int *)p; }
__device__ __forceinline__ unsigned int vloadu(const unsigned int *p) { return *(volatile const unsigned int *)p; }

// Entries after position p of a run in ascending order (ending at `end`)
// that are <= hi, given a[p] <= hi: galloping search from p.
__device__ __forceinline__ int64_t run_tail(const int32_t *__restrict__ a, int64_t p, int64_t end, int32_t hi,
                                            unsigned long long &probes) {
    int64_t lo = p, step = 1, hi_pos = end;
    while (true) {
        int64_t q = lo + step;
        if (q >= end) break;
        probes++;
        if (__ldg(a + q) <= hi) { lo = q; step <<= 1; } else { hi_pos = q; break; }
    }
    while (hi_pos - lo > 1) {
        int64_t mid = lo + ((hi_pos - lo) >> 1);
        probes++;
        if (__ldg(a + mid) <= hi) lo = mid; else hi_pos = mid;
    }
    return lo - p;
}

// kExt: the extended schedules (thread tier, sibling splitting, multi-offload)
// are compiled in; the default kernel leaves them out.
template <bool kStats, bool kExt>
struct Miner {
    const Params &p;
    WarpState &ws;
    unsigned long long *s_cnt;
    int lane;
    Work w;
    int64_t ri;                        // root index of the current work (per-root outputs)
    int polls;                         // chunk loads since the last look at the idle counter
    int split_h;                       // planned slices for the current root's first-level lists
    uint64_t rmask;                    // queries served by the current root
    unsigned long long acc;            // this lane's deferred star-leaf count (drain of one frame)
    int32_t acc_ref;                   // ref index whose counts are deferred, or -1
    int32_t cap;                       // last edge id any of those queries' windows reaches
    int32_t gsame;                     // star frames: this lane's later same-endpoint survivors, or -1

    __device__ Miner(const Params &pp, WarpState &s, unsigned long long *c, int l)
        : p(pp), ws(s), s_cnt(c), lane(l), polls(0), split_h(0), rmask(~0ull), acc(0), acc_ref(-1), cap(INT32_MAX),
          gsame(-1) {
        for (int i = 0; i < kStatFields; i++) w.v[i] = 0;
    }

    // The checking build's test of an index; always true otherwise.
    __device__ __forceinline__ bool chk(bool ok) const {
        if (kCheck && !ok) {
            atomicOr(&p.q->error, kErrCheck);
            return false;
        }
        return true;
    }

    // ws.ehi[d], d an index into the window table
    __device__ __forceinline__ int32_t ehi(int d) const {
        return chk(d >= 0 && d < TM_NDELTAS) ? ws.ehi[d] : -1;
    }

    __device__ __forceinline__ void add_count(int32_t counter, unsigned long long c) {
        // called by one lane
        if (c == 0) return;
        if (!chk(counter >= 0 && counter < TM_NCOUNTERS)) return;
        if (p.smem_counters == 2) s_cnt[counter] += c;          // the warp's own slice
        else if (p.smem_counters) atomicAdd(&s_cnt[counter], c);
        else atomicAdd(&p.counts[counter], c);
        if (p.per_root_counts)
            atomicAdd((unsigned long long *)&p.per_root_counts[ri * TM_NCOUNTERS + counter], c);
    }

    // value of motif label l for a lane whose level-k candidate maps (uk -> cs, vk -> cd)
    __device__ __forceinline__ int32_t lab(int l, int uk, int vk, int32_t cs, int32_t cd) const {
        return l == uk ? cs : (l == vk ? cd : ws.m2g[l]);
    }

    // Count, for one lane, the candidates of leaf edge `lv` of node L that
    // end a match by edge id hi, after the lane's candidate (cs -> cd, id
    // last) at level lv - 1.
    __device__ int64_t leaf_count(const DevNode &L, int lv, int uk, int vk, int32_t cs, int32_t cd, int32_t last,
                                  int32_t hi) {
        const int nv = L.nvb[lv];                       // labels mapped before the leaf edge
        int32_t img[kMaxV];
#pragma unroll
        for (int l = 0; l < kMaxV; l++) img[l] = (l < nv) ? lab(l, uk, vk, cs, cd) : -1;
        return leaf_count_img(L, lv, img, cs, cd, last, hi);
    }

    // The same for a full mapping img[0 .. L.nvb[lv]) of the motif labels
    // (cs -> cd: the endpoints of edge `last`).
    __device__ int64_t leaf_count_img(const DevNode &L, int lv, const int32_t *img, int32_t cs, int32_t cd,
                                      int32_t last, int32_t hi) {
        const DevGraph &g = p.g;
        const int u = L.eu[lv], v = L.ev[lv];
        const int nv = L.nvb[lv];                       // labels mapped before the leaf edge
        const bool um = u < nv, vm = v < nv;
        unsigned long long hp = 0, pp = 0, lp = 0, sc = 0;
        int64_t c = 0;
        if (um && vm) {
            c = pair_count(g, img[u], img[v], last, hi, hp, pp);
        } else {
            const bool out = um;
            const int32_t x = out ? img[u] : img[v];
            const int2 *adj = out ? g.out_adj : g.in_adj;
            const int64_t *off = out ? g.out_off : g.in_off;
            int64_t b0 = __ldg(off + x), b1 = __ldg(off + x + 1);
            int64_t a = after_pos(g, out, x, last, cs, cd);
            if (a < 0) a = lane_upper(adj, b0, b1, last, lp);
            int64_t b = lane_gallop(adj, a, b1, hi, lp);
            if (b - a <= kLaneScanMax) {
                for (int64_t i = a; i < b; i++) {
                    int32_t y = __ldg(&adj[i].x);
                    bool bad = false;
#pragma unroll
                    for (int l = 0; l < kMaxV; l++) bad |= (l < nv) & (y == img[l]);
                    c += !bad;
                }
                sc = (unsigned long long)(b - a);
            } else {
                c = b - a;
#pragma unroll
                for (int l = 0; l < kMaxV; l++) {
                    if (l < nv) c -= out ? pair_count(g, x, img[l], last, hi, hp, pp)
                                         : pair_count(g, img[l], x, last, hi, hp, pp);
                }
            }
        }
        if (kStats) {
            w.v[kStHashProbe] += hp;
            w.v[kStPairProbe] += pp;
            w.v[kStListProbe] += lp;
            w.v[kStCand] += sc;
            w.v[kStLeaf] += 1;
        }
        return c;
    }

    // Leaf node L's last level for all survivor lanes S of level k, one ref at a time.
    // A star leaf whose window is the frame's own counts from the frame:
    // the later survivors of level k (suffix count `suf` of the chunk) minus
    // the later edges of the lane's own (src, dst) run inside the window.
    // S: lanes that evaluate; Sall: every survivor of the chunk (for the star count).
    // The leaf edge's two endpoints were mapped before level k, so every lane
    // counts edges of one pair, xu -> xv, in (its candidate, hi]: lane 0 finds
    // the run and the part of it inside (eid[k-1], hi] once (cached per warp
    // while the pair, the window end and the frame start stay the same), and
    // each lane searches only that part.
    __device__ void uniform_pair_window(const DevNode &L, int lv, int k, int32_t hi, const int32_t **run,
                                        int32_t *wlo, int32_t *whi) {
        const int32_t xu = ws.m2g[L.eu[lv]], xv = ws.m2g[L.ev[lv]];
        const int32_t flast = ws.eid[k - 1];
        const unsigned long long k1 = (unsigned long long)(uint32_t)xu | ((unsigned long long)(uint32_t)xv << 32);
        const unsigned long long k2 = (unsigned long long)(uint32_t)hi | ((unsigned long long)(uint32_t)flast << 32);
        __syncwarp();
        if (lane == 0 && (ws.pc_k1 != k1 || ws.pc_k2 != k2)) {
            int64_t st, len;
            unsigned long long hp = 0, pp = 0;
            pair_run(p.g, xu, xv, &st, &len, hp);
            const int32_t *r = p.g.pair_eid + st;
            const int64_t a = lane_upper_e(r, 0, len, flast, pp);
            const int64_t b = lane_gallop_e(r, a, len, hi, pp);
            ws.pc_k1 = k1;
            ws.pc_k2 = k2;
            ws.pc_st = st;
            ws.pc_wlo = (int32_t)a;
            ws.pc_whi = (int32_t)b;
            if (kStats) {
                w.v[kStHashProbe] += hp;
                w.v[kStPairProbe] += pp;
            }
        }
        __syncwarp();
        *run = p.g.pair_eid + ws.pc_st;
        *wlo = ws.pc_wlo;
        *whi = ws.pc_whi;
    }

    __device__ void leaf_batch(const DevNode &L, int k, uint32_t S, int uk, int vk, int32_t cs, int32_t cd,
                               int32_t last, int32_t fhi, int64_t suf, int32_t y, uint32_t peers, uint32_t Sall) {
        const bool star = (L.flags & kNodeStarLeaf) && ws.star[k];
        const uint32_t above = (lane == 31) ? 0u : ~((2u << lane) - 1u);       // lanes after this one
        const int lv = k + 1;
        const bool uni = k >= 1 && L.eu[lv] < L.nvb[k] && L.ev[lv] < L.nvb[k];   // same pair for every lane
        for (int i = 0; i < L.n_ref; i++) {
            const DevRef ref = TM_REF(L.ref_begin + i);
            if (!((rmask >> ref.query) & 1ull)) continue;
            const int32_t hi = ehi(ref.delta);
            unsigned long long c = 0;
            const int32_t *urun = nullptr;
            int32_t uwlo = 0, uwhi = 0;
            if (uni) uniform_pair_window(L, lv, k, hi, &urun, &uwlo, &uwhi);
            if (((S >> lane) & 1u) && last < hi) {
                if (uni) {
                    unsigned long long pp = 0;
                    c = (unsigned long long)(uwhi - lane_upper_e(urun, uwlo, uwhi, last, pp));
                    if (kStats) {
                        w.v[kStPairProbe] += pp;
                        w.v[kStLeaf] += 1;
                    }
                } else if (star && hi == fhi) {
                    unsigned long long pr = 0;
                    const int64_t later = suf + __popc(Sall & above);
                    int64_t same;
                    const int8_t sm = ws.same_mode[k];
                    const uint32_t slot = ((uint32_t)y * 2654435761u) >> kSlotShift;
                    const unsigned long long ent = sm == kSameTable ? ws.cslot[slot] : 0ull;
                    const uint32_t key = (uint32_t)(ent >> 32);
                    if (sm == kSameChunk) {
                        same = __popc(peers & above);
                    } else if (sm == kSameTable && key == (uint32_t)y) {
                        same = (int64_t)(uint32_t)ent + __popc(peers & above);
                    } else if (sm == kSameTable && key == kCacheEmpty) {
                        // a value seen above would have claimed this empty slot
                        same = __popc(peers & above);
                    } else {
                        same = run_tail(p.g.pair_eid, __ldg(p.g.pr_pos + last), __ldg(p.g.pr_end + last), hi, pr);
                        pr += 2;
                    }
                    c = (unsigned long long)(later - same);
                    gsame = (int32_t)same;
                    if (kStats) {
                        w.v[kStPairProbe] += pr;
                        w.v[kStLeaf] += 1;
                    }
                } else {
                    c = (unsigned long long)leaf_count(L, k + 1, uk, vk, cs, cd, last, hi);
                }
            }
            if (L.ref_begin + i == acc_ref) {           // summed once when the frame is drained
                acc += c;
                continue;
            }
            c = warp_sum_u64(c);
            if (lane == 0) add_count(ref.counter, c);
        }
    }

    // Chunk-level work for survivors S of level k of node N: count the refs
    // of a completed node, count single-edge leaves lane-parallel; returns
    // the survivors to descend.
    __device__ uint32_t survivors(int k, const DevNode &N, uint32_t S, int2 c, int64_t suf, uint32_t peers) {
        if (S == 0) return 0;
        const int uk = N.eu[k], vk = N.ev[k];
        int32_t cs, cd;
        const int8_t lt = ws.ltype[k];
        if (lt == kListOut || lt == kListPair) { cs = ws.lvert[k]; cd = c.x; }
        else if (lt == kListIn) { cs = c.x; cd = ws.lvert[k]; }
        else {                                             // the root edge, or a global-window level
            const bool mine = (S >> lane) & 1u;
            cs = mine ? __ldg(p.g.src + c.y) : 0;
            cd = mine ? __ldg(p.g.dst + c.y) : 0;
        }
        const bool complete = (k == N.k_end - 1);
        if (complete && N.n_ref > 0) {                     // Q_N counted (Algorithm 3)
            for (int i = 0; i < N.n_ref; i++) {
                const DevRef ref = TM_REF(N.ref_begin + i);
                if (!((rmask >> ref.query) & 1ull)) continue;
                uint32_t in = __ballot_sync(0xffffffffu, c.y <= ehi(ref.delta)) & S;
                if (lane == 0) add_count(ref.counter, (unsigned long long)__popc(in));
            }
        }
        if (complete && N.n_par > 0) {
            for (int ci = 0; ci < N.n_par; ci++) {
                const DevNode &L = TM_NODE(N.child_begin + N.n_seq + ci);
                if (!(L.qmask & rmask)) continue;
                uint32_t S2 = __ballot_sync(0xffffffffu, c.y < min(ehi(L.dmax), cap)) & S;
                if (S2) leaf_batch(L, k, S2, uk, vk, cs, cd, c.y, frame_hi(N), suf, c.x, peers, S);
            }
        }
        const bool par_self = (N.flags & kNodeParLeaf) && (k == N.k_end - 2);
        if (par_self) {
            uint32_t S2 = __ballot_sync(0xffffffffu, c.y < frame_hi(N)) & S;
            if (S2) leaf_batch(N, k, S2, uk, vk, cs, cd, c.y, frame_hi(N), suf, c.x, peers, S);
        }
        return ws.seq[k] ? S : 0u;
    }

    // Candidate list of level k of node N under the current mapping.
    __device__ __forceinline__ void list_of(const DevNode &N, int k, int8_t &lt, int32_t &x, int32_t &far) const {
        const int u = N.eu[k], v = N.ev[k], nv = N.nvb[k];
        const bool um = u < nv, vm = v < nv;
        x = 0;
        far = 0;
        if (um && vm) { lt = kListPair; x = ws.m2g[u]; far = ws.m2g[v]; }   // exactly the x -> far edges
        else if (um) { lt = kListOut; x = ws.m2g[u]; }
        else if (vm) { lt = kListIn; x = ws.m2g[v]; }
        else { lt = kListGlobal; }
    }

    __device__ __forceinline__ bool seq_of(const DevNode &N, int k) const {
        const bool complete = (k == N.k_end - 1);
        const bool par_self = (N.flags & kNodeParLeaf) && (k == N.k_end - 2);
        return complete ? (N.n_seq > 0) : !par_self;
    }

    __device__ void set_frame(int k, int node, int sib_end, int8_t lt, int32_t x, int64_t pos, int64_t end, bool seq,
                              int64_t wend, bool star, int64_t suf) {
        __syncwarp();
        if (lane == 0) {
            ws.node[k] = (int16_t)node;
            ws.sib_end[k] = (int16_t)sib_end;
            ws.ltype[k] = lt;
            ws.lvert[k] = x;
            ws.pos[k] = pos;
            ws.end[k] = end;
            ws.mask[k] = 0;
            ws.seq[k] = seq ? 1 : 0;
            ws.wend[k] = wend;
            ws.star[k] = star ? 1 : 0;
            ws.suf[k] = suf;
        }
        __syncwarp();
    }

    // Star leaves are counted from level k of node N.
    __device__ __forceinline__ bool star_of(const DevNode &N, int k) const {
        return ((N.flags & kNodeStarLeaf) && (N.flags & kNodeParLeaf) && k == N.k_end - 2) ||
               ((N.flags & kNodeStarKids) && k == N.k_end - 1);
    }

    // The per-warp table of later-occurrence counts belongs to the star
    // frame at level k from now on (empty), if no other frame holds it.
    __device__ void cache_claim(int k) {
        if (ws.cache_owner >= 0) return;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < kSlots / 32; i++) ws.cslot[lane + 32 * i] = kSlotEmpty;
        if (lane == 0) ws.cache_owner = k;
        __syncwarp();
    }

    __device__ void cache_release(int k) {
        __syncwarp();
        if (lane == 0 && ws.cache_owner == k) ws.cache_owner = -1;
        __syncwarp();
    }

    // Add the survivors of one chunk (groups of equal endpoint `peers`) to the
    // table.  `known`: for the lowest survivor of a group, its later survivors
    // with the same endpoint (exact), or -1.  A slot held by another endpoint
    // goes to the group's endpoint when its count so far (known + 1) is larger:
    // the hot endpoints keep their slots.  Every slot update is one
    // compare-and-swap of the whole (endpoint, count) word, so a count is
    // never added to an endpoint it was not taken for.
    __device__ void cache_add(uint32_t S, int32_t y, uint32_t peers, int32_t known) {
        if (((S >> lane) & 1u) && lane == __ffs(peers) - 1) {
            const uint32_t slot = ((uint32_t)y * 2654435761u) >> kSlotShift;
            const unsigned long long n = (unsigned long long)__popc(peers);
            unsigned long long e = ws.cslot[slot];
            while (true) {
                const uint32_t key = (uint32_t)(e >> 32);
                unsigned long long v;
                if (key == (uint32_t)y) v = e + n;
                // an empty slot: y was not seen above (it would have claimed the slot)
                else if (key == kCacheEmpty) v = ((unsigned long long)(uint32_t)y << 32) | n;
                else if (known >= 0 && (unsigned long long)known + 1 > (e & 0xffffffffull))
                    v = ((unsigned long long)(uint32_t)y << 32) | (unsigned long long)(known + 1);
                else break;
                const unsigned long long o = atomicCAS(&ws.cslot[slot], e, v);
                if (o == e) break;
                e = o;
            }
        }
        __syncwarp();
    }

    // Survivors of level k of node N in [pos, wend) (the filter of load_chunk);
    // with `fill`, also their endpoints into the table this frame owns.
    __device__ int64_t count_survivors(const DevNode &N, int k, int8_t lt, int64_t pos, int64_t wend, bool fill) {
        const int2 *adj = lt == kListOut ? p.g.out_adj : p.g.in_adj;
        const int32_t last = ws.eid[k - 1];
        const int32_t hi = frame_hi(N);
        const int nv = N.nvb[k];
        int64_t n = 0;
        for (int64_t b = pos; b < wend; b += 32) {
            const int64_t i = b + lane;
            bool ok = false;
            int2 c = make_int2(0, 0);
            if (i < wend) {
                c = __ldg(adj + i);
                bool bad = false;
#pragma unroll
                for (int l = 0; l < kMaxV; l++) bad |= (l < nv) & (c.x == ws.m2g[l]);
                ok = !bad && c.y > last && c.y <= hi;
            }
            const uint32_t S = __ballot_sync(0xffffffffu, ok);
            n += __popc(S);
            if (fill) cache_add(S, c.x, __match_any_sync(0xffffffffu, ok ? c.x : -1), -1);
            if (kStats && lane == 0) w.v[kStCand] += (unsigned long long)((wend - b) < 32 ? (wend - b) : 32);
        }
        return n;
    }

    // End of a pair run's window: run[rel..len) relative to base b0, the first
    // position whose edge id exceeds hi; one lane gallops, the warp gets it.
    __device__ int64_t lane_gallop_warp(int64_t rel, int64_t len, int64_t b0, int32_t hi) {
        int64_t r = 0;
        unsigned long long pr = 0;
        if (lane == 0) r = lane_gallop_e(p.g.pair_eid + b0, rel, len, hi, pr);
        if (kStats && lane == 0) w.v[kStPairProbe] += pr;
        return __shfl_sync(0xffffffffu, r, 0);
    }

    // Open level k for node `node` (siblings up to sib_end): the slice of
    // its list with edge ids in (eid[k-1], ehi].
    __device__ void open(int k, int node, int sib_end) {
        cache_release(k);                               // a sibling re-opening this level
        if (!chk(node >= 0 && node < TM_NNODES && sib_end <= TM_NNODES)) {
            set_frame(k, 0, 0, kListGlobal, 0, 0, 0, false, 0, false, 0);   // an empty frame
            return;
        }
        const DevNode &N = TM_NODE(node);
        if (!(N.qmask & rmask)) {                       // no query of this root below this node
            set_frame(k, node, sib_end, kListGlobal, 0, 0, 0, false, 0, false, 0);
            return;
        }
        const int32_t last = ws.eid[k - 1];
        const int32_t hi = frame_hi(N);
        int8_t lt;
        int32_t x, far;
        list_of(N, k, lt, x, far);
        int64_t start, end;
        int64_t deg = p.g.E;                            // length of the list searched
        if (kHasGlobal && lt == kListGlobal) {
            start = (int64_t)last + 1;
            end = (int64_t)hi + 1;
        } else if (lt == kListPair) {                   // both endpoints mapped: the x -> far run
            int64_t st = 0, len = 0;
            unsigned long long hp = 0;
            if (lane == 0) pair_run(p.g, x, far, &st, &len, hp);
            st = __shfl_sync(0xffffffffu, st, 0);
            len = __shfl_sync(0xffffffffu, len, 0);
            if (kStats && lane == 0) w.v[kStHashProbe] += hp;
            const int64_t b0 = st, b1 = st + len;
            deg = len;
            start = (len <= 32) ? b0 : warp_upper_e(p.g.pair_eid, b0, b1, last, lane, w.v[kStPairProbe]);
            end = (b1 - start <= 32) ? b1 : b0 + lane_gallop_warp(start - b0, b1 - b0, b0, hi);
        } else {
            const int64_t *off = lt == kListOut ? p.g.out_off : p.g.in_off;
            const int2 *adj = lt == kListOut ? p.g.out_adj : p.g.in_adj;
            const int64_t b0 = __ldg(off + x), b1 = __ldg(off + x + 1);
            deg = b1 - b0;
            // the list of an endpoint of the previous match starts right after it (per-edge index)
            const int64_t ap = after_pos(p.g, lt == kListOut, x, last, ws.m2g[N.eu[k - 1]], ws.m2g[N.ev[k - 1]]);
            if (ap >= 0) start = ap;
            else if (b1 - b0 <= 32) start = b0;                 // the chunk mask drops ids <= last
            else start = warp_upper(adj, b0, b1, last, lane, w.v[kStListProbe]);
            end = (b1 - start <= 32) ? b1 : warp_gallop(adj, start, b1, hi, lane, w.v[kStListProbe]);
        }
        const bool star = (lt == kListOut || lt == kListIn) && star_of(N, k);
        if (lane == 0) ws.lfar[k] = far;
        set_frame(k, node, sib_end, lt, x, start, end, seq_of(N, k), end, star, 0);
        if (star) {
            int8_t sm = kSameGallop;
            if (end - start <= 32) sm = kSameChunk;      // every later entry is in this one chunk
            else if (ws.cache_owner < 0) { cache_claim(k); sm = kSameTable; }
            if (lane == 0) ws.same_mode[k] = sm;
            __syncwarp();
        }
        if (kStats && lane == 0) {
            w.v[kStExp]++;
            w.v[kStLogDeg] += (unsigned long long)(64 - __clzll((unsigned long long)deg));   // ceil(log2(deg + 1))
        }
        if (k == 1 && split_h > 1) force_split(k, split_h);
    }

    // Planned split: cut the unscanned part of level k into `parts` slices of
    // whole chunks, keep the first, queue the rest.
    __device__ void force_split(int k, int parts) {
        const int64_t pos = ws.pos[k], end = ws.end[k];
        const int64_t rem = end - pos;
        if (rem <= 32) return;
        int64_t sz = (rem + parts - 1) / parts;
        sz = (sz + 31) & ~31ll;
        if (ws.star[k]) {                              // scanned top-down: keep the top slice
            const int64_t keep = end - sz;
            for (int64_t lo = pos; lo < keep; lo += sz)
                if (!push_task(k, lo, min(keep, lo + sz))) return;
            __syncwarp();
            if (lane == 0) ws.pos[k] = keep;
            __syncwarp();
            return;
        }
        for (int64_t lo = pos + sz; lo < end; lo += sz)
            if (!push_task(k, lo, min(end, lo + sz))) return;
        __syncwarp();
        if (lane == 0) ws.end[k] = pos + sz;
        __syncwarp();
    }

    // ---------------------------------------------------------------- tasks

    // Publish the slice [lo, hi) of level k under the current partial match;
    // false when the queue is full (the caller keeps the work).
    __device__ bool push_task(int k, int64_t lo, int64_t hi) {
        unsigned int slot = 0;
        if (lane == 0) slot = atomicAdd(&p.q->tail, 1u);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= (unsigned int)kQueueCap) return false;
        Task *tk = p.tasks + slot;
        if (lane < kMaxE) tk->eid[lane] = lane < k ? ws.eid[lane] : -1;
        if (lane == 0) {
            tk->ri = (int32_t)ri;
            tk->node = ws.node[k];
            tk->k = (int8_t)k;
            tk->lo = lo;
            tk->hi = hi;
            tk->wend = ws.wend[k];
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            for (int i = 0; i < TM_TEST_PUBLISH_PAUSE; i++) __nanosleep(1000);
            atomicExch(p.ready + slot, 1);
        }
        if (kStats && lane == 0) w.v[kStSplit]++;
        __syncwarp();
        return true;
    }

    // Sibling splitting (the paper's GPU load balancing): the children
    // [first + 1, end) of the current partial match go to the queue as one
    // task each, when warps are idle (or always, for tests); returns the end
    // of the children this warp keeps (first + 1 when every push succeeded).
    __device__ int split_siblings(int k, int first, int end) {
        int idle = 0;
        if (lane == 0 && !p.sib_always) idle = vload(&p.q->idle);
        idle = __shfl_sync(0xffffffffu, idle, 0);
        if (!p.sib_always && idle <= 0) return end;
        for (int c = end - 1; c > first; c--) {      // the last child first: the warp keeps a prefix
            if (!push_task_node(k, c)) return c + 1;
            end = c;
        }
        return end;
    }

    // Publish "open node `node` at level k" under the current partial match.
    __device__ bool push_task_node(int k, int node) {
        unsigned int slot = 0;
        if (lane == 0) slot = atomicAdd(&p.q->tail, 1u);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= (unsigned int)kQueueCap) return false;
        Task *tk = p.tasks + slot;
        if (lane < kMaxE) tk->eid[lane] = lane < k ? ws.eid[lane] : -1;
        if (lane == 0) {
            tk->ri = (int32_t)ri;
            tk->node = (int16_t)node;
            tk->k = (int8_t)k;
            tk->lo = -1;
            tk->hi = -1;
            tk->wend = 0;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            for (int i = 0; i < TM_TEST_PUBLISH_PAUSE; i++) __nanosleep(1000);
            atomicExch(p.ready + slot, 1);
        }
        if (kStats && lane == 0) w.v[kStSplit]++;
        __syncwarp();
        return true;
    }

    // Multi-offload: hand up to min(idle warps, offload_max) pieces of whole
    // chunks of level kb's unscanned slice to the queue at once, keeping one
    // piece; returns false when nothing was handed over.
    __device__ bool offload(int kb, int idle) {
        const int64_t pos = ws.pos[kb], end = ws.end[kb];
        const int64_t rem = end - pos;
        const int64_t minsz = ws.seq[kb] ? p.donate_seq : p.donate_leaf;
        int pieces = min(idle, p.offload_max);
        pieces = (int)min((int64_t)pieces, rem / max(minsz, (int64_t)32) - 1);
        if (pieces < 1) pieces = 1;
        const int64_t sz = ((rem + pieces) / (pieces + 1) + 31) & ~31ll;
        if (ws.star[kb]) {                           // scanned top-down: keep the top piece
            const int64_t keep = max(pos, end - sz);
            int64_t cur = pos;
            for (int i = 0; i < pieces && cur < keep; i++) {
                const int64_t hi = min(keep, cur + sz);
                if (!push_task(kb, cur, hi)) break;
                cur = hi;
            }
            __syncwarp();
            if (lane == 0) ws.pos[kb] = cur;
            __syncwarp();
            return cur > pos;
        }
        const int64_t keep = min(end, pos + sz);      // keep the bottom piece
        int64_t cur = end;
        for (int i = 0; i < pieces && cur > keep; i++) {
            const int64_t lo = max(keep, cur - sz);
            if (!push_task(kb, lo, cur)) break;
            cur = lo;
        }
        __syncwarp();
        if (lane == 0) ws.end[kb] = cur;
        __syncwarp();
        return cur < end;
    }

    // Hand [mid, end) of the shallowest long slice in levels [kbase, top] to the queue.
    __device__ void maybe_donate(int kbase, int top) {
        int idle = 0;
        unsigned int tail = 0;
        if (lane == 0) {
            idle = vload(&p.q->idle);
            tail = vloadu(&p.q->tail);
        }
        idle = __shfl_sync(0xffffffffu, idle, 0);
        tail = __shfl_sync(0xffffffffu, tail, 0);
        if (idle <= 0 || tail >= (unsigned int)(kQueueCap - 64)) return;
        for (int kb = max(kbase, 1); kb <= top; kb++) {
            const int64_t pos = ws.pos[kb], end = ws.end[kb];
            const int64_t rem = end - pos;
            if (rem < (ws.seq[kb] ? p.donate_seq : p.donate_leaf)) continue;
            if (kExt && p.siblings) {                  // multi-offload
                offload(kb, idle);
                return;
            }
            const int64_t mid = pos + (((rem >> 1) + 31) & ~31ll);
            if (ws.star[kb]) {                         // scanned top-down: hand over the bottom part
                if (push_task(kb, pos, mid)) {
                    __syncwarp();
                    if (lane == 0) ws.pos[kb] = mid;
                    __syncwarp();
                }
            } else if (push_task(kb, mid, end)) {
                __syncwarp();
                if (lane == 0) ws.end[kb] = mid;
                __syncwarp();
            }
            return;
        }
    }

    // Claim a published task; false if none (or a bounded wait expired).
    __device__ bool pop(Task &tk) {
        int slot = -1;
        if (lane == 0) {
            while (true) {
                unsigned int h = vloadu(&p.q->head);
                unsigned int t = min(vloadu(&p.q->tail), (unsigned int)kQueueCap);
                if (h >= t) break;
                if (atomicCAS(&p.q->head, h, h + 1) == h) { slot = (int)h; break; }
            }
            if (slot >= 0) {
                long long spins = 0;
                while (vload(p.ready + slot) == 0) {
                    if (++spins > kReadySpins) { atomicOr(&p.q->error, kErrTimeout); slot = -2; break; }
                    __nanosleep(64);
                }
                __threadfence();
            }
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot < 0) return false;
        __syncwarp();
        const Task *src = p.tasks + slot;
        tk.ri = src->ri;
        tk.node = src->node;
        tk.k = src->k;
#pragma unroll
        for (int i = 0; i < kMaxE; i++) tk.eid[i] = src->eid[i];
        tk.lo = src->lo;
        tk.hi = src->hi;
        tk.wend = src->wend;
        return true;
    }

    // Idle: wait (bounded) until a task is published or all work is done.
    // Returns true when a task may be available.
    __device__ bool wait_for_work() {
        int r = 0;
        if (lane == 0) {
            atomicSub(&p.q->busy, 1);
            atomicAdd(&p.q->idle, 1);
            bool done = false;
            for (long long it = 0; it < kIdleSpins; it++) {
                unsigned int h = vloadu(&p.q->head);
                unsigned int t = min(vloadu(&p.q->tail), (unsigned int)kQueueCap);
                if (h < t) {
                    atomicAdd(&p.q->busy, 1);
                    r = 1;
                    break;
                }
                if (vload(&p.q->busy) == 0) {
                    __threadfence();
                    h = vloadu(&p.q->head);
                    t = min(vloadu(&p.q->tail), (unsigned int)kQueueCap);
                    if (h >= t) { done = true; break; }  // nothing queued, nobody working: done
                }
                __nanosleep(256);
            }
            // the wait ran out while other warps still held work: this warp
            // leaves (their work stays theirs, so counts are unaffected)
            if (!r && !done) atomicAdd(&p.q->idle_expired, 1);
            atomicSub(&p.q->idle, 1);
        }
        return __shfl_sync(0xffffffffu, r, 0) != 0;
    }

    // ---------------------------------------------------------------- mining

    // Windows of every distinct delta for root r.
    __device__ void windows(int32_t r) {
        const int64_t tr0 = __ldg(p.g.t + r);
        for (int j = lane; j < TM_NDELTAS; j += 32) {
            unsigned long long pr = 0;
            ws.ehi[j] = window_end(p.g.t, p.g.E, r, sat_add(tr0, TM_DELTA(j)), pr);
            if (kStats) w.v[kStListProbe] += pr;
        }
        __syncwarp();
        // with request masks, no frame of this root scans past its own requests' largest window
        cap = INT32_MAX;
        if (rmask != ~0ull) {
            int32_t c = -1;
            const int q = lane, q2 = lane + 32;
            if ((rmask >> q) & 1ull) { const int d = TM_QDMAX(q); if (d >= 0) c = max(c, ehi(d)); }
            if ((rmask >> q2) & 1ull) { const int d = TM_QDMAX(q2); if (d >= 0) c = max(c, ehi(d)); }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
            cap = c < 0 ? INT32_MAX : c;
        }
    }

    __device__ __forceinline__ int32_t frame_hi(const DevNode &N) const { return min(ehi(N.dmax), cap); }

    // First position of level k's next chunk (star frames run from the top).
    __device__ __forceinline__ int64_t chunk_base(int k) const {
        return ws.star[k] ? max(ws.pos[k], ws.end[k] - 32) : ws.pos[k];
    }

    // This lane's entry of the chunk of level k starting at `base` (lists end at `end`).
    __device__ __forceinline__ int2 fetch(int8_t lt, int64_t base, int64_t end, int32_t far) const {
        const int64_t i = base + lane;
        int2 c = make_int2(0, 0);
        if (i < end) {
            if (lt == kListOut) c = __ldg(&p.g.out_adj[i]);
            else if (lt == kListIn) c = __ldg(&p.g.in_adj[i]);
            else if (lt == kListPair) c = make_int2(far, __ldg(p.g.pair_eid + i));
            else if (kHasGlobal) c = make_int2(0, (int32_t)i);
        }
        return c;
    }

    // Filter the chunk of level k at `base` (entries c, valid below `end`):
    // advance the frame, count and evaluate its survivors, keep those to
    // descend in mask[k].
    __device__ void step(int k, int64_t base, int64_t end, int2 c) {
        const DevNode &N = TM_NODE(ws.node[k]);
        const int8_t lt = ws.ltype[k];
        const bool down = ws.star[k];                   // star frames run from the top
        const int64_t i = base + lane;
        const int32_t last = ws.eid[k - 1];
        const int32_t hi = frame_hi(N);
        bool valid = i < end;
        const bool inwin = c.y <= hi;
        const uint32_t outw = __ballot_sync(0xffffffffu, valid && !inwin);
        valid = valid && inwin && c.y > last;
        // structural predicate (reading 3), branch-free over the mapped labels
        const int u = N.eu[k], v = N.ev[k], nv = N.nvb[k];
        const bool um = u < nv, vm = v < nv;
        bool ok;
        if (kHasGlobal && lt == kListGlobal) {
            int32_t s = valid ? __ldg(p.g.src + c.y) : 0, d = valid ? __ldg(p.g.dst + c.y) : 0;
            bool bad = (s == d);
#pragma unroll
            for (int l = 0; l < kMaxV; l++) bad |= (l < nv) & ((s == ws.m2g[l]) | (d == ws.m2g[l]));
            ok = !bad;
        } else if (um && vm) {
            ok = lt == kListPair || c.x == (lt == kListOut ? ws.m2g[v] : ws.m2g[u]);
        } else {
            bool bad = false;
#pragma unroll
            for (int l = 0; l < kMaxV; l++) bad |= (l < nv) & (c.x == ws.m2g[l]);
            ok = !bad;
        }
        const uint32_t S = __ballot_sync(0xffffffffu, valid && ok);
        const uint32_t VB = __ballot_sync(0xffffffffu, valid);
        if (kStats && lane == 0) w.v[kStCand] += (unsigned long long)__popc(VB);
        ws.cand[k][lane] = c;
        const int64_t suf = ws.suf[k];
        __syncwarp();
        if (lane == 0) {
            ws.cbase[k] = base;
            if (down) {
                ws.end[k] = min(ws.end[k], base);
                ws.suf[k] = suf + __popc(S);
            } else {
                ws.pos[k] = outw ? ws.end[k] : max(ws.pos[k], base + 32);
            }
        }
        const uint32_t peers = down ? __match_any_sync(0xffffffffu, ((S >> lane) & 1u) ? c.x : -1) : 0u;
        gsame = -1;
        uint32_t D = survivors(k, N, S, c, suf, peers);
        if (down && ws.cache_owner == k) cache_add(S, c.x, peers, gsame);
        __syncwarp();
        if (lane == 0) ws.mask[k] = D;
        __syncwarp();
    }

    // Load and filter the next chunk of level k.
    __device__ void load_chunk(int k) {
        const int64_t base = chunk_base(k);
        const int64_t end = ws.end[k];
        step(k, base, end, fetch(ws.ltype[k], base, end, ws.lfar[k]));
    }

    // The hot case of drain: a counting-only star frame whose work per
    // survivor is one star leaf with one ref and, on the node's last level,
    // the node's own refs, all counted in the frame's own window (the last
    // two edges of an out- or in-star; the 3-star that is the 4-star's
    // prefix).  Every survivor matches such a node ref, so those refs get the
    // frame's survivor total at the end.  The frame's cursor, end and
    // survivor suffix stay in registers and the mapped labels are read once;
    // the shared-memory frame is brought up to date around a donation and at
    // the end.  Counts, work counters and donations are those of the general
    // loop.  Returns false (nothing done) when the level is not of that form.
    __device__ bool drain_star(int k, int kbase) {
        if (!ws.star[k]) return false;
        const DevNode &N = TM_NODE(ws.node[k]);
        const int32_t fhi = frame_hi(N);
        const bool complete = (k == N.k_end - 1);
        const DevNode *L = nullptr;
        if (!complete) {
            if ((N.flags & kNodeParLeaf) && k == N.k_end - 2) L = &N;
        } else if (N.n_par == 1) {
            L = &TM_NODE(N.child_begin + N.n_seq);
            for (int i = 0; i < N.n_ref; i++) {
                const DevRef r = TM_REF(N.ref_begin + i);
                if (((rmask >> r.query) & 1ull) && ehi(r.delta) != fhi) return false;
            }
        }
        if (!L || !(L->flags & kNodeStarLeaf) || L->n_ref != 1) return false;
        const DevRef ref = TM_REF(L->ref_begin);
        if (!((rmask >> ref.query) & 1ull) || ehi(ref.delta) != fhi) return false;

        const int2 *adj = ws.ltype[k] == kListOut ? p.g.out_adj : p.g.in_adj;
        const int nv = N.nvb[k];
        int32_t lab[kMaxV];
#pragma unroll
        for (int l = 0; l < kMaxV; l++) lab[l] = l < nv ? ws.m2g[l] : -1;   // -1 is no vertex
        const int8_t sm = ws.same_mode[k];
        const bool own = ws.cache_owner == k;
        const uint32_t above = (lane == 31) ? 0u : ~((2u << lane) - 1u);
        // positions and counts fit 32 bits (lists and windows below 2^31 entries)
        int32_t pos = (int32_t)ws.pos[k], end = (int32_t)ws.end[k], suf = (int32_t)ws.suf[k];
        const int32_t suf0 = suf;
        unsigned long long acc_l = 0;
        int32_t cb = max(pos, end - 32), ce = end;       // the chunk [cb, ce), scanned from the top
        int2 c = (cb + lane < ce) ? __ldg(adj + cb + lane) : make_int2(0, 0);
        while (true) {
            end = cb;                                    // claimed: a donation cannot hand it out
            if (p.react && ++polls >= p.poll_every) {
                polls = 0;
                __syncwarp();
                if (lane == 0) {
                    ws.end[k] = end;
                    ws.pos[k] = pos;
                }
                __syncwarp();
                maybe_donate(kbase, k);
                pos = (int32_t)ws.pos[k];                // a donation hands over the bottom part
            }
            const bool more = pos < end;
            int32_t nb = 0;
            int2 nc = make_int2(0, 0);
            if (more) {
                nb = max(pos, end - 32);
                if (nb + lane < end) nc = __ldg(adj + nb + lane);
            }
            const bool valid = cb + lane < ce;
            bool bad = false;
#pragma unroll
            for (int l = 0; l < kMaxV; l++) bad |= (c.x == lab[l]);
            const bool ok = valid && !bad;
            const uint32_t S = __ballot_sync(0xffffffffu, ok);
            const uint32_t peers = (sm != kSameGallop) ? __match_any_sync(0xffffffffu, ok ? c.x : -1) : 0u;
            int32_t known = -1;
            if (ok) {
                const int32_t later = suf + __popc(S & above);
                int32_t same;
                if (sm == kSameChunk) {
                    same = __popc(peers & above);
                } else {
                    const uint32_t slot = ((uint32_t)c.x * 2654435761u) >> kSlotShift;
                    const unsigned long long ent = sm == kSameTable ? ws.cslot[slot] : 0ull;
                    const uint32_t key = (uint32_t)(ent >> 32);
                    if (sm == kSameTable && key == (uint32_t)c.x) {
                        same = (int32_t)(uint32_t)ent + __popc(peers & above);
                    } else if (sm == kSameTable && key == kCacheEmpty) {
                        same = __popc(peers & above);    // a value seen above would have claimed the slot
                    } else {
                        unsigned long long pr = 0;
                        same = (int32_t)run_tail(p.g.pair_eid, __ldg(p.g.pr_pos + c.y), __ldg(p.g.pr_end + c.y), fhi, pr);
                        if (kStats) w.v[kStPairProbe] += pr + 2;
                    }
                }
                acc_l += (unsigned long long)(uint32_t)(later - same);
                known = same;
                if (kStats) w.v[kStLeaf] += 1;
            }
            if (kStats) {
                const uint32_t VB = __ballot_sync(0xffffffffu, valid);     // every lane votes
                if (lane == 0) w.v[kStCand] += (unsigned long long)__popc(VB);
            }
            suf += __popc(S);
            if (own) cache_add(S, c.x, peers, known);
            if (!more) break;
            ce = cb;
            cb = nb;
            c = nc;
        }
        __syncwarp();
        if (lane == 0) {
            ws.pos[k] = pos;
            ws.end[k] = end;
            ws.suf[k] = suf;
            ws.mask[k] = 0;
        }
        __syncwarp();
        const unsigned long long tot = warp_sum_u64(acc_l);
        if (lane == 0) {
            add_count(ref.counter, tot);
            if (complete) {                              // Q_N: every survivor of the frame matches
                for (int i = 0; i < N.n_ref; i++) {
                    const DevRef r = TM_REF(N.ref_begin + i);
                    if ((rmask >> r.query) & 1ull) add_count(r.counter, (unsigned long long)(suf - suf0));
                }
            }
        }
        return true;
    }

    // A level whose survivors are only counted (nothing to descend): run all
    // its chunks, fetching the next chunk before filtering the current one.
    __device__ void drain(int k, int kbase) {
        if (drain_star(k, kbase)) return;
        const int8_t lt = ws.ltype[k];
        int64_t base = chunk_base(k);
        int64_t end = ws.end[k];
        const int32_t far = ws.lfar[k];
        int2 c = fetch(lt, base, end, far);
        // a star frame counting one star leaf with one ref: sum that ref's
        // counts in registers across chunks and add them once
        const DevNode &N = TM_NODE(ws.node[k]);
        acc = 0;
        acc_ref = -1;
        if (ws.star[k]) {
            const DevNode *Ls = nullptr;
            if ((N.flags & kNodeParLeaf) && k == N.k_end - 2) Ls = &N;
            else if (k == N.k_end - 1 && N.n_par == 1) Ls = &TM_NODE(N.child_begin + N.n_seq);
            if (Ls && (Ls->flags & kNodeStarLeaf) && Ls->n_ref == 1) acc_ref = Ls->ref_begin;
        }
        while (true) {
            // claim the current chunk so a donation cannot hand it out
            __syncwarp();
            if (lane == 0) {
                if (ws.star[k]) ws.end[k] = base;
                else ws.pos[k] = base + 32;
            }
            __syncwarp();
            if (p.react && ++polls >= p.poll_every) {
                polls = 0;
                maybe_donate(kbase, k);
            }
            const bool more = ws.pos[k] < ws.end[k];
            int64_t nbase = 0, nend = 0;
            int2 nc = make_int2(0, 0);
            if (more) {
                nbase = chunk_base(k);
                nend = ws.end[k];
                nc = fetch(lt, nbase, nend, far);
            }
            step(k, base, end, c);
            if (!more || ws.pos[k] >= ws.end[k]) break;   // done, or the window ended in this chunk
            base = nbase;
            end = nend;
            c = nc;
        }
        if (acc_ref >= 0) {
            const unsigned long long tot = warp_sum_u64(acc);
            if (lane == 0) add_count(TM_REF(acc_ref).counter, tot);
            acc_ref = -1;
            acc = 0;
        }
    }

    // Depth-first walk of the frames from level `kbase` up.
    __device__ void run(int kbase) {
        const DevGraph &g = p.g;
        int k = kbase;
        while (k >= kbase) {
            uint32_t m = ws.mask[k];
            if (m) {
                const int j = __ffs(m) - 1;
                const int2 cj = ws.cand[k][j];
                const DevNode &N = TM_NODE(ws.node[k]);
                const int8_t lt = ws.ltype[k];
                int32_t cs, cd;
                if (lt == kListOut || lt == kListPair) { cs = ws.lvert[k]; cd = cj.x; }
                else if (lt == kListIn) { cs = cj.x; cd = ws.lvert[k]; }
                else { cs = __ldg(g.src + cj.y); cd = __ldg(g.dst + cj.y); }   // root edge or global window
                __syncwarp();
                if (lane == 0) {
                    ws.mask[k] = m & (m - 1);
                    ws.eid[k] = cj.y;
                    ws.mpos[k] = ws.cbase[k] + j;
                    if (chk(N.eu[k] < kMaxV && N.ev[k] < kMaxV)) {
                        ws.m2g[N.eu[k]] = cs;
                        ws.m2g[N.ev[k]] = cd;
                    }
                }
                __syncwarp();
                // (the checking build: no frame beyond the deepest level)
                if (k == N.k_end - 1) {
                    if (N.n_seq > 0 && chk(k + 1 < kMaxE)) {
                        int sib_end = N.child_begin + N.n_seq;
                        if (kExt && p.siblings && N.n_seq > 1) sib_end = split_siblings(k + 1, N.child_begin, sib_end);
                        open(k + 1, N.child_begin, sib_end);
                        k++;
                    }
                } else if (chk(k + 1 < kMaxE)) {
                    open(k + 1, ws.node[k], ws.node[k] + 1);
                    k++;
                }
                continue;
            }
            if (ws.pos[k] < ws.end[k]) {
                if (!ws.seq[k] && ws.end[k] - ws.pos[k] > 32) {   // counted only, several chunks: pipelined
                    drain(k, kbase);
                    continue;
                }
                if (p.react && ++polls >= p.poll_every) {
                    polls = 0;
                    maybe_donate(kbase, k);
                }
                load_chunk(k);
                continue;
            }
            if (ws.node[k] + 1 < ws.sib_end[k]) {        // next sibling from the same partial match
                open(k, ws.node[k] + 1, ws.sib_end[k]);
                continue;
            }
            cache_release(k);
            k--;
        }
    }

    // Root edge r as the first motif edge (Algorithm 1, first call).
    __device__ void root(int32_t r) {
        const DevGraph &g = p.g;
        const int32_t a = __ldg(g.src + r), b = __ldg(g.dst + r);
        if (a == b) return;                             // injective map needs a != b
        windows(r);
        if (lane == 0) {
            ws.cache_owner = -1;
            ws.pc_k1 = ~0ull;                           // no uniform pair window cached
        }
        const DevNode &N0 = TM_NODE(0);
        set_frame(0, 0, 1, kListGlobal, -1, 0, 0, seq_of(N0, 0), 0, false, 0);
        if (lane == 0) ws.cbase[0] = r;
        // level 0: the root edge as a one-candidate chunk on lane 0
        int2 c = make_int2(lane == 0 ? b : 0, lane == 0 ? r : 0);
        ws.cand[0][lane] = c;
        __syncwarp();
        uint32_t D = survivors(0, N0, 1u, c, 0, 0u);
        __syncwarp();
        if (lane == 0) ws.mask[0] = D;
        __syncwarp();
        run(0);
    }

    // ---------------------------------------------------------------- thread tier

    // Counts of one lane's root go to the shared counters with atomics (the
    // lanes of the warp add at once).
    __device__ __forceinline__ void add_count_lane(int32_t counter, unsigned long long c) {
        if (c == 0) return;
        if (!chk(counter >= 0 && counter < TM_NCOUNTERS)) return;
        if (p.smem_counters) atomicAdd(&s_cnt[counter], c);
        else atomicAdd(&p.counts[counter], c);
        if (p.per_root_counts)
            atomicAdd((unsigned long long *)&p.per_root_counts[ri * TM_NCOUNTERS + counter], c);
    }

    // The lane's frames of its own walk: per level, the node, its siblings'
    // end, the list kind and the unscanned positions [pos, end).
    struct LaneFrames {
        int16_t node[kMaxE], sib[kMaxE];
        int8_t lt[kMaxE];
        int32_t pos[kMaxE], end[kMaxE];
        int32_t eid[kMaxE];
        int32_t m2g[kMaxV];
        int32_t eh[kLaneDeltas];
    };

    // Open level k of `node` (siblings up to sib) on the lane's own frames:
    // the slice of its candidate list with edge ids in (eid[k-1], window end].
    __device__ void lane_open(LaneFrames &F, int k, int node, int sib) {
        const DevNode &N = TM_NODE(node);
        F.node[k] = (int16_t)node;
        F.sib[k] = (int16_t)sib;
        F.pos[k] = 0;
        F.end[k] = 0;
        F.lt[k] = kListGlobal;
        if (!(N.qmask & rmask)) return;
        const int32_t last = F.eid[k - 1];
        const int32_t hi = F.eh[N.dmax];
        const int u = N.eu[k], v = N.ev[k], nv = N.nvb[k];
        const bool um = u < nv, vm = v < nv;
        int8_t lt = kListGlobal;
        int32_t x = 0;
        if (um && vm) {
            const int32_t xu = F.m2g[u], xv = F.m2g[v];
            const int64_t du = __ldg(p.g.out_off + xu + 1) - __ldg(p.g.out_off + xu);
            const int64_t dv = __ldg(p.g.in_off + xv + 1) - __ldg(p.g.in_off + xv);
            if (du <= dv) { lt = kListOut; x = xu; } else { lt = kListIn; x = xv; }
        } else if (um) { lt = kListOut; x = F.m2g[u]; }
        else if (vm) { lt = kListIn; x = F.m2g[v]; }
        F.lt[k] = lt;
        if (lt == kListGlobal) {
            F.pos[k] = last + 1;
            F.end[k] = hi + 1;
            return;
        }
        const bool out = lt == kListOut;
        const int64_t *off = out ? p.g.out_off : p.g.in_off;
        const int2 *adj = out ? p.g.out_adj : p.g.in_adj;
        const int64_t b0 = __ldg(off + x), b1 = __ldg(off + x + 1);
        unsigned long long lp = 0;
        int64_t a = after_pos(p.g, out, x, last, F.m2g[N.eu[k - 1]], F.m2g[N.ev[k - 1]]);
        if (a < 0) a = lane_upper(adj, b0, b1, last, lp);
        const int64_t b = lane_gallop(adj, a, b1, hi, lp);
        F.pos[k] = (int32_t)a;
        F.end[k] = (int32_t)b;
        if (kStats) {
            w.v[kStListProbe] += lp;
            w.v[kStExp]++;
            w.v[kStLogDeg] += (unsigned long long)(64 - __clzll((unsigned long long)(b1 - b0)));
        }
    }

    // Level k of `node` has just been matched (F.eid[k], F.m2g): count what
    // completes here and open the next level; returns the deepest open level.
    __device__ int lane_matched(LaneFrames &F, int k, int node) {
        const DevNode &N = TM_NODE(node);
        const int32_t last = F.eid[k];
        const int32_t cs = F.m2g[N.eu[k]], cd = F.m2g[N.ev[k]];
        if (k == N.k_end - 1) {                         // C_N complete: Q_N, then the children
            for (int i = 0; i < N.n_ref; i++) {
                const DevRef ref = TM_REF(N.ref_begin + i);
                if (((rmask >> ref.query) & 1ull) && last <= F.eh[ref.delta]) add_count_lane(ref.counter, 1);
            }
            for (int ci = 0; ci < N.n_par; ci++) {
                const DevNode &L = TM_NODE(N.child_begin + N.n_seq + ci);
                for (int i = 0; i < L.n_ref; i++) {
                    const DevRef ref = TM_REF(L.ref_begin + i);
                    const int32_t hi = F.eh[ref.delta];
                    if (((rmask >> ref.query) & 1ull) && last < hi)
                        add_count_lane(ref.counter, (unsigned long long)leaf_count_img(L, k + 1, F.m2g, cs, cd, last, hi));
                }
            }
            if (N.n_seq > 0 && chk(k + 1 < kMaxE)) {
                lane_open(F, k + 1, N.child_begin, N.child_begin + N.n_seq);
                return k + 1;
            }
            return k;
        }
        if ((N.flags & kNodeParLeaf) && k == N.k_end - 2) {   // N's last edge counted from here
            for (int i = 0; i < N.n_ref; i++) {
                const DevRef ref = TM_REF(N.ref_begin + i);
                const int32_t hi = F.eh[ref.delta];
                if (((rmask >> ref.query) & 1ull) && last < hi)
                    add_count_lane(ref.counter, (unsigned long long)leaf_count_img(N, k + 1, F.m2g, cs, cd, last, hi));
            }
            return k;
        }
        if (!chk(k + 1 < kMaxE)) return k;
        lane_open(F, k + 1, node, node + 1);
        return k + 1;
    }

    // Root edge r on this lane alone: Algorithm 3 as a serial depth-first
    // walk over the lane's own frames (no warp collectives), the single-edge
    // leaves counted by the same window arithmetic as the warp tier.
    __device__ void lane_root(int32_t r) {
        const DevGraph &g = p.g;
        const int32_t a = __ldg(g.src + r), b = __ldg(g.dst + r);
        if (a == b) return;                             // injective map needs a != b
        LaneFrames F;
        const int64_t t0 = __ldg(g.t + r);
#pragma unroll
        for (int d = 0; d < kLaneDeltas; d++) {
            F.eh[d] = -1;
            if (d < TM_NDELTAS) {
                unsigned long long pr = 0;
                F.eh[d] = window_end(g.t, g.E, r, sat_add(t0, TM_DELTA(d)), pr);
                if (kStats) w.v[kStListProbe] += pr;
            }
        }
#pragma unroll
        for (int l = 0; l < kMaxV; l++) F.m2g[l] = -1;
        F.m2g[0] = a;                                   // the root edge is canonical 0 -> 1
        F.m2g[1] = b;
        F.eid[0] = r;
        int k = lane_matched(F, 0, 0);
        while (k >= 1) {
            if (F.pos[k] < F.end[k]) {
                const int32_t i = F.pos[k]++;
                const DevNode &N = TM_NODE(F.node[k]);
                const int u = N.eu[k], v = N.ev[k], nv = N.nvb[k];
                int32_t e, s, d;
                if (F.lt[k] == kListOut) {
                    const int2 c = __ldg(p.g.out_adj + i);
                    e = c.y; s = F.m2g[u]; d = c.x;
                } else if (F.lt[k] == kListIn) {
                    const int2 c = __ldg(p.g.in_adj + i);
                    e = c.y; s = c.x; d = F.m2g[v];
                } else {
                    e = i; s = __ldg(g.src + i); d = __ldg(g.dst + i);
                }
                if (kStats) w.v[kStCand]++;
                // structure with full injectivity (reading 3)
                bool ok = (u >= nv || s == F.m2g[u]) && (v >= nv || d == F.m2g[v]) && (u < nv || v < nv || s != d);
#pragma unroll
                for (int l = 0; l < kMaxV; l++)
                    if (l < nv) ok &= (u < nv || s != F.m2g[l]) && (v < nv || d != F.m2g[l]);
                if (!ok) continue;
                F.eid[k] = e;
                F.m2g[u] = s;
                F.m2g[v] = d;
                k = lane_matched(F, k, F.node[k]);
                continue;
            }
            if (F.node[k] + 1 < F.sib[k]) {                 // next sibling from the same partial match
                lane_open(F, k, F.node[k] + 1, F.sib[k]);
                continue;
            }
            k--;
        }
    }

    // A donated slice: rebuild the partial match, then walk its subtree.
    __device__ void task(const Task &tk) {
        const DevGraph &g = p.g;
        const int k = tk.k;
        if (!chk(k >= 1 && k < kMaxE && tk.node >= 0 && tk.node < TM_NNODES && tk.lo <= tk.hi &&
                 tk.eid[0] >= 0 && tk.eid[0] < g.E))
            return;
        windows(tk.eid[0]);
        const DevNode &N = TM_NODE(tk.node);
        if (lane == 0) {
            for (int i = 0; i < k; i++) {
                const int32_t e = tk.eid[i];
                ws.eid[i] = e;
                ws.m2g[N.eu[i]] = __ldg(g.src + e);
                ws.m2g[N.ev[i]] = __ldg(g.dst + e);
            }
        }
        __syncwarp();
        if (kExt && tk.lo < 0) {                       // a sibling task: this node's subtree alone
            if (lane == 0) ws.cache_owner = -1;
            __syncwarp();
            open(k, tk.node, tk.node + 1);
            run(k);
            return;
        }
        int8_t lt;
        int32_t x, far;
        list_of(N, k, lt, x, far);
        const bool star = (lt == kListOut || lt == kListIn) && star_of(N, k);
        if (lane == 0) {
            ws.cache_owner = -1;
            ws.lfar[k] = far;
        }
        __syncwarp();
        if (star) cache_claim(k);
        // a top-down slice needs the survivors above it, up to the window's end
        const int64_t suf = star ? count_survivors(N, k, lt, tk.hi, tk.wend, true) : 0;
        set_frame(k, tk.node, tk.node + 1, lt, x, tk.lo, tk.hi, seq_of(N, k), tk.wend, star, suf);
        if (lane == 0) ws.same_mode[k] = kSameTable;
        __syncwarp();
        run(k);
    }
};

template <bool kStats, bool kExt>
__device__ void flush_work(Miner<kStats, kExt> &M, const Work &before, const Params &p, int lane) {
    if (!kStats || !p.per_root_work) return;
    unsigned long long d[4];
    d[0] = warp_sum_u64(M.w.v[kStCand] - before.v[kStCand]);
    d[1] = warp_sum_u64(M.w.v[kStExp] - before.v[kStExp]);
    d[2] = warp_sum_u64(M.w.v[kStListProbe] + M.w.v[kStHashProbe] + M.w.v[kStPairProbe] -
                        before.v[kStListProbe] - before.v[kStHashProbe] - before.v[kStPairProbe]);
    d[3] = warp_sum_u64(M.w.v[kStLeaf] - before.v[kStLeaf]);
    if (lane == 0)
        for (int f = 0; f < 4; f++)
            if (d[f]) atomicAdd((unsigned long long *)&p.per_root_work[M.ri * TM_WORK_FIELDS + f], d[f]);
}

// kExt: the launch may use the extended schedules (a thread tier,
// TM_SCHED_TIERS; sibling splitting and multi-offload, TM_SCHED_SIBLINGS);
// only such launches carry their code.
template <bool kStats, bool kExt>
#ifndef TM_MIN_BLOCKS
#define TM_MIN_BLOCKS 3   // CTAs per SM the register budget is sized for (80 registers per thread)
#endif
__global__ void __launch_bounds__(kThreads, TM_MIN_BLOCKS) k_mine(Params p) {
    extern __shared__ unsigned long long s_cnt[];
    __shared__ WarpState s_ws[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_cnt = TM_NCOUNTERS;
    const int n_smem = p.smem_counters == 2 ? kWarps * n_cnt : (p.smem_counters ? n_cnt : 0);
    for (int i = threadIdx.x; i < n_smem; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    Miner<kStats, kExt> M(p, s_ws[warp], s_cnt + (p.smem_counters == 2 ? warp * n_cnt : 0), lane);
    if (lane == 0) s_ws[warp].pc_k1 = ~0ull;            // no uniform pair window cached yet
    __syncwarp();
    if (p.dynamic && lane == 0) atomicAdd(&p.q->busy, 1);
    // stats launch: this warp's cycles spent other than waiting for work
    const long long t_begin = kStats ? clock64() : 0;
    long long idle = 0;
    while (true) {
        if (p.dynamic) {
            Task tk;
            const long long tp = kStats ? clock64() : 0;
            const bool got = M.pop(tk);
            if (kStats && !got) idle += clock64() - tp;
            if (got) {
                M.ri = tk.ri;
                M.split_h = 0;
                M.rmask = p.root_qmask ? __ldg(p.root_qmask + tk.ri) : ~0ull;
                Work before = M.w;
                M.task(tk);
                flush_work(M, before, p, lane);
                continue;
            }
        }
        // warp tier: roots [0, n_warp); the thread tier takes the rest
        const int64_t n_warp = (kExt && p.tiers) ? min((int64_t)p.q->lane_from, p.n_roots) : p.n_roots;
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(&p.q->root_cursor, (unsigned long long)p.chunk);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (first < (unsigned long long)n_warp) {
            const int64_t last = min((int64_t)first + p.chunk, n_warp);
            for (int64_t ri = (int64_t)first; ri < last; ri++) {
                M.ri = ri;
                M.split_h = p.split ? __ldg(p.split + ri) : 0;
                M.rmask = p.root_qmask ? __ldg(p.root_qmask + ri) : ~0ull;
                const int32_t r = p.roots ? __ldg(p.roots + ri) : (int32_t)(p.root_lo + ri);
                if (r < 0 || r >= p.g.E) {                  // a device root list is not checked on the host
                    if (lane == 0) atomicOr(&p.q->error, kErrBadRoot);
                    continue;
                }
                Work before = M.w;
                if (kStats && lane == 0 && M.split_h > 1) M.w.v[kStSplitRoots]++;
                M.root(r);
                if (kStats && lane == 0) M.w.v[kStRoots]++;
                flush_work(M, before, p, lane);
            }
            continue;
        }
        if (kExt && p.tiers) {                           // thread tier: 32 roots, one per lane
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(&p.q->lane_cursor, 32ull);
            b = __shfl_sync(0xffffffffu, b, 0);
            const int64_t base = n_warp + (int64_t)b;
            if (base < p.n_roots) {
                const int64_t ri = base + lane;
                if (ri < p.n_roots) {
                    const int32_t r = p.roots ? __ldg(p.roots + ri) : (int32_t)(p.root_lo + ri);
                    if (r < 0 || r >= p.g.E) {
                        atomicOr(&p.q->error, kErrBadRoot);
                    } else {
                        M.ri = ri;
                        M.rmask = p.root_qmask ? __ldg(p.root_qmask + ri) : ~0ull;
                        Work before = M.w;
                        M.lane_root(r);
                        if (kStats) {
                            M.w.v[kStRoots]++;
                            M.w.v[kStLaneRoots]++;
                            if (p.per_root_work) {              // this lane's root alone
                                unsigned long long d[4] = {
                                    M.w.v[kStCand] - before.v[kStCand], M.w.v[kStExp] - before.v[kStExp],
                                    M.w.v[kStListProbe] + M.w.v[kStHashProbe] + M.w.v[kStPairProbe] -
                                        before.v[kStListProbe] - before.v[kStHashProbe] - before.v[kStPairProbe],
                                    M.w.v[kStLeaf] - before.v[kStLeaf]};
                                for (int f = 0; f < 4; f++)
                                    if (d[f]) atomicAdd((unsigned long long *)&p.per_root_work[ri * TM_WORK_FIELDS + f], d[f]);
                            }
                        }
                    }
                }
                __syncwarp();
                continue;
            }
        }
        if (!p.dynamic) break;
        const long long tw = kStats ? clock64() : 0;
        const bool more = M.wait_for_work();
        if (kStats) idle += clock64() - tw;
        if (!more) break;
    }
    if (kStats && lane == 0) {
        const unsigned long long busy = (unsigned long long)max(0ll, clock64() - t_begin - idle);
        atomicMax(&p.stats[kStatFields + kBusyMax], busy);
        atomicAdd(&p.stats[kStatFields + kBusySum], busy);
        atomicAdd(&p.stats[kStatFields + kBusyWarps], 1ull);
    }
    if (kStats) {
        for (int f = 0; f < kStatFields; f++) {
            unsigned long long s = warp_sum_u64(M.w.v[f]);
            if (lane == 0 && s) atomicAdd(&p.stats[f], s);
        }
    }
    __syncthreads();
    if (p.smem_counters)
        for (int i = threadIdx.x; i < n_cnt; i += blockDim.x) {
            unsigned long long c = s_cnt[i];
            if (p.smem_counters == 2)
                for (int wi = 1; wi < kWarps; wi++) c += s_cnt[wi * n_cnt + i];
            if (c) atomicAdd(&p.counts[i], c);
        }
}

}  // namespace dev
}  // namespace tmo
