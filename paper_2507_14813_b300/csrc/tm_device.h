// Device-side data structures shared by the library and its kernels.
//
// This header is compiled by nvcc (with the rest of the library) and by the
// runtime compiler (NVRTC) for kernels specialised to one MG-Tree, which see
// no host headers: it includes nothing but the public header on the host
// side, and the runtime compilation defines the few limits it needs itself.
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#ifndef INT32_MAX
#define INT32_MAX 2147483647
#endif
#ifndef INT64_MAX
#define INT64_MAX 9223372036854775807LL
#endif
#else
#include <stdint.h>
#include "../../include/tmotif.h"
#endif

#ifndef TM_K_MAXE
#define TM_K_MAXE TM_MAX_EDGES
#endif
#ifndef TM_K_MAXV
#define TM_K_MAXV TM_MAX_VERTICES
#endif

namespace tmo {

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


// ---------------------------------------------------------------- device tree
// Array sizes of the device structures: the library's limits, or the tree's
// own depth and vertex count in a kernel compiled for one tree.
static constexpr int kMaxE = TM_K_MAXE;
static constexpr int kMaxV = TM_K_MAXV;

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

}  // namespace tmo
