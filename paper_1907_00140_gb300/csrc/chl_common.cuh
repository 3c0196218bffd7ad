// Internal declarations shared by the translation units of libchl.so.
// Nothing here is part of the public ABI (include/chl.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/chl.h"

// the labels object behind the opaque ABI handle
struct chl_labels {
    uint32_t n = 0;
    uint64_t total = 0;
    uint64_t *offsets = nullptr;
    uint32_t *hub = nullptr;
    uint32_t *hubpos = nullptr;
    uint32_t *dist = nullptr;
    uint32_t *parent = nullptr;  // SPT parent per label (caller id), or null
    uint64_t bytes = 0;
    chl_build_stats stats{};
    int device = 0;
};

namespace chl {

// ------------------------------------------------------------------ graph in rank order
// The input graph renumbered by rank position: vertex p of this graph is the
// vertex of rank position p (R = n-1-p) of the caller's graph.
struct RankGraph {
    uint32_t n = 0;
    uint64_t m2 = 0;             // arcs
    uint64_t *row = nullptr;     // [n+1]
    uint2 *arc = nullptr;        // [m2] {neighbour pos, weight}
    uint32_t *vert_at = nullptr; // [n] pos -> caller vertex id
    uint32_t *pos_of = nullptr;  // [n] caller vertex id -> pos
    uint32_t w_max = 0, w_min = 0;
    double w_mean = 0.0;
};

// ------------------------------------------------------------------ tree kernel interface
struct TreeLaunch {
    // graph (rank order)
    uint32_t n;
    const uint64_t *row;
    const uint2 *arc;
    const uint32_t *vert_at;
    // roots: pos ids root_list[i] (if non-null) or root_begin + i, i < root_count
    const uint32_t *root_list;
    uint32_t root_begin;
    uint32_t root_count;
    const uint32_t *count_dev;  // non-null: the root count is read here (written by an earlier kernel)
    const int *stop;            // non-null: no root is claimed once *stop != 0
    // search parameters
    uint32_t delta;
    int delta_shift;    // log2(delta) when delta is a power of two, else -1
    uint32_t nwin;
    uint32_t w_min;     // lightest arc weight
    uint32_t round_limit;  // expansion rounds per tree before ERR_ROUND_LIMIT
    uint32_t fin_words; // settled-filter bitmap words in dynamic shared memory
    uint32_t fin_bits;  // vertices (pos) the bitmap covers: min(n, 32 * fin_words)
    // Common Label Table (Sec. 5.3), or hc = null: hc[v * hc_stride + c] =
    // d(v, c) for table hub c (pos c < hc_hubs) when (c, d) is a label of v,
    // else all ones; hc_stride = hc_hubs rounded up to a multiple of 4
    const uint32_t *hc;
    uint32_t hc_hubs;
    uint32_t hc_stride;
    // label table of the earlier phases of a hybrid build, or lt_off = null:
    // all labels of the hubs of rank position in [hc_hubs, lt_hubs) (the
    // Common Label Table answers for the hubs below hc_hubs), CSR by vertex
    // rank position (offsets [n+1]) of {hub position, distance} entries, each
    // vertex's entries in no particular order (see LabelTable)
    const uint64_t *lt_off;
    const uint2 *lt_e;     // {hub position, distance}
    uint32_t lt_hubs;
    uint32_t aux_bytes;    // dynamic shared memory after the settled bitmap (multiple of 128):
                           // the staging area, or the root's table distances by hub position
    uint32_t stage_bytes;  // aux_bytes when the queried lists are staged there, else 0
    // per slot [n], all ones when idle, or null: the root's table labels by
    // hub position, for roots with more of them than the shared-memory hash holds
    uint32_t *lt_root;
    uint32_t lt_hash_max;  // roots with more table labels than this use lt_root
    // slot state: slot s owns [s*n, (s+1)*n) of each array
    void *key;          // tree keys, all ones when idle (see chl_tree.cu)
    int key_bytes;      // 4 (distances provably < 2^31 - 1) or 8
    uint32_t *rtag;     // per slot: round id that last listed the vertex in nxt
    uint32_t *lists;    // per slot: round lists l0, l1, far, touched, then nwin bucket lists
    uint32_t *slot_ctr; // [slot][4] persistent per-slot words: [0] round id, [1] held by a CTA
    int dyn_slots;      // 1: a CTA takes any free slot of [0, nslots) (launches may overlap), 0: slot = CTA
    uint32_t nslots;    // slots of the launch (its grid size)
    // label output (structure of arrays)
    uint32_t *out_v;    // caller vertex id of the labelled vertex
    uint32_t *out_h;    // hub pos id
    uint32_t *out_d;    // distance
    uint32_t *out_p;    // SPT parent (caller vertex id), or null: no parents
    unsigned long long out_cap;
    unsigned long long *out_count;  // next free record (may pass out_cap once a tree failed)
    unsigned long long *out_valid;  // records written, set by the first tree that failed
    // control
    unsigned int *next_root;
    uint32_t *failed;          // roots whose labels did not fit
    unsigned int *failed_count;
    int *flags;                // [0] error code, [1] output full
    unsigned long long *stats; // [0] expanded [1] arcs [2] trivial [3] trees [4] rounds [5] buckets [6] pruned
};

enum : int { ERR_NONE = 0, ERR_DIST_OVERFLOW = 1, ERR_ROUND_LIMIT = 2, ERR_WAIT_LIMIT = 3 };

// launches (defined in chl_tree.cu)
cudaError_t launch_plant_trees(const TreeLaunch &p, int threads_per_tree, int slots,
                               cudaStream_t s);
// CTAs per SM of a launch with that bitmap and auxiliary area
int plant_max_slots_per_sm(int threads_per_tree, uint32_t fin_words, uint32_t aux_bytes);
// roots [begin, begin + count): the label of every trivial root is written to
// the output (p.out_*, p.out_count; the caller guarantees room for count
// records), the other roots are appended to list (*list_n of them)
cudaError_t launch_split_trivial(const TreeLaunch &p, uint32_t begin, uint32_t count, uint32_t *list,
                                 unsigned int *list_n, cudaStream_t s);
// dynamic shared memory per CTA (bytes) that keeps the CTAs per SM of a launch
// without any
uint32_t plant_dyn_budget(int threads_per_tree);
// that budget split between the auxiliary area of phases that prune with the
// label table (at most aux_want bytes, at most half the budget) and the
// settled-filter bitmap (at most one bit per vertex)
void plant_smem_split(int threads_per_tree, uint32_t n, uint32_t aux_want, uint32_t *fin_words,
                      uint32_t *aux_bytes);
// Common Label Table entries from label records (those of hub positions < hubs)
cudaError_t launch_clt_fill(const uint32_t *out_v, const uint32_t *out_h, const uint32_t *out_d,
                            unsigned long long count, const uint32_t *pos_of, uint32_t *hc,
                            uint32_t stride, uint32_t hubs, cudaStream_t s);

// label assembly (chl_labels.cu)
struct LabelCSR {
    uint64_t *offsets = nullptr; // [n+1] by caller vertex id
    uint32_t *hub = nullptr;     // caller vertex id
    uint32_t *hubpos = nullptr;  // rank position of hub (ascending per vertex, but see assemble_table)
    uint32_t *dist = nullptr;
};
// builds CSR from T label triples; returns error status via cudaError_t, sets
// *too_long when a vertex holds more labels than the sorter handles
cudaError_t assemble_labels(uint32_t n, uint64_t T, const uint32_t *in_v, const uint32_t *in_h,
                            const uint32_t *in_d, const uint32_t *vert_at, LabelCSR &out,
                            int *too_long, cudaStream_t s, int *launches);

// The same records as a table for the distance queries of label pruning:
// offsets [n+1] by rank position (pos_of maps caller ids to positions), entries
// {hub position, distance} interleaved, each vertex's entries in no particular
// order. Records of hubs below min_hub are left out. The entry array has two
// spare entries past the last (all ones), so a read widened to 16-byte
// boundaries stays inside it.
struct LabelTable {
    uint64_t *offsets = nullptr;
    uint2 *e = nullptr;
};
cudaError_t assemble_table(uint32_t n, uint64_t T, const uint32_t *in_v, const uint32_t *in_h,
                           const uint32_t *in_d, const uint32_t *pos_of, uint32_t min_hub,
                           LabelTable &out, cudaStream_t s, int *launches);

// a table from assemble_table of records [0, T0) grown by records [T0, T):
// each vertex keeps its old entries first (lt is replaced; on success the old
// arrays are freed on s, or handed to *keep_old when that is non-null)
cudaError_t grow_table(uint32_t n, LabelTable &lt, uint64_t T0, uint64_t T, const uint32_t *in_v,
                       const uint32_t *in_h, const uint32_t *in_d, const uint32_t *pos_of,
                       uint32_t min_hub, cudaStream_t s, int *launches, LabelTable *keep_old = nullptr);
void free_table(LabelTable &t, cudaStream_t s);

// parents of label records into the slots of the assembled CSR (parent[T])
cudaError_t place_parents(uint64_t T, const uint32_t *in_v, const uint32_t *in_h, const uint32_t *in_p,
                          const LabelCSR &csr, uint32_t *parent, cudaStream_t s, int *launches);

// queries (chl_query.cu)
// bad is set to 1 when a pair holds a vertex id >= n (that answer is UINT32_MAX)
cudaError_t launch_query(uint32_t n, const uint64_t *offsets, const uint32_t *hubpos,
                         const uint32_t *dist, const uint32_t *pairs, uint64_t q, uint32_t *out,
                         int *bad, cudaStream_t s);
// shortest paths from parents stored with the labels; bad = 1 for an id >= n,
// 2 for a broken parent chain
cudaError_t launch_paths(uint32_t n, const uint64_t *offsets, const uint32_t *hubpos,
                         const uint32_t *dist, const uint32_t *hub, const uint32_t *parent,
                         const uint32_t *pairs, uint64_t q, uint32_t max_len, uint32_t *paths,
                         uint32_t *lens, int *bad, cudaStream_t s);
// one resident label set as the query kernels read it: its lists, or (nparts
// > 0) its hub partitions, a device array of nparts sets over the same n
// vertices whose answer is the minimum of theirs
struct QuerySet {
    uint32_t n;
    const uint64_t *offsets;
    const uint32_t *hubpos;
    const uint32_t *dist;
    uint32_t nparts;
    const QuerySet *parts;
};
// a batch whose pair i asks set set_of[i] (sets: device array, *nsets in device
// memory; set id 0xFFFF = padding, skipped); perm (or null) is the order in
// which the pairs are answered (launch_group_order)
cudaError_t launch_query_sets(const QuerySet *sets, const uint32_t *nsets, const uint32_t *pairs,
                              const uint16_t *set_of, const uint32_t *perm, uint64_t q, uint32_t *out,
                              int *bad, int max_blocks, cudaStream_t s);
// grouped order of a batch: perm[0..q) = the pairs sorted by the block pair of
// their two vertices (64 blocks per set); set_of may be null (all set 0);
// scratch holds 4096 counters
constexpr uint32_t GROUP_SCRATCH_WORDS = 4096;
cudaError_t launch_group_order(const QuerySet *sets, const uint32_t *nsets, const uint32_t *pairs,
                               const uint16_t *set_of, uint64_t q, uint32_t *scratch, uint32_t *perm,
                               cudaStream_t s);

// exclusive prefix sum of n uint64 values (out may alias in); chl_graph.cu
cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                               int *launches);

// graph preparation (chl_graph.cu)
// validates the caller CSR (device copy) and rank; builds the rank-ordered graph
// returns CHL_OK / CHL_EINVAL (with message) / CHL_ECUDA / CHL_ENOMEM
chl_status prepare_graph(uint32_t n, uint64_t m2, const uint64_t *row, const uint32_t *col,
                         const uint32_t *w, const uint32_t *rank, RankGraph &g, cudaStream_t s,
                         int *launches);
void free_graph(RankGraph &g, cudaStream_t s);

// errors (chl_api.cu)
chl_status set_error(chl_status st, const char *fmt, ...);
// a failed CUDA call as a status (CHL_ENOMEM for an allocation failure, else
// CHL_ECUDA) with its message; clears the thread's CUDA last-error state
chl_status cuda_status(cudaError_t e, const char *what);

// stream-ordered device allocation from the library's pool of the current
// device (free with cudaFreeAsync or cudaFree)
cudaError_t dmalloc(void **ptr, size_t bytes, cudaStream_t s);
template <typename T>
cudaError_t dmalloc(T **ptr, size_t bytes, cudaStream_t s) {
    return dmalloc(reinterpret_cast<void **>(ptr), bytes, s);
}

// SMs of the current device (queried once per device; 1 if the query fails),
// for sizing grid-stride launches
int device_sms();

}  // namespace chl
