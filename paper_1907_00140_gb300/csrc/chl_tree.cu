// PLaNT shortest-path trees on the GPU (Sec. 5.2, Algorithm 3).
//
// One persistent launch builds every tree of a root range. Each CTA owns a
// tree "slot" (dense per-vertex state in global memory) and repeatedly claims
// the next root in rank order with a global atomic counter, the dynamic
// root claiming of Sec. 4.1 (threads pop the most important remaining root).
//
// Per tree the search is a bucketed label-correcting Dijkstra (delta-stepping,
// bucket width delta) over packed keys (see "Keys" below): an atomicMin keeps
// the shortest distance and, at equal distance, prefers a path through a
// vertex that outranks the root (Algorithm 3, equal-distance branch). Every
// vertex that is expanded relaxes all its arcs, labelled or not: PLaNT does
// not prune trees (Sec. 1, Sec. 5.2); a vertex outranked by its ancestor only
// gets no label.
//
// Pending vertices (keys in later buckets) are held per bucket:
//   sub[s]   one list per bucket of the current window of `nwin` buckets
//            (bucket win_base + s); a vertex is listed once per bucket it
//            enters (keys only decrease, so an earlier entry is then stale)
//   far      vertices whose bucket lies beyond the window; when the window is
//            used up it restarts at the nearest far bucket
//   nxt      vertices improved inside the current bucket during a round
// plus `touched`, every vertex that got a finite key (for emission and for
// resetting only what the tree modified, footnote of Sec. 4.1).
// The value an atomicMin replaces says which lists already hold the vertex,
// since buckets only move down: a window bucket is joined iff the old key was
// in another bucket, far iff the old key was unreached (a key beyond the
// window was far-listed when it was set, and keys never rise back past the
// window). Only the per-round nxt list needs a tag (rtag, the round id).
//
// Early termination (Sec. 5.2). The paper stops when every vertex in
// Dijkstra's queue is outranked; Algorithm 3 keeps the count `cnt` of queued
// vertices whose ancestor is the root. Here `cnt` counts the live vertices
// whose key lies beyond the current bucket: every successful atomicMin on a
// key adds f(new) - f(old), f(K) = [K live and beyond the current bucket].
// atomicMin serialises the updates of one key, so the sum telescopes to the
// exact count whatever the order of the atomic adds; entering a bucket
// subtracts its live vertices. After a bucket converges all keys below its
// end are final, so the tree stops when cnt = 0: exact at bucket granularity.
//
// Labels: after a tree stops, every touched vertex whose key is live gets
// (vertex, root, dist); the tree reserves its output range with one
// atomicAdd. Ranges are handed out in increasing order, so those that fit the
// buffer are a prefix of it: the first range that does not fit records where
// that prefix ends, and it and every later tree give up their labels whole
// (no partial tree is kept); the host rebuilds those roots after growing the
// buffer.
#include <algorithm>
#include <cstdio>

#include "chl_common.cuh"

namespace chl {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t NWIN_MAX = 64;
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t CLT_MAX = 64;  // largest Common Label Table (hubs)
constexpr uint32_t LTH_SLOTS = 1024;  // hash of the root's labels in the label table
constexpr uint32_t LTH_MAX = 512;     // most root labels the hash holds
constexpr int QSTEPS = 4;             // label-table query from global memory: loads in flight per lane
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // polls of a staging barrier before it counts as hung
#ifndef SMEM_CAP_BYTES
#define SMEM_CAP_BYTES (132u << 10)
#endif

// ------------------------------------------------------------------ keys
// Vertices are numbered by rank position (pos 0 = most important), so in the
// tree of root h a vertex outranks h iff its pos is below h. Algorithm 3 keeps
// per vertex its distance and the highest-ranked vertex a[v] on its shortest
// paths; the label decision only asks whether a[v] is h itself, and a[v] can
// never rank below h (every path starts at h). So one bit carries it:
//   key = dist << 1 | clean
// clean = 1 iff no vertex before v on the best known paths outranks h. Under
// unsigned min a shorter distance wins and, at equal distance, clean = 0
// wins: a vertex is outranked as soon as one of its shortest paths is (the
// equal-distance branch of Algorithm 3; Sec. 5.2's example, a[v5] = v1).
// v is live (would get the label (h, d)) iff clean and v >= h, and the bit
// it passes on to its out-neighbours is exactly its own liveness.
// Three layouts (K below is one of these traits; K::T is the stored word):
//   KeyN  uint32  dist << 1 | clean            when every tentative distance is
//                                              provably below 2^31 - 1 (the host
//                                              checks w_max * n)
//   KeyW  uint64  dist << 1 | clean            otherwise
//   KeyP  uint64  dist << 32 | clean << 31 | parent, for path recovery (the
//                 SPT parent stored with each label, Sec. 5.4 (Extensions)):
//                 among equal (dist, clean) the smallest parent id wins, so
//                 the parent is the lowest-numbered tight predecessor, a
//                 deterministic choice. A candidate carries its source
//                 vertex in the parent field.
// All ones is "unreached".
// U: arcs a lane relaxes per step of the arc pass (its loads in flight); the
// 8-byte layouts take two, so that a thread's probe state fits its registers
// at 1024 threads per SM.
struct KeyN { using T = uint32_t; static constexpr int S = 1; static constexpr int U = 4; };
struct KeyW { using T = uint64_t; static constexpr int S = 1; static constexpr int U = 2; };
struct KeyP { using T = uint64_t; static constexpr int S = 32; static constexpr int U = 2; };

template <typename K>
__device__ __forceinline__ typename K::T key_inf() { return ~typename K::T(0); }
template <typename K>
__device__ __forceinline__ typename K::T make_key(uint64_t dist, bool clean, uint32_t parent) {
    using KS = typename K::T;
    return (KS(dist) << K::S) | (KS(clean) << (K::S - 1)) | (K::S > 1 ? KS(parent) : KS(0));
}
template <typename K>
__device__ __forceinline__ uint32_t key_dist(typename K::T k) { return uint32_t(k >> K::S); }
template <typename K>
__device__ __forceinline__ bool key_clean(typename K::T k) { return (k >> (K::S - 1)) & 1; }
template <typename K>
__device__ __forceinline__ uint32_t key_parent(typename K::T k) {
    return K::S > 1 ? uint32_t(k & 0x7FFFFFFFu) : 0u;
}
// largest distance a key holds below key_inf
template <typename K>
__device__ __forceinline__ uint64_t key_dist_limit() {
    return sizeof(typename K::T) == 4 ? 0x7FFFFFFEull : 0xFFFFFFFEull;
}

struct Shared {
    uint32_t root;
    uint32_t cur_n, nxt_n, far_n, touch_n;
    uint32_t rid;
    uint32_t sel;          // round lists: cur = sel ? l1 : l0 (rounds after the first)
    uint32_t cur_slot;     // window slot expanded in the bucket's first round, NONE after
    uint32_t bcur;         // current bucket
    uint32_t win_base;     // bucket of window slot 0
    int cnt;               // live vertices with keys beyond the current bucket
    uint64_t t_lo, t_hi;   // current bucket [t_lo, t_hi)
    uint64_t w_hi;         // end of the window
    uint32_t min_b;
    uint32_t out_n;
    int abort;
    int ok;
    int live_sum;
    int fuse_live;         // the current list's first stage also counts its live entries
    int prune;             // this tree prunes by the Common Label Table
    int lt_prune;          // ... and by the label table of earlier phases
    int lt_dense;          // the root's table labels: 0 hashed, 1 in p.lt_root, 2 in the shared array
    uint32_t qn;           // table queries queued by the current chunk
    uint32_t stage_used;   // bytes of the staging area reserved by the current batch
    uint32_t bn;           // queries staged in the current batch
    unsigned long long mbar;  // barrier that counts the staging copies of a batch
    uint32_t hch[CLT_MAX]; // table row of the root: d(h, c) per table hub c
    // the root's labels in the label table, hashed by hub position (key + 1)
    uint32_t lth_key[LTH_SLOTS];
    uint32_t lth_val[LTH_SLOTS];
    unsigned long long base;
    uint32_t sub_n[NWIN_MAX];
    uint32_t slot;         // the tree slot this CTA holds
    // launch statistics of this CTA, reported once at exit (kept here, not in
    // registers, which the arc pass needs)
    unsigned long long n_exp, n_arcs, n_pruned, n_rounds, n_buckets;
    uint64_t lt_a, lt_b;   // the root's entries in the label table
    uint32_t n_trees, n_trivial;
};

// bucket of a distance: a shift when the width is a power of two
__device__ __forceinline__ uint32_t bucket_of(const TreeLaunch &p, uint32_t d) {
    return p.delta_shift >= 0 ? d >> p.delta_shift : d / p.delta;
}

// A slot's lists sit back to back, n entries each: l0, l1, far, touch, then
// the nwin window lists; their addresses are formed where used (fewer
// registers held across the tree than one pointer per list).
template <typename K>
struct Slot {
    typename K::T *key;
    uint32_t *rtag;
    uint32_t *lists;
    uint32_t n;
    __device__ __forceinline__ uint32_t *l0() const { return lists; }
    __device__ __forceinline__ uint32_t *l1() const { return lists + n; }
    __device__ __forceinline__ uint32_t *far() const { return lists + 2 * size_t(n); }
    __device__ __forceinline__ uint32_t *touch() const { return lists + 3 * size_t(n); }
    __device__ __forceinline__ uint32_t *sub(uint32_t s) const { return lists + (4 + size_t(s)) * n; }
};

template <typename K>
__device__ __forceinline__ bool is_live(typename K::T k, uint32_t v, uint32_t h) {
    return key_clean<K>(k) && v >= h;
}

// warp-aggregated append to a list counted by a shared-memory counter
__device__ __forceinline__ void warp_append(bool pred, uint32_t val, uint32_t *list,
                                            uint32_t *counter) {
    const unsigned m = __ballot_sync(FULL, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
    base = __shfl_sync(FULL, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1))] = val;
}

// list a pending vertex in bucket b of the window
template <typename K>
__device__ __forceinline__ void sub_append(Shared &S, const Slot<K> &sl, uint32_t n, uint32_t u,
                                           uint32_t b) {
    const uint32_t s = b - S.win_base;
    sl.sub(s)[atomicAdd(&S.sub_n[s], 1u)] = u;
}

// Relaxation of one arc (v -> u, weight w) of a vertex expanded with distance
// dv and liveness lv (the clean bit it passes on), in two stages so that a
// lane can have several key loads in flight:
//   probe:  form the candidate key and load the target's key from L2 (keys
//           only decrease, so a stale read never hides an improvement)
//   commit: if the candidate is smaller, atomicMin; on improvement, update
//           the live-pending count, record the vertex as touched and list it
//           for the bucket it now falls in
template <typename K>
struct Probe {
    typename K::T cand;
    typename K::T seen;
    uint32_t u;
    bool live;  // still worth committing
};

__device__ __forceinline__ uint32_t atomic_min_key(uint32_t *a, uint32_t v) { return atomicMin(a, v); }
// atomicMin under a predicate, as one predicated instruction (no branch
// around it); returns `none` where the predicate is false
__device__ __forceinline__ uint32_t atomic_min_key_if(bool on, uint32_t *a, uint32_t v, uint32_t none) {
    uint32_t old = none;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\t@p atom.global.min.u32 %0, [%1], %2;\n\t}"
        : "+r"(old)
        : "l"(a), "r"(v), "r"(uint32_t(on))
        : "memory");
    return old;
}
__device__ __forceinline__ uint64_t atomic_min_key_if(bool on, uint64_t *a, uint64_t v, uint64_t none) {
    uint64_t old = none;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\t@p atom.global.min.u64 %0, [%1], %2;\n\t}"
        : "+l"(old)
        : "l"(a), "l"(v), "r"(uint32_t(on))
        : "memory");
    return old;
}
__device__ __forceinline__ uint64_t atomic_min_key(uint64_t *a, uint64_t v) {
    return atomicMin((unsigned long long *)a, (unsigned long long)v);
}
__device__ __forceinline__ void atomic_set_key(uint32_t *a, uint32_t v) { atomicExch(a, v); }
__device__ __forceinline__ void atomic_set_key(uint64_t *a, uint64_t v) {
    atomicExch((unsigned long long *)a, (unsigned long long)v);
}

// Settled filter (dynamic shared memory, one bit per vertex pos below
// p.fin_bits): a vertex expanded with distance below t_lo + w_min, t_lo the
// start of the current bucket, holds its final key. Buckets below t_lo are
// settled, so any later relaxation starts from a distance >= t_lo and offers
// at least t_lo + w_min; hence no later candidate can lower (or tie) that
// key, and a probe of a marked target skips its key load. Bits are set when a
// vertex is expanded and cleared per tree; a probe that misses a fresh bit
// only does a load it could have saved.
extern __shared__ __align__(128) uint32_t fin_bitmap[];

// The staging area of the label-table queries follows the bitmap in dynamic
// shared memory, at the next multiple of 128 bytes.
__device__ __forceinline__ uint32_t stage_offset(uint32_t fin_words) { return (fin_words * 4u + 127u) & ~127u; }

// ---- shared-memory barrier and bulk copy (PTX mbarrier, cp.async.bulk)
__device__ __forceinline__ uint32_t smem_addr(const void *ptr) {
    return uint32_t(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(unsigned long long *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
    // make the initialised barrier visible to the copy engine's proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *m) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_addr(m))
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *m, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            smem_addr(m)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *m, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return done != 0;
}
// global -> shared copy by the copy engine; both addresses 16-byte aligned,
// bytes a multiple of 16; completion counted on barrier m
__device__ __forceinline__ void bulk_to_shared(void *dst, const void *src, uint32_t bytes,
                                               unsigned long long *m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(m))
        : "memory");
}

// kv = make_key(dv, lv) of the expanded vertex: the candidate through arc
// (u, w) is kv + 2w (the clean bit rides along in bit 0). With 4-byte keys
// the host has proven every tentative distance below the key limit
// (w_max * n < 2^31 - 1), so only the wide form checks for overflow.
// Written without early exits (predicates instead), so that a step's K::U
// probes form no divergent regions; valid: the lane has an arc at this index.
template <typename K>
__device__ __forceinline__ void probe(const TreeLaunch &p, Shared &S, const Slot<K> &sl,
                                      typename K::T kv, uint2 a, bool valid, Probe<K> &q) {
    using KS = typename K::T;
    q.u = a.x;
    if (sizeof(KS) == 8 && valid && uint64_t(key_dist<K>(kv)) + a.y > key_dist_limit<K>()) {
        atomicExch(&p.flags[0], ERR_DIST_OVERFLOW);
        S.abort = 1;
        valid = false;
    }
    const uint32_t word = valid && q.u < p.fin_bits ? fin_bitmap[q.u >> 5] : 0u;
    q.live = valid && !((word >> (q.u & 31)) & 1u);
    q.cand = kv + (KS(a.y) << K::S);
    q.seen = q.live ? __ldcg(&sl.key[q.u]) : KS(0);
}

// Frontier staging of one chunk of up to TPB list entries, compacted to the
// entries that are expanded (stale ones dropped): each row's start (with the
// vertex's liveness in bit 63), its distance, and the exclusive prefix of the
// degrees. The chunk's arcs then form one flat index range [0, total), cut
// into one contiguous piece per warp, whatever the degree mix (a hub's row
// and a thousand short rows alike). Every staged row has at least one arc
// (a zero-degree vertex is never expanded: it is unreachable or a trivial
// root), so row starts are distinct flat positions.
template <int TPB, typename K>
struct Frontier {
    uint64_t base[TPB];  // row start minus degree prefix: arc index = base + flat position
    uint64_t pre[TPB];   // exclusive degree prefix
    typename K::T kv[TPB];  // make_key(distance, liveness, vertex) of the row's vertex
    uint32_t wrows[TPB / 32];
    uint64_t wdeg[TPB / 32];
    // per warp: improvements waiting to be classified (vertex, new key, old key)
    uint32_t iu[TPB / 32][32];
    typename K::T ic[TPB / 32][32];
    typename K::T io[TPB / 32][32];
};

// Commit of one warp step, called by all 32 lanes. The atomicMins of all
// K::U probes are issued together (independent, so their round trips
// overlap). The improvements (typically a few per step of 128 arcs) are
// appended to the warp's shared buffer, and classified 32 at a time, one per
// lane: the appends to the touched list, nxt, far and the window buckets then
// take one shared atomic per warp and list (per bucket for the window), the
// live-pending count one per warp. Each improvement is classified once with
// its own old and new key, so the order of classification does not matter;
// what it appends is read only after the chunk's last barrier, before which
// the warp classifies what its buffer still holds.
template <typename K>
__device__ __forceinline__ void commit_one(const TreeLaunch &p, Shared &S, const Slot<K> &sl,
                                           uint32_t h, bool has, uint32_t u, typename K::T cand,
                                           typename K::T old) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    uint32_t cls = 0;  // 0 none, 1 nxt (current bucket), 2 window bucket, 3 far
    uint32_t sx = NONE;
    bool touch = false;
    int dcnt = 0;
    if (has) {
        const bool unreached = old == key_inf<K>();
        const uint32_t nb = bucket_of(p, key_dist<K>(cand));
        const uint32_t ob = unreached ? NONE : bucket_of(p, key_dist<K>(old));
        const bool f_new = nb > S.bcur && is_live<K>(cand, u, h);
        const bool f_old = !unreached && ob > S.bcur && is_live<K>(old, u, h);
        dcnt = int(f_new) - int(f_old);
        if (nb == S.bcur) {
            if (atomicExch(&sl.rtag[u], S.rid) != S.rid) cls = 1;
        } else if (key_dist<K>(cand) < S.w_hi) {
            if (ob != nb) {
                cls = 2;
                sx = nb - S.win_base;
            }
        } else if (unreached) {
            cls = 3;
        }
        touch = unreached;
    }
    const int dsum = __reduce_add_sync(FULL, dcnt);
    const unsigned mt = __ballot_sync(FULL, touch);
    const unsigned mn = __ballot_sync(FULL, cls == 1);
    const unsigned mf = __ballot_sync(FULL, cls == 3);
    const unsigned mw = __ballot_sync(FULL, cls == 2);
    uint32_t bt = 0, bn = 0, bf = 0;
    if (lane == 0) {
        if (dsum) atomicAdd(&S.cnt, dsum);
        if (mt) bt = atomicAdd(&S.touch_n, uint32_t(__popc(mt)));
        if (mn) bn = atomicAdd(&S.nxt_n, uint32_t(__popc(mn)));
        if (mf) bf = atomicAdd(&S.far_n, uint32_t(__popc(mf)));
    }
    if (mt) {
        bt = __shfl_sync(FULL, bt, 0);
        if (touch) sl.touch()[bt + __popc(mt & lt)] = u;
    }
    if (mn) {
        bn = __shfl_sync(FULL, bn, 0);
        uint32_t *nxt = S.sel ? sl.l0() : sl.l1();
        if (cls == 1) nxt[bn + __popc(mn & lt)] = u;
    }
    if (mf) {
        bf = __shfl_sync(FULL, bf, 0);
        if (cls == 3) sl.far()[bf + __popc(mf & lt)] = u;
    }
    if (mw) {
        // lanes joining the same window bucket share one counter update
        const unsigned g = __match_any_sync(FULL, sx);
        const int ld = __ffs(g) - 1;
        uint32_t base = 0;
        if (cls == 2 && lane == ld) base = atomicAdd(&S.sub_n[sx], uint32_t(__popc(g)));
        base = __shfl_sync(FULL, base, ld);
        if (cls == 2) sl.sub(sx)[base + __popc(g & lt)] = u;
    }
}

// classify the first cnt entries of the warp's buffer
template <int TPB, typename K>
__device__ __forceinline__ void commit_buffer(const TreeLaunch &p, Shared &S, Frontier<TPB, K> &F,
                                              const Slot<K> &sl, uint32_t h, uint32_t cnt) {
    using KS = typename K::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncwarp();  // every lane's entries are written
    const bool has = uint32_t(lane) < cnt;
    uint32_t u = 0;
    KS cand = 0, o = 0;
    if (has) {
        u = F.iu[warp][lane];
        cand = F.ic[warp][lane];
        o = F.io[warp][lane];
    }
    __syncwarp();  // the buffer is free again
    commit_one<K>(p, S, sl, h, has, u, cand, o);
}

// returns the warp's new buffer count (bn before the step, warp-uniform)
template <int TPB, typename K>
__device__ __forceinline__ uint32_t commit_step(const TreeLaunch &p, Shared &S, Frontier<TPB, K> &F,
                                                const Slot<K> &sl, uint32_t h,
                                                const Probe<K> (&q)[K::U], uint32_t bn) {
    using KS = typename K::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1;
    KS old[K::U];
    unsigned im = 0;
#pragma unroll
    for (int k = 0; k < K::U; ++k)
        old[k] = atomic_min_key_if(q[k].live && q[k].cand < q[k].seen, &sl.key[q[k].u], q[k].cand, KS(0));
#pragma unroll
    for (int k = 0; k < K::U; ++k)
        if (q[k].live && q[k].cand < q[k].seen && q[k].cand < old[k]) im |= 1u << k;
    if (!__any_sync(FULL, im != 0)) return bn;
#pragma unroll
    for (int k = 0; k < K::U; ++k) {
        const bool has = (im >> k) & 1u;
        const unsigned m = __ballot_sync(FULL, has);
        if (!m) continue;
        const uint32_t cnt = __popc(m);
        int pos = int(bn + __popc(m & lt));
        if (has && pos < 32) {
            F.iu[warp][pos] = q[k].u;
            F.ic[warp][pos] = q[k].cand;
            F.io[warp][pos] = old[k];
        }
        if (bn + cnt >= 32) {
            // the buffer is full: classify it, then keep what did not fit
            commit_buffer<TPB, K>(p, S, F, sl, h, 32);
            pos -= 32;
            if (has && pos >= 0) {
                F.iu[warp][pos] = q[k].u;
                F.ic[warp][pos] = q[k].cand;
                F.io[warp][pos] = old[k];
            }
            bn = bn + cnt - 32;
        } else {
            bn += cnt;
        }
    }
    return bn;
}

// largest o in [lo, hi) with pre[o] <= j, given pre[lo] <= j
template <int TPB, typename K>
__device__ __forceinline__ uint32_t owner(const Frontier<TPB, K> &F, uint64_t j, uint32_t lo,
                                          uint32_t hi) {
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (F.pre[mid] <= j) lo = mid; else hi = mid;
    }
    return lo;
}

// Common Label Table pruning (Sec. 5.3): the distance query between the root
// and v over the table hubs, min_c d(h, c) + d(c, v); the table row of v is
// read as 16-byte vectors (rows are padded to a multiple of 4 hubs)
__device__ __forceinline__ uint64_t clt_query(const TreeLaunch &p, const Shared &S, uint32_t v) {
    const uint4 *row = reinterpret_cast<const uint4 *>(p.hc + size_t(v) * p.hc_stride);
    uint64_t best = ~0ull;
    for (uint32_t c4 = 0; c4 < p.hc_stride / 4; ++c4) {
        const uint4 x = __ldg(&row[c4]);
        const uint32_t b[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t a = S.hch[c4 * 4 + j];
            if (a != 0xFFFFFFFFu && b[j] != 0xFFFFFFFFu && uint64_t(a) + b[j] < best) best = uint64_t(a) + b[j];
        }
    }
    return best;
}

// Label table of earlier phases (hybrid pruning): every label of every hub of
// rank position below p.lt_hubs, as CSR by vertex rank position (entries of a
// vertex unordered). min over shared hubs c of d(h,c) + d(c,v) <= dv means a
// vertex outranking h lies on a shortest h-v path, as for the Common Label
// Table: the table is complete for a rank-closed set of hubs (Sec. 5.3). The
// query must see every table label of h and of v: a vertex reached only past a
// pruned one is left with a wrong distance and ancestor unless it is pruned
// too, which the complete query guarantees (a partial one would not). The
// root's table labels are hashed in shared memory, or, when more than the hash
// holds, written into the slot's dense array p.lt_root by hub position.
__device__ __forceinline__ uint32_t lth_slot(uint32_t hp) { return (hp * 2654435761u) >> 22; }

// does table entry (c, dc) of v witness dv: d(h, c) + dc <= dv for a hub c of
// the root (its distance from the hash, or from the slot's dense array rootd)
__device__ __forceinline__ bool lt_hit(const Shared &S, const uint32_t *rootd, uint32_t c, uint32_t dc,
                                       uint32_t dv) {
    if (dc > dv) return false;  // also every filler entry (all ones)
    if (rootd) {
        // written by this CTA at tree start: a plain load
        const uint32_t dhc = rootd[c];
        return dhc != NONE && uint64_t(dhc) + dc <= dv;
    }
    for (uint32_t sx = lth_slot(c);; sx = (sx + 1) & (LTH_SLOTS - 1)) {
        const uint32_t key = S.lth_key[sx];
        if (key == 0) return false;  // the hash holds at most half its slots
        if (key == c + 1) return uint64_t(S.lth_val[sx]) + dc <= dv;
    }
}

// One warp answers the query of one vertex whose table labels are entries
// [a, b) in global memory: each lane takes every 32nd of them (coalesced),
// QSTEPS steps of 32 are loaded before any is looked up, and the warp stops
// at the first step where some lane found a witness.
__device__ __forceinline__ bool lt_prunes_warp(const TreeLaunch &p, const Shared &S,
                                               const uint32_t *rootd, uint64_t a, uint64_t b,
                                               uint32_t dv, int lane) {
    for (uint64_t j0 = a; j0 < b; j0 += 32 * QSTEPS) {
        uint2 x[QSTEPS];
#pragma unroll
        for (int u = 0; u < QSTEPS; ++u) {
            const uint64_t j = j0 + uint64_t(u) * 32 + lane;
            x[u] = j < b ? __ldg(&p.lt_e[j]) : make_uint2(0, NONE);
        }
        bool hit = false;
        if (rootd) {
            // the root's distances by hub position: one predicated load per
            // entry (no divergent region); fillers and entries beyond dv
            // read nothing
#pragma unroll
            for (int u = 0; u < QSTEPS; ++u) {
                const bool near = x[u].y <= dv;
                const uint32_t dhc = near ? rootd[x[u].x] : NONE;
                hit |= dhc != NONE && uint64_t(dhc) + x[u].y <= dv;
            }
        } else {
#pragma unroll
            for (int u = 0; u < QSTEPS; ++u) hit |= lt_hit(S, rootd, x[u].x, x[u].y, dv);
        }
        if (__any_sync(0xffffffffu, hit)) return true;
    }
    return false;
}

// The same query over len entries already staged in shared memory.
__device__ __forceinline__ bool lt_prunes_staged(const Shared &S, const uint32_t *rootd, const uint2 *e,
                                                 uint32_t len, uint32_t dv, int lane) {
    for (uint32_t j0 = 0; j0 < len; j0 += 32) {
        const uint32_t j = j0 + lane;
        bool hit = false;
        if (j < len) {
            const uint2 x = e[j];
            hit = lt_hit(S, rootd, x.x, x.y, dv);
        }
        if (__any_sync(0xffffffffu, hit)) return true;
    }
    return false;
}

// Wait for the current phase of the staging barrier, bounded: past WAIT_LIMIT
// polls the error flag is set and the tree aborts; the wait goes on for as
// long again, so that copies still in flight land before the area is reused.
__device__ __forceinline__ void stage_wait(const TreeLaunch &p, Shared &S, uint32_t parity) {
    for (uint32_t it = 0; !mbar_try_wait(&S.mbar, parity); ++it) {
        if (it == WAIT_LIMIT) {
            atomicExch(&p.flags[0], ERR_WAIT_LIMIT);
            S.abort = 1;
        }
        if (it >= 2 * WAIT_LIMIT) break;
    }
}

// Answers the chunk's qn queued label-table queries (query q: its list starts
// at F.base[q], F.pre[q] = length << 32 | distance); the answer (1 = pruned)
// replaces F.pre[q]. The lists are copied into the shared staging area by the
// copy engine, as many per batch as fit, each widened to 16-byte boundaries
// (entries are 8 bytes, so one spare entry at either end): thread q issues the
// copy of query q, the batch's barrier counts the bytes, and then each warp
// answers whole queries from shared memory. No registers hold loads in flight,
// so a batch keeps hundreds of lists in flight per CTA. A list longer than
// the staging area is answered from global memory afterwards.
template <int TPB, typename K>
__device__ void lt_answer(const TreeLaunch &p, Shared &S, Frontier<TPB, K> &F, uint32_t qn,
                          uint8_t *stage, uint32_t &parity) {
    constexpr int NW = TPB / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t = threadIdx.x;
    const uint32_t *rootd = S.lt_dense == 1 ? p.lt_root + size_t(S.slot) * p.n
                            : S.lt_dense == 2 ? reinterpret_cast<const uint32_t *>(stage)
                                              : nullptr;
    // the batch's staged queries; the staging keys are free during stage A
    uint32_t *blist = reinterpret_cast<uint32_t *>(F.kv);
    uint64_t la = 0;
    uint32_t bytes = 0;
    bool todo = false;
    if (t < qn) {
        la = F.base[t];
        const uint64_t len = F.pre[t] >> 32;
        bytes = uint32_t((((la + len + 1) & ~1ull) - (la & ~1ull)) * 8u);
        todo = bytes <= p.stage_bytes;
        if (!todo) F.pre[t] |= 1ull << 63;  // answered from global memory
    }
    while (__syncthreads_or(todo)) {
        if (t == 0) {
            S.stage_used = 0;
            S.bn = 0;
        }
        __syncthreads();
        bool issued = false;
        if (todo) {
            // the first reservation of a batch always fits
            const uint32_t off = atomicAdd(&S.stage_used, bytes);
            if (off + bytes <= p.stage_bytes) {
                issued = true;
                todo = false;
                blist[atomicAdd(&S.bn, 1u)] = t;
                F.base[t] = (uint64_t(off) << 1) | (la & 1);
                mbar_arrive_expect_tx(&S.mbar, bytes);
                bulk_to_shared(stage + off, p.lt_e + (la & ~1ull), bytes, &S.mbar);
            }
        }
        if (!issued) mbar_arrive(&S.mbar);  // every thread arrives once per batch
        stage_wait(p, S, parity);
        parity ^= 1u;
        __syncthreads();  // blist and S.bn
        const uint32_t bn = S.bn;
        for (uint32_t i = warp; i < bn; i += NW) {
            const uint32_t q = blist[i];
            const uint64_t b = F.base[q], e = F.pre[q];
            const uint2 *ent = reinterpret_cast<const uint2 *>(stage + (b >> 1)) + (b & 1);
            const bool hit = lt_prunes_staged(S, rootd, ent, uint32_t(e >> 32), uint32_t(e), lane);
            __syncwarp();  // every lane has read the entry before lane 0 rewrites it
            if (lane == 0) F.pre[q] = hit;
        }
        __syncthreads();  // the next batch reuses the staging area
    }
    for (uint32_t q = warp; q < qn; q += NW) {
        const uint64_t e = F.pre[q];
        if (!(e >> 63)) continue;
        const uint64_t a = F.base[q];
        const bool hit =
            lt_prunes_warp(p, S, rootd, a, a + ((e >> 32) & 0x7FFFFFFFu), uint32_t(e), lane);
        __syncwarp();
        if (lane == 0) F.pre[q] = hit;
    }
}

// Expand the current list once, in chunks of TPB entries. In the first round
// of a bucket the list is the bucket's window list, whose stale entries (keys
// since lowered into an earlier bucket) are skipped.
//
// Arc pass: a warp walks its piece in steps of STEP = 32 * K::U consecutive
// arcs [i0, i0 + STEP). The rows starting inside a step are found with one
// ballot per 32 rows and recorded as a STEP-bit mask of start positions; the
// row of position q is then oa + (set bits at positions <= q), oa being the
// row that covers i0 (the last row of the previous step). Lanes first load
// K::U arcs, then K::U keys, then commit, so each lane has K::U
// independent loads in flight at each stage.
template <int TPB, typename K>
__device__ void expand_round(const TreeLaunch &p, Shared &S, Frontier<TPB, K> &F, const Slot<K> &sl,
                             uint32_t h, uint8_t *stage, uint32_t &parity) {
    using KS = typename K::T;
    constexpr int NW = TPB / 32;
    constexpr uint32_t STEP = 32 * K::U;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // The round's list, its length and the bucket start do not change during
    // the round; they are read from shared memory per chunk rather than held
    // in registers across the arc pass.
    for (uint32_t cb = 0; cb < S.cur_n; cb += TPB) {
        // ---- stage the chunk: rows, distances, liveness, degree prefix
        const uint32_t n_cur = S.cur_n;
        const uint64_t t_lo = S.t_lo;
        const uint32_t *cur = S.cur_slot != NONE ? sl.sub(S.cur_slot) : (S.sel ? sl.l1() : sl.l0());
        const uint32_t i = cb + threadIdx.x;
        uint64_t deg = 0, rs = 0;
        uint32_t dv = 0, vid = 0;
        bool lv = false, clean = false, cut = false, ask = false, ex = false;
        if (i < n_cur) {
            const uint32_t v = cur[i];
            const KS k = __ldcg(&sl.key[v]);
            vid = v;
            if (key_dist<K>(k) >= t_lo) {  // else stale: expanded in an earlier bucket
                dv = key_dist<K>(k);
                rs = __ldg(&p.row[v]);
                deg = __ldg(&p.row[v + 1]) - rs;
                lv = is_live<K>(k, v, h);
                clean = key_clean<K>(k);
                if (v < p.fin_bits && uint64_t(dv) < t_lo + p.w_min)
                    atomicOr(&fin_bitmap[v >> 5], 1u << (v & 31));
                ex = true;
                cut = S.prune && clt_query(p, S, v) <= dv;
                // a hub of the label table meets the root at the top vertex of
                // their shortest paths, which outranks v and so is a table hub
                // too: the complete query would find it
                if (!cut && S.lt_prune) {
                    if (v < p.lt_hubs) cut = true;
                    else ask = true;
                }
            }
        }
        if (S.lt_prune) {  // uniform over the CTA
            // queue the table queries with their label ranges; then each warp
            // answers whole queries
            uint64_t la = 0, lb = 0;
            if (ask) {
                la = __ldg(&p.lt_off[vid]);
                lb = __ldg(&p.lt_off[vid + 1]);
                ask = lb > la;  // no table label: nothing to find
            }
            const unsigned qm = __ballot_sync(FULL, ask);
            uint32_t qs = 0;
            if (qm) {
                const int leader = __ffs(qm) - 1;
                if (lane == leader) qs = atomicAdd(&S.qn, uint32_t(__popc(qm)));
                qs = __shfl_sync(FULL, qs, leader) + __popc(qm & ((1u << lane) - 1));
                if (ask) {
                    F.base[qs] = la;
                    F.pre[qs] = ((lb - la) << 32) | dv;
                }
            }
            __syncthreads();
            const uint32_t qn = S.qn;
            if (qn) lt_answer<TPB, K>(p, S, F, qn, stage, parity);
            __syncthreads();
            if (threadIdx.x == 0) S.qn = 0;  // read again only after the chunk's next barrier
            if (ask) cut = F.pre[qs] != 0;
        }
        if (cut) {
            // a table hub, which outranks h, lies on a shortest h-v path:
            // v gets no label and is not expanded (Sec. 5.3)
            deg = 0;
            if (clean) atomic_min_key(&sl.key[vid], make_key<K>(dv, false, 0));
        }
        const bool ok = deg != 0;
        const unsigned okm = __ballot_sync(FULL, ok);
        {
            const unsigned em = __ballot_sync(FULL, ex), pm = __ballot_sync(FULL, cut);
            if (lane == 0 && em) atomicAdd(&S.n_exp, (unsigned long long)__popc(em));
            if (lane == 0 && pm) atomicAdd(&S.n_pruned, (unsigned long long)__popc(pm));
        }
        // the bucket's live entries stop counting as pending when it is entered;
        // for a list of one chunk this stage counts them (no commit has run yet)
        if (S.fuse_live) {
            const int c = __popc(__ballot_sync(FULL, lv));
            if (lane == 0 && c) atomicSub(&S.cnt, c);
        }
        uint64_t inc = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) {
            F.wdeg[warp] = inc;
            F.wrows[warp] = __popc(okm);
        }
        __syncthreads();
        // every warp sums the warp totals itself: its offsets and the chunk totals
        uint64_t dl = 0, da = 0;
        uint32_t rl = 0, ra = 0;
        if (lane < NW) {
            const uint64_t x = F.wdeg[lane];
            const uint32_t r = F.wrows[lane];
            da = x;
            ra = r;
            if (lane < warp) { dl = x; rl = r; }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            dl += __shfl_xor_sync(FULL, dl, o);
            da += __shfl_xor_sync(FULL, da, o);
            rl += __shfl_xor_sync(FULL, rl, o);
            ra += __shfl_xor_sync(FULL, ra, o);
        }
        if (ok) {
            const uint32_t c = rl + __popc(okm & ((1u << lane) - 1));
            const uint64_t pre = dl + inc - deg;
            F.base[c] = rs - pre;  // wraps: base + position = rs + (position - pre)
            F.kv[c] = make_key<K>(dv, lv, vid);
            F.pre[c] = pre;
        }
        const uint64_t total = da;
        const uint32_t nrows = ra;
        __syncthreads();

        // ---- relax the chunk's arcs: warp w takes [lo, hi) of [0, total)
        const uint64_t per = (total + NW - 1) / NW;
        const uint64_t lo = per * warp;
        const uint64_t hi = lo + per < total ? lo + per : total;
        if (lo < hi) {
            if (lane == 0) atomicAdd(&S.n_arcs, (unsigned long long)(hi - lo));
            uint32_t oa = owner(F, lo, 0, nrows);
            uint32_t bn = 0;  // improvements in the warp's buffer
            for (uint64_t i0 = lo; i0 < hi; i0 += STEP) {
                const uint32_t span = hi - i0 < STEP ? uint32_t(hi - i0) : STEP;  // positions in this step
                uint2 a[K::U];
                KS kv[K::U];
#pragma unroll
                for (int k = 0; k < K::U; ++k) {
                    a[k] = make_uint2(0, 0);
                    kv[k] = 0;
                }
                uint32_t ob = oa;
                const uint64_t next = oa + 1 < nrows ? F.pre[oa + 1] : ~0ull;
                if (next >= i0 + span) {
                    // the whole step lies in row oa (long rows: hubs)
                    const uint64_t base = F.base[oa] + i0;
                    const KS k0 = F.kv[oa];
#pragma unroll
                    for (int k = 0; k < K::U; ++k) {
                        const uint32_t q = k * 32 + lane;
                        kv[k] = k0;
                        if (q < span) a[k] = __ldg(&p.arc[base + q]);
                    }
                } else {
                    // start positions (0..span-1) of rows oa+1, oa+2, ... inside the step
                    uint32_t wm[K::U];
#pragma unroll
                    for (int k = 0; k < K::U; ++k) wm[k] = 0;
                    for (;;) {
                        const uint32_t o = ob + 1 + lane;
                        uint32_t q = STEP;
                        if (o < nrows) {
                            const uint64_t st = F.pre[o];
                            if (st < i0 + span) q = uint32_t(st - i0);
                        }
                        const unsigned m = __ballot_sync(FULL, q < STEP);
#pragma unroll
                        for (int k = 0; k < K::U; ++k)
                            wm[k] |= __reduce_or_sync(FULL, (q >> 5) == uint32_t(k) ? 1u << (q & 31) : 0u);
                        ob += __popc(m);
                        if (m != FULL) break;
                    }
                    // every lane's row index stays below nrows (only row starts
                    // inside the span are counted), so the shared-memory reads
                    // need no guard; the arc load does
                    uint32_t cum = 0;
#pragma unroll
                    for (int k = 0; k < K::U; ++k) {
                        const uint32_t q = k * 32 + lane;
                        const uint32_t o = oa + cum + __popc(wm[k] & ((2u << lane) - 1u));
                        kv[k] = F.kv[o];
                        const uint64_t ai = F.base[o] + i0 + q;
                        if (q < span) a[k] = __ldg(&p.arc[ai]);
                        cum += __popc(wm[k]);
                    }
                }
                Probe<K> pr[K::U];
#pragma unroll
                for (int k = 0; k < K::U; ++k)
                    probe(p, S, sl, kv[k], a[k], uint32_t(k * 32 + lane) < span, pr[k]);
                bn = commit_step<TPB, K>(p, S, F, sl, h, pr, bn);
                oa = ob;
            }
            if (bn) commit_buffer<TPB, K>(p, S, F, sl, h, bn);
        }
        __syncthreads();  // the next chunk rewrites the staging arrays
    }
}

__device__ __forceinline__ uint32_t warp_min(uint32_t x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x = min(x, __shfl_xor_sync(FULL, x, o));
    return x;
}

// Far list pass with in-place compaction. Entries whose bucket is below
// `drop_below` are stale (listed in the window or expanded) and are dropped;
// with `move` set, entries whose bucket is below S.win_base + nwin move to
// the window lists; the minimum bucket of the remaining entries goes to
// S.min_b. Tags of removed entries are cleared so the vertex can be listed
// again.
template <int TPB, typename K>
__device__ void far_pass(const TreeLaunch &p, Shared &S, const Slot<K> &sl, uint32_t drop_below,
                         bool move) {
    const uint32_t n_in = S.far_n;
    __syncthreads();
    if (threadIdx.x == 0) {
        S.out_n = 0;
        S.min_b = NONE;
    }
    __syncthreads();
    const uint32_t win_end = S.win_base + p.nwin;
    uint32_t mn = NONE;
    for (uint32_t base = 0; base < n_in; base += TPB) {
        const uint32_t i = base + threadIdx.x;
        bool keep = false;
        uint32_t u = 0;
        if (i < n_in) {
            u = sl.far()[i];
            const uint32_t b = bucket_of(p, key_dist<K>(__ldcg(&sl.key[u])));
            if (b < drop_below) {
                // stale: lowered into the window (and listed there) or expanded
            } else if (move && b < win_end) {
                sub_append(S, sl, p.n, u, b);
            } else {
                keep = true;
                mn = min(mn, b);
            }
        }
        __syncthreads();  // every entry of this chunk is read before any is rewritten
        warp_append(keep, u, sl.far(), &S.out_n);
    }
    __syncthreads();
    mn = warp_min(mn);
    if ((threadIdx.x & 31) == 0) atomicMin(&S.min_b, mn);
    __syncthreads();
    if (threadIdx.x == 0) S.far_n = S.out_n;
    __syncthreads();
}

// live vertices among the window list of bucket b (entries whose key is in b)
template <int TPB, typename K>
__device__ void count_live_in_bucket(const TreeLaunch &p, Shared &S, const Slot<K> &sl, uint32_t h,
                                     uint32_t slot, uint32_t b) {
    __syncthreads();
    if (threadIdx.x == 0) S.live_sum = 0;
    __syncthreads();
    const uint32_t *lst = sl.sub(slot);
    const uint32_t cnt = S.sub_n[slot];
    int c = 0;
    for (uint32_t i = threadIdx.x; i < cnt; i += TPB) {
        const uint32_t u = lst[i];
        const typename K::T k = __ldcg(&sl.key[u]);
        c += (bucket_of(p, key_dist<K>(k)) == b && is_live<K>(k, u, h));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&S.live_sum, c);
    __syncthreads();
}

// Register bound: 1024 threads per SM (64 registers a thread). A 32-thread
// block asks for half that many blocks: shared memory holds fewer than 32 such
// CTAs per SM anyway, and the thread gets the registers its probe state needs.
template <int TPB, typename K>
__global__ void __launch_bounds__(TPB, TPB >= 64 ? 1024 / TPB : 16) plant_trees_kernel(TreeLaunch p) {
    __shared__ Shared S;
    __shared__ Frontier<TPB, K> F;
    const uint32_t n = p.n;
    // The CTA's tree slot: its own index, or (when launches share the slots)
    // any slot no running CTA holds. A CTA becomes resident only once another
    // has left its SM, and every CTA gives its slot back before it exits, so
    // a free slot exists; a CTA that finds none leaves its roots to the others.
    if (threadIdx.x == 0) {
        uint32_t got = NONE;
        if (p.dyn_slots) {
            for (uint32_t i = 0; i < p.nslots; ++i) {
                const uint32_t c = (blockIdx.x + i) % p.nslots;
                if (atomicCAS(&p.slot_ctr[c * 4 + 1], 0u, 1u) == 0u) {
                    got = c;
                    break;
                }
            }
        } else {
            got = blockIdx.x;
        }
        S.slot = got;
    }
    __syncthreads();
    if (S.slot == NONE) return;
    const size_t so = size_t(S.slot) * n;
    Slot<K> sl;
    sl.key = (typename K::T *)p.key + so;
    sl.rtag = p.rtag + so;
    sl.lists = p.lists + so * (4 + p.nwin);
    sl.n = n;

    uint8_t *stage = reinterpret_cast<uint8_t *>(fin_bitmap) + stage_offset(p.fin_words);
    uint32_t parity = 0;  // phase of S.mbar the next staging batch completes
    if (threadIdx.x == 0) {
        S.rid = p.slot_ctr[S.slot * 4 + 0];
        mbar_init(&S.mbar, TPB);
        S.n_exp = S.n_arcs = S.n_pruned = S.n_rounds = S.n_buckets = 0;
        S.n_trees = S.n_trivial = 0;
    }

    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t r = NONE;
            if (!p.flags[1] && !p.flags[0] && !(p.stop && *(volatile const int *)p.stop)) {
                const uint32_t cnt = p.count_dev ? *(volatile const uint32_t *)p.count_dev : p.root_count;
                const uint32_t i = atomicAdd(p.next_root, 1u);
                if (i < cnt) r = p.root_list ? p.root_list[i] : p.root_begin + i;
            }
            S.root = r;
        }
        __syncthreads();
        const uint32_t h = S.root;
        if (h == NONE) break;
        if (threadIdx.x == 0) ++S.n_trees;

        // trivial tree: every neighbour outranks the root, so after the root is
        // popped no queued vertex has the root as ancestor (cnt = 0)
        bool lower = false;
        {
            const uint64_t rs = p.row[h], re = p.row[h + 1];
            for (uint64_t e = rs + threadIdx.x; e < re; e += TPB) lower |= (__ldg(&p.arc[e]).x > h);
        }
        const bool nontrivial = __syncthreads_or(lower);

        uint32_t nlab = 0;
        if (!nontrivial) {
            if (threadIdx.x == 0) ++S.n_trivial;
            if (threadIdx.x == 0) {
                S.out_n = 1;
                sl.l0()[0] = h;
                sl.l1()[0] = 0;
                sl.far()[0] = h;  // the root is its own parent
            }
            __syncthreads();
            nlab = 1;
        } else {
            // ---- tree search
            for (uint32_t s = threadIdx.x; s < p.nwin; s += TPB) S.sub_n[s] = 0;
            for (uint32_t i = threadIdx.x; i < p.fin_words; i += TPB) fin_bitmap[i] = 0;
            // trees of roots outside the table prune with it; the table's own
            // trees (which built it) do not
            const bool prune = p.hc && h >= p.hc_hubs;
            if (prune)
                for (uint32_t c = threadIdx.x; c < p.hc_stride; c += TPB)
                    S.hch[c] = __ldg(&p.hc[size_t(h) * p.hc_stride + c]);
            if (threadIdx.x == 0) S.prune = prune;
            // the label table of earlier phases: the root's labels in it, as
            // distances by hub position in shared memory when the table's hubs
            // fit the auxiliary area (no staging), else hashed or (more than
            // the hash holds) in the slot's dense array
            bool lt_prune = p.lt_off && h >= p.lt_hubs;
            bool lt_dense = false;
            const bool lt_shared = lt_prune && !p.stage_bytes && p.lt_hubs <= p.aux_bytes / 4;
            uint64_t lt_a = 0, lt_b = 0;
            if (lt_prune) {
                lt_a = __ldg(&p.lt_off[h]);
                lt_b = __ldg(&p.lt_off[h + 1]);
                lt_dense = !lt_shared && lt_b - lt_a > min(LTH_MAX, p.lt_hash_max);  // uniform over the CTA
                lt_prune = !lt_dense || p.lt_root;
                lt_dense = lt_dense && lt_prune;
            }
            if (lt_shared) {
                uint32_t *rs = reinterpret_cast<uint32_t *>(stage);
                for (uint32_t c = threadIdx.x; c < p.lt_hubs; c += TPB) rs[c] = NONE;
                __syncthreads();
                for (uint64_t j = lt_a + threadIdx.x; j < lt_b; j += TPB) {
                    const uint2 e = __ldg(&p.lt_e[j]);  // hub positions of the table lie below lt_hubs
                    rs[e.x] = e.y;
                }
            } else if (lt_dense) {
                uint32_t *rootd = p.lt_root + so;
                for (uint64_t j = lt_a + threadIdx.x; j < lt_b; j += TPB) {
                    const uint2 e = __ldg(&p.lt_e[j]);
                    rootd[e.x] = e.y;
                }
            } else if (lt_prune) {
                for (uint32_t i = threadIdx.x; i < LTH_SLOTS; i += TPB) S.lth_key[i] = 0;
                __syncthreads();
                const uint64_t a = lt_a;
                const uint32_t cnt = uint32_t(lt_b - lt_a);
                for (uint32_t i = threadIdx.x; i < cnt; i += TPB) {
                    const uint2 e = __ldg(&p.lt_e[a + i]);
                    for (uint32_t sx = lth_slot(e.x);; sx = (sx + 1) & (LTH_SLOTS - 1)) {
                        if (atomicCAS(&S.lth_key[sx], 0u, e.x + 1) == 0u) {
                            S.lth_val[sx] = e.y;
                            break;
                        }
                    }
                }
            }
            if (threadIdx.x == 0) {
                S.lt_prune = lt_prune;
                S.lt_dense = lt_shared ? 2 : lt_dense ? 1 : 0;
                S.lt_a = lt_a;
                S.lt_b = lt_b;
            }
            if (threadIdx.x == 0) {
                S.cur_n = 1;
                S.nxt_n = 0;
                S.far_n = 0;
                S.touch_n = 1;
                S.sel = 0;
                S.cur_slot = NONE;
                S.rid += 1;
                S.bcur = 0;
                S.win_base = 0;
                S.cnt = 0;
                S.t_lo = 0;
                S.t_hi = p.delta;
                S.w_hi = uint64_t(p.delta) * p.nwin;
                S.abort = 0;
                S.fuse_live = 0;
                S.qn = 0;
                sl.l0()[0] = h;
                sl.touch()[0] = h;
                atomic_set_key(&sl.key[h], make_key<K>(0, true, h));
            }
            __syncthreads();
            uint32_t rounds = 0;
            for (;;) {
                expand_round<TPB, K>(p, S, F, sl, h, stage, parity);  // ends with a barrier
                if (S.abort) break;
                if (threadIdx.x == 0) ++S.n_rounds;
                if (++rounds > p.round_limit) {
                    if (threadIdx.x == 0) atomicExch(&p.flags[0], ERR_ROUND_LIMIT);
                    break;
                }
                if (S.nxt_n) {  // the current bucket is not settled yet
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        S.sel ^= 1u;  // the next round reads the list this round appended to
                        S.cur_slot = NONE;
                        S.fuse_live = 0;
                        S.cur_n = S.nxt_n;
                        S.nxt_n = 0;
                        S.rid += 1;
                    }
                    __syncthreads();
                    continue;
                }
                // bucket settled: every key below t_hi is final. Warp 0 marks
                // its list consumed and finds the next non-empty window bucket.
                if (threadIdx.x < 32) {
                    const uint32_t s0 = S.bcur >= S.win_base ? S.bcur - S.win_base + 1 : 0;
                    uint32_t found = NONE;
                    for (uint32_t b0 = 0; b0 < p.nwin; b0 += 32) {
                        const uint32_t sx = b0 + threadIdx.x;
                        const unsigned m = __ballot_sync(FULL, sx >= s0 && sx < p.nwin && S.sub_n[sx] != 0);
                        if (m) { found = S.win_base + b0 + __ffs(m) - 1; break; }
                    }
                    __syncwarp();
                    if (threadIdx.x == 0) {
                        if (S.bcur >= S.win_base) S.sub_n[S.bcur - S.win_base] = 0;  // consumed
                        S.cur_slot = NONE;
                        S.min_b = found;
                    }
                }
                __syncthreads();
                if (S.cnt == 0) break;  // no pending vertex can still receive the root as hub
                if (S.min_b == NONE) {
                    // window used up: restart it at the nearest far bucket
                    far_pass<TPB, K>(p, S, sl, S.win_base + p.nwin, false);
                    if (S.far_n == 0) break;  // nothing pending at all
                    if (threadIdx.x == 0) {
                        S.win_base = S.min_b;
                        S.w_hi = uint64_t(S.win_base + p.nwin) * p.delta;
                        for (uint32_t s = 0; s < p.nwin; ++s) S.sub_n[s] = 0;
                    }
                    __syncthreads();
                    far_pass<TPB, K>(p, S, sl, 0, true);
                    if (threadIdx.x == 0) S.min_b = S.win_base;
                    __syncthreads();
                }
                // enter bucket min_b: its live vertices stop counting as pending
                const uint32_t nb = S.min_b, slot = nb - S.win_base;
                if (threadIdx.x == 0) ++S.n_buckets;
                const bool fuse = S.sub_n[slot] <= TPB;
                if (!fuse) count_live_in_bucket<TPB, K>(p, S, sl, h, slot, nb);
                if (threadIdx.x == 0) {
                    if (!fuse) S.cnt -= S.live_sum;
                    S.fuse_live = fuse;
                    S.bcur = nb;
                    S.t_lo = uint64_t(nb) * p.delta;
                    S.t_hi = S.t_lo + p.delta;
                    S.cur_slot = slot;
                    S.cur_n = S.sub_n[slot];
                    S.rid += 1;
                }
                __syncthreads();
            }
            __syncthreads();
            if (S.abort) {
                // reset and give up on this tree; the host reports the error
                for (uint32_t i = threadIdx.x; i < S.touch_n; i += TPB) sl.key[sl.touch()[i]] = key_inf<K>();
                if (S.lt_dense == 1)
                    for (uint64_t j = S.lt_a + threadIdx.x; j < S.lt_b; j += TPB) p.lt_root[so + __ldg(&p.lt_e[j]).x] = NONE;
                __threadfence();
                __syncthreads();
                break;
            }
            // ---- label emission: live touched vertices, staged in l0 (vertex) / l1 (dist)
            if (threadIdx.x == 0) {
                S.out_n = 0;
            }
            __syncthreads();
            const uint32_t nt = S.touch_n;
            for (uint32_t base = 0; base < nt; base += TPB) {
                const uint32_t i = base + threadIdx.x;
                bool lv = false;
                uint32_t u = 0, d = 0, par = 0;
                if (i < nt) {
                    u = sl.touch()[i];
                    const typename K::T k = __ldcg(&sl.key[u]);
                    lv = is_live<K>(k, u, h);
                    d = key_dist<K>(k);
                    par = key_parent<K>(k);
                }
                const unsigned m = __ballot_sync(FULL, lv);
                if (m) {
                    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                    uint32_t b = 0;
                    if (lane == leader) b = atomicAdd(&S.out_n, (uint32_t)__popc(m));
                    b = __shfl_sync(FULL, b, leader);
                    if (lv) {
                        const uint32_t o = b + __popc(m & ((1u << lane) - 1));
                        sl.l0()[o] = u;
                        sl.l1()[o] = d;
                        if (p.out_p) sl.far()[o] = par;  // far is free once the tree stopped
                    }
                }
            }
            __syncthreads();
            nlab = S.out_n;
            // reset exactly what this tree modified
            for (uint32_t i = threadIdx.x; i < nt; i += TPB) sl.key[sl.touch()[i]] = key_inf<K>();
            if (S.lt_dense == 1)
                for (uint64_t j = S.lt_a + threadIdx.x; j < S.lt_b; j += TPB) p.lt_root[so + __ldg(&p.lt_e[j]).x] = NONE;
            // the next tree reads keys with L2 loads and L2 atomics: the plain
            // reset stores must be visible there first, not only inside the CTA
            __threadfence();
        }

        // ---- reserve an all-or-nothing output range and copy the labels out
        if (threadIdx.x == 0) {
            const unsigned long long old = atomicAdd(p.out_count, (unsigned long long)nlab);
            S.ok = old + nlab <= p.out_cap;
            S.base = old;
            if (!S.ok) {
                // nlab >= 1, so only the first range past the end starts within it
                if (old <= p.out_cap) *p.out_valid = old;
                p.failed[atomicAdd(p.failed_count, 1u)] = h;
                atomicExch(&p.flags[1], 1);
            }
        }
        __syncthreads();
        if (S.ok) {
            const unsigned long long b = S.base;
            for (uint32_t i = threadIdx.x; i < nlab; i += TPB) {
                p.out_v[b + i] = __ldg(&p.vert_at[sl.l0()[i]]);
                p.out_h[b + i] = h;
                p.out_d[b + i] = sl.l1()[i];
                if (p.out_p) p.out_p[b + i] = __ldg(&p.vert_at[sl.far()[i]]);
            }
        }
        __syncthreads();
    }

    // counters (every warp's shared-memory adds came before the last barrier)
    if (threadIdx.x == 0) {
        atomicAdd(&p.stats[0], S.n_exp);
        atomicAdd(&p.stats[1], S.n_arcs);
        if (S.n_pruned) atomicAdd(&p.stats[6], S.n_pruned);
        atomicAdd(&p.stats[2], (unsigned long long)S.n_trivial);
        atomicAdd(&p.stats[3], (unsigned long long)S.n_trees);
        atomicAdd(&p.stats[4], S.n_rounds);
        atomicAdd(&p.stats[5], S.n_buckets);
        p.slot_ctr[S.slot * 4 + 0] = S.rid;
        if (p.dyn_slots) {
            // the slot is idle again (every key and root array entry reset)
            __threadfence();
            atomicExch(&p.slot_ctr[S.slot * 4 + 1], 0u);
        }
    }
}

// both key widths may take up to the opt-in maximum of dynamic shared memory
template <typename F>
cudaError_t allow_smem_of(F kernel, int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (!e) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - int(fa.sharedSizeBytes));
    return e;
}

template <int TPB>
cudaError_t allow_smem() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!e) e = allow_smem_of(plant_trees_kernel<TPB, KeyN>, optin);
    if (!e) e = allow_smem_of(plant_trees_kernel<TPB, KeyW>, optin);
    if (!e) e = allow_smem_of(plant_trees_kernel<TPB, KeyP>, optin);
    return e;
}

// dynamic shared memory of a launch: the settled bitmap, then (label-pruned
// phases) the staging area at the next multiple of 128 bytes
size_t dyn_bytes(uint32_t fin_words, uint32_t aux_bytes) {
    return aux_bytes ? ((size_t(fin_words) * 4 + 127) & ~size_t(127)) + aux_bytes : size_t(fin_words) * 4;
}

template <int TPB>
cudaError_t launch_t(const TreeLaunch &p, int slots, cudaStream_t s) {
    cudaError_t e = allow_smem<TPB>();
    if (e) return e;
    const size_t smem = dyn_bytes(p.fin_words, p.aux_bytes);
    if (p.out_p)
        plant_trees_kernel<TPB, KeyP><<<slots, TPB, smem, s>>>(p);
    else if (p.key_bytes == 4)
        plant_trees_kernel<TPB, KeyN><<<slots, TPB, smem, s>>>(p);
    else if (p.key_bytes == 8)
        plant_trees_kernel<TPB, KeyW><<<slots, TPB, smem, s>>>(p);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// CTAs per SM with `bytes` of dynamic shared memory; all key layouts are built
// under the same register cap, the smallest of the three is returned
template <int TPB>
int occ(size_t bytes) {
    if (allow_smem<TPB>()) return 0;
    int b = 0, b4 = 0, bp = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, plant_trees_kernel<TPB, KeyW>, TPB, bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b4, plant_trees_kernel<TPB, KeyN>, TPB, bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bp, plant_trees_kernel<TPB, KeyP>, TPB, bytes);
    b = b < b4 ? b : b4;
    return b < bp ? b : bp;
}

// Shared memory per SM that the tree launches may take. The SM's L1 and
// shared memory are one store: what shared memory does not take is L1, which
// the kernel's read-only loads (arcs, rows, table rows and entries) go
// through. Measured on rmat21 (1024-thread slots, one per SM): a settled
// bitmap of all 1.24M vertices (155 KB) plus a 2-39 KB table area made the
// label-pruned phases 1.5x slower than the bitmap alone, and a bitmap capped
// at 100 KB was 11% faster than the whole one.
constexpr uint32_t SMEM_PER_SM_CAP = SMEM_CAP_BYTES;

// the most dynamic shared memory (a multiple of 128 bytes) that keeps the
// register-limited number of CTAs per SM, within SMEM_PER_SM_CAP per SM
template <int TPB>
uint32_t dyn_budget_t() {
    const int full = occ<TPB>(0);
    if (full <= 0) return 0;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))
        return 0;
    uint32_t lo = 0, hi = uint32_t(optin) & ~127u;  // occ(lo) == full holds for lo = 0
    if (occ<TPB>(hi) >= full) {
        lo = hi;
    } else {
        while (hi - lo > 128) {
            const uint32_t mid = (lo + (hi - lo) / 2) & ~127u;
            if (mid <= lo) break;
            if (occ<TPB>(mid) >= full) lo = mid; else hi = mid;
        }
    }
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, plant_trees_kernel<TPB, KeyN>)) return lo;
    // per CTA: the cap's share, less the static part and the 1 KiB the SM reserves per CTA
    const int64_t cap = int64_t(SMEM_PER_SM_CAP) / full - int64_t(fa.sharedSizeBytes) - 1024;
    const uint32_t c = cap > 0 ? uint32_t(cap) & ~127u : 0u;
    return c < lo ? c : lo;
}

}  // namespace

cudaError_t launch_plant_trees(const TreeLaunch &pl, int tpt, int slots, cudaStream_t s) {
    TreeLaunch p = pl;
    p.nslots = uint32_t(slots);
    if (p.nwin < 2 || p.nwin > NWIN_MAX) return cudaErrorInvalidValue;
    // the staging copies read the label table in 16-byte units
    if (p.lt_off && ((reinterpret_cast<uintptr_t>(p.lt_e) & 15) || (p.stage_bytes & 15)))
        return cudaErrorMisalignedAddress;
    if (p.stage_bytes > p.aux_bytes) return cudaErrorInvalidValue;
    switch (tpt) {
        case 32: return launch_t<32>(p, slots, s);
        case 64: return launch_t<64>(p, slots, s);
        case 128: return launch_t<128>(p, slots, s);
        case 256: return launch_t<256>(p, slots, s);
        case 512: return launch_t<512>(p, slots, s);
        case 1024: return launch_t<1024>(p, slots, s);
        default: return cudaErrorInvalidValue;
    }
}

int plant_max_slots_per_sm(int tpt, uint32_t fin_words, uint32_t aux_bytes) {
    const size_t bytes = dyn_bytes(fin_words, aux_bytes);
    switch (tpt) {
        case 32: return occ<32>(bytes);
        case 64: return occ<64>(bytes);
        case 128: return occ<128>(bytes);
        case 256: return occ<256>(bytes);
        case 512: return occ<512>(bytes);
        case 1024: return occ<1024>(bytes);
        default: return 0;
    }
}

uint32_t plant_dyn_budget(int tpt) {
    switch (tpt) {
        case 32: return dyn_budget_t<32>();
        case 64: return dyn_budget_t<64>();
        case 128: return dyn_budget_t<128>();
        case 256: return dyn_budget_t<256>();
        case 512: return dyn_budget_t<512>();
        case 1024: return dyn_budget_t<1024>();
        default: return 0;
    }
}

void plant_smem_split(int tpt, uint32_t n, uint32_t aux_want, uint32_t *fin_words,
                      uint32_t *aux_bytes) {
    const uint32_t budget = plant_dyn_budget(tpt);
    const uint32_t want = (n + 31) / 32;
    const uint32_t stage = std::min<uint32_t>(budget / 2, aux_want) & ~127u;
    const uint32_t room = budget > stage + 128 ? budget - stage - 128 : 0;
    uint32_t fw = std::min<uint32_t>(want, room / 4);
    if (fw < want) fw &= ~31u;
    *fin_words = fw;
    *aux_bytes = stage;
}

}  // namespace chl

namespace chl {
namespace {

// Common Label Table from label records: record i is (caller vertex out_v[i],
// hub pos out_h[i], distance out_d[i]); those of hubs below `hubs` go in
__global__ void clt_fill_kernel(const uint32_t *out_v, const uint32_t *out_h, const uint32_t *out_d,
                                unsigned long long count, const uint32_t *pos_of, uint32_t *hc,
                                uint32_t stride, uint32_t hubs) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t c = out_h[i];
        if (c < hubs) hc[size_t(pos_of[out_v[i]]) * stride + c] = out_d[i];
    }
}

}  // namespace

cudaError_t launch_clt_fill(const uint32_t *out_v, const uint32_t *out_h, const uint32_t *out_d,
                            unsigned long long count, const uint32_t *pos_of, uint32_t *hc,
                            uint32_t stride, uint32_t hubs, cudaStream_t s) {
    if (!count) return cudaSuccess;
    unsigned long long blocks = (count + 255) / 256;
    if (blocks > uint64_t(device_sms()) * 32) blocks = uint64_t(device_sms()) * 32;
    clt_fill_kernel<<<unsigned(blocks), 256, 0, s>>>(out_v, out_h, out_d, count, pos_of, hc, stride,
                                                     hubs);
    return cudaGetLastError();
}

namespace {

// A root all of whose neighbours outrank it is a trivial tree: once the root
// is popped no queued vertex has it as ancestor (Algorithm 3 stops), so its
// only label is (h, h, 0). One thread per root of [begin, begin + count):
// trivial roots get that label here (one output reservation per warp), the
// others are listed for the tree launch.
__global__ void split_trivial_kernel(TreeLaunch p, uint32_t begin, uint32_t count, uint32_t *list,
                                     unsigned int *list_n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool triv = false;
    const uint32_t h = begin + i;
    if (i < count) {
        triv = true;
        const uint64_t rs = __ldg(&p.row[h]), re = __ldg(&p.row[h + 1]);
        for (uint64_t e = rs; e < re && triv; ++e) triv = __ldg(&p.arc[e]).x <= h;
    }
    const unsigned tm = __ballot_sync(0xffffffffu, triv);
    const unsigned om = __ballot_sync(0xffffffffu, i < count && !triv);
    const unsigned below = (1u << lane) - 1;
    if (tm) {
        unsigned long long b = 0;
        if (lane == 0) {
            b = atomicAdd(p.out_count, (unsigned long long)__popc(tm));
            atomicAdd(&p.stats[2], (unsigned long long)__popc(tm));
            atomicAdd(&p.stats[3], (unsigned long long)__popc(tm));
        }
        b = __shfl_sync(0xffffffffu, b, 0);
        if (triv) {
            const unsigned long long o = b + __popc(tm & below);
            const uint32_t cv = __ldg(&p.vert_at[h]);
            p.out_v[o] = cv;
            p.out_h[o] = h;
            p.out_d[o] = 0;
            if (p.out_p) p.out_p[o] = cv;  // the root is its own parent
        }
    }
    if (om) {
        unsigned b = 0;
        if (lane == 0) b = atomicAdd(list_n, unsigned(__popc(om)));
        b = __shfl_sync(0xffffffffu, b, 0);
        if (i < count && !triv) list[b + __popc(om & below)] = h;
    }
}

}  // namespace

cudaError_t launch_split_trivial(const TreeLaunch &p, uint32_t begin, uint32_t count, uint32_t *list,
                                 unsigned int *list_n, cudaStream_t s) {
    if (!count) return cudaSuccess;
    split_trivial_kernel<<<(count + 255) / 256, 256, 0, s>>>(p, begin, count, list, list_n);
    return cudaGetLastError();
}

}  // namespace chl
