// PLaNT shortest-path trees on the GPU (Sec. 4.2, Algorithm 3).
//
// One persistent launch builds every tree of a root range. Each CTA owns a
// tree "slot" (dense per-vertex state in global memory) and repeatedly claims
// the next root in rank order with a global atomic counter, the dynamic
// root claiming of Sec. 3.1 (threads pop the most important remaining root).
//
// Per tree the search is a bucketed label-correcting Dijkstra (delta-stepping,
// bucket width delta) over packed keys (see "Keys" below): an atomicMin keeps
// the shortest distance and, at equal distance, prefers a path through a
// vertex that outranks the root (Algorithm 3, equal-distance branch). Every
// vertex that is expanded relaxes all its arcs, labelled or not: PLaNT does
// not prune trees (Sec. 1, Sec. 4.2); a vertex outranked by its ancestor only
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
// resetting only what the tree modified, footnote of Sec. 3.1).
//
// Early termination (Sec. 4.2). The paper stops when every vertex in
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
// (vertex, root, dist); the tree reserves its output range with one CAS
// (all-or-nothing, so a full buffer loses no partial tree), and the host
// rebuilds failed roots after growing the buffer.
#include <cstdio>

#include "chl_common.cuh"

namespace chl {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t MAX_ROUNDS_PER_TREE = 1u << 26;
constexpr uint32_t RESERVE_TRIES = 1u << 20;
constexpr int LARGE_DEG = 32;
constexpr uint32_t NWIN_MAX = 64;
constexpr int UNROLL = 4;
constexpr uint32_t CHUNK = 32 * UNROLL;  // arcs one warp relaxes per step
constexpr uint32_t HUB_DEG = 4 * CHUNK;  // rows this long are shared by all warps
constexpr uint32_t HUBQ = 128;           // queued hub rows per round
constexpr uint32_t NONE = 0xFFFFFFFFu;

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
// equal-distance branch of Algorithm 3; Sec. 4.2's example, a[v5] = v1).
// v is live (would get the label (h, d)) iff clean and v >= h, and the bit
// it passes on to its out-neighbours is exactly its own liveness.
// K = uint32_t when every tentative distance is provably below 2^31 - 1 (the
// host checks w_max * n), else uint64_t. All ones is "unreached".
template <typename K>
__device__ __forceinline__ K key_inf() { return ~K(0); }
template <typename K>
__device__ __forceinline__ K make_key(uint64_t dist, bool clean) { return (K(dist) << 1) | K(clean); }
template <typename K>
__device__ __forceinline__ uint32_t key_dist(K k) { return uint32_t(k >> 1); }
// largest distance a key of type K holds below key_inf
template <typename K>
__device__ __forceinline__ uint64_t key_dist_limit() {
    return sizeof(K) == 4 ? 0x7FFFFFFEull : 0xFFFFFFFEull;
}

struct Shared {
    uint32_t root;
    uint32_t cur_n, nxt_n, far_n, touch_n;
    uint32_t rid, fid;
    uint32_t sel;          // round lists: cur = sel ? l1 : l0 (rounds after the first)
    uint32_t cur_slot;     // window slot expanded in the bucket's first round, NONE after
    uint32_t bcur;         // current bucket
    uint32_t win_base;     // bucket of window slot 0
    uint32_t bid_base;     // tag of bucket b is bid_base + b + 1
    uint32_t bid_top;      // one past the largest bucket tagged in this tree
    int cnt;               // live vertices with keys beyond the current bucket
    uint64_t t_lo, t_hi;   // current bucket [t_lo, t_hi)
    uint64_t w_hi;         // end of the window
    uint32_t min_b;
    uint32_t out_n;
    int abort;
    int ok;
    int live_sum;
    unsigned long long base;
    uint32_t sub_n[NWIN_MAX];
    // high-degree rows queued for CTA-wide processing in the current round
    uint32_t hub_n, hub_next;
    uint32_t hub_dv[HUBQ], hub_av[HUBQ], hub_deg[HUBQ], hub_pre[HUBQ + 1];
    uint64_t hub_rs[HUBQ];
};

template <typename K>
struct Slot {
    K *key;
    uint32_t *rtag, *wtag, *ftag;
    uint32_t *l0, *l1, *far, *touch, *sub;  // sub: nwin lists of n entries
};

template <typename K>
__device__ __forceinline__ bool is_live(K k, uint32_t v, uint32_t h) {
    return (k & 1) && v >= h;
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

// list a pending vertex in bucket b of the window (the tag dedups per bucket)
template <typename K>
__device__ __forceinline__ void sub_append(Shared &S, const Slot<K> &sl, uint32_t n, uint32_t u,
                                           uint32_t b) {
    const uint32_t s = b - S.win_base;
    const uint32_t tag = S.bid_base + b + 1;
    if (atomicExch(&sl.wtag[u], tag) != tag) sl.sub[size_t(s) * n + atomicAdd(&S.sub_n[s], 1u)] = u;
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
    K cand;
    K seen;
    uint32_t u;
    bool live;  // still worth committing
};

__device__ __forceinline__ uint32_t atomic_min_key(uint32_t *a, uint32_t v) { return atomicMin(a, v); }
__device__ __forceinline__ uint64_t atomic_min_key(uint64_t *a, uint64_t v) {
    return atomicMin((unsigned long long *)a, (unsigned long long)v);
}
__device__ __forceinline__ void atomic_set_key(uint32_t *a, uint32_t v) { atomicExch(a, v); }
__device__ __forceinline__ void atomic_set_key(uint64_t *a, uint64_t v) {
    atomicExch((unsigned long long *)a, (unsigned long long)v);
}

template <typename K>
__device__ __forceinline__ void probe(const TreeLaunch &p, Shared &S, const Slot<K> &sl, uint32_t dv,
                                      bool lv, uint2 a, Probe<K> &q) {
    q.u = a.x;
    const uint64_t nd = uint64_t(dv) + a.y;
    if (nd > key_dist_limit<K>()) {
        atomicExch(&p.flags[0], ERR_DIST_OVERFLOW);
        S.abort = 1;
        q.live = false;
        return;
    }
    q.cand = make_key<K>(nd, lv);
    q.seen = __ldcg(&sl.key[q.u]);
    q.live = true;
}

template <typename K>
__device__ __forceinline__ void commit(const TreeLaunch &p, Shared &S, const Slot<K> &sl, uint32_t h,
                                       const Probe<K> &q) {
    if (q.cand >= q.seen) return;
    const uint32_t u = q.u;
    const K old = atomic_min_key(&sl.key[u], q.cand);
    if (q.cand >= old) return;
    if (old == key_inf<K>()) sl.touch[atomicAdd(&S.touch_n, 1u)] = u;
    const uint32_t nb = key_dist(q.cand) / p.delta;
    const bool f_new = nb > S.bcur && is_live(q.cand, u, h);
    const bool f_old = old != key_inf<K>() && key_dist(old) / p.delta > S.bcur && is_live(old, u, h);
    if (f_new != f_old) atomicAdd(&S.cnt, f_new ? 1 : -1);
    if (nb == S.bcur) {
        if (atomicExch(&sl.rtag[u], S.rid) != S.rid) {
            uint32_t *nxt = S.sel ? sl.l0 : sl.l1;
            nxt[atomicAdd(&S.nxt_n, 1u)] = u;
        }
    } else if (key_dist(q.cand) < S.w_hi) {
        sub_append(S, sl, p.n, u, nb);
    } else if (atomicExch(&sl.ftag[u], S.fid) != S.fid) {
        sl.far[atomicAdd(&S.far_n, 1u)] = u;
    }
}

// relax arcs [j0, min(j0 + CHUNK, deg)) of one row, UNROLL arcs per lane in flight
template <typename K>
__device__ __forceinline__ void relax_chunk(const TreeLaunch &p, Shared &S, const Slot<K> &sl,
                                            uint32_t h, uint32_t dv, bool lv, uint64_t rs,
                                            uint32_t deg, uint32_t j0, unsigned long long &arcs) {
    const int lane = threadIdx.x & 31;
    Probe<K> q[UNROLL];
    uint2 a[UNROLL];
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
        const uint32_t j = j0 + k * 32 + lane;
        if (j < deg) a[k] = __ldg(&p.arc[rs + j]);
    }
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
        const uint32_t j = j0 + k * 32 + lane;
        q[k].live = false;
        if (j < deg) {
            ++arcs;
            probe(p, S, sl, dv, lv, a[k], q[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < UNROLL; ++k)
        if (q[k].live) commit(p, S, sl, h, q[k]);
}

// Expand the current list once. In the first round of a bucket the list is
// the bucket's window list, whose stale entries (keys since lowered into an
// earlier bucket) are skipped. Rows shorter than 32 arcs are packed densely
// over the lanes of a warp; rows of 32..HUB_DEG-1 arcs are walked by the warp
// that met them; longer rows (hubs of scale-free graphs) are queued and split
// into CHUNK-arc pieces that all warps claim, so one hub does not hold the
// whole CTA at the round barrier.
template <int TPB, typename K>
__device__ void expand_round(const TreeLaunch &p, Shared &S, const Slot<K> &sl, uint32_t h,
                             unsigned long long &expanded, unsigned long long &arcs) {
    constexpr int NW = TPB / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t *cur = S.cur_slot != NONE ? sl.sub + size_t(S.cur_slot) * p.n
                                             : (S.sel ? sl.l1 : sl.l0);
    const uint32_t n_cur = S.cur_n;
    const uint64_t t_lo = S.t_lo;
    for (uint32_t base = warp * 32; base < n_cur; base += NW * 32) {
        const uint32_t i = base + lane;
        uint32_t dv = 0, av = 0, deg = 0;  // av: liveness of v as 0/1
        uint64_t rs = 0;
        if (i < n_cur) {
            const uint32_t v = cur[i];
            const K k = __ldcg(&sl.key[v]);
            if (key_dist(k) >= t_lo) {  // else stale: expanded in an earlier bucket
                dv = key_dist(k);
                av = is_live(k, v, h);
                rs = __ldg(&p.row[v]);
                deg = uint32_t(__ldg(&p.row[v + 1]) - rs);
                ++expanded;
            }
        }
        bool queued = false;
        if (deg >= HUB_DEG) {
            const uint32_t slot = atomicAdd(&S.hub_n, 1u);
            if (slot < HUBQ) {
                S.hub_dv[slot] = dv;
                S.hub_av[slot] = av;
                S.hub_deg[slot] = deg;
                S.hub_rs[slot] = rs;
                queued = true;
            }
        }
        // rows of 32+ arcs not queued: the whole warp walks the row
        unsigned big = __ballot_sync(FULL, deg >= LARGE_DEG && !queued);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t bd = __shfl_sync(FULL, dv, src);
            const uint32_t ba = __shfl_sync(FULL, av, src);
            const uint64_t brs = __shfl_sync(FULL, rs, src);
            const uint32_t bdeg = __shfl_sync(FULL, deg, src);
            for (uint32_t j0 = 0; j0 < bdeg; j0 += CHUNK)
                relax_chunk(p, S, sl, h, bd, ba != 0, brs, bdeg, j0, arcs);
        }
        // low-degree vertices: pack their arcs densely over the lanes
        const uint32_t ds = deg < LARGE_DEG ? deg : 0;
        uint32_t incl = ds;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        const uint32_t excl = incl - ds;
        for (uint32_t jb = 0; jb < total; jb += 32) {
            const uint32_t j = jb + lane;
            int o = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int c = o + step;
                const uint32_t ex = __shfl_sync(FULL, excl, c);
                if (ex <= j) o = c;
            }
            const uint32_t od = __shfl_sync(FULL, dv, o);
            const uint32_t oa = __shfl_sync(FULL, av, o);
            const uint32_t oex = __shfl_sync(FULL, excl, o);
            const uint64_t ors = __shfl_sync(FULL, rs, o);
            if (j < total) {
                Probe<K> q;
                ++arcs;
                probe(p, S, sl, od, oa != 0, __ldg(&p.arc[ors + (j - oex)]), q);
                if (q.live) commit(p, S, sl, h, q);
            }
        }
    }
    __syncthreads();
    // queued hub rows: CHUNK-arc pieces claimed by any warp
    const uint32_t nh = min(S.hub_n, HUBQ);
    if (nh) {
        if (warp == 0) {
            uint32_t run = 0;
            for (uint32_t b = 0; b < nh; b += 32) {
                const uint32_t it = b + lane;
                const uint32_t c = it < nh ? (S.hub_deg[it] + CHUNK - 1) / CHUNK : 0;
                uint32_t inc = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(FULL, inc, o);
                    if (lane >= o) inc += t;
                }
                if (it < nh) S.hub_pre[it] = run + inc - c;
                run += __shfl_sync(FULL, inc, 31);
            }
            if (lane == 0) {
                S.hub_pre[nh] = run;
                S.hub_next = 0;
            }
        }
        __syncthreads();
        const uint32_t chunks = S.hub_pre[nh];
        for (;;) {
            uint32_t c = 0;
            if (lane == 0) c = atomicAdd(&S.hub_next, 1u);
            c = __shfl_sync(FULL, c, 0);
            if (c >= chunks) break;
            uint32_t lo = 0, hi = nh;  // largest item with hub_pre[item] <= c
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (S.hub_pre[mid] <= c) lo = mid; else hi = mid;
            }
            relax_chunk(p, S, sl, h, S.hub_dv[lo], S.hub_av[lo] != 0, S.hub_rs[lo], S.hub_deg[lo],
                        (c - S.hub_pre[lo]) * CHUNK, arcs);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) S.hub_n = 0;
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
            u = sl.far[i];
            const uint32_t b = key_dist(__ldcg(&sl.key[u])) / p.delta;
            if (b < drop_below) {
                sl.ftag[u] = 0;
            } else if (move && b < win_end) {
                sl.ftag[u] = 0;
                sub_append(S, sl, p.n, u, b);
            } else {
                keep = true;
                mn = min(mn, b);
            }
        }
        __syncthreads();  // every entry of this chunk is read before any is rewritten
        warp_append(keep, u, sl.far, &S.out_n);
    }
    // tag resets above are plain stores, while tags are later updated by
    // atomics performed in L2: publish them device-wide before the barrier
    __threadfence();
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
    const uint32_t *lst = sl.sub + size_t(slot) * p.n;
    const uint32_t cnt = S.sub_n[slot];
    int c = 0;
    for (uint32_t i = threadIdx.x; i < cnt; i += TPB) {
        const uint32_t u = lst[i];
        const K k = __ldcg(&sl.key[u]);
        c += (key_dist(k) / p.delta == b && is_live(k, u, h));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&S.live_sum, c);
    __syncthreads();
}

template <int TPB, typename K>
__global__ void __launch_bounds__(TPB, 1024 / TPB) plant_trees_kernel(TreeLaunch p) {
    __shared__ Shared S;
    const uint32_t n = p.n;
    const size_t so = size_t(blockIdx.x) * n;
    Slot<K> sl;
    sl.key = (K *)p.key + so;
    sl.rtag = p.rtag + so;
    sl.wtag = p.wtag + so;
    sl.ftag = p.ftag + so;
    uint32_t *lb = p.lists + so * (4 + p.nwin);
    sl.l0 = lb;
    sl.l1 = lb + n;
    sl.far = lb + 2 * size_t(n);
    sl.touch = lb + 3 * size_t(n);
    sl.sub = lb + 4 * size_t(n);

    unsigned long long expanded = 0, arcs = 0, trivial = 0, trees = 0;
    if (threadIdx.x == 0) {
        S.hub_n = 0;
        S.rid = p.slot_ctr[blockIdx.x * 4 + 0];
        S.bid_base = p.slot_ctr[blockIdx.x * 4 + 1];
        S.fid = p.slot_ctr[blockIdx.x * 4 + 2];
    }

    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t r = NONE;
            if (!p.flags[1] && !p.flags[0]) {
                const uint32_t i = atomicAdd(p.next_root, 1u);
                if (i < p.root_count) r = p.root_list ? p.root_list[i] : p.root_begin + i;
            }
            S.root = r;
        }
        __syncthreads();
        const uint32_t h = S.root;
        if (h == NONE) break;
        ++trees;

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
            ++trivial;
            if (threadIdx.x == 0) {
                S.out_n = 1;
                sl.l0[0] = h;
                sl.l1[0] = 0;
            }
            __syncthreads();
            nlab = 1;
        } else {
            // ---- tree search
            for (uint32_t s = threadIdx.x; s < p.nwin; s += TPB) S.sub_n[s] = 0;
            if (threadIdx.x == 0) {
                S.cur_n = 1;
                S.nxt_n = 0;
                S.far_n = 0;
                S.touch_n = 1;
                S.sel = 0;
                S.cur_slot = NONE;
                S.rid += 1;
                S.fid += 1;
                S.bcur = 0;
                S.win_base = 0;
                S.bid_top = p.nwin;
                S.cnt = 0;
                S.t_lo = 0;
                S.t_hi = p.delta;
                S.w_hi = uint64_t(p.delta) * p.nwin;
                S.abort = 0;
                sl.l0[0] = h;
                sl.touch[0] = h;
                atomic_set_key(&sl.key[h], make_key<K>(0, true));
            }
            __syncthreads();
            uint32_t rounds = 0;
            for (;;) {
                expand_round<TPB, K>(p, S, sl, h, expanded, arcs);
                __syncthreads();
                if (S.abort) break;
                if (++rounds > MAX_ROUNDS_PER_TREE) {
                    if (threadIdx.x == 0) atomicExch(&p.flags[0], ERR_ROUND_LIMIT);
                    break;
                }
                if (S.nxt_n) {  // the current bucket is not settled yet
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        S.sel ^= 1u;  // the next round reads the list this round appended to
                        S.cur_slot = NONE;
                        S.cur_n = S.nxt_n;
                        S.nxt_n = 0;
                        S.rid += 1;
                    }
                    __syncthreads();
                    continue;
                }
                // bucket settled: every key below t_hi is final
                __syncthreads();
                if (threadIdx.x == 0) {
                    if (S.bcur >= S.win_base) S.sub_n[S.bcur - S.win_base] = 0;  // consumed
                    S.cur_slot = NONE;
                    S.min_b = NONE;
                }
                __syncthreads();
                if (S.cnt == 0) break;  // no pending vertex can still receive the root as hub
                // next non-empty bucket of the window
                if (threadIdx.x == 0) {
                    const uint32_t s0 = S.bcur >= S.win_base ? S.bcur - S.win_base + 1 : 0;
                    for (uint32_t s = s0; s < p.nwin; ++s)
                        if (S.sub_n[s]) { S.min_b = S.win_base + s; break; }
                }
                __syncthreads();
                if (S.min_b == NONE) {
                    // window used up: restart it at the nearest far bucket
                    far_pass<TPB, K>(p, S, sl, S.win_base + p.nwin, false);
                    if (S.far_n == 0) break;  // nothing pending at all
                    if (threadIdx.x == 0) {
                        S.win_base = S.min_b;
                        S.w_hi = uint64_t(S.win_base + p.nwin) * p.delta;
                        if (S.win_base + p.nwin > S.bid_top) S.bid_top = S.win_base + p.nwin;
                        for (uint32_t s = 0; s < p.nwin; ++s) S.sub_n[s] = 0;
                    }
                    __syncthreads();
                    far_pass<TPB, K>(p, S, sl, 0, true);
                    if (threadIdx.x == 0) S.min_b = S.win_base;
                    __syncthreads();
                }
                // enter bucket min_b: its live vertices stop counting as pending
                const uint32_t nb = S.min_b, slot = nb - S.win_base;
                count_live_in_bucket<TPB, K>(p, S, sl, h, slot, nb);
                if (threadIdx.x == 0) {
                    S.cnt -= S.live_sum;
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
                for (uint32_t i = threadIdx.x; i < S.touch_n; i += TPB) sl.key[sl.touch[i]] = key_inf<K>();
                __threadfence();
                __syncthreads();
                break;
            }
            // ---- label emission: live touched vertices, staged in l0 (vertex) / l1 (dist)
            if (threadIdx.x == 0) {
                S.out_n = 0;
                S.bid_base += S.bid_top + 2;  // fresh window tags for the next tree
            }
            __syncthreads();
            const uint32_t nt = S.touch_n;
            for (uint32_t base = 0; base < nt; base += TPB) {
                const uint32_t i = base + threadIdx.x;
                bool lv = false;
                uint32_t u = 0, d = 0;
                if (i < nt) {
                    u = sl.touch[i];
                    const K k = __ldcg(&sl.key[u]);
                    lv = is_live(k, u, h);
                    d = key_dist(k);
                }
                const unsigned m = __ballot_sync(FULL, lv);
                if (m) {
                    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                    uint32_t b = 0;
                    if (lane == leader) b = atomicAdd(&S.out_n, (uint32_t)__popc(m));
                    b = __shfl_sync(FULL, b, leader);
                    if (lv) {
                        const uint32_t o = b + __popc(m & ((1u << lane) - 1));
                        sl.l0[o] = u;
                        sl.l1[o] = d;
                    }
                }
            }
            __syncthreads();
            nlab = S.out_n;
            // reset exactly what this tree modified
            for (uint32_t i = threadIdx.x; i < nt; i += TPB) sl.key[sl.touch[i]] = key_inf<K>();
            // the next tree reads keys with L2 loads and L2 atomics: the plain
            // reset stores must be visible there first, not only inside the CTA
            __threadfence();
        }

        // ---- reserve an all-or-nothing output range and copy the labels out
        if (threadIdx.x == 0) {
            S.ok = 0;
            unsigned long long old = *((volatile unsigned long long *)p.out_count);
            uint32_t t = 0;
            for (; t < RESERVE_TRIES; ++t) {
                if (old + nlab > p.out_cap) break;
                const unsigned long long prev = atomicCAS(p.out_count, old, old + nlab);
                if (prev == old) { S.ok = 1; break; }
                old = prev;
            }
            if (t == RESERVE_TRIES) atomicExch(&p.flags[0], ERR_RESERVE_LIMIT);
            S.base = old;
            if (!S.ok) {
                p.failed[atomicAdd(p.failed_count, 1u)] = h;
                atomicExch(&p.flags[1], 1);
            }
        }
        __syncthreads();
        if (S.ok) {
            const unsigned long long b = S.base;
            for (uint32_t i = threadIdx.x; i < nlab; i += TPB) {
                p.out_v[b + i] = __ldg(&p.vert_at[sl.l0[i]]);
                p.out_h[b + i] = h;
                p.out_d[b + i] = sl.l1[i];
            }
        }
        __syncthreads();
    }

    // counters
    for (int o = 16; o; o >>= 1) {
        expanded += __shfl_xor_sync(FULL, expanded, o);
        arcs += __shfl_xor_sync(FULL, arcs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&p.stats[0], expanded);
        atomicAdd(&p.stats[1], arcs);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&p.stats[2], trivial);
        atomicAdd(&p.stats[3], trees);
        p.slot_ctr[blockIdx.x * 4 + 0] = S.rid;
        p.slot_ctr[blockIdx.x * 4 + 1] = S.bid_base;
        p.slot_ctr[blockIdx.x * 4 + 2] = S.fid;
    }
}

template <int TPB>
cudaError_t launch_t(const TreeLaunch &p, int slots, cudaStream_t s) {
    if (p.key_bytes == 4)
        plant_trees_kernel<TPB, uint32_t><<<slots, TPB, 0, s>>>(p);
    else if (p.key_bytes == 8)
        plant_trees_kernel<TPB, uint64_t><<<slots, TPB, 0, s>>>(p);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// both key widths are built under the same register cap, so they share the
// occupancy of the wide form
template <int TPB>
int occ() {
    int b = 0, b4 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, plant_trees_kernel<TPB, uint64_t>, TPB, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b4, plant_trees_kernel<TPB, uint32_t>, TPB, 0);
    return b < b4 ? b : b4;
}

}  // namespace

cudaError_t launch_plant_trees(const TreeLaunch &p, int tpt, int slots, cudaStream_t s) {
    if (p.nwin < 2 || p.nwin > NWIN_MAX) return cudaErrorInvalidValue;
    switch (tpt) {
        case 32: return launch_t<32>(p, slots, s);
        case 64: return launch_t<64>(p, slots, s);
        case 128: return launch_t<128>(p, slots, s);
        case 256: return launch_t<256>(p, slots, s);
        case 512: return launch_t<512>(p, slots, s);
        default: return cudaErrorInvalidValue;
    }
}

int plant_max_slots_per_sm(int tpt) {
    switch (tpt) {
        case 32: return occ<32>();
        case 64: return occ<64>();
        case 128: return occ<128>();
        case 256: return occ<256>();
        case 512: return occ<512>();
        default: return 0;
    }
}

}  // namespace chl
