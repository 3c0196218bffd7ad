// PLaNT shortest-path trees on the GPU (Sec. 4.2, Algorithm 3).
//
// One persistent launch builds every tree of a root range. Each CTA owns a
// tree "slot" (dense per-vertex state in global memory) and repeatedly claims
// the next root in rank order with a global atomic counter, the dynamic
// root claiming of Sec. 3.1 (threads pop the most important remaining root).
//
// Per tree the search is a bucketed label-correcting Dijkstra (delta-stepping)
// over packed keys dist<<32 | anc (see chl_common.cuh): a 64-bit atomicMin
// keeps the shortest distance and, at equal distance, the highest-ranked
// ancestor (Algorithm 3, equal-distance branch). Every vertex that is
// expanded relaxes all its arcs, labelled or not: PLaNT does not prune trees
// (Sec. 1, Sec. 4.2); a vertex outranked by its ancestor only gets no label.
//
// Early termination (Sec. 4.2): the paper stops a tree when every vertex in
// Dijkstra's queue is outranked (cnt = 0). Here the pending vertices are the
// ones whose key lies in a later bucket; after a bucket converges, all keys
// below its upper bound are final, and the tree stops once no pending vertex
// is live. The test is exact at bucket granularity: the lists that hold
// pending vertices are scanned (the far list only when a live key was ever
// sent there).
//
// Pending vertices sit in four deduplicated lists per slot:
//   cur  vertices of the current bucket to expand this round
//   nxt  vertices of the current bucket improved during this round
//   win  vertices in later buckets of the current window (nwin buckets)
//   far  vertices beyond the window
// plus `touched`, every vertex that got a finite key (for emission and
// for resetting only what the tree modified, footnote of Sec. 3.1).
//
// Labels: after a tree stops, every touched vertex whose key is live gets
// (vertex, root, dist); the tree reserves its output range with one CAS
// (the range is all-or-nothing, so a full buffer loses no partial tree), and
// the host rebuilds failed roots after growing the buffer.
#include <cstdio>

#include "chl_common.cuh"

namespace chl {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t MAX_ROUNDS_PER_TREE = 1u << 26;
constexpr uint32_t RESERVE_TRIES = 1u << 20;
constexpr int LARGE_DEG = 32;

struct Shared {
    uint32_t root;
    uint32_t cur_n, nxt_n, win_n, far_n, touch_n;
    uint32_t rid, wid, fid;
    uint32_t sel;          // which of list 0/1 is cur
    uint64_t t_hi, w_hi;   // bucket and window upper bounds (exclusive)
    uint32_t min_d;
    uint32_t out_n;
    int far_live;
    int live;
    int tmp_live;
    uint32_t tmp_min;
    int abort;
    int ok;
    unsigned long long base;
};

struct Slot {
    uint64_t *key;
    uint32_t *rtag, *wtag, *ftag;
    uint32_t *l0, *l1, *win, *far, *touch;
};

__device__ __forceinline__ bool is_live(uint64_t k, uint32_t v, uint32_t h) {
    return key_anc(k) == h && v >= h;
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

// Relaxation of one arc (v -> u, weight w) of a vertex expanded with distance
// dv and inclusive ancestor av = min(anc(v), v), in two stages so that a lane
// can have several key loads in flight:
//   probe:  form the candidate key and load the target's key from L2 (keys
//           only decrease, so a stale read never hides an improvement)
//   commit: if the candidate is smaller, atomicMin; on improvement, record
//           the vertex as touched and list it for the bucket it now falls in

struct Probe {
    uint64_t cand;
    uint64_t seen;
    uint32_t u;
    bool live;  // still worth committing
};

__device__ __forceinline__ void probe(const TreeLaunch &p, Shared &S, const Slot &sl, uint32_t dv,
                                      uint32_t av, uint2 a, Probe &q) {
    q.u = a.x;
    const uint64_t nd = uint64_t(dv) + a.y;
    if (nd >= 0xFFFFFFFFull) {
        atomicExch(&p.flags[0], ERR_DIST_OVERFLOW);
        S.abort = 1;
        q.live = false;
        return;
    }
    q.cand = make_key(uint32_t(nd), av);
    q.seen = __ldcg(&sl.key[q.u]);
    q.live = true;
}

__device__ __forceinline__ void commit(Shared &S, const Slot &sl, uint32_t h, uint32_t av,
                                       const Probe &q) {
    const uint32_t u = q.u;
    if (q.cand >= q.seen) return;
    const uint64_t old = atomicMin((unsigned long long *)&sl.key[u], (unsigned long long)q.cand);
    if (q.cand >= old) return;
    if (old == KEY_INF) sl.touch[atomicAdd(&S.touch_n, 1u)] = u;
    const uint64_t nd = key_dist(q.cand);
    if (nd < S.t_hi) {
        if (atomicExch(&sl.rtag[u], S.rid) != S.rid) {
            uint32_t *nxt = S.sel ? sl.l0 : sl.l1;
            nxt[atomicAdd(&S.nxt_n, 1u)] = u;
        }
    } else if (nd < S.w_hi) {
        if (atomicExch(&sl.wtag[u], S.wid) != S.wid) sl.win[atomicAdd(&S.win_n, 1u)] = u;
    } else {
        if (atomicExch(&sl.ftag[u], S.fid) != S.fid) sl.far[atomicAdd(&S.far_n, 1u)] = u;
        if (av == h && u > h) S.far_live = 1;
    }
}

constexpr int UNROLL = 4;

// expand every vertex of the current list once
template <int TPB>
__device__ void expand_round(const TreeLaunch &p, Shared &S, const Slot &sl, uint32_t h,
                             unsigned long long &expanded, unsigned long long &arcs) {
    constexpr int NW = TPB / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t *cur = S.sel ? sl.l1 : sl.l0;
    const uint32_t n_cur = S.cur_n;
    for (uint32_t base = warp * 32; base < n_cur; base += NW * 32) {
        const uint32_t i = base + lane;
        uint32_t dv = 0, av = 0, deg = 0;
        uint64_t rs = 0;
        if (i < n_cur) {
            const uint32_t v = cur[i];
            const uint64_t k = __ldcg(&sl.key[v]);
            dv = key_dist(k);
            av = min(key_anc(k), v);
            rs = __ldg(&p.row[v]);
            deg = uint32_t(__ldg(&p.row[v + 1]) - rs);
            ++expanded;
        }
        // high-degree vertices: the whole warp walks the row, 32 arcs per step
        unsigned big = __ballot_sync(FULL, deg >= LARGE_DEG);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t bd = __shfl_sync(FULL, dv, src);
            const uint32_t ba = __shfl_sync(FULL, av, src);
            const uint64_t brs = __shfl_sync(FULL, rs, src);
            const uint32_t bdeg = __shfl_sync(FULL, deg, src);
            for (uint32_t j0 = 0; j0 < bdeg; j0 += 32 * UNROLL) {
                Probe q[UNROLL];
                uint2 a[UNROLL];
#pragma unroll
                for (int k = 0; k < UNROLL; ++k) {
                    const uint32_t j = j0 + k * 32 + lane;
                    if (j < bdeg) a[k] = __ldg(&p.arc[brs + j]);
                }
#pragma unroll
                for (int k = 0; k < UNROLL; ++k) {
                    const uint32_t j = j0 + k * 32 + lane;
                    q[k].live = false;
                    if (j < bdeg) {
                        ++arcs;
                        probe(p, S, sl, bd, ba, a[k], q[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < UNROLL; ++k)
                    if (q[k].live) commit(S, sl, h, ba, q[k]);
            }
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
                Probe q;
                ++arcs;
                probe(p, S, sl, od, oa, __ldg(&p.arc[ors + (j - oex)]), q);
                if (q.live) commit(S, sl, h, oa, q);
            }
        }
    }
}

// block-wide min / or helpers (result valid in all threads after return)
__device__ __forceinline__ uint32_t warp_min(uint32_t x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x = min(x, __shfl_xor_sync(FULL, x, o));
    return x;
}

// Pass over a pending list (win or far) with in-place compaction.
//   mode 0: drop entries with dist < drop_below (stale); report live / min of the rest
//   mode 1: entries with dist < take_below move to `dst` (dst tag set to dst_tag);
//           the rest stay; report live / min of the rest
// Tags of removed entries are cleared so the vertex can be listed again.
template <int TPB>
__device__ void list_pass(Shared &S, const Slot &sl, uint32_t h, uint32_t *list, uint32_t *count,
                          uint32_t *tag, int mode, uint64_t bound, uint32_t *dst,
                          uint32_t *dst_count, uint32_t *dst_tagarr, uint32_t dst_tag,
                          int *live_out, uint32_t *min_out) {
    const uint32_t n_in = *count;
    if (threadIdx.x == 0) S.out_n = 0;
    __syncthreads();
    bool live = false;
    uint32_t mn = 0xFFFFFFFFu;
    for (uint32_t base = 0; base < n_in; base += TPB) {
        const uint32_t i = base + threadIdx.x;
        bool keep = false, move = false;
        uint32_t u = 0;
        if (i < n_in) {
            u = list[i];
            const uint64_t k = __ldcg(&sl.key[u]);
            const uint32_t d = key_dist(k);
            if (d < bound) {
                tag[u] = 0;
                move = (mode == 1);
                if (move && dst_tagarr) dst_tagarr[u] = dst_tag;
            } else {
                keep = true;
                live |= is_live(k, u, h);
                mn = min(mn, d);
            }
        }
        __syncthreads();  // every entry of this chunk is read before any is rewritten
        warp_append(keep, u, list, &S.out_n);
        if (mode == 1) warp_append(move, u, dst, dst_count);
    }
    // the tag resets above are plain stores, while tags are later updated by
    // atomics performed in L2: publish them device-wide before the barrier
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *count = S.out_n;
    mn = warp_min(mn);
    if ((threadIdx.x & 31) == 0) atomicMin(min_out, mn);
    live = __syncthreads_or(live);
    if (threadIdx.x == 0 && live) *live_out = 1;
    __syncthreads();
}

template <int TPB>
__global__ void __launch_bounds__(TPB) plant_trees_kernel(TreeLaunch p) {
    __shared__ Shared S;
    const uint32_t n = p.n;
    const size_t so = size_t(blockIdx.x) * n;
    Slot sl;
    sl.key = p.key + so;
    sl.rtag = p.rtag + so;
    sl.wtag = p.wtag + so;
    sl.ftag = p.ftag + so;
    uint32_t *lb = p.lists + so * 5;
    sl.l0 = lb;
    sl.l1 = lb + n;
    sl.win = lb + 2 * size_t(n);
    sl.far = lb + 3 * size_t(n);
    sl.touch = lb + 4 * size_t(n);

    unsigned long long expanded = 0, arcs = 0, trivial = 0, trees = 0;
    if (threadIdx.x == 0) {
        S.rid = p.slot_ctr[blockIdx.x * 4 + 0];
        S.wid = p.slot_ctr[blockIdx.x * 4 + 1];
        S.fid = p.slot_ctr[blockIdx.x * 4 + 2];
    }

    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t r = 0xFFFFFFFFu;
            if (!p.flags[1] && !p.flags[0]) {
                const uint32_t i = atomicAdd(p.next_root, 1u);
                if (i < p.root_count) r = p.root_list ? p.root_list[i] : p.root_begin + i;
            }
            S.root = r;
        }
        __syncthreads();
        const uint32_t h = S.root;
        if (h == 0xFFFFFFFFu) break;
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
            if (threadIdx.x == 0) {
                S.cur_n = 1;
                S.nxt_n = 0;
                S.win_n = 0;
                S.far_n = 0;
                S.touch_n = 1;
                S.sel = 0;
                S.rid += 1;
                S.wid += 1;
                S.fid += 1;
                S.t_hi = p.delta;
                S.w_hi = uint64_t(p.delta) * p.nwin;
                S.far_live = 0;
                S.abort = 0;
                sl.l0[0] = h;
                sl.touch[0] = h;
                atomicExch((unsigned long long *)&sl.key[h], (unsigned long long)make_key(0, h));
            }
            __syncthreads();
            uint32_t rounds = 0;
            for (;;) {
                expand_round<TPB>(p, S, sl, h, expanded, arcs);
                __syncthreads();
                if (S.abort) break;
                if (++rounds > MAX_ROUNDS_PER_TREE) {
                    if (threadIdx.x == 0) atomicExch(&p.flags[0], ERR_ROUND_LIMIT);
                    break;
                }
                if (S.nxt_n) {  // the current bucket is not settled yet
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        S.sel ^= 1u;
                        S.cur_n = S.nxt_n;
                        S.nxt_n = 0;
                        S.rid += 1;
                    }
                    __syncthreads();
                    continue;
                }
                // bucket settled: all keys below t_hi are final.
                // 1) pending vertices of the window: drop stale ones, find live / min
                if (threadIdx.x == 0) { S.live = 0; S.min_d = 0xFFFFFFFFu; }
                __syncthreads();
                list_pass<TPB>(S, sl, h, sl.win, &S.win_n, sl.wtag, 0, S.t_hi, nullptr, nullptr,
                               nullptr, 0, &S.live, &S.min_d);
                // 2) beyond the window: scanned only if a live key was ever sent there
                if (!S.live && S.far_live) {
                    if (threadIdx.x == 0) { S.tmp_live = 0; S.tmp_min = 0xFFFFFFFFu; }
                    __syncthreads();
                    list_pass<TPB>(S, sl, h, sl.far, &S.far_n, sl.ftag, 0, S.w_hi, nullptr,
                                   nullptr, nullptr, 0, &S.tmp_live, &S.tmp_min);
                    if (threadIdx.x == 0) { S.far_live = S.tmp_live; S.live = S.tmp_live; }
                    __syncthreads();
                }
                if (!S.live) break;  // no pending vertex can still receive the root as hub
                // 3) the window is empty: open the next window at the nearest far entry
                if (S.win_n == 0) {
                    if (threadIdx.x == 0) { S.tmp_live = 0; S.tmp_min = 0xFFFFFFFFu; }
                    __syncthreads();
                    list_pass<TPB>(S, sl, h, sl.far, &S.far_n, sl.ftag, 0, S.w_hi, nullptr,
                                   nullptr, nullptr, 0, &S.tmp_live, &S.tmp_min);
                    if (S.far_n == 0) break;
                    if (threadIdx.x == 0) {
                        S.min_d = S.tmp_min;
                        const uint64_t wlo = (uint64_t(S.min_d) / p.delta) * p.delta;
                        S.w_hi = wlo + uint64_t(p.delta) * p.nwin;
                        S.wid += 1;
                        S.tmp_live = 0;
                        S.tmp_min = 0xFFFFFFFFu;
                    }
                    __syncthreads();
                    list_pass<TPB>(S, sl, h, sl.far, &S.far_n, sl.ftag, 1, S.w_hi, sl.win,
                                   &S.win_n, sl.wtag, S.wid, &S.tmp_live, &S.tmp_min);
                    if (threadIdx.x == 0) S.far_live = S.tmp_live;  // live among what stays far
                    __syncthreads();
                }
                // 4) the next non-empty bucket becomes current: move its entries to cur
                if (threadIdx.x == 0) {
                    const uint64_t tlo = (uint64_t(S.min_d) / p.delta) * p.delta;
                    S.t_hi = tlo + p.delta;
                    S.rid += 1;
                    S.cur_n = 0;
                    S.tmp_live = 0;
                    S.tmp_min = 0xFFFFFFFFu;
                }
                __syncthreads();
                list_pass<TPB>(S, sl, h, sl.win, &S.win_n, sl.wtag, 1, S.t_hi,
                               S.sel ? sl.l1 : sl.l0, &S.cur_n, nullptr, 0, &S.tmp_live,
                               &S.tmp_min);
            }
            __syncthreads();
            if (S.abort) {
                // reset and give up on this tree; the host reports the error
                for (uint32_t i = threadIdx.x; i < S.touch_n; i += TPB) sl.key[sl.touch[i]] = KEY_INF;
                __threadfence();
                __syncthreads();
                break;
            }
            // ---- label emission: live touched vertices, staged in l0 (vertex) / l1 (dist)
            if (threadIdx.x == 0) S.out_n = 0;
            __syncthreads();
            const uint32_t nt = S.touch_n;
            for (uint32_t base = 0; base < nt; base += TPB) {
                const uint32_t i = base + threadIdx.x;
                bool lv = false;
                uint32_t u = 0, d = 0;
                if (i < nt) {
                    u = sl.touch[i];
                    const uint64_t k = __ldcg(&sl.key[u]);
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
            for (uint32_t i = threadIdx.x; i < nt; i += TPB) sl.key[sl.touch[i]] = KEY_INF;
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
        p.slot_ctr[blockIdx.x * 4 + 1] = S.wid;
        p.slot_ctr[blockIdx.x * 4 + 2] = S.fid;
    }
}

template <int TPB>
cudaError_t launch_t(const TreeLaunch &p, int slots, cudaStream_t s) {
    plant_trees_kernel<TPB><<<slots, TPB, 0, s>>>(p);
    return cudaGetLastError();
}

template <int TPB>
int occ() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, plant_trees_kernel<TPB>, TPB, 0);
    return b;
}

}  // namespace

cudaError_t launch_plant_trees(const TreeLaunch &p, int tpt, int slots, cudaStream_t s) {
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
