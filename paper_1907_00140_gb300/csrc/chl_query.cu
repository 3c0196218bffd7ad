// PPSD queries by merge-intersection of rank-sorted label lists.
//
// d(u,v) = min over hubs h in L_u and L_v of d(u,h) + d(v,h) (Sec. 1, cover
// property); the paper's single-node mode merges the two hub-rank-sorted lists
// (Sec. 6 QLSN, footnote of Sec. 7.2 on linear-merge querying).
//
// One warp per query. Both lists are read in 32-entry chunks with coalesced
// loads (hub rank position, ascending). Each lane takes one entry of the L_u
// chunk and looks it up in the L_v chunk by a 5-step binary search over lanes
// (shuffles); matches contribute d(u,h)+d(v,h). The chunk whose last entry is
// smaller is consumed entirely and the other advances past every entry not
// larger than that, which is a merge on 32-wide blocks: every common hub is
// met exactly once. Sums are 64-bit and saturate at UINT32_MAX; a pair without
// a common hub (different components) answers UINT32_MAX.
#include "chl_common.cuh"

namespace chl {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint64_t min64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// d(u, v) by one warp (all 32 lanes call it with the same u, v)
__device__ __forceinline__ uint32_t merge_query(const uint64_t *__restrict__ off,
                                                const uint32_t *__restrict__ hp,
                                                const uint32_t *__restrict__ dd, uint32_t u,
                                                uint32_t v) {
    const int lane = threadIdx.x & 31;
    const uint64_t a0 = __ldg(&off[u]), la = __ldg(&off[u + 1]) - a0;
    const uint64_t b0 = __ldg(&off[v]), lb = __ldg(&off[v + 1]) - b0;
    uint64_t ia = 0, ib = 0;
    uint64_t best = 0xFFFFFFFFull;
    while (ia < la && ib < lb) {
        const bool va = ia + lane < la, vb = ib + lane < lb;
        const uint32_t x = va ? __ldg(&hp[a0 + ia + lane]) : 0xFFFFFFFFu;
        const uint32_t y = vb ? __ldg(&hp[b0 + ib + lane]) : 0xFFFFFFFFu;
        // largest lane l with y[l] <= x (y ascending across lanes)
        int o = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int c = o + step;
            if (__shfl_sync(FULL, y, c) <= x) o = c;
        }
        const uint32_t yo = __shfl_sync(FULL, y, o);
        const bool hit = va && yo == x;
        const unsigned hits = __ballot_sync(FULL, hit);
        if (hits) {
            // fetch both distances only for matching lanes
            uint64_t s = 0xFFFFFFFFull;
            if (hit) s = uint64_t(__ldg(&dd[a0 + ia + lane])) + __ldg(&dd[b0 + ib + o]);
            best = min64(best, s);
        }
        const uint32_t lastA = __shfl_sync(FULL, x, int(min64(la - ia, 32) - 1));
        const uint32_t lastB = __shfl_sync(FULL, y, int(min64(lb - ib, 32) - 1));
        if (lastA <= lastB) {
            ia += min64(la - ia, 32);
            ib += __popc(__ballot_sync(FULL, vb && y <= lastA));
        } else {
            ib += min64(lb - ib, 32);
            ia += __popc(__ballot_sync(FULL, va && x <= lastB));
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) best = min64(best, __shfl_xor_sync(FULL, best, o));
    return uint32_t(min64(best, 0xFFFFFFFFull));
}

__global__ void query_kernel(uint32_t n, const uint64_t *__restrict__ off,
                             const uint32_t *__restrict__ hp, const uint32_t *__restrict__ dd,
                             const uint32_t *__restrict__ pairs, uint64_t q,
                             uint32_t *__restrict__ out, int *bad) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t i = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < q; i += warps) {
        const uint32_t u = __ldg(&pairs[2 * i]), v = __ldg(&pairs[2 * i + 1]);
        if (u >= n || v >= n) {
            if (lane == 0) {
                out[i] = 0xFFFFFFFFu;
                atomicExch(bad, 1);
            }
            continue;
        }
        const uint32_t d = merge_query(off, hp, dd, u, v);
        if (lane == 0) out[i] = d;
    }
}

// The best common hub of u and v: the smallest (d(u,h) + d(v,h), hub position)
// packed as sum << 31 | position (all ones: no common hub). At equal sums the
// highest-ranked hub wins, the canonical hub of the pair (the max-rank vertex
// on its shortest paths). All 32 lanes call it; every lane gets the result.
__device__ __forceinline__ uint64_t merge_best(const uint64_t *__restrict__ off,
                                               const uint32_t *__restrict__ hp,
                                               const uint32_t *__restrict__ dd, uint32_t u, uint32_t v) {
    const int lane = threadIdx.x & 31;
    const uint64_t a0 = __ldg(&off[u]), la = __ldg(&off[u + 1]) - a0;
    const uint64_t b0 = __ldg(&off[v]), lb = __ldg(&off[v + 1]) - b0;
    uint64_t ia = 0, ib = 0;
    uint64_t best = ~0ull;
    while (ia < la && ib < lb) {
        const bool va = ia + lane < la, vb = ib + lane < lb;
        const uint32_t x = va ? __ldg(&hp[a0 + ia + lane]) : 0xFFFFFFFFu;
        const uint32_t y = vb ? __ldg(&hp[b0 + ib + lane]) : 0xFFFFFFFFu;
        int o = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int c = o + step;
            if (__shfl_sync(FULL, y, c) <= x) o = c;
        }
        const uint32_t yo = __shfl_sync(FULL, y, o);
        const bool hit = va && yo == x;
        if (__ballot_sync(FULL, hit) && hit) {
            const uint64_t sum = uint64_t(__ldg(&dd[a0 + ia + lane])) + __ldg(&dd[b0 + ib + o]);
            best = min64(best, (sum << 31) | x);
        }
        const uint32_t lastA = __shfl_sync(FULL, x, int(min64(la - ia, 32) - 1));
        const uint32_t lastB = __shfl_sync(FULL, y, int(min64(lb - ib, 32) - 1));
        if (lastA <= lastB) {
            ia += min64(la - ia, 32);
            ib += __popc(__ballot_sync(FULL, vb && y <= lastA));
        } else {
            ib += min64(lb - ib, 32);
            ia += __popc(__ballot_sync(FULL, va && x <= lastB));
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) best = min64(best, __shfl_xor_sync(FULL, best, o));
    return best;
}

// entry of hub position hpos in w's list (ascending hub positions), or ~0
__device__ __forceinline__ uint64_t find_hub(const uint64_t *__restrict__ off,
                                             const uint32_t *__restrict__ hp, uint32_t w,
                                             uint32_t hpos) {
    uint64_t lo = __ldg(&off[w]), hi = __ldg(&off[w + 1]);
    if (lo == hi) return ~0ull;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (__ldg(&hp[mid]) <= hpos) lo = mid; else hi = mid;
    }
    return __ldg(&hp[lo]) == hpos ? lo : ~0ull;
}

// Shortest paths by following the SPT parents stored with the labels (Sec. 5.4,
// Extensions): from u and from v towards their canonical hub H, each step the
// parent stored with w's label of H. One warp per pair (merge), lane 0 walks.
__global__ void paths_kernel(uint32_t n, const uint64_t *__restrict__ off,
                             const uint32_t *__restrict__ hp, const uint32_t *__restrict__ dd,
                             const uint32_t *__restrict__ hub, const uint32_t *__restrict__ par,
                             const uint32_t *__restrict__ pairs, uint64_t q, uint32_t max_len,
                             uint32_t *__restrict__ paths, uint32_t *__restrict__ lens, int *bad) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t i = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < q; i += warps) {
        const uint32_t u = __ldg(&pairs[2 * i]), v = __ldg(&pairs[2 * i + 1]);
        if (u >= n || v >= n) {
            if (lane == 0) {
                lens[i] = 0;
                atomicExch(bad, 1);
            }
            continue;
        }
        const uint64_t best = merge_best(off, hp, dd, u, v);
        if (lane != 0) continue;
        if (best == ~0ull) {  // different components
            lens[i] = 0;
            continue;
        }
        const uint32_t hpos = uint32_t(best & 0x7FFFFFFFu);
        uint32_t *out = paths + i * uint64_t(max_len);
        bool ok = true;
        // u side: u, parent, ..., H at positions 0 .. lu - 1
        uint32_t lu = 0, w = u;
        for (uint32_t guard = 0; guard <= n; ++guard) {
            if (lu < max_len) out[lu] = w;
            ++lu;
            const uint64_t j = find_hub(off, hp, w, hpos);
            if (j == ~0ull) { ok = false; break; }
            if (__ldg(&hub[j]) == w) break;
            w = __ldg(&par[j]);
        }
        // v side: count, then write v at the end back to the vertex after H
        uint32_t lv = 0;
        w = v;
        for (uint32_t guard = 0; ok && guard <= n; ++guard) {
            ++lv;
            const uint64_t j = find_hub(off, hp, w, hpos);
            if (j == ~0ull) { ok = false; break; }
            if (__ldg(&hub[j]) == w) break;
            w = __ldg(&par[j]);
        }
        if (!ok) {
            lens[i] = 0;
            atomicExch(bad, 2);
            continue;
        }
        const uint32_t total = lu + lv - 1;
        w = v;
        for (uint32_t pos = total - 1; pos >= lu; --pos) {
            if (pos < max_len) out[pos] = w;
            w = __ldg(&par[find_hub(off, hp, w, hpos)]);
        }
        lens[i] = total;
    }
}

// d(u, v) over a label set: its own lists, or, for a set held as hub
// partitions (QFDL-style, Sec. 6: every partition holds the labels of a
// disjoint hub range for all vertices), the minimum of the partial merges
__device__ __forceinline__ uint32_t set_query(const QuerySet &S, uint32_t u, uint32_t v) {
    if (!S.nparts) return merge_query(S.offsets, S.hubpos, S.dist, u, v);
    uint32_t d = 0xFFFFFFFFu;
    for (uint32_t k = 0; k < S.nparts; ++k) {
        const QuerySet P = S.parts[k];
        const uint32_t x = merge_query(P.offsets, P.hubpos, P.dist, u, v);
        d = x < d ? x : d;
    }
    return d;
}

// a batch mixing label sets: pair i asks set set_of[i]
// (the set count is read from device memory, so a captured launch stays valid
// as sets are added; set id 0xFFFF marks padding that is skipped). With perm,
// the j-th pair answered is perm[j] (grouped order); its answer still goes to
// out[perm[j]].
__global__ void query_sets_kernel(const QuerySet *__restrict__ sets, const uint32_t *nsets_p,
                                  const uint32_t *__restrict__ pairs,
                                  const uint16_t *__restrict__ set_of, const uint32_t *__restrict__ perm,
                                  uint64_t q, uint32_t *__restrict__ out, int *bad) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint32_t nsets = *nsets_p;
    for (uint64_t j = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; j < q; j += warps) {
        const uint64_t i = perm ? __ldg(&perm[j]) : j;
        const uint32_t k = set_of ? __ldg(&set_of[i]) : 0u;
        if (k == 0xFFFFu) continue;
        const uint32_t u = __ldg(&pairs[2 * i]), v = __ldg(&pairs[2 * i + 1]);
        const QuerySet S = sets[k < nsets ? k : 0];
        if (k >= nsets || u >= S.n || v >= S.n) {
            if (lane == 0) {
                out[i] = 0xFFFFFFFFu;
                atomicExch(bad, 1);
            }
            continue;
        }
        const uint32_t d = set_query(S, u, v);
        if (lane == 0) out[i] = d;
    }
}

// ---- grouped order (QDOL-style, Sec. 6: queries sorted and grouped by the
// vertex partitions they touch, answers rearranged back into arrival order).
// On one GPU a partition is a block of vertex ids: a pair's key is the block
// pair (min(u, v), max(u, v)) over GROUP_BLOCKS blocks per label set, so pairs
// that read the lists of the same two blocks run together. The order is a
// counting sort by key: count, one-CTA exclusive scan, scatter of indices.
// Pairs of an unknown set or with an id >= n go to key 0 (the query kernel
// reports them).
constexpr uint32_t GROUP_BLOCKS = 64;
constexpr uint32_t GROUP_KEYS = GROUP_BLOCKS * GROUP_BLOCKS;

__device__ __forceinline__ uint32_t group_key(const QuerySet *sets, uint32_t nsets, const uint32_t *pairs,
                                              const uint16_t *set_of, uint64_t i) {
    const uint32_t k = set_of ? __ldg(&set_of[i]) : 0;
    if (k >= nsets) return 0;
    const uint32_t n = sets[k].n;
    uint32_t u = __ldg(&pairs[2 * i]), v = __ldg(&pairs[2 * i + 1]);
    if (u >= n || v >= n) return 0;
    if (u > v) {
        const uint32_t t = u;
        u = v;
        v = t;
    }
    const uint32_t bu = uint32_t(uint64_t(u) * GROUP_BLOCKS / n), bv = uint32_t(uint64_t(v) * GROUP_BLOCKS / n);
    return bu * GROUP_BLOCKS + bv;
}

__global__ void group_count_kernel(const QuerySet *sets, const uint32_t *nsets_p, const uint32_t *pairs,
                                   const uint16_t *set_of, uint64_t q, uint32_t *cnt) {
    const uint32_t nsets = *nsets_p;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < q;
         i += uint64_t(gridDim.x) * blockDim.x)
        atomicAdd(&cnt[group_key(sets, nsets, pairs, set_of, i)], 1u);
}

// exclusive prefix of the GROUP_KEYS counts, in place (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024) group_scan_kernel(uint32_t *cnt) {
    constexpr uint32_t PER = GROUP_KEYS / 1024;
    __shared__ uint32_t wsum[32];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t x[PER], s = 0;
#pragma unroll
    for (uint32_t k = 0; k < PER; ++k) {
        x[k] = cnt[t * PER + k];
        s += x[k];
    }
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= uint32_t(o)) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, wi, o);
            if (lane >= uint32_t(o)) wi += y;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + inc - s;
#pragma unroll
    for (uint32_t k = 0; k < PER; ++k) {
        cnt[t * PER + k] = run;
        run += x[k];
    }
}

__global__ void group_scatter_kernel(const QuerySet *sets, const uint32_t *nsets_p, const uint32_t *pairs,
                                     const uint16_t *set_of, uint64_t q, uint32_t *fill, uint32_t *perm) {
    const uint32_t nsets = *nsets_p;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < q;
         i += uint64_t(gridDim.x) * blockDim.x)
        perm[atomicAdd(&fill[group_key(sets, nsets, pairs, set_of, i)], 1u)] = uint32_t(i);
}

}  // namespace

cudaError_t launch_group_order(const QuerySet *sets, const uint32_t *nsets, const uint32_t *pairs,
                               const uint16_t *set_of, uint64_t q, uint32_t *scratch, uint32_t *perm,
                               cudaStream_t s) {
    if (q == 0) return cudaSuccess;
    if (q > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(scratch, 0, GROUP_KEYS * sizeof(uint32_t), s);
    if (e) return e;
    uint64_t blocks = (q + 255) / 256;
    if (blocks > uint64_t(device_sms()) * 8) blocks = uint64_t(device_sms()) * 8;
    group_count_kernel<<<unsigned(blocks), 256, 0, s>>>(sets, nsets, pairs, set_of, q, scratch);
    group_scan_kernel<<<1, 1024, 0, s>>>(scratch);
    group_scatter_kernel<<<unsigned(blocks), 256, 0, s>>>(sets, nsets, pairs, set_of, q, scratch, perm);
    return cudaGetLastError();
}

cudaError_t launch_query_sets(const QuerySet *sets, const uint32_t *nsets, const uint32_t *pairs,
                              const uint16_t *set_of, const uint32_t *perm, uint64_t q, uint32_t *out,
                              int *bad, int max_blocks, cudaStream_t s) {
    if (q == 0) return cudaSuccess;
    uint64_t blocks = (q * 32 + 255) / 256;
    if (blocks > uint64_t(max_blocks)) blocks = uint64_t(max_blocks);
    query_sets_kernel<<<unsigned(blocks), 256, 0, s>>>(sets, nsets, pairs, set_of, perm, q, out, bad);
    return cudaGetLastError();
}

cudaError_t launch_paths(uint32_t n, const uint64_t *offsets, const uint32_t *hubpos,
                         const uint32_t *dist, const uint32_t *hub, const uint32_t *parent,
                         const uint32_t *pairs, uint64_t q, uint32_t max_len, uint32_t *paths,
                         uint32_t *lens, int *bad, cudaStream_t s) {
    if (q == 0) return cudaSuccess;
    uint64_t blocks = (q * 32 + 255) / 256;
    if (blocks > uint64_t(device_sms()) * 64) blocks = uint64_t(device_sms()) * 64;
    paths_kernel<<<unsigned(blocks), 256, 0, s>>>(n, offsets, hubpos, dist, hub, parent, pairs, q,
                                                   max_len, paths, lens, bad);
    return cudaGetLastError();
}

cudaError_t launch_query(uint32_t n, const uint64_t *offsets, const uint32_t *hubpos,
                         const uint32_t *dist, const uint32_t *pairs, uint64_t q, uint32_t *out,
                         int *bad, cudaStream_t s) {
    if (q == 0) return cudaSuccess;
    uint64_t blocks = (q * 32 + 255) / 256;
    if (blocks > uint64_t(device_sms()) * 64) blocks = uint64_t(device_sms()) * 64;
    query_kernel<<<unsigned(blocks), 256, 0, s>>>(n, offsets, hubpos, dist, pairs, q, out, bad);
    return cudaGetLastError();
}

}  // namespace chl
