// Input validation and renumbering of the graph by rank position.
//
// The paper's input is an undirected graph with positive edge weights
// (Sec. 2) and a total order R (Sec. 1). chl_build checks the CSR on the GPU
// (row bounds, ids, weights >= 1, sorted rows without duplicates or
// self-loops, an equal-weight reverse for every arc) and that R is a
// permutation, then renumbers vertices by rank position p = n-1-R(v): the
// vertex with the highest rank becomes 0. In that numbering the ancestor with
// the highest rank is the smallest id, so "highest-ranked ancestor" in
// Algorithm 3 becomes an unsigned min inside the packed search key, and the
// trees of the most important roots (the largest ones, Sec. 5.1 label counts
// per tree) come first in the claim order.
#include <cstdio>

#include "chl_common.cuh"

namespace chl {

// ------------------------------------------------------------------ scan
namespace {

constexpr int SCAN_TPB = 1024;

__global__ void scan_blocks_kernel(const uint64_t *in, uint64_t *out, uint64_t *block_sums,
                                   uint64_t n) {
    __shared__ uint64_t warp_tot[32];
    const uint64_t i = uint64_t(blockIdx.x) * SCAN_TPB + threadIdx.x;
    const uint64_t x = i < n ? in[i] : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t t = warp_tot[lane];
        uint64_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        warp_tot[lane] = s - t;  // exclusive prefix of warp totals
        if (lane == 31 && block_sums) block_sums[blockIdx.x] = s;
    }
    __syncthreads();
    if (i < n) out[i] = incl - x + warp_tot[warp];
}

__global__ void scan_add_kernel(uint64_t *out, const uint64_t *block_prefix, uint64_t n) {
    const uint64_t i = uint64_t(blockIdx.x) * SCAN_TPB + threadIdx.x;
    if (i < n) out[i] += block_prefix[blockIdx.x];
}

}  // namespace

// exclusive scan of n uint64 values; out may alias in
cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                               int *launches) {
    if (n == 0) return cudaSuccess;
    const uint64_t nb = (n + SCAN_TPB - 1) / SCAN_TPB;
    if (nb == 1) {
        scan_blocks_kernel<<<1, SCAN_TPB, 0, s>>>(in, out, nullptr, n);
        if (launches) *launches += 1;
        return cudaGetLastError();
    }
    uint64_t *sums = nullptr;
    cudaError_t e = dmalloc(&sums, nb * sizeof(uint64_t), s);
    if (e != cudaSuccess) return e;
    scan_blocks_kernel<<<unsigned(nb), SCAN_TPB, 0, s>>>(in, out, sums, n);
    if (launches) *launches += 1;
    e = exclusive_scan_u64(sums, sums, nb, s, launches);
    if (e == cudaSuccess) {
        scan_add_kernel<<<unsigned(nb), SCAN_TPB, 0, s>>>(out, sums, n);
        if (launches) *launches += 1;
        e = cudaGetLastError();
    }
    cudaFreeAsync(sums, s);
    return e;
}

// ------------------------------------------------------------------ validation
namespace {

enum : uint32_t {
    BAD_ROWPTR = 1u << 0,
    BAD_COL = 1u << 1,
    BAD_WEIGHT = 1u << 2,
    BAD_ORDER = 1u << 3,
    BAD_SELF = 1u << 4,
    BAD_SYMM = 1u << 5,
    BAD_RANK = 1u << 6,
};

struct Check {
    uint32_t bits;
    uint32_t where;  // a vertex where the first failure was seen (any)
    unsigned long long fp;  // symmetry fingerprint: sum of h(v, u, w) - h(u, v, w) over the arcs
};

__device__ void fail(Check *c, uint32_t bit, uint32_t v) {
    if (!(atomicOr(&c->bits, bit) & bit)) atomicExch(&c->where, v);
}

__global__ void check_rows_kernel(uint32_t n, uint64_t m2, const uint64_t *row, Check *c) {
    for (uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t a = row[v], b = row[v + 1];
        if (a > b || b > m2 || (v == 0 && a != 0) || (v == n - 1 && b != m2)) fail(c, BAD_ROWPTR, uint32_t(v));
    }
}

// 64-bit mix of an arc (the splitmix64 finaliser of Steele, Lea and Flood)
__device__ __forceinline__ unsigned long long arc_hash(uint32_t a, uint32_t b, uint32_t wt) {
    unsigned long long x = ((unsigned long long)a << 32 | b) ^ ((unsigned long long)wt * 0x9E3779B97F4A7C15ull);
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// One warp per vertex: ids, weights, strictly increasing rows, no self-loop,
// in one streaming pass. Symmetry by fingerprint: the arcs (v, u, w) form
// the same multiset as their reverses (u, v, w) iff the graph is undirected
// with equal weights both ways, so the sum of h(v, u, w) - h(u, v, w) is 0
// for every undirected graph; any other sum proves an arc without its
// reverse, which check_symm_kernel then locates.
__global__ void check_arcs_kernel(uint32_t n, const uint64_t *row, const uint32_t *col,
                                  const uint32_t *w, Check *c) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    unsigned long long fp = 0;
    for (uint64_t v = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint64_t a = row[v], b = row[v + 1];
        for (uint64_t e = a + lane; e < b; e += 32) {
            const uint32_t u = col[e], wt = w[e];
            if (u >= n) { fail(c, BAD_COL, uint32_t(v)); continue; }
            if (wt == 0) fail(c, BAD_WEIGHT, uint32_t(v));
            if (u == v) fail(c, BAD_SELF, uint32_t(v));
            if (e > a && col[e - 1] >= u) fail(c, BAD_ORDER, uint32_t(v));
            fp += arc_hash(uint32_t(v), u, wt) - arc_hash(u, uint32_t(v), wt);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) fp += __shfl_xor_sync(0xffffffffu, fp, o);
    if (lane == 0 && fp) atomicAdd(&c->fp, fp);
}

// exact symmetry check, run only when the fingerprint is not 0: the reverse
// arc with the same weight by binary search in the target row
__global__ void check_symm_kernel(uint32_t n, const uint64_t *row, const uint32_t *col,
                                  const uint32_t *w, Check *c) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t v = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint64_t a = row[v], b = row[v + 1];
        for (uint64_t e = a + lane; e < b; e += 32) {
            const uint32_t u = col[e], wt = w[e];
            if (u >= n) continue;
            uint64_t lo = row[u], hi = row[u + 1];
            bool found = false;
            while (lo < hi) {
                const uint64_t mid = lo + (hi - lo) / 2;
                const uint32_t x = col[mid];
                if (x == v) { found = (w[mid] == wt); break; }
                if (x < v) lo = mid + 1; else hi = mid;
            }
            if (!found) fail(c, BAD_SYMM, uint32_t(v));
        }
    }
}

__global__ void rank_count_kernel(uint32_t n, const uint32_t *rank, uint32_t *cnt, Check *c) {
    for (uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t r = rank[v];
        if (r >= n) fail(c, BAD_RANK, uint32_t(v));
        else atomicAdd(&cnt[r], 1u);
    }
}

__global__ void rank_perm_kernel(uint32_t n, const uint32_t *rank, const uint32_t *cnt,
                                 uint32_t *pos_of, uint32_t *vert_at, Check *c) {
    for (uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += uint64_t(gridDim.x) * blockDim.x) {
        if (cnt[v] != 1) fail(c, BAD_RANK, uint32_t(v));
        const uint32_t r = rank[v];
        if (r < n) {
            const uint32_t p = n - 1 - r;
            pos_of[v] = p;
            vert_at[p] = uint32_t(v);
        }
    }
}

// degrees in rank order, and weight statistics
__global__ void rank_degree_kernel(uint32_t n, const uint64_t *row, const uint32_t *vert_at,
                                   uint64_t *deg) {
    for (uint64_t p = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
         p += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = vert_at[p];
        deg[p] = row[v + 1] - row[v];
    }
}

struct WStats {
    uint32_t wmax, wmin;
    unsigned long long wsum;
};

// one warp per vertex: copy its row with neighbours renumbered
__global__ void rank_arcs_kernel(uint32_t n, const uint64_t *row, const uint32_t *col,
                                 const uint32_t *w, const uint32_t *vert_at,
                                 const uint32_t *pos_of, const uint64_t *nrow, uint2 *arc,
                                 WStats *ws) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    uint32_t wmax = 0, wmin = 0xFFFFFFFFu;
    unsigned long long wsum = 0;
    for (uint64_t p = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
        const uint32_t v = vert_at[p];
        const uint64_t a = row[v], b = row[v + 1], o = nrow[p];
        for (uint64_t e = a + lane; e < b; e += 32) {
            const uint32_t wt = w[e];
            arc[o + (e - a)] = make_uint2(pos_of[col[e]], wt);
            wmax = max(wmax, wt);
            wmin = min(wmin, wt);
            wsum += wt;
        }
    }
    for (int o = 16; o; o >>= 1) {
        wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        wmin = min(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
        wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    }
    if (lane == 0) {
        atomicMax(&ws->wmax, wmax);
        atomicMin(&ws->wmin, wmin);
        atomicAdd(&ws->wsum, wsum);
    }
}

int grid_for(uint64_t work, int tpb) {
    uint64_t b = (work + tpb - 1) / tpb;
    if (b > uint64_t(device_sms()) * 32) b = uint64_t(device_sms()) * 32;
    if (b < 1) b = 1;
    return int(b);
}

}  // namespace

#define CK(x)                                                                   \
    do {                                                                        \
        cudaError_t e__ = (x);                                                  \
        if (e__ != cudaSuccess) {                                               \
            st = cuda_status(e__, #x);                                          \
            goto done;                                                          \
        }                                                                       \
    } while (0)

chl_status prepare_graph(uint32_t n, uint64_t m2, const uint64_t *row, const uint32_t *col,
                         const uint32_t *w, const uint32_t *rank, RankGraph &g, cudaStream_t s,
                         int *launches) {
    chl_status st = CHL_OK;
    Check *chk = nullptr;
    Check hchk{0, 0, 0};
    uint32_t *cnt = nullptr;
    uint64_t *deg = nullptr;
    WStats *ws = nullptr;
    WStats hws{0, 0xFFFFFFFFu, 0};
    g = RankGraph{};
    g.n = n;
    g.m2 = m2;
    CK(dmalloc(&chk, sizeof(Check), s));
    CK(cudaMemsetAsync(chk, 0, sizeof(Check), s));
    CK(dmalloc(&cnt, size_t(n) * sizeof(uint32_t), s));
    CK(cudaMemsetAsync(cnt, 0, size_t(n) * sizeof(uint32_t), s));
    CK(dmalloc(&g.pos_of, size_t(n) * sizeof(uint32_t), s));
    CK(dmalloc(&g.vert_at, size_t(n) * sizeof(uint32_t), s));
    check_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, m2, row, chk);
    rank_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, rank, cnt, chk);
    rank_perm_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, rank, cnt, g.pos_of, g.vert_at, chk);
    *launches += 3;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&hchk, chk, sizeof(Check), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hchk.bits & BAD_ROWPTR) {
        st = set_error(CHL_EINVAL, "row_ptr is not a valid CSR offset array (vertex %u)", hchk.where);
        goto done;
    }
    if (hchk.bits & BAD_RANK) {
        st = set_error(CHL_EINVAL, "rank is not a permutation of [0,n) (vertex %u)", hchk.where);
        goto done;
    }
    check_arcs_kernel<<<grid_for(uint64_t(n) * 32, 256), 256, 0, s>>>(n, row, col, w, chk);
    *launches += 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&hchk, chk, sizeof(Check), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!(hchk.bits & BAD_COL) && hchk.fp) {
        // some arc has no reverse of equal weight: find a vertex that shows it
        check_symm_kernel<<<grid_for(uint64_t(n) * 32, 256), 256, 0, s>>>(n, row, col, w, chk);
        *launches += 1;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&hchk, chk, sizeof(Check), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!hchk.bits) hchk.bits = BAD_SYMM;  // (a non-zero sum always has a cause)
    }
    if (hchk.bits) {
        const char *what = (hchk.bits & BAD_COL)      ? "a neighbour id is >= n"
                           : (hchk.bits & BAD_WEIGHT) ? "a weight is 0 (weights must be positive)"
                           : (hchk.bits & BAD_SELF)   ? "a self-loop is present"
                           : (hchk.bits & BAD_ORDER)  ? "a row is not strictly increasing (unsorted or duplicate arcs)"
                                                      : "an arc has no reverse arc of equal weight (graph must be undirected)";
        st = set_error(CHL_EINVAL, "invalid graph: %s (vertex %u)", what, hchk.where);
        goto done;
    }
    // renumber by rank position
    CK(dmalloc(&deg, (size_t(n) + 1) * sizeof(uint64_t), s));
    CK(dmalloc(&g.row, (size_t(n) + 1) * sizeof(uint64_t), s));
    CK(dmalloc(&g.arc, (m2 ? m2 : 1) * sizeof(uint2), s));
    CK(dmalloc(&ws, sizeof(WStats), s));
    CK(cudaMemcpyAsync(ws, &hws, sizeof(WStats), cudaMemcpyHostToDevice, s));
    rank_degree_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, row, g.vert_at, deg);
    *launches += 1;
    CK(cudaMemsetAsync(deg + n, 0, sizeof(uint64_t), s));
    CK(exclusive_scan_u64(deg, g.row, uint64_t(n) + 1, s, launches));
    rank_arcs_kernel<<<grid_for(uint64_t(n) * 32, 256), 256, 0, s>>>(n, row, col, w, g.vert_at,
                                                                     g.pos_of, g.row, g.arc, ws);
    *launches += 1;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&hws, ws, sizeof(WStats), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    g.w_max = m2 ? hws.wmax : 1;
    g.w_min = m2 ? hws.wmin : 1;
    g.w_mean = m2 ? double(hws.wsum) / double(m2) : 1.0;
done:
    if (chk) cudaFreeAsync(chk, s);
    if (cnt) cudaFreeAsync(cnt, s);
    if (deg) cudaFreeAsync(deg, s);
    if (ws) cudaFreeAsync(ws, s);
    if (st != CHL_OK) free_graph(g, s);
    return st;
}

void free_graph(RankGraph &g, cudaStream_t s) {
    if (g.row) cudaFreeAsync(g.row, s);
    if (g.arc) cudaFreeAsync(g.arc, s);
    if (g.vert_at) cudaFreeAsync(g.vert_at, s);
    if (g.pos_of) cudaFreeAsync(g.pos_of, s);
    g.row = nullptr;
    g.arc = nullptr;
    g.vert_at = nullptr;
    g.pos_of = nullptr;
}

}  // namespace chl
