// Label assembly: from the (vertex, hub, dist) records the trees emit, in
// whatever order the trees finished, to per-vertex lists sorted by hub rank
// (Algorithm 2, "sort labels in L_v using hub rank"; the lists are stored
// per vertex only, as in the footnote of Sec. 7.2).
//
//   1. count labels per vertex (atomic histogram)
//   2. exclusive scan -> offsets
//   3. scatter (hubpos << 32 | dist) into each vertex's segment
//   4. sort every segment by hubpos (= descending R of the hub) in shared
//      memory: one warp per segment up to 32 labels, one CTA per segment up
//      to MAX_SEGMENT labels (bitonic networks)
//   5. split into hub (caller id), hubpos and dist arrays
#include "chl_common.cuh"

namespace chl {

cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                               int *launches);

namespace {

constexpr uint32_t MAX_SEGMENT = 16384;

__global__ void count_kernel(uint64_t T, const uint32_t *v, uint64_t *cnt) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < T;
         i += uint64_t(gridDim.x) * blockDim.x)
        atomicAdd((unsigned long long *)&cnt[v[i]], 1ull);
}

// unsorted table by rank position: (hubpos, dist) straight into each
// vertex's segment; records of hubs below min_hub are left out (the dense
// Common Label Table answers for those hubs)
__global__ void count_table_kernel(uint64_t T, const uint32_t *v, const uint32_t *h,
                                   const uint32_t *pos_of, uint32_t min_hub, uint64_t *cnt) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < T;
         i += uint64_t(gridDim.x) * blockDim.x)
        if (h[i] >= min_hub) atomicAdd((unsigned long long *)&cnt[pos_of[v[i]]], 1ull);
}

__global__ void scatter_table_kernel(uint64_t T, const uint32_t *v, const uint32_t *h,
                                     const uint32_t *d, const uint32_t *pos_of, uint32_t min_hub,
                                     const uint64_t *off, uint64_t *fill, uint2 *e) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < T;
         i += uint64_t(gridDim.x) * blockDim.x) {
        if (h[i] < min_hub) continue;
        const uint32_t x = pos_of[v[i]];
        const uint64_t k = off[x] + atomicAdd((unsigned long long *)&fill[x], 1ull);
        e[k] = make_uint2(h[i], d[i]);
    }
}

// entries per vertex of the grown table: its old entries plus the new ones
__global__ void grown_count_kernel(uint32_t n, const uint64_t *old_off, uint64_t *cnt) {
    for (uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += uint64_t(gridDim.x) * blockDim.x)
        cnt[v] += old_off[v + 1] - old_off[v];
}

// one warp per vertex: its old entries to the front of its new segment
__global__ void copy_segments_kernel(uint32_t n, const uint64_t *old_off, const uint2 *old_e,
                                     const uint64_t *new_off, uint2 *e) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t v = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint64_t a = old_off[v], len = old_off[v + 1] - a, o = new_off[v];
        for (uint64_t i = lane; i < len; i += 32) e[o + i] = old_e[a + i];
    }
}

// new records after each vertex's old entries
__global__ void scatter_new_kernel(uint64_t T0, uint64_t T, const uint32_t *v, const uint32_t *h,
                                   const uint32_t *d, const uint32_t *pos_of, uint32_t min_hub,
                                   const uint64_t *old_off, const uint64_t *off, uint64_t *fill,
                                   uint2 *e) {
    for (uint64_t i = T0 + uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < T;
         i += uint64_t(gridDim.x) * blockDim.x) {
        if (h[i] < min_hub) continue;
        const uint32_t x = pos_of[v[i]];
        const uint64_t k = off[x] + (old_off[x + 1] - old_off[x]) +
                           atomicAdd((unsigned long long *)&fill[x], 1ull);
        e[k] = make_uint2(h[i], d[i]);
    }
}

__global__ void scatter_kernel(uint64_t T, const uint32_t *v, const uint32_t *h, const uint32_t *d,
                               const uint64_t *off, uint64_t *fill, uint64_t *tmp) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < T;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t x = v[i];
        const uint64_t k = off[x] + atomicAdd((unsigned long long *)&fill[x], 1ull);
        tmp[k] = (uint64_t(h[i]) << 32) | d[i];
    }
}

// classify segments by length into three work lists; record the longest
__global__ void classify_kernel(uint32_t n, const uint64_t *off, uint32_t *small_list,
                                uint32_t *mid_list, uint32_t *big_list, uint32_t *counts,
                                unsigned long long *max_len) {
    for (uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t len = off[v + 1] - off[v];
        if (len <= 1) continue;
        atomicMax(max_len, (unsigned long long)len);
        if (len <= 32) small_list[atomicAdd(&counts[0], 1u)] = uint32_t(v);
        else if (len <= 1024) mid_list[atomicAdd(&counts[1], 1u)] = uint32_t(v);
        else if (len <= MAX_SEGMENT) big_list[atomicAdd(&counts[2], 1u)] = uint32_t(v);
    }
}

// one warp per segment of <= 32 keys: bitonic network in registers
__global__ void sort_small_kernel(const uint32_t *list, const uint32_t *count, const uint64_t *off,
                                  uint64_t *tmp) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < *count; w += warps) {
        const uint32_t v = list[w];
        const uint64_t a = off[v], len = off[v + 1] - a;
        uint64_t x = lane < len ? tmp[a + lane] : ~0ull;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint64_t y = __shfl_xor_sync(0xffffffffu, x, j);
                const bool up = ((lane & k) == 0);
                const bool lower = ((lane & j) == 0);
                // keep min in the lower lane of an ascending pair
                x = (lower == up) ? min(x, y) : max(x, y);
            }
        }
        if (lane < len) tmp[a + lane] = x;
    }
}

// one CTA per segment: bitonic sort in shared memory (size rounded up to a power of two)
template <int TPB>
__global__ void sort_block_kernel(const uint32_t *list, const uint32_t *count, const uint64_t *off,
                                  uint64_t *tmp) {
    extern __shared__ uint64_t sm[];
    for (uint32_t s = blockIdx.x; s < *count; s += gridDim.x) {
        const uint32_t v = list[s];
        const uint64_t a = off[v];
        const uint32_t len = uint32_t(off[v + 1] - a);
        uint32_t P = 1;
        while (P < len) P <<= 1;
        for (uint32_t i = threadIdx.x; i < P; i += TPB) sm[i] = i < len ? tmp[a + i] : ~0ull;
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = threadIdx.x; i < P; i += TPB) {
                    const uint32_t ix = i ^ j;
                    if (ix > i) {
                        const uint64_t x = sm[i], y = sm[ix];
                        const bool up = ((i & k) == 0);
                        if ((x > y) == up) {
                            sm[i] = y;
                            sm[ix] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = threadIdx.x; i < len; i += TPB) tmp[a + i] = sm[i];
        __syncthreads();
    }
}

__global__ void split_kernel(uint64_t T, const uint64_t *tmp, const uint32_t *vert_at,
                             uint32_t *hub, uint32_t *hubpos, uint32_t *dist) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < T;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t k = tmp[i];
        const uint32_t hp = uint32_t(k >> 32);
        hubpos[i] = hp;
        dist[i] = uint32_t(k);
        hub[i] = vert_at[hp];
    }
}

int grid_for(uint64_t work, int tpb) {
    uint64_t b = (work + tpb - 1) / tpb;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return int(b);
}

}  // namespace

#define CKE(x)                                   \
    do {                                         \
        e = (x);                                 \
        if (e != cudaSuccess) goto done;         \
    } while (0)

cudaError_t assemble_labels(uint32_t n, uint64_t T, const uint32_t *in_v, const uint32_t *in_h,
                            const uint32_t *in_d, const uint32_t *vert_at, LabelCSR &out,
                            int *too_long, cudaStream_t s, int *launches) {
    cudaError_t e = cudaSuccess;
    uint64_t *cnt = nullptr, *tmp = nullptr;
    uint32_t *lists = nullptr, *counts = nullptr;
    unsigned long long *maxlen = nullptr;
    unsigned long long hmax = 0;
    *too_long = 0;
    out = LabelCSR{};
    const size_t Tb = (T ? T : 1);
    CKE(cudaMallocAsync(&out.offsets, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(cudaMallocAsync(&out.hub, Tb * sizeof(uint32_t), s));
    CKE(cudaMallocAsync(&out.hubpos, Tb * sizeof(uint32_t), s));
    CKE(cudaMallocAsync(&out.dist, Tb * sizeof(uint32_t), s));
    CKE(cudaMallocAsync(&cnt, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(cudaMallocAsync(&tmp, Tb * sizeof(uint64_t), s));
    CKE(cudaMallocAsync(&lists, 3 * size_t(n) * sizeof(uint32_t), s));
    CKE(cudaMallocAsync(&counts, 4 * sizeof(uint32_t), s));
    CKE(cudaMallocAsync(&maxlen, sizeof(unsigned long long), s));
    CKE(cudaMemsetAsync(cnt, 0, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(cudaMemsetAsync(counts, 0, 4 * sizeof(uint32_t), s));
    CKE(cudaMemsetAsync(maxlen, 0, sizeof(unsigned long long), s));
    count_kernel<<<grid_for(T, 256), 256, 0, s>>>(T, in_v, cnt);
    *launches += 1;
    CKE(cudaGetLastError());
    CKE(exclusive_scan_u64(cnt, out.offsets, uint64_t(n) + 1, s, launches));
    CKE(cudaMemsetAsync(cnt, 0, (size_t(n) + 1) * sizeof(uint64_t), s));
    scatter_kernel<<<grid_for(T, 256), 256, 0, s>>>(T, in_v, in_h, in_d, out.offsets, cnt, tmp);
    classify_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, out.offsets, lists, lists + n,
                                                     lists + 2 * size_t(n), counts, maxlen);
    *launches += 2;
    CKE(cudaGetLastError());
    CKE(cudaMemcpyAsync(&hmax, maxlen, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    CKE(cudaStreamSynchronize(s));
    if (hmax > MAX_SEGMENT) {
        *too_long = 1;
        goto done;
    }
    sort_small_kernel<<<152 * 8, 256, 0, s>>>(lists, counts, out.offsets, tmp);
    sort_block_kernel<256><<<152 * 8, 256, 1024 * sizeof(uint64_t), s>>>(lists + n, counts + 1,
                                                                         out.offsets, tmp);
    *launches += 2;
    if (hmax > 1024) {
        static bool attr_set = false;
        if (!attr_set) {
            CKE(cudaFuncSetAttribute(sort_block_kernel<1024>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(MAX_SEGMENT * sizeof(uint64_t))));
            attr_set = true;
        }
        sort_block_kernel<1024><<<152, 1024, MAX_SEGMENT * sizeof(uint64_t), s>>>(
            lists + 2 * size_t(n), counts + 2, out.offsets, tmp);
        *launches += 1;
    }
    split_kernel<<<grid_for(T, 256), 256, 0, s>>>(T, tmp, vert_at, out.hub, out.hubpos, out.dist);
    *launches += 1;
    CKE(cudaGetLastError());
done:
    if (cnt) cudaFreeAsync(cnt, s);
    if (tmp) cudaFreeAsync(tmp, s);
    if (lists) cudaFreeAsync(lists, s);
    if (counts) cudaFreeAsync(counts, s);
    if (maxlen) cudaFreeAsync(maxlen, s);
    if (e != cudaSuccess || *too_long) {
        if (out.offsets) cudaFreeAsync(out.offsets, s);
        if (out.hub) cudaFreeAsync(out.hub, s);
        if (out.hubpos) cudaFreeAsync(out.hubpos, s);
        if (out.dist) cudaFreeAsync(out.dist, s);
        out = LabelCSR{};
    }
    return e;
}

// Entries are allocated with two spare ones past the last, so that a read
// widened to 16-byte boundaries (two entries) stays inside the array.
cudaError_t assemble_table(uint32_t n, uint64_t T, const uint32_t *in_v, const uint32_t *in_h,
                           const uint32_t *in_d, const uint32_t *pos_of, uint32_t min_hub,
                           LabelTable &out, cudaStream_t s, int *launches) {
    cudaError_t e = cudaSuccess;
    uint64_t *cnt = nullptr;
    out = LabelTable{};
    CKE(cudaMallocAsync(&out.offsets, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(cudaMallocAsync(&out.e, (size_t(T) + 2) * sizeof(uint2), s));
    CKE(cudaMemsetAsync(out.e, 0xFF, (size_t(T) + 2) * sizeof(uint2), s));
    CKE(cudaMallocAsync(&cnt, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(cudaMemsetAsync(cnt, 0, (size_t(n) + 1) * sizeof(uint64_t), s));
    count_table_kernel<<<grid_for(T, 256), 256, 0, s>>>(T, in_v, in_h, pos_of, min_hub, cnt);
    *launches += 1;
    CKE(cudaGetLastError());
    CKE(exclusive_scan_u64(cnt, out.offsets, uint64_t(n) + 1, s, launches));
    CKE(cudaMemsetAsync(cnt, 0, (size_t(n) + 1) * sizeof(uint64_t), s));
    scatter_table_kernel<<<grid_for(T, 256), 256, 0, s>>>(T, in_v, in_h, in_d, pos_of, min_hub,
                                                          out.offsets, cnt, out.e);
    *launches += 1;
    CKE(cudaGetLastError());
done:
    if (cnt) cudaFreeAsync(cnt, s);
    if (e != cudaSuccess) {
        if (out.offsets) cudaFreeAsync(out.offsets, s);
        if (out.e) cudaFreeAsync(out.e, s);
        out = LabelTable{};
    }
    return e;
}

cudaError_t grow_table(uint32_t n, LabelTable &lt, uint64_t T0, uint64_t T, const uint32_t *in_v,
                       const uint32_t *in_h, const uint32_t *in_d, const uint32_t *pos_of,
                       uint32_t min_hub, cudaStream_t s, int *launches) {
    cudaError_t e = cudaSuccess;
    uint64_t *cnt = nullptr;
    LabelTable out;
    const uint64_t dT = T - T0;
    CKE(cudaMallocAsync(&out.offsets, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(cudaMallocAsync(&out.e, (size_t(T) + 2) * sizeof(uint2), s));
    CKE(cudaMemsetAsync(out.e, 0xFF, (size_t(T) + 2) * sizeof(uint2), s));
    CKE(cudaMallocAsync(&cnt, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(cudaMemsetAsync(cnt, 0, (size_t(n) + 1) * sizeof(uint64_t), s));
    if (dT) {
        count_table_kernel<<<grid_for(dT, 256), 256, 0, s>>>(dT, in_v + T0, in_h + T0, pos_of, min_hub,
                                                             cnt);
        *launches += 1;
    }
    grown_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, lt.offsets, cnt);
    *launches += 1;
    CKE(cudaGetLastError());
    CKE(exclusive_scan_u64(cnt, out.offsets, uint64_t(n) + 1, s, launches));
    copy_segments_kernel<<<grid_for(uint64_t(n) * 32, 256), 256, 0, s>>>(n, lt.offsets, lt.e,
                                                                         out.offsets, out.e);
    *launches += 1;
    CKE(cudaGetLastError());
    if (dT) {
        CKE(cudaMemsetAsync(cnt, 0, (size_t(n) + 1) * sizeof(uint64_t), s));
        scatter_new_kernel<<<grid_for(dT, 256), 256, 0, s>>>(T0, T, in_v, in_h, in_d, pos_of, min_hub,
                                                             lt.offsets, out.offsets, cnt, out.e);
        *launches += 1;
        CKE(cudaGetLastError());
    }
done:
    if (cnt) cudaFreeAsync(cnt, s);
    if (e != cudaSuccess) {
        if (out.offsets) cudaFreeAsync(out.offsets, s);
        if (out.e) cudaFreeAsync(out.e, s);
        return e;
    }
    cudaFreeAsync(lt.offsets, s);
    cudaFreeAsync(lt.e, s);
    lt = out;
    return e;
}

void free_table(LabelTable &t, cudaStream_t s) {
    if (t.offsets) cudaFreeAsync(t.offsets, s);
    if (t.e) cudaFreeAsync(t.e, s);
    t = LabelTable{};
}

namespace {

// record i's parent goes to the slot of its hub in its vertex's sorted list
// (hub positions are unique within a list)
__global__ void place_parents_kernel(uint64_t T, const uint32_t *in_v, const uint32_t *in_h,
                                     const uint32_t *in_p, const uint64_t *off,
                                     const uint32_t *hubpos, uint32_t *parent) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < T;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = in_v[i], hp = in_h[i];
        uint64_t lo = off[v], hi = off[v + 1];  // hubpos[lo..hi) ascending, contains hp
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (hubpos[mid] <= hp) lo = mid; else hi = mid;
        }
        parent[lo] = in_p[i];
    }
}

}  // namespace

cudaError_t place_parents(uint64_t T, const uint32_t *in_v, const uint32_t *in_h, const uint32_t *in_p,
                          const LabelCSR &csr, uint32_t *parent, cudaStream_t s, int *launches) {
    if (!T) return cudaSuccess;
    place_parents_kernel<<<grid_for(T, 256), 256, 0, s>>>(T, in_v, in_h, in_p, csr.offsets,
                                                           csr.hubpos, parent);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace chl
