// Label assembly: from the (vertex, hub, dist) records the trees emit, in
// whatever order the trees finished, to per-vertex lists sorted by hub rank
// (Algorithm 2, "sort labels in L_v using hub rank"; the lists are stored
// per vertex only, as in the footnote of Sec. 7.2).
//
//   1. count labels per vertex (atomic histogram)
//   2. exclusive scan -> offsets
//   3. scatter (hubpos << 32 | dist) into each vertex's segment
//   4. sort every segment by hubpos (= descending R of the hub): one warp per
//      segment up to 32 labels, one CTA per segment up to MAX_SEGMENT labels
//      (bitonic networks in shared memory); a longer segment (one CTA each) is
//      sorted in chunks in shared memory, then the sorted runs are merged
//      pairwise in global memory
//   5. split into hub (caller id), hubpos and dist arrays
#include "chl_common.cuh"

namespace chl {

cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                               int *launches);

namespace {

constexpr uint32_t MAX_SEGMENT = 16384;  // longest segment sorted in shared memory at once
constexpr uint32_t LONG_CHUNK = 4096;    // chunk of a longer segment sorted in shared memory

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

// classify segments by length into four work lists; record the longest
__global__ void classify_kernel(uint32_t n, const uint64_t *off, uint32_t *small_list,
                                uint32_t *mid_list, uint32_t *big_list, uint32_t *long_list,
                                uint32_t *counts, unsigned long long *max_len) {
    for (uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t len = off[v + 1] - off[v];
        if (len <= 1) continue;
        atomicMax(max_len, (unsigned long long)len);
        if (len <= 32) small_list[atomicAdd(&counts[0], 1u)] = uint32_t(v);
        else if (len <= 1024) mid_list[atomicAdd(&counts[1], 1u)] = uint32_t(v);
        else if (len <= MAX_SEGMENT) big_list[atomicAdd(&counts[2], 1u)] = uint32_t(v);
        else long_list[atomicAdd(&counts[3], 1u)] = uint32_t(v);
    }
}

// One CTA per segment longer than MAX_SEGMENT: its chunks of LONG_CHUNK keys
// are sorted in shared memory (bitonic), then runs of width w, 2w, 4w, ...
// are merged pairwise between tmp and tmp2 (each thread writes an equal share
// of a merged pair, starting where the merge path of its first output crosses
// the two runs); the sorted segment ends in tmp. Keys (hubpos << 32 | dist)
// are distinct within a segment (one label per hub), so the order is unique.
__global__ void __launch_bounds__(1024) sort_long_kernel(const uint32_t *list, const uint32_t *count,
                                                         const uint64_t *off, uint64_t *tmp,
                                                         uint64_t *tmp2) {
    __shared__ uint64_t sm[LONG_CHUNK];
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    for (uint32_t sidx = blockIdx.x; sidx < *count; sidx += gridDim.x) {
        const uint32_t v = list[sidx];
        const uint64_t a = off[v], len = off[v + 1] - a;
        for (uint64_t c0 = 0; c0 < len; c0 += LONG_CHUNK) {
            const uint32_t cl = uint32_t(len - c0 < LONG_CHUNK ? len - c0 : LONG_CHUNK);
            for (uint32_t i = tid; i < LONG_CHUNK; i += nt) sm[i] = i < cl ? tmp[a + c0 + i] : ~0ull;
            __syncthreads();
            for (uint32_t k = 2; k <= LONG_CHUNK; k <<= 1) {
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    for (uint32_t i = tid; i < LONG_CHUNK; i += nt) {
                        const uint32_t ix = i ^ j;
                        if (ix > i) {
                            const uint64_t x = sm[i], y = sm[ix];
                            if ((x > y) == ((i & k) == 0)) {
                                sm[i] = y;
                                sm[ix] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (uint32_t i = tid; i < cl; i += nt) tmp[a + c0 + i] = sm[i];
            __syncthreads();
        }
        uint64_t *src = tmp + a, *dst = tmp2 + a;
        for (uint64_t w = LONG_CHUNK; w < len; w *= 2) {
            for (uint64_t p0 = 0; p0 < len; p0 += 2 * w) {
                const uint64_t na = len - p0 < w ? len - p0 : w;
                const uint64_t nb = len - p0 > w ? (len - p0 - w < w ? len - p0 - w : w) : 0;
                const uint64_t m = na + nb;
                const uint64_t *A = src + p0, *B = A + na;
                const uint64_t k0 = m * tid / nt, k1 = m * (tid + 1) / nt;
                if (k0 >= k1) continue;
                // i = keys of A among the first k0 outputs (smallest i with A[i] > B[k0 - i - 1])
                uint64_t lo = k0 > nb ? k0 - nb : 0, hi = k0 < na ? k0 : na;
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    if (A[mid] <= B[k0 - mid - 1]) lo = mid + 1; else hi = mid;
                }
                uint64_t i = lo, j = k0 - lo;
                for (uint64_t k = k0; k < k1; ++k) {
                    const bool take_a = j >= nb || (i < na && A[i] <= B[j]);
                    dst[p0 + k] = take_a ? A[i++] : B[j++];
                }
            }
            __syncthreads();
            uint64_t *t = src;
            src = dst;
            dst = t;
        }
        if (src != tmp + a)
            for (uint64_t i = tid; i < len; i += nt) tmp[a + i] = src[i];
        __syncthreads();
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
    const uint64_t cap = uint64_t(device_sms()) * 32;
    if (b > cap) b = cap;
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
    uint64_t *cnt = nullptr, *tmp = nullptr, *tmp2 = nullptr;
    uint32_t *lists = nullptr, *counts = nullptr;
    unsigned long long *maxlen = nullptr;
    unsigned long long hmax = 0;
    const int sms = device_sms();
    *too_long = 0;
    out = LabelCSR{};
    const size_t Tb = (T ? T : 1);
    CKE(dmalloc(&out.offsets, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(dmalloc(&out.hub, Tb * sizeof(uint32_t), s));
    CKE(dmalloc(&out.hubpos, Tb * sizeof(uint32_t), s));
    CKE(dmalloc(&out.dist, Tb * sizeof(uint32_t), s));
    CKE(dmalloc(&cnt, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(dmalloc(&tmp, Tb * sizeof(uint64_t), s));
    CKE(dmalloc(&lists, 4 * size_t(n) * sizeof(uint32_t), s));
    CKE(dmalloc(&counts, 4 * sizeof(uint32_t), s));
    CKE(dmalloc(&maxlen, sizeof(unsigned long long), s));
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
                                                     lists + 2 * size_t(n), lists + 3 * size_t(n),
                                                     counts, maxlen);
    *launches += 2;
    CKE(cudaGetLastError());
    CKE(cudaMemcpyAsync(&hmax, maxlen, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    CKE(cudaStreamSynchronize(s));
    sort_small_kernel<<<sms * 8, 256, 0, s>>>(lists, counts, out.offsets, tmp);
    sort_block_kernel<256><<<sms * 8, 256, 1024 * sizeof(uint64_t), s>>>(lists + n, counts + 1,
                                                                         out.offsets, tmp);
    *launches += 2;
    if (hmax > 1024) {
        // the attribute belongs to the current device: set on every call
        CKE(cudaFuncSetAttribute(sort_block_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(MAX_SEGMENT * sizeof(uint64_t))));
        sort_block_kernel<1024><<<sms, 1024, MAX_SEGMENT * sizeof(uint64_t), s>>>(
            lists + 2 * size_t(n), counts + 2, out.offsets, tmp);
        *launches += 1;
    }
    if (hmax > MAX_SEGMENT) {
        CKE(dmalloc(&tmp2, Tb * sizeof(uint64_t), s));
        sort_long_kernel<<<sms, 1024, 0, s>>>(lists + 3 * size_t(n), counts + 3, out.offsets, tmp, tmp2);
        *launches += 1;
        CKE(cudaGetLastError());
    }
    split_kernel<<<grid_for(T, 256), 256, 0, s>>>(T, tmp, vert_at, out.hub, out.hubpos, out.dist);
    *launches += 1;
    CKE(cudaGetLastError());
done:
    if (cnt) cudaFreeAsync(cnt, s);
    if (tmp) cudaFreeAsync(tmp, s);
    if (tmp2) cudaFreeAsync(tmp2, s);
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
    CKE(dmalloc(&out.offsets, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(dmalloc(&out.e, (size_t(T) + 2) * sizeof(uint2), s));
    CKE(cudaMemsetAsync(out.e, 0xFF, (size_t(T) + 2) * sizeof(uint2), s));
    CKE(dmalloc(&cnt, (size_t(n) + 1) * sizeof(uint64_t), s));
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
                       uint32_t min_hub, cudaStream_t s, int *launches, LabelTable *keep_old) {
    cudaError_t e = cudaSuccess;
    uint64_t *cnt = nullptr;
    LabelTable out;
    const uint64_t dT = T - T0;
    CKE(dmalloc(&out.offsets, (size_t(n) + 1) * sizeof(uint64_t), s));
    CKE(dmalloc(&out.e, (size_t(T) + 2) * sizeof(uint2), s));
    CKE(cudaMemsetAsync(out.e, 0xFF, (size_t(T) + 2) * sizeof(uint2), s));
    CKE(dmalloc(&cnt, (size_t(n) + 1) * sizeof(uint64_t), s));
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
    if (keep_old) {
        *keep_old = lt;  // still read by trees on another stream: the caller frees it after them
    } else {
        cudaFreeAsync(lt.offsets, s);
        cudaFreeAsync(lt.e, s);
    }
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
