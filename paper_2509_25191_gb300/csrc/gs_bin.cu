// Tile binning and per-tile depth sort.
//
// Every projected record with radius > 0 touches the tiles of its float32
// rectangle (tile_rect in gs_common.cuh). Instead of a global radix sort of
// (tile, depth) keys over all instances, the instances are bucketed by tile
// (count -> scan -> scatter with per-tile cursors) and each tile's bucket is
// then sorted on chip by the 64-bit key (float32 depth bits << 32 | slot).
// The slot in the low bits makes every key unique, so the order inside a
// tile is the total order (depth, slot) whatever order the scatter's atomics
// produced: the result is deterministic. Depths are > near_z > 0, so their
// IEEE bits sort like the values.
//
// Kernels:
//   k_bin_count    one thread per slot, atomic per-tile counts
//   k_bin_scan     one block: tile ranges, cursors, instance total, capacity
//                  check, and a work order of tiles by decreasing count
//   k_bin_scatter  one thread per slot, writes keys at per-tile cursors
//   k_sort_small   persistent; tiles of <= 2047 instances, bitonic in smem
//   k_sort_large   persistent; larger tiles: bitonic on 16384-key chunks in
//                  smem, then merge-path merges through keys_tmp
#include "gs_common.cuh"

namespace gsk {

constexpr int SORT_SMALL_CAP = 2048;    // padded size (instances <= 2047)
constexpr int SORT_SMALL_THREADS = 256;
constexpr int SORT_LARGE_CAP = 16384;   // 128 KB of keys
constexpr int SORT_LARGE_THREADS = 1024;
constexpr int LARGE_BUCKET = 12;        // bucket of counts >= 2048

__global__ void __launch_bounds__(256) k_bin_count(const Launch L, const float4 *__restrict__ proj,
                                                   int *__restrict__ tile_count) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= L.n_slots) return;
    const float4 r2 = proj[4 * p + 2];
    if (!(r2.w > 0.f)) return;
    const float4 r0 = proj[4 * p];
    const int v = view_of_slot(L, p);
    const ViewDesc &vd = L.v[v];
    int x0, x1, y0, y1;
    tile_rect(r0.x, r0.y, r2.w, 1.f / (float)L.tw, 1.f / (float)L.th, vd.Gx, vd.Gy, x0, x1, y0, y1);
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) atomicAdd(tile_count + vd.tile_base + ty * vd.Gx + tx, 1);
}

__device__ __forceinline__ int count_bucket(int c) { return c <= 0 ? 0 : 32 - __clz(c); }

__global__ void __launch_bounds__(1024) k_bin_scan(const Launch L, long long capacity, int *__restrict__ tile_count,
                                                   int2 *__restrict__ ranges, int *__restrict__ order,
                                                   int *__restrict__ counters, int *__restrict__ status) {
    __shared__ long long s_warp[32];
    __shared__ int s_hist[34];
    __shared__ int s_base[34];
    __shared__ long long s_total;
    const int T = L.n_tiles;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunk = (T + nt - 1) / nt;
    const int beg = min(T, tid * chunk), end = min(T, beg + chunk);
    if (tid < 34) s_hist[tid] = 0;
    long long local = 0;
    int local_max = 0;
    for (int t = beg; t < end; ++t) {
        int c = tile_count[t];
        local += c;
        local_max = max(local_max, c);
    }
    // block exclusive scan of the per-thread sums
    const int lane = tid & 31, wid = tid >> 5;
    long long incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (nt >> 5) ? s_warp[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long n = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += n;
        }
        s_warp[lane] = wi - w;   // exclusive warp offsets
        if (lane == 31) s_total = wi;
    }
    __syncthreads();
    long long run = s_warp[wid] + incl - local;
    const long long total = s_total;
    const bool too_many = total > 0x7fffffffLL;
    const bool abort = too_many || total > capacity;
    for (int t = beg; t < end; ++t) {
        int c = tile_count[t];
        int st = (int)min(run, 0x7fffffffLL);
        run += c;
        ranges[t] = make_int2(st, (int)min(run, 0x7fffffffLL));
        tile_count[t] = st;   // becomes the scatter cursor
        atomicAdd(&s_hist[count_bucket(c)], 1);
    }
    // max tile count
    int m = local_max;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(counters + CNT_MAX_TILE, m);
    __syncthreads();
    if (tid == 0) {
        int acc = 0, large = 0;
        for (int b = 33; b >= 0; --b) {   // decreasing counts first
            s_base[b] = acc;
            acc += s_hist[b];
            if (b >= LARGE_BUCKET) large += s_hist[b];
        }
        counters[CNT_INSTANCES] = (int)min(total, 0x7fffffffLL);
        counters[CNT_ABORT] = abort ? 1 : 0;
        counters[CNT_Q_FWD] = 0;
        counters[CNT_Q_BWD] = 0;
        counters[CNT_Q_SORT] = 0;
        counters[CNT_Q_SORT_L] = 0;
        counters[CNT_LARGE_TILES] = large;
        if (abort && status) {
            status[0] = too_many ? GS_ERR_OVERFLOW : GS_ERR_CAPACITY;
            status[1] = (int)(total & 0xffffffffLL);
            status[2] = (int)(total >> 32);
        }
    }
    __syncthreads();
    for (int t = beg; t < end; ++t) {
        int c = ranges[t].y - ranges[t].x;
        int pos = atomicAdd(&s_base[count_bucket(c)], 1);
        order[pos] = t;
    }
}

__global__ void __launch_bounds__(256) k_bin_scatter(const Launch L, const float4 *__restrict__ proj,
                                                     int *__restrict__ cursor,
                                                     unsigned long long *__restrict__ keys,
                                                     const int *__restrict__ counters) {
    if (counters[CNT_ABORT]) return;
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= L.n_slots) return;
    const float4 r2 = proj[4 * p + 2];
    if (!(r2.w > 0.f)) return;
    const float4 r0 = proj[4 * p];
    const float depth = proj[4 * p + 3].x;
    const int v = view_of_slot(L, p);
    const ViewDesc &vd = L.v[v];
    int x0, x1, y0, y1;
    tile_rect(r0.x, r0.y, r2.w, 1.f / (float)L.tw, 1.f / (float)L.th, vd.Gx, vd.Gy, x0, x1, y0, y1);
    const unsigned long long key =
        ((unsigned long long)__float_as_uint(depth) << 32) | (unsigned long long)(unsigned int)p;
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) {
            int pos = atomicAdd(cursor + vd.tile_base + ty * vd.Gx + tx, 1);
            keys[pos] = key;
        }
}

// ascending bitonic sort of s[0..n2), n2 a power of two, by the whole block
__device__ __forceinline__ void block_bitonic(unsigned long long *s, int n2) {
    const int half = n2 >> 1;
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < half; i += blockDim.x) {
                const int a = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                const int b = a | j;
                const unsigned long long ka = s[a], kb = s[b];
                const bool up = (a & k) == 0;
                if ((ka > kb) == up) { s[a] = kb; s[b] = ka; }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int next_pow2(int n) { return n <= 1 ? 1 : 1 << (32 - __clz(n - 1)); }

__device__ __forceinline__ void sort_in_smem(unsigned long long *s, unsigned long long *keys, int st, int n) {
    const int n2 = next_pow2(n);
    for (int i = threadIdx.x; i < n2; i += blockDim.x) s[i] = i < n ? keys[st + i] : ~0ull;
    __syncthreads();
    block_bitonic(s, n2);
    for (int i = threadIdx.x; i < n; i += blockDim.x) keys[st + i] = s[i];
    __syncthreads();
}

__device__ __forceinline__ void write_ids(const unsigned long long *keys, unsigned int *ids, int st, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) ids[st + i] = (unsigned int)(keys[st + i] & 0xffffffffu);
}

__global__ void __launch_bounds__(SORT_SMALL_THREADS) k_sort_small(const Launch L, const int2 *__restrict__ ranges,
                                                                   const int *__restrict__ order,
                                                                   unsigned long long *__restrict__ keys,
                                                                   unsigned int *__restrict__ ids,
                                                                   int *__restrict__ counters) {
    __shared__ unsigned long long s[SORT_SMALL_CAP];
    __shared__ int s_item;
    if (counters[CNT_ABORT]) return;
    const int first = counters[CNT_LARGE_TILES];
    for (;;) {
        if (threadIdx.x == 0) s_item = first + atomicAdd(counters + CNT_Q_SORT, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= L.n_tiles) break;
        const int2 r = ranges[order[item]];
        const int n = r.y - r.x;
        if (n > 1) sort_in_smem(s, keys, r.x, n);
        write_ids(keys, ids, r.x, n);
    }
}

// merge sorted a[0..na) and b[0..nb) into out[0..na+nb) with the whole block
__device__ void block_merge(const unsigned long long *a, int na, const unsigned long long *b, int nb,
                            unsigned long long *out) {
    const int total = na + nb;
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int d0 = min(total, (int)threadIdx.x * per), d1 = min(total, d0 + per);
    if (d0 >= d1) return;
    // merge path: number of a-elements among the first d0 outputs
    int lo = max(0, d0 - nb), hi = min(d0, na);
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < b[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    int ia = lo, ib = d0 - lo;
    for (int d = d0; d < d1; ++d) {
        bool take_a = ib >= nb || (ia < na && a[ia] < b[ib]);
        out[d] = take_a ? a[ia++] : b[ib++];
    }
}

__global__ void __launch_bounds__(SORT_LARGE_THREADS) k_sort_large(const Launch L, const int2 *__restrict__ ranges,
                                                                   const int *__restrict__ order,
                                                                   unsigned long long *__restrict__ keys,
                                                                   unsigned long long *__restrict__ keys_tmp,
                                                                   unsigned int *__restrict__ ids,
                                                                   int *__restrict__ counters) {
    extern __shared__ unsigned long long s_large[];
    __shared__ int s_item;
    if (counters[CNT_ABORT]) return;
    const int n_large = counters[CNT_LARGE_TILES];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counters + CNT_Q_SORT_L, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_large) break;
        const int2 r = ranges[order[item]];
        const int n = r.y - r.x;
        for (int c = 0; c < n; c += SORT_LARGE_CAP) sort_in_smem(s_large, keys, r.x + c, min(SORT_LARGE_CAP, n - c));
        // pairwise merges of sorted runs, ping-pong between keys and keys_tmp
        unsigned long long *src = keys + r.x, *dst = keys_tmp + r.x;
        for (int w = SORT_LARGE_CAP; w < n; w <<= 1) {
            for (int m = 0; m < n; m += 2 * w) {
                const int na = min(w, n - m), nb = max(0, min(w, n - m - w));
                block_merge(src + m, na, src + m + na, nb, dst + m);
            }
            __syncthreads();
            unsigned long long *t = src; src = dst; dst = t;
        }
        if (src != keys + r.x) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) keys[r.x + i] = src[i];
            __syncthreads();
        }
        write_ids(keys, ids, r.x, n);
        __syncthreads();
    }
}

int launch_bin_sort(const Launch &L, const float *proj, const gs_bins *b, int32_t *status, cudaStream_t st) {
    const float4 *p = reinterpret_cast<const float4 *>(proj);
    if (cudaMemsetAsync(b->tile_scratch, 0, sizeof(int) * (size_t)L.n_tiles, st) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(b->counters, 0, sizeof(int) * GS_NUM_COUNTERS, st) != cudaSuccess) return GS_ERR_CUDA;
    const int bs = 256;
    const long long nb = (L.n_slots + bs - 1) / bs;
    if (nb > 0) k_bin_count<<<nb, bs, 0, st>>>(L, p, b->tile_scratch);
    k_bin_scan<<<1, 1024, 0, st>>>(L, b->capacity, b->tile_scratch, reinterpret_cast<int2 *>(b->tile_ranges),
                                   b->tile_order, b->counters, status);
    if (nb > 0)
        k_bin_scatter<<<nb, bs, 0, st>>>(L, p, b->tile_scratch, reinterpret_cast<unsigned long long *>(b->keys),
                                         b->counters);
    static int smem_set = 0;
    const int large_smem = SORT_LARGE_CAP * (int)sizeof(unsigned long long);
    if (!smem_set) {
        if (cudaFuncSetAttribute(k_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, large_smem) != cudaSuccess)
            return GS_ERR_CUDA;
        smem_set = 1;
    }
    const int sms = num_sms();
    k_sort_large<<<sms, SORT_LARGE_THREADS, large_smem, st>>>(
        L, reinterpret_cast<const int2 *>(b->tile_ranges), b->tile_order,
        reinterpret_cast<unsigned long long *>(b->keys), reinterpret_cast<unsigned long long *>(b->keys_tmp),
        b->ids, b->counters);
    k_sort_small<<<sms * 8, SORT_SMALL_THREADS, 0, st>>>(L, reinterpret_cast<const int2 *>(b->tile_ranges),
                                                         b->tile_order, reinterpret_cast<unsigned long long *>(b->keys),
                                                         b->ids, b->counters);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gsk
