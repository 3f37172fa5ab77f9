// Tile binning and per-tile depth sort.
//
// Every projected record with radius > 0 touches the tiles of its float32
// rectangle (tile_rect in gs_common.cuh), built from its reach extents. Instead of a global radix sort of
// (tile, depth) keys over all instances, the instances are bucketed by tile
// (count -> scan -> scatter with per-tile cursors) and each tile's bucket is
// then sorted on chip by the 64-bit key (float32 depth bits << 32 | slot).
// The slot in the low bits makes every key unique, so the order inside a
// tile is the total order (depth, slot) whatever order the scatter's atomics
// produced: the result is deterministic. Depths are > near_z > 0, so their
// IEEE bits sort like the values.
//
// Kernels:
//   k_bin_count    per-tile counts, block-aggregated in shared memory; one
//                  global atomic per (block, tile) reserves the block's
//                  range in the tile (kept in a table when it fits)
//   k_bin_scan     one block: tile ranges, cursors, instance total, capacity
//                  check, and a work order of tiles by decreasing count
//   k_bin_scatter  writes keys inside the reserved ranges, placement by
//                  shared-memory atomics
//   k_split_large  tiles far above the sort's work per block: partitioned
//                  by depth into runs of bins, listed for the sort
//   k_sort_tiles   persistent, one queue: the runs, then the other tiles
//                  largest first; radix sort on chip
#include "gs_common.cuh"

namespace gsk {

// Slots are processed in chunks of BIN_CHUNK per block. Within a chunk, the
// tile counts of each view segment are first gathered in a shared-memory
// histogram and then added to global memory once per (block, tile), which
// removes almost all same-address contention on the per-tile counters.
// Views with more tiles than BIN_SMEM_TILES fall back to direct atomics.
constexpr int BIN_THREADS = 512;
constexpr int BIN_CHUNK = 2048;
constexpr int BIN_SMEM_TILES = 12288;   // at most 48 KB of int counters, sized per launch

// The first float4 of a record holds everything binning needs (one sector);
// culled records are all zero, valid ones have positive extents.
__device__ __forceinline__ bool slot_rect(const Launch &L, const float4 &r0, const ViewDesc &vd, int &x0, int &x1,
                                          int &y0, int &y1) {
    if (!(r0.z > 0.f)) return false;
    tile_rect(r0.x, r0.y, r0.z, r0.w, 1.f / (float)L.tw, 1.f / (float)L.th, vd.Gx, vd.Gy, x0, x1, y0, y1);
    return true;
}

// a slot's binning record (zeros past the segment end)
__device__ __forceinline__ float4 slot_head(const float4 *__restrict__ proj, long long p, long long end) {
    return p < end ? proj[4 * p] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Warp-cooperative walk over the tiles of the 32 lanes' rectangles: the
// lanes' tile counts are prefix-summed across the warp and the flattened
// list of (lane, tile) items is processed 32 at a time, so every lane stays
// busy whatever the mix of rectangle sizes (a per-lane loop over its own
// rectangle leaves most lanes idle). For each item, f(tile index in the view,
// the owner lane's payload words a, b) runs on the lane that took it. All 32
// lanes must call this.
template <typename F>
__device__ __forceinline__ void warp_rect_walk(bool valid, int x0, int x1, int y0, int y1, int gx, unsigned int pa,
                                               unsigned int pb, F &&f) {
    const int lane = threadIdx.x & 31;
    const int w = valid ? x1 - x0 : 0;
    const int n = valid ? w * (y1 - y0) : 0;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - n;
    const float rw = w > 0 ? 1.f / (float)w : 0.f;
    for (int base = 0; base < total; base += 32) {
        const int fi = base + lane;
        // owner = number of lanes whose inclusive count is <= fi
        int own = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, own + step - 1);
            if (v <= fi) own += step;
        }
        const int ox0 = __shfl_sync(0xffffffffu, x0, own);
        const int oy0 = __shfl_sync(0xffffffffu, y0, own);
        const int ow = __shfl_sync(0xffffffffu, w, own);
        const int oex = __shfl_sync(0xffffffffu, excl, own);
        const float orw = __shfl_sync(0xffffffffu, rw, own);
        const unsigned int opa = __shfl_sync(0xffffffffu, pa, own);
        const unsigned int opb = __shfl_sync(0xffffffffu, pb, own);
        if (fi < total) {
            const int local = fi - oex;
            int dy = (int)(((float)local + 0.5f) * orw);   // exact after the correction below
            if (dy * ow > local) --dy;
            else if ((dy + 1) * ow <= local) ++dy;
            const int dx = local - dy * ow;
            f((oy0 + dy) * gx + ox0 + dx, opa, opb);
        }
    }
}

// next view segment [seg, seg_end) of a chunk that ends at c1
__device__ __forceinline__ long long segment_end(const Launch &L, int v, long long c1) {
    const long long e = (v + 1 < L.n_views) ? L.v[v + 1].slot_base : L.n_slots;
    return e < c1 ? e : c1;
}

// With a reservation table (table != nullptr), the block also keeps the
// value each (block, tile) atomic returned: the start of the block's range
// inside the tile, relative to the tile's first instance. The scatter then
// places its instances without counting again. Row blockIdx.x of the table
// holds the on-chip segments of the block's chunk one after another.
__global__ void __launch_bounds__(BIN_THREADS) k_bin_count(const Launch L, const float4 *__restrict__ proj,
                                                           int *__restrict__ tile_count, int smem_tiles,
                                                           int *__restrict__ table, int table_row) {
    extern __shared__ int s_cnt[];
    const long long c0 = (long long)blockIdx.x * BIN_CHUNK;
    const long long c1 = c0 + BIN_CHUNK < L.n_slots ? c0 + BIN_CHUNK : L.n_slots;
    int *trow = table ? table + (long long)blockIdx.x * table_row : nullptr;
    for (long long seg = c0; seg < c1;) {
        const int v = view_of_slot(L, seg);
        const long long seg_end = segment_end(L, v, c1);
        const ViewDesc &vd = L.v[v];
        const int Tv = vd.Gx * vd.Gy;
        const bool on_chip = Tv <= smem_tiles;
        if (on_chip) {
            for (int t = threadIdx.x; t < Tv; t += BIN_THREADS) s_cnt[t] = 0;
            __syncthreads();
        }
        // uniform trip count: whole warps walk; the next slot's record is
        // loaded while the current one's tiles are walked
        float4 rec = slot_head(proj, seg + threadIdx.x, seg_end);
        for (long long pb = seg; pb < seg_end; pb += BIN_THREADS) {
            const float4 cur = rec;
            rec = slot_head(proj, pb + BIN_THREADS + threadIdx.x, seg_end);
            int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
            const bool valid = slot_rect(L, cur, vd, x0, x1, y0, y1);
            warp_rect_walk(valid, x0, x1, y0, y1, vd.Gx, 0u, 0u, [&](int t, unsigned int, unsigned int) {
                if (on_chip) atomicAdd(s_cnt + t, 1);
                else atomicAdd(tile_count + vd.tile_base + t, 1);
            });
        }
        if (on_chip) {
            __syncthreads();
            for (int t = threadIdx.x; t < Tv; t += BIN_THREADS) {
                const int c = s_cnt[t];
                if (c) {
                    const int at = atomicAdd(tile_count + vd.tile_base + t, c);
                    if (trow) trow[t] = at;
                }
            }
            if (trow) trow += Tv;
            __syncthreads();
        }
        seg = seg_end;
    }
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
        int acc = 0;
        for (int b = 33; b >= 0; --b) {   // decreasing counts first
            s_base[b] = acc;
            acc += s_hist[b];
        }
        counters[CNT_INSTANCES] = (int)min(total, 0x7fffffffLL);
        counters[CNT_ABORT] = abort ? 1 : 0;
        counters[CNT_Q_FWD] = 0;
        counters[CNT_Q_BWD] = 0;
        counters[CNT_Q_SORT] = 0;
        counters[CNT_RUN_RES] = 0;
        counters[CNT_Q_SPLIT] = 0;
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

// Same chunking as k_bin_count: each block owns one contiguous range per
// (block, tile), taken from the count kernel's reservation table or (without
// one) reserved here by counting again and one global atomic per (block,
// tile); it places its instances inside the range with shared-memory atomics.
__global__ void __launch_bounds__(BIN_THREADS) k_bin_scatter(const Launch L, const float4 *__restrict__ proj,
                                                             int *__restrict__ cursor,
                                                             unsigned long long *__restrict__ keys,
                                                             const int *__restrict__ counters, int smem_tiles,
                                                             const int *__restrict__ table, int table_row) {
    extern __shared__ int s_cnt[];
    if (counters[CNT_ABORT]) return;
    const long long c0 = (long long)blockIdx.x * BIN_CHUNK;
    const long long c1 = c0 + BIN_CHUNK < L.n_slots ? c0 + BIN_CHUNK : L.n_slots;
    const int *trow = table ? table + (long long)blockIdx.x * table_row : nullptr;
    for (long long seg = c0; seg < c1;) {
        const int v = view_of_slot(L, seg);
        const long long seg_end = segment_end(L, v, c1);
        const ViewDesc &vd = L.v[v];
        const int Tv = vd.Gx * vd.Gy;
        const bool on_chip = Tv <= smem_tiles;
        if (on_chip && trow) {
            // the block's range in each tile, reserved by the count kernel
            // (entries of tiles the block does not touch are never read back)
            for (int t = threadIdx.x; t < Tv; t += BIN_THREADS) s_cnt[t] = cursor[vd.tile_base + t] + trow[t];
            trow += Tv;
            __syncthreads();
        } else if (on_chip) {
            for (int t = threadIdx.x; t < Tv; t += BIN_THREADS) s_cnt[t] = 0;
            __syncthreads();
            for (long long pb = seg; pb < seg_end; pb += BIN_THREADS) {
                const long long p = pb + threadIdx.x;
                int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
                const bool valid = slot_rect(L, slot_head(proj, p, seg_end), vd, x0, x1, y0, y1);
                warp_rect_walk(valid, x0, x1, y0, y1, vd.Gx, 0u, 0u,
                               [&](int t, unsigned int, unsigned int) { atomicAdd(s_cnt + t, 1); });
            }
            __syncthreads();
            for (int t = threadIdx.x; t < Tv; t += BIN_THREADS) {
                const int c = s_cnt[t];
                if (c) s_cnt[t] = atomicAdd(cursor + vd.tile_base + t, c);
            }
            __syncthreads();
        }
        // the next slot's record and depth are loaded while the current
        // one's instances are written
        float4 rec = slot_head(proj, seg + threadIdx.x, seg_end);
        float dep = seg + threadIdx.x < seg_end ? proj[4 * (seg + threadIdx.x) + 3].z : 0.f;
        for (long long pb = seg; pb < seg_end; pb += BIN_THREADS) {
            const long long p = pb + threadIdx.x;
            const float4 cur = rec;
            const float cdep = dep;
            const long long pn = p + BIN_THREADS;
            rec = slot_head(proj, pn, seg_end);
            dep = pn < seg_end ? proj[4 * pn + 3].z : 0.f;
            int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
            const bool valid = slot_rect(L, cur, vd, x0, x1, y0, y1);
            const unsigned int dbits = valid ? __float_as_uint(cdep) : 0u;
            const unsigned int pl = (unsigned int)p;
            // payload: the owner's key = (depth bits << 32) | slot
            warp_rect_walk(valid, x0, x1, y0, y1, vd.Gx, dbits, pl, [&](int t, unsigned int hi, unsigned int lo) {
                const int pos = on_chip ? atomicAdd(s_cnt + t, 1) : atomicAdd(cursor + vd.tile_base + t, 1);
                keys[pos] = ((unsigned long long)hi << 32) | lo;
            });
        }
        if (on_chip) __syncthreads();
        seg = seg_end;
    }
}

// ---------------------------------------------------------------------------
// per-tile sort: stable block-wide LSD radix sort (8-bit digits) of a 16-bit
// monotone compression of the depth bits, carrying the slot, then a fix-up
// that orders each run of equal compressed keys by (depth bits, slot). The
// result is the unique (depth, slot) order. Tiles longer than SORT_CAP
// are sorted in chunks and merged (merge path) through keys_tmp.
// ---------------------------------------------------------------------------
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_CAP = 4096;      // ~74 KB of shared memory: 3 blocks per SM (228 KB with the per-block reserve)
constexpr int SORT_SEG_MIN = 128;   // at least this many keys per active warp

struct SortSmem {
    unsigned int key[2][SORT_CAP];
    unsigned int val[2][SORT_CAP];
    unsigned int hist[256][SORT_WARPS + 1];   // [digit][warp] counts, then running offsets (odd pitch)
    unsigned int part[SORT_WARPS];   // per-warp partial sums of the histogram scan
    unsigned int kmin, kmax;
    int item;
    unsigned int moff[257];          // large tiles: bin offsets within the tile
};
// (the per-bin counts and cursors of a large tile's partition pass live in
// hist, unused until the segments are sorted)

// exclusive scan of the (digit, warp)-ordered counts hist[d][w], w < nwa:
// thread d owns digit d (SORT_THREADS == 256 digits), sums its row, the block
// scans the 256 row sums, and each row is rewritten as running offsets
static_assert(SORT_THREADS == 256, "one thread per 8-bit digit");
__device__ __forceinline__ void scan_hist(SortSmem &S, int nwa) {
    const int d = threadIdx.x;
    unsigned int sum = 0;
    for (int w = 0; w < nwa; ++w) sum += S.hist[d][w];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) S.part[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned int w = lane < SORT_WARPS ? S.part[lane] : 0, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < SORT_WARPS) S.part[lane] = wi - w;
    }
    __syncthreads();
    unsigned int run = S.part[wid] + incl - sum;
    for (int w = 0; w < nwa; ++w) {
        const unsigned int c = S.hist[d][w];
        S.hist[d][w] = run;
        run += c;
    }
    __syncthreads();
}

constexpr int FIX_RUN = 32;   // longest run of equal compressed keys one thread orders alone
static_assert(2 * (SORT_CAP / (FIX_RUN + 1)) + 1 <= 256 * (SORT_WARPS + 1), "the long-run list fits the histogram");

// Order key[0..L), val[0..L) (shared memory) by (key, val) with the whole
// block: a sorting network of ascending compare-exchanges over the next power
// of two P >= L (each merge of two sorted halves starts with the mirrored
// pairs i, size-1-i and continues with half-cleaners), so positions >= L act
// as +infinity and are never touched.
__device__ void block_sort_run(unsigned int *key, unsigned int *val, int L) {
    int P = 1;
    while (P < L) P <<= 1;
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (P >> 1); t += SORT_THREADS) {
                int i, j;
                if (stride == (size >> 1)) {   // mirrored pairs of the two halves
                    const int blk = t / stride, off = t % stride;
                    i = blk * size + off;
                    j = blk * size + size - 1 - off;
                } else {
                    const int blk = t / stride, off = t % stride;
                    i = blk * 2 * stride + off;
                    j = i + stride;
                }
                if (j < L) {
                    const unsigned int ki = key[i], kj = key[j], vi = val[i], vj = val[j];
                    if (ki > kj || (ki == kj && vi > vj)) {
                        key[i] = kj; key[j] = ki;
                        val[i] = vj; val[j] = vi;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// sort src[st .. st+n) (n <= SORT_CAP) by (depth, slot) into keys[st ..]
// (src may be keys itself)
__device__ void radix_sort_tile(SortSmem &S, const unsigned long long *src, unsigned long long *keys,
                                unsigned int *__restrict__ ids, int st, int n, bool write_ids) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) { S.kmin = 0xffffffffu; S.kmax = 0u; }
    __syncthreads();
    unsigned int lmin = 0xffffffffu, lmax = 0u;
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += SORT_THREADS) {
        const unsigned long long k = src[st + i];
        const unsigned int d = (unsigned int)(k >> 32);
        S.key[0][i] = d;
        S.val[0][i] = (unsigned int)(k & 0xffffffffu);
        lmin = min(lmin, d);
        lmax = max(lmax, d);
    }
    lmin = __reduce_min_sync(0xffffffffu, lmin);
    lmax = __reduce_max_sync(0xffffffffu, lmax);
    if (lane == 0) {
        atomicMin(&S.kmin, lmin);
        atomicMax(&S.kmax, lmax);
    }
    __syncthreads();
    // Radix-sort a 16-bit monotone compression of the depth bits,
    // (bits - kmin) >> shift, then order each run of equal compressed keys by
    // the full (depth bits, slot): the same total order in at most 2 passes.
    const unsigned int kmin = S.kmin, range = S.kmax - S.kmin;
    const int nbits = range ? 32 - __clz(range) : 0;
    const int shift = nbits > 16 ? nbits - 16 : 0;
    const int passes = (min(nbits, 16) + 7) / 8;
    const int nwa = max(1, min(SORT_WARPS, (n + SORT_SEG_MIN - 1) / SORT_SEG_MIN));
    const int seg = ((n + nwa - 1) / nwa + 31) & ~31;
    const int s0 = wid * seg, s1 = min(n, s0 + seg);
    const unsigned int lt_mask = (1u << lane) - 1u;
    int cur = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const int dshift = shift + 8 * pass;
        for (int w = 0; w < nwa; ++w) S.hist[threadIdx.x][w] = 0;
        __syncthreads();
        if (wid < nwa) {
            // counts only: order does not matter, plain shared atomics
            for (int i = s0 + lane; i < s1; i += 32)
                atomicAdd(&S.hist[((S.key[cur][i] - kmin) >> dshift) & 255u][wid], 1u);
        }
        __syncthreads();
        scan_hist(S, nwa);
        if (wid < nwa) {
            for (int b = s0; b < s1; b += 32) {
                const int i = b + lane;
                const bool act = i < s1;
                const unsigned int key = act ? S.key[cur][i] : 0u;
                const unsigned int d = ((key - kmin) >> dshift) & 255u;
                // lanes holding the same digit, from one ballot per digit bit
                unsigned int peers = __ballot_sync(0xffffffffu, act);
#pragma unroll
                for (int bit = 0; bit < 8; ++bit) {
                    const unsigned int ones = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
                    peers &= ((d >> bit) & 1u) ? ones : ~ones;
                }
                unsigned int pos = 0;
                if (act) pos = S.hist[d][wid] + __popc(peers & lt_mask);
                __syncwarp();
                if (act && lane == __ffs(peers) - 1) S.hist[d][wid] += __popc(peers);
                if (act) {
                    S.key[cur ^ 1][pos] = key;
                    S.val[cur ^ 1][pos] = S.val[cur][i];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    // runs of equal compressed key: up to FIX_RUN keys are ordered by
    // (depth bits, slot) by the thread that finds the run (insertion sort);
    // a longer run (many equal or nearly equal depths) is recorded and then
    // sorted by the whole block, so no thread sorts thousands of keys alone
    // (the histogram is free after the passes and holds the list)
    unsigned int *nlong = &S.hist[0][0], *lrun = &S.hist[0][1];
    if (threadIdx.x == 0) *nlong = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += SORT_THREADS) {
        const unsigned int c = (S.key[cur][i] - kmin) >> shift;
        if ((i == 0 || ((S.key[cur][i - 1] - kmin) >> shift) != c) && i + 1 < n &&
            ((S.key[cur][i + 1] - kmin) >> shift) == c) {
            int e = i + 1;
            while (e < n && ((S.key[cur][e] - kmin) >> shift) == c) ++e;
            if (e - i > FIX_RUN) {
                const unsigned int q = atomicAdd(nlong, 1u);   // at most n / (FIX_RUN + 1) runs
                lrun[2 * q] = (unsigned int)i;
                lrun[2 * q + 1] = (unsigned int)(e - i);
                continue;
            }
            for (int a = i + 1; a < e; ++a) {
                const unsigned int ka = S.key[cur][a], va = S.val[cur][a];
                int b = a - 1;
                while (b >= i && (S.key[cur][b] > ka || (S.key[cur][b] == ka && S.val[cur][b] > va))) {
                    S.key[cur][b + 1] = S.key[cur][b];
                    S.val[cur][b + 1] = S.val[cur][b];
                    --b;
                }
                S.key[cur][b + 1] = ka;
                S.val[cur][b + 1] = va;
            }
        }
    }
    __syncthreads();
    const unsigned int n_long = *nlong;
    for (unsigned int q = 0; q < n_long; ++q)
        block_sort_run(S.key[cur] + lrun[2 * q], S.val[cur] + lrun[2 * q], (int)lrun[2 * q + 1]);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += SORT_THREADS) {
        const unsigned int v = S.val[cur][i];
        keys[st + i] = ((unsigned long long)S.key[cur][i] << 32) | v;
        if (write_ids) ids[st + i] = v;
    }
    __syncthreads();
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

// Sort a segment longer than SORT_CAP whose keys are in tmp[st .. st+n):
// chunks of SORT_CAP sorted on chip into keys, then pairwise merges
// (ping-pong between keys and tmp over the same index range); the result,
// with its ids, ends in keys.
__device__ void sort_segment_merge(SortSmem &S, unsigned long long *keys, unsigned long long *tmp,
                                   unsigned int *__restrict__ ids, int st, int n) {
    for (int c = 0; c < n; c += SORT_CAP) radix_sort_tile(S, tmp, keys, ids, st + c, min(SORT_CAP, n - c), false);
    unsigned long long *src = keys + st, *dst = tmp + st;
    for (int w = SORT_CAP; w < n; w <<= 1) {
        for (int m = 0; m < n; m += 2 * w) {
            const int na = min(w, n - m), nb = max(0, min(w, n - m - w));
            block_merge(src + m, na, src + m + na, nb, dst + m);
        }
        __syncthreads();
        unsigned long long *t = src;
        src = dst;
        dst = t;
    }
    for (int i = threadIdx.x; i < n; i += SORT_THREADS) {
        const unsigned long long k = src[i];
        if (src != keys + st) keys[st + i] = k;
        ids[st + i] = (unsigned int)(k & 0xffffffffu);
    }
    __syncthreads();
}

// Large tiles (above SORT_CAP instances) are cut into runs of consecutive
// depth bins that are sorted independently, so that one large tile is sorted
// by many blocks at once (sorted by its own block, the largest tile alone set
// the sort's length). k_split_large partitions each large tile by the top 8
// bits of (depth bits - tile minimum) into keys_tmp (bins in depth order) and
// appends its runs -- stretches of consecutive bins of about SORT_SPLIT_RUN
// keys (see list_runs) -- to a list of (start, length) pairs. k_sort_tiles,
// launched after it, takes the runs first and then the other tiles, largest
// first, from one queue. A large tile whose runs do not fit the list is left
// whole and sorted by one block.
constexpr int SORT_SPLIT_RUN = 2048;
constexpr int SPLIT_THREADS = 1024;   // a large tile's partition: a few keys per thread

// partition of the large tile [r0, r0 + n) of keys into keys_tmp by the top 8
// bits of its depth range; moff[0..256] receives the bin offsets (relative to
// r0). mcnt is 256 words of scratch, part SORT_WARPS words. Whole block of NT
// (>= 256) threads; ends with the keys_tmp writes visible to the block.
template <int NT>
__device__ void partition_tile(const unsigned long long *__restrict__ keys, unsigned long long *__restrict__ keys_tmp,
                               int r0, int n, unsigned int *mcnt, unsigned int *moff, unsigned int *part,
                               unsigned int *kmin_s, unsigned int *kmax_s) {
    static_assert(NT >= 256 && NT % 32 == 0, "one thread per bin in the scan");
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        *kmin_s = 0xffffffffu;
        *kmax_s = 0u;
    }
    for (int b = tid; b < 256; b += NT) mcnt[b] = 0;
    __syncthreads();
    {
        unsigned int lmin = 0xffffffffu, lmax = 0u;
#pragma unroll 4
        for (int i = tid; i < n; i += NT) {
            const unsigned int d = (unsigned int)(keys[r0 + i] >> 32);
            lmin = min(lmin, d);
            lmax = max(lmax, d);
        }
        lmin = __reduce_min_sync(0xffffffffu, lmin);
        lmax = __reduce_max_sync(0xffffffffu, lmax);
        if (lane == 0) {
            atomicMin(kmin_s, lmin);
            atomicMax(kmax_s, lmax);
        }
    }
    __syncthreads();
    const unsigned int kmin = *kmin_s, range = *kmax_s - kmin;
    const int nbits = range ? 32 - __clz(range) : 0;
    const int mshift = nbits > 8 ? nbits - 8 : 0;
#pragma unroll 4
    for (int i = tid; i < n; i += NT)
        atomicAdd(&mcnt[(((unsigned int)(keys[r0 + i] >> 32)) - kmin) >> mshift], 1u);
    __syncthreads();
    // exclusive scan of the 256 bin counts, thread b < 256 owning bin b; the
    // offsets become the scatter cursors
    unsigned int c = 0u, incl = 0u;
    if (tid < 256) {
        c = mcnt[tid];
        incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) part[wid] = incl;
    }
    __syncthreads();
    if (wid == 0) {
        const unsigned int w = lane < SORT_WARPS ? part[lane] : 0u;
        unsigned int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < SORT_WARPS) part[lane] = wi - w;
    }
    __syncthreads();
    if (tid < 256) {
        const unsigned int excl = part[wid] + incl - c;
        moff[tid] = excl;
        mcnt[tid] = excl;
        if (tid == 255) moff[256] = excl + c;
    }
    __syncthreads();
#pragma unroll 4
    for (int i = tid; i < n; i += NT) {
        const unsigned long long k = keys[r0 + i];
        const unsigned int b = (((unsigned int)(k >> 32)) - kmin) >> mshift;
        keys_tmp[r0 + atomicAdd(&mcnt[b], 1u)] = k;
    }
    __syncthreads();   // the block's global writes are visible to the block after the barrier
}

// end of the run that starts at bin b0 (exclusive): the longest stretch of
// bins from b0 holding at most `limit` keys, at least one bin
__device__ __forceinline__ int run_end(const unsigned int *moff, int b0, int limit) {
    int b1 = b0 + 1;
    while (b1 < 256 && moff[b1 + 1] - moff[b0] <= (unsigned int)limit) ++b1;
    return b1;
}

struct SplitSmem {
    unsigned int mcnt[256];
    unsigned int moff[257];
    unsigned int part[SORT_WARPS];
    unsigned int starts[257];   // run starts (relative to the tile), then the end
    unsigned int wmax[SORT_WARPS], wcnt[SORT_WARPS];
    unsigned int kmin, kmax;
    int item, base, k;
};

// Runs of a partitioned tile, one thread per bin: a non-empty bin starts a run
// if it is the first, if its start lies in another SORT_SPLIT_RUN window of
// the tile than the previous non-empty bin's start, or if it or that bin holds
// more than half a window (so a large bin is a run of its own). A run then
// holds at most two windows' worth of keys unless one bin is larger.
constexpr int SPLIT_SHIFT = 11;   // log2(SORT_SPLIT_RUN)
static_assert((1 << SPLIT_SHIFT) == SORT_SPLIT_RUN, "window of the run rule");
__device__ void list_runs(SplitSmem &S) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned int o = 0u, sz = 0u, ps = 0u;
    if (tid < 256) {
        o = S.moff[tid];
        sz = S.moff[tid + 1] - o;
        // start of the previous non-empty bin: exclusive max-scan of the
        // non-empty bins' starts (plus one, so that "none" is 0)
        const unsigned int mine = sz ? o + 1u : 0u;
        unsigned int incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl = max(incl, t);
        }
        if (lane == 31) S.wmax[wid] = incl;
        ps = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) ps = 0u;
    }
    __syncthreads();
    bool start = false;
    if (tid < 256) {
        for (int w = 0; w < wid; ++w) ps = max(ps, S.wmax[w]);
        if (sz) {
            if (ps == 0u) {
                start = true;   // the first non-empty bin (start 0)
            } else {
                const unsigned int prev = ps - 1u;
                start = (o >> SPLIT_SHIFT) != (prev >> SPLIT_SHIFT) || sz > (unsigned int)(SORT_SPLIT_RUN / 2) ||
                        o - prev > (unsigned int)(SORT_SPLIT_RUN / 2);
            }
        }
        const unsigned int bal = __ballot_sync(0xffffffffu, start);
        if (lane == 0) S.wcnt[wid] = __popc(bal);
        S.part[wid] = bal;   // (only read back by this warp)
    }
    __syncthreads();
    if (tid < 256) {
        unsigned int j = __popc(S.part[wid] & ((1u << lane) - 1u));
        for (int w = 0; w < wid; ++w) j += S.wcnt[w];
        if (start) S.starts[j] = o;
        if (tid == 255) {
            const unsigned int k = j + (start ? 1u : 0u);
            S.k = (int)k;
            S.starts[k] = S.moff[256];
        }
    }
    __syncthreads();
}

// Partition the large tiles (the head of the work order: decreasing count
// buckets) and list their runs. A tile is split only if it is large against
// the sort's share of work per block: above SORT_CAP instances and above half
// of (instances / sort blocks) -- a tile below that is not the sort's last
// item to finish, and where most tiles are large (many views of a dense
// scene) splitting them only adds a pass. runq holds (start, length) int
// pairs, at most run_cap of them; flags[t] = -1 marks tile t as split (flags
// is the scatter's cursor array, non-negative until then).
__global__ void __launch_bounds__(SPLIT_THREADS) k_split_large(const int2 *__restrict__ ranges,
                                                              const int *__restrict__ order, int n_tiles,
                                                              unsigned long long *__restrict__ keys,
                                                              unsigned long long *__restrict__ keys_tmp,
                                                              unsigned int *__restrict__ ids,
                                                              int *__restrict__ counters, int *__restrict__ flags,
                                                              int *__restrict__ runq, int run_cap, int sort_blocks) {
    __shared__ SplitSmem S;
    if (counters[CNT_ABORT]) return;
    const int thr = max(SORT_CAP + 1, (int)((long long)counters[CNT_INSTANCES] / (2LL * sort_blocks)));
    const int thr_bucket = count_bucket(thr);
    for (;;) {
        if (threadIdx.x == 0) S.item = atomicAdd(counters + CNT_Q_SPLIT, 1);
        __syncthreads();
        const int item = S.item;
        __syncthreads();
        if (item >= n_tiles) break;
        const int t = order[item];
        const int2 r = ranges[t];
        const int n = r.y - r.x;
        if (count_bucket(n) < thr_bucket) break;   // the order is by count bucket: no tile to split follows
        if (n < thr) continue;
        partition_tile<SPLIT_THREADS>(keys, keys_tmp, r.x, n, S.mcnt, S.moff, S.part, &S.kmin, &S.kmax);
        list_runs(S);
        const int k = S.k;
        if (threadIdx.x == 0) {
            // one atomic add per tile (a compare-and-swap loop would retry once
            // per competing block); pairs past run_cap do not exist, so a
            // reservation that does not fit whole marks its pairs below
            // run_cap empty and the tile is sorted whole
            int base = atomicAdd(counters + CNT_RUN_RES, k);
            if (base + k > run_cap) {
                for (int j = base; j < run_cap; ++j) runq[2 * j + 1] = 0;
                base = -1;
            } else {
                flags[t] = -1;
            }
            S.base = base;
        }
        __syncthreads();
        const int base = S.base;
        if (base >= 0) {
            for (int j = threadIdx.x; j < k; j += SPLIT_THREADS) {
                runq[2 * (base + j)] = r.x + (int)S.starts[j];
                runq[2 * (base + j) + 1] = (int)(S.starts[j + 1] - S.starts[j]);
            }
        }
        __syncthreads();   // starts, k and base are read before the next item
    }
}

// Persistent, one queue: items [0, R) are the runs listed by k_split_large
// (R = the pairs reserved, at most run_cap; empty pairs are skipped), then the
// tiles in work order (largest first); split tiles are skipped.
__global__ void __launch_bounds__(SORT_THREADS, 3) k_sort_tiles(const Launch L, const int2 *__restrict__ ranges,
                                                             const int *__restrict__ order,
                                                             unsigned long long *__restrict__ keys,
                                                             unsigned long long *__restrict__ keys_tmp,
                                                             unsigned int *__restrict__ ids,
                                                             int *__restrict__ counters,
                                                             const int *__restrict__ flags,
                                                             const int *__restrict__ runq, int run_cap) {
    extern __shared__ __align__(16) unsigned char sort_smem[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(sort_smem);
    if (counters[CNT_ABORT]) return;
    const int R = min(counters[CNT_RUN_RES], run_cap);
    for (;;) {
        if (threadIdx.x == 0) S.item = atomicAdd(counters + CNT_Q_SORT, 1);
        __syncthreads();
        const int item = S.item;
        __syncthreads();
        if (item < R) {
            const int st = runq[2 * item], len = runq[2 * item + 1];
            if (len == 0) continue;   // a slot of a reservation that did not fit
            if (len == 1) {
                if (threadIdx.x == 0) {
                    const unsigned long long k = keys_tmp[st];
                    keys[st] = k;
                    ids[st] = (unsigned int)(k & 0xffffffffu);
                }
                continue;
            }
            if (len <= SORT_CAP) radix_sort_tile(S, keys_tmp, keys, ids, st, len, true);
            else sort_segment_merge(S, keys, keys_tmp, ids, st, len);
            continue;
        }
        if (item - R >= L.n_tiles) break;
        const int t = order[item - R];
        const int2 r = ranges[t];
        const int n = r.y - r.x;
        if (n <= 1) {
            if (n == 1 && threadIdx.x == 0) ids[r.x] = (unsigned int)(keys[r.x] & 0xffffffffu);
            continue;
        }
        if (n <= SORT_CAP) {
            radix_sort_tile(S, keys, keys, ids, r.x, n, true);
            continue;
        }
        if (flags[t] < 0) continue;   // split: its runs were items of this queue
        // a large tile left whole: partition, then sort runs of bins that fit
        // on chip one after another (a single bin larger than that takes the
        // chunk-and-merge path). The result is the same (depth, slot) order.
        partition_tile<SORT_THREADS>(keys, keys_tmp, r.x, n, &S.hist[0][0], S.moff, S.part, &S.kmin, &S.kmax);
        for (int b0 = 0; b0 < 256;) {
            const int b1 = run_end(S.moff, b0, SORT_CAP);
            const int s0 = (int)S.moff[b0], len = (int)(S.moff[b1] - S.moff[b0]);
            if (len == 1 && threadIdx.x == 0) {
                const unsigned long long k = keys_tmp[r.x + s0];
                keys[r.x + s0] = k;
                ids[r.x + s0] = (unsigned int)(k & 0xffffffffu);
            } else if (len > 1 && len <= SORT_CAP) {
                radix_sort_tile(S, keys_tmp, keys, ids, r.x + s0, len, true);
            } else if (len > SORT_CAP) {
                sort_segment_merge(S, keys, keys_tmp, ids, r.x + s0, len);
            }
            __syncthreads();
            b0 = b1;
        }
    }
}

int launch_bin_sort(const Launch &L, const float *proj, const gs_bins *b, int32_t *status, cudaStream_t st) {
    const float4 *p = reinterpret_cast<const float4 *>(proj);
    // tile_scratch [5T]: the tile cursors (then the split flags), then up to
    // 2T (start, length) runs of split large tiles
    if (cudaMemsetAsync(b->tile_scratch, 0, sizeof(int) * (size_t)L.n_tiles, st) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(b->counters, 0, sizeof(int) * GS_NUM_COUNTERS, st) != cudaSuccess) return GS_ERR_CUDA;
    const long long nb = (L.n_slots + BIN_CHUNK - 1) / BIN_CHUNK;
    int smem_tiles = 0;
    for (int v = 0; v < L.n_views; ++v) smem_tiles = max(smem_tiles, L.v[v].Gx * L.v[v].Gy);
    smem_tiles = min(smem_tiles, BIN_SMEM_TILES);
    const size_t bin_smem = sizeof(int) * (size_t)max(smem_tiles, 1);
    // reservation table in keys_tmp (free until the sort): one row per block
    // covering the on-chip view segments of its chunk, if it fits
    long long row = 0;
    for (int v = 0; v < L.n_views; ++v) {
        // the chunk that holds the view's first slot may also hold the ends
        // of earlier views and the starts of later ones
        const long long c0 = (L.v[v].slot_base / BIN_CHUNK) * BIN_CHUNK, c1 = c0 + BIN_CHUNK;
        long long sum = 0;
        for (int u = 0; u < L.n_views; ++u) {
            const long long u0 = L.v[u].slot_base, u1 = u0 + L.v[u].g_count;
            const int Tu = L.v[u].Gx * L.v[u].Gy;
            if (u1 > c0 && u0 < c1 && Tu <= smem_tiles) sum += Tu;
        }
        row = max(row, sum);
    }
    int *table = nullptr;
    if (nb > 0 && row > 0 && row < 0x7fffffffLL && (unsigned long long)nb * (unsigned long long)row * 4ULL <=
                                                    (unsigned long long)b->capacity * 8ULL)
        table = reinterpret_cast<int *>(b->keys_tmp);
    const int table_row = table ? (int)row : 0;
    if (nb > 0) k_bin_count<<<nb, BIN_THREADS, bin_smem, st>>>(L, p, b->tile_scratch, smem_tiles, table, table_row);
    k_bin_scan<<<1, 1024, 0, st>>>(L, b->capacity, b->tile_scratch, reinterpret_cast<int2 *>(b->tile_ranges),
                                   b->tile_order, b->counters, status);
    if (nb > 0)
        k_bin_scatter<<<nb, BIN_THREADS, bin_smem, st>>>(L, p, b->tile_scratch,
                                                         reinterpret_cast<unsigned long long *>(b->keys), b->counters,
                                                         smem_tiles, table, table_row);
    static int sort_blocks = 0;
    const int smem = (int)sizeof(SortSmem);
    if (!sort_blocks) {
        if (cudaFuncSetAttribute(k_sort_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return GS_ERR_CUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_tiles, SORT_THREADS, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        sort_blocks = per_sm * num_sms();
    }
    const int2 *ranges = reinterpret_cast<const int2 *>(b->tile_ranges);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(b->keys);
    unsigned long long *keys_tmp = reinterpret_cast<unsigned long long *>(b->keys_tmp);
    int *runq = b->tile_scratch + L.n_tiles;
    k_split_large<<<num_sms(), SPLIT_THREADS, 0, st>>>(ranges, b->tile_order, (int)L.n_tiles, keys, keys_tmp,
                                                          b->ids, b->counters, b->tile_scratch, runq,
                                                          2 * (int)L.n_tiles, sort_blocks);
    k_sort_tiles<<<sort_blocks, SORT_THREADS, smem, st>>>(L, ranges, b->tile_order, keys, keys_tmp, b->ids,
                                                          b->counters, b->tile_scratch, runq, 2 * (int)L.n_tiles);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gsk
