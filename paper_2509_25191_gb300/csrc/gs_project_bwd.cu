// Backward of the projection: per-slot 2D gradients -> raw Gaussian
// parameters and camera poses.
//
// One thread per Gaussian (fixed grid, grid-stride; for one-view calls one
// thread per Gaussian with a nonzero 2D gradient: see COMPACT), looping over
// the views of its scene: the Gaussian's parameters are read once, its
// gradients are summed over views in registers and written once (overwritten,
// or added to the caller's values when the configuration accumulates). For degree-3 SH the block's
// first-view 2D-gradient rows arrive by a tensor copy, the SH rows are staged
// in shared memory, and the block's SH-coefficient gradients leave by tensor
// stores (see PbStage). Each view's pose
// gradient (dL/dR, dL/dt; Section 3.4 needs it for the pose residuals) is
// summed over a warp with shuffles, kept per warp in shared memory, and
// written as one partial per block; k_pose_reduce then sums the partials in a
// fixed order, so the pose gradient is deterministic given grad2d.
//
// Chain (FP32, exact derivative of the forward in gs_project.cu):
//   dilated 2D covariance (its gradient comes from the raster backward),
//   Sigma' = T Sigma T^T with
//   T = J R_v, J with the tangent clamp (zero derivative through a clamped
//   tangent), mean2D = f x / z + c, m = R_v mu + t_v, Sigma = M M^T with
//   M = R(q) diag(exp l), q normalised, o = sigmoid, colour = max(0,
//   sum f_k Y_k(d) + 0.5), d = normalise(mu - C_v), C_v = -R_v^T t_v.
#include <string.h>

#include "gs_common.cuh"

namespace gsk {

constexpr int PB_THREADS = 128;   // 128 registers: 4 blocks per SM, no spills

// a parameter gradient: written (overwrite) or added to the caller's value
__device__ __forceinline__ void put(float *p, float v, bool acc) { *p = acc ? *p + v : v; }
constexpr int PB_WARPS = PB_THREADS / 32;

// Staging of a block's 128 Gaussians on the degree-3 path: the SH rows arrive
// as a 32-float box with the 128-byte swizzle and a 16-float box with the
// 64-byte swizzle (a thread reads its own row 16 bytes at a time without bank
// conflicts) by two tensor copies for the whole block, and the SH-coefficient
// gradients are summed over views in the same layout and leave by two tensor
// stores.
struct PbStage {
    float4 shA[PB_THREADS * 8];
    float4 shB[PB_THREADS * 4];
    float4 gA[PB_THREADS * 8];
    float4 gB[PB_THREADS * 4];
    float4 g2d[PB_THREADS * 3];   // the first view's 2D-gradient rows (48-byte rows: conflict-free)
    unsigned long long bar;
};

// COMPACT (one-view calls): most Gaussians of a dense scene get no 2D
// gradient in one view (they are hidden behind saturated pixels), and a
// thread per Gaussian left most lanes idle. Instead each block takes a
// contiguous range of Gaussians, finds those with a nonzero 2D-gradient row
// (PB_SUB at a time, listed in shared memory in an order fixed by their
// indices) and runs the chain over the list with full warps. Each range's
// parameter-gradient rows are zeroed by its block, coalesced, when the range
// is listed, and the listed Gaussians' rows written again after a barrier
// (accumulating, the others are left as they are). The pose partials stay
// per block over a fixed range, so the pose gradient is deterministic. With
// several views most Gaussians contribute somewhere and the block-wide
// tensor copies are faster.
constexpr int PB_SUB = 1024;   // Gaussians compacted at a time (8 per thread)

// List the Gaussians (thread indices) in [g0, g1) with a nonzero 2D-gradient
// row in their (single) view into s_list; returns the count. Thread t checks
// g0 + j * PB_THREADS + t (coalesced rows) and lists its hits in j order
// after those of lower threads. Whole block; starts and ends with a barrier.
__device__ __forceinline__ int compact_range(const Launch &L, const float4 *__restrict__ grad2d, long long g0,
                                             long long g1, int *s_list, int *s_wsum) {
    constexpr int PER = PB_SUB / PB_THREADS;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();   // the previous list has been read
    unsigned int hits = 0u;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const long long g = g0 + (long long)j * PB_THREADS + threadIdx.x;
        if (g < g1) {
            const int sc = scene_of_thread(L, g);
            const long long slot = L.v[L.s[sc].v_begin].slot_base + (g - L.s[sc].thread_base);
            const float4 a4 = grad2d[3 * slot], b4 = grad2d[3 * slot + 1];
            const float c0 = reinterpret_cast<const float *>(grad2d)[12 * slot + 8];
            // nonzero iff some value has nonzero magnitude bits
            const unsigned int bits = __float_as_uint(a4.x) | __float_as_uint(a4.y) | __float_as_uint(a4.z) |
                                      __float_as_uint(a4.w) | __float_as_uint(b4.x) | __float_as_uint(b4.y) |
                                      __float_as_uint(b4.z) | __float_as_uint(b4.w) | __float_as_uint(c0);
            if (bits & 0x7fffffffu) hits |= 1u << j;
        }
    }
    const int cnt = __popc(hits);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_wsum[wid] = incl;
    __syncthreads();
    int at = incl - cnt, total = 0;
#pragma unroll
    for (int w = 0; w < PB_WARPS; ++w) {
        const int ws = s_wsum[w];
        if (w < wid) at += ws;
        total += ws;
    }
#pragma unroll
    for (int j = 0; j < PER; ++j)
        if (hits >> j & 1u) s_list[at++] = j * PB_THREADS + (int)threadIdx.x;
    __syncthreads();
    return total;
}

// Zero the parameter-gradient rows of Gaussians [i0, i0 + cnt) (K SH
// coefficients per colour channel) with the whole block, coalesced; float4
// stores where a span is 16-byte aligned and a whole number of float4.
__device__ __forceinline__ void zero_span(float *__restrict__ p, long long count) {
    if (((uintptr_t)p & 15u) == 0 && (count & 3) == 0) {
        float4 *q = reinterpret_cast<float4 *>(p);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (long long e = threadIdx.x; e < (count >> 2); e += PB_THREADS) q[e] = z;
    } else {
        for (long long e = threadIdx.x; e < count; e += PB_THREADS) p[e] = 0.f;
    }
}
template <int K>
__device__ __forceinline__ void zero_rows(long long i0, long long cnt, float *__restrict__ g_means,
                                          float *__restrict__ g_log_scales, float *__restrict__ g_quats,
                                          float *__restrict__ g_logits, float *__restrict__ g_sh) {
    zero_span(g_means + 3 * i0, 3 * cnt);
    zero_span(g_log_scales + 3 * i0, 3 * cnt);
    zero_span(g_quats + 4 * i0, 4 * cnt);
    zero_span(g_logits + i0, cnt);
    zero_span(g_sh + 3LL * K * i0, 3LL * K * cnt);
}

template <int DEG, bool GAUSS, bool TMA, bool COMPACT>
__global__ void __launch_bounds__(PB_THREADS, 4) k_project_bwd(
    const Launch L, const float *__restrict__ means, const float *__restrict__ log_scales,
    const float *__restrict__ quats, const float *__restrict__ logits, const float *__restrict__ sh,
    const float *__restrict__ viewmats, const float *__restrict__ intr, const float4 *__restrict__ proj,
    const float4 *__restrict__ grad2d, float *__restrict__ g_means, float *__restrict__ g_log_scales,
    float *__restrict__ g_quats, float *__restrict__ g_logits, float *__restrict__ g_sh,
    float *__restrict__ pose_partials, const __grid_constant__ CUtensorMap tm_shA,
    const __grid_constant__ CUtensorMap tm_shB, const __grid_constant__ CUtensorMap tm_gA,
    const __grid_constant__ CUtensorMap tm_gB, const __grid_constant__ CUtensorMap tm_g2d,
    int *__restrict__ status) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int GP = 3 * K + 1;   // odd row pitch: conflict-free column access
    static_assert(!TMA || DEG == 3, "the staged path is for 48-float SH rows");
    static_assert(!(TMA && COMPACT), "the compacted path reads rows per thread");
    // per-warp pose partials [PB_WARPS][n_views][12] (dynamic: sized by the launch)
    extern __shared__ float s_pose[];
    // per-thread SH-coefficient gradients, summed over views here and written
    // out by the whole block with coalesced stores (per-thread path)
    __shared__ float s_gf[GAUSS && !TMA ? PB_THREADS * GP : 1];
    __shared__ long long s_row[GAUSS && !TMA ? PB_THREADS : 1];
    __shared__ __align__(1024) PbStage S[1];   // (removed by the compiler where unused)
    __shared__ int s_list[COMPACT ? PB_SUB : 1];   // offsets from the range's current start
    __shared__ int s_wsum[PB_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nv = L.n_views;
    for (int i = threadIdx.x; i < PB_WARPS * nv * 12; i += PB_THREADS) s_pose[i] = 0.f;
    if (TMA && threadIdx.x == 0) mbar_init(&S[0].bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    const int r = threadIdx.x;   // this thread's row of the staging boxes

    const long long stride = (long long)gridDim.x * PB_THREADS;
    // COMPACT: this block's range [c_next, c_end), the current list of c_cnt
    // offsets from c_at, and how far it has been taken
    long long c_next = 0, c_end = 0, c_at = 0;
    int c_cnt = 0, c_pos = 0;
    if constexpr (COMPACT) {
        const long long per = (L.n_threads + gridDim.x - 1) / gridDim.x;
        c_next = min((long long)L.n_threads, (long long)blockIdx.x * per);
        c_end = min((long long)L.n_threads, c_next + per);
    }
    for (long long base = (long long)blockIdx.x * PB_THREADS;; base += stride) {
        long long gid;
        bool valid;
        if constexpr (COMPACT) {
            while (c_pos >= c_cnt && c_next < c_end) {   // (uniform over the block)
                const long long g1 = min(c_end, c_next + PB_SUB);
                c_cnt = compact_range(L, grad2d, c_next, g1, s_list, s_wsum);
                if (GAUSS && !L.accumulate) {
                    // this range's rows, zero; the listed Gaussians' rows are
                    // written again below by this block, after a barrier (one
                    // view: the range's Gaussians are contiguous)
                    const int sc = scene_of_thread(L, c_next);
                    zero_rows<K>(L.s[sc].g_begin + (c_next - L.s[sc].thread_base), g1 - c_next, g_means,
                                 g_log_scales, g_quats, g_logits, g_sh);
                    __syncthreads();
                }
                c_at = c_next;
                c_next = g1;
                c_pos = 0;
            }
            if (c_pos >= c_cnt) break;
            valid = c_pos + (int)threadIdx.x < c_cnt;
            gid = valid ? c_at + s_list[c_pos + threadIdx.x] : 0;
            c_pos += PB_THREADS;
        } else {
            if (base >= L.n_threads) break;
            gid = base + threadIdx.x;
            valid = gid < L.n_threads;
        }
        const int s = valid ? scene_of_thread(L, gid) : 0;
        const long long li = valid ? gid - L.s[s].thread_base : 0;
        const long long i = L.s[s].g_begin + li;
        const int vb = valid ? L.s[s].v_begin : 0x7fffffff, ve = valid ? L.s[s].v_end : 0;
        const int wvb = __reduce_min_sync(0xffffffffu, vb), wve = __reduce_max_sync(0xffffffffu, ve);

        // a block iteration is "full" when its 128 threads are Gaussians of one
        // scene: its SH rows (and gradient rows) are then contiguous boxes
        bool full = false;
        int row0 = 0, v_first = -1;
        if constexpr (TMA) {
            const long long last = base + PB_THREADS - 1;
            if (last < L.n_threads) {
                const int s0 = scene_of_thread(L, base);
                full = scene_of_thread(L, last) == s0 && (smem_u32(S[0].shA) & 1023u) == 0;
                row0 = (int)(L.s[s0].g_begin + base - L.s[s0].thread_base);
                v_first = L.s[s0].v_begin;
            }
            // with accumulation the SH-gradient rows start from the caller's
            // values (loaded like the SH rows), otherwise from zero
            const bool acc_rows = GAUSS && L.accumulate;
            if (threadIdx.x == 0) {
                // the previous iteration's gradient stores have read the staging
                if (GAUSS) bulk_wait_read_all();
                if (full) {
                    fence_async_smem();
                    mbar_expect_tx(&S[0].bar, PB_THREADS * ((acc_rows ? 48 : 0) + 48 + 12) * 4);
                    tma_load_2d(S[0].shA, &tm_shA, 0, row0, &S[0].bar);
                    tma_load_2d(S[0].shB, &tm_shB, 32, row0, &S[0].bar);
                    const int srow = (int)(L.v[v_first].slot_base + base - L.s[scene_of_thread(L, base)].thread_base);
                    tma_load_2d(S[0].g2d, &tm_g2d, 0, srow, &S[0].bar);
                    if (acc_rows) {
                        tma_load_2d(S[0].gA, &tm_gA, 0, row0, &S[0].bar);
                        tma_load_2d(S[0].gB, &tm_gB, 32, row0, &S[0].bar);
                    }
                }
            }
            __syncthreads();
            if (!full && valid) {
                // a partial iteration stages its rows itself, in the same layout
                const float4 *src = reinterpret_cast<const float4 *>(sh + 48LL * i);
#pragma unroll
                for (int c = 0; c < 8; ++c) S[0].shA[swz128(r, c)] = src[c];
#pragma unroll
                for (int c = 0; c < 4; ++c) S[0].shB[swz64(r, c)] = src[8 + c];
            }
            if (GAUSS && !(full && acc_rows)) {
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 *cur = reinterpret_cast<const float4 *>(g_sh + 48LL * i);
                const bool load = acc_rows && valid;
#pragma unroll
                for (int c = 0; c < 8; ++c) S[0].gA[swz128(r, c)] = load ? cur[c] : z;
#pragma unroll
                for (int c = 0; c < 4; ++c) S[0].gB[swz64(r, c)] = load ? cur[8 + c] : z;
            }
        }

        // The Gaussian's parameters are read, and its activations formed, only
        // if some view gives it a nonzero 2D gradient: most Gaussians of a
        // dense scene are hidden behind saturated pixels in every view and
        // only get (zero) gradients written. Otherwise the values below give
        // exact zeros in the gradient formulas.
        float mx = 0.f, my = 0.f, mz = 0.f, sc[3] = {0.f, 0.f, 0.f}, qn[4] = {1.f, 0.f, 0.f, 0.f}, qlen = 1.f;
        float Rq[9], M[9], S00 = 0, S01 = 0, S02 = 0, S11 = 0, S12 = 0, S22 = 0, opac = 0.f;
        bool loaded = false;
        // SH coefficients are read per view where needed (L1-resident or
        // staged), not held in registers
        const float *f = sh + (long long)3 * K * (valid ? i : 0);

        // accumulators over views
        float gm[3] = {0.f, 0.f, 0.f}, go = 0.f;
        float GS00 = 0, GS01 = 0, GS02 = 0, GS11 = 0, GS12 = 0, GS22 = 0;   // full-matrix entries, symmetric
        float *gf = s_gf + (GAUSS && !TMA ? threadIdx.x * GP : 0);
        if (GAUSS && !TMA) {
#pragma unroll
            for (int k = 0; k < 3 * K; ++k) gf[k] = 0.f;
            s_row[threadIdx.x] = valid ? i : -1;
        }
        if constexpr (TMA) {
            if (full) {
                const bool ok = __syncthreads_and(mbar_wait(&S[0].bar, phase));
                phase ^= 1;
                if (!ok) {
                    if (threadIdx.x == 0) {
                        if (status) {
                            atomicCAS(status, 0, GS_ERR_TIMEOUT);
                            atomicExch(status + 1, (int)blockIdx.x);
                        }
                        mbar_wait(&S[0].bar, phase ^ 1);   // give the copy in flight (bounded) time to land
                    }
                    // this block's pose partials are zero, not left from an earlier call
                    for (int e = threadIdx.x; e < nv * 12; e += PB_THREADS)
                        pose_partials[((long long)(e / 12) * gridDim.x + blockIdx.x) * 12 + e % 12] = 0.f;
                    return;
                }
            } else {
                __syncthreads();   // the partial iteration's gradient rows are initialised
            }
        }

        // (listed Gaussians of the compacted path all have a gradient)
        loaded = valid;
        // only the loads are conditional; the activations are formed from the
        // loaded values or from defaults that make every gradient term zero
        float l3[3] = {0.f, 0.f, 0.f}, lg = 0.f;
        float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
        if (loaded) {
            mx = means[3 * i]; my = means[3 * i + 1]; mz = means[3 * i + 2];
#pragma unroll
            for (int a = 0; a < 3; ++a) l3[a] = log_scales[3 * i + a];
            q = reinterpret_cast<const float4 *>(quats)[i];
            lg = logits[i];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) sc[a] = loaded ? expf(l3[a]) : 0.f;
        qlen = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        {
            const float iq = 1.f / qlen;
            qn[0] = q.x * iq; qn[1] = q.y * iq; qn[2] = q.z * iq; qn[3] = q.w * iq;
        }
        opac = loaded ? 1.f / (1.f + expf(-lg)) : 0.f;
        quat_rot(qn[0], qn[1], qn[2], qn[3], Rq);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) M[3 * a + b] = Rq[3 * a + b] * sc[b];
        S00 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
        S01 = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
        S02 = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
        S11 = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
        S12 = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
        S22 = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];

        for (int v = wvb; v < wve; ++v) {
            float pg[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) pg[c] = 0.f;
            bool contrib = false;
            if (v >= vb && v < ve) {
                const long long slot = L.v[v].slot_base + li;
                const bool staged = TMA && full && v == v_first;
                const float4 ga4 = staged ? S[0].g2d[3 * r] : grad2d[3 * slot];
                const float4 gb4 = staged ? S[0].g2d[3 * r + 1] : grad2d[3 * slot + 1];
                const float4 gc4 = staged ? S[0].g2d[3 * r + 2] : grad2d[3 * slot + 2];
                contrib = ga4.x != 0.f || ga4.y != 0.f || ga4.z != 0.f || ga4.w != 0.f || gb4.x != 0.f ||
                          gb4.y != 0.f || gb4.z != 0.f || gb4.w != 0.f || gc4.x != 0.f;
                if (contrib) {
                    const float gx = ga4.x, gy = ga4.y, gsa = ga4.z, gsb = ga4.w, gsc = gb4.x, gop = gb4.y;
                    const float grgb[3] = {gb4.z, gb4.w, gc4.x};
                    const int clamp_bits = __float_as_int(proj[4 * slot + 3].w);
                    const ViewDesc &vd = L.v[v];
                    const float *vm = viewmats + 12 * v;
                    float R[9], t[3];
#pragma unroll
                    for (int a = 0; a < 9; ++a) R[a] = __ldg(vm + a);
#pragma unroll
                    for (int a = 0; a < 3; ++a) t[a] = __ldg(vm + 9 + a);
                    const float fx = __ldg(intr + 4 * v), fy = __ldg(intr + 4 * v + 1);
                    const float x = R[0] * mx + R[1] * my + R[2] * mz + t[0];
                    const float y = R[3] * mx + R[4] * my + R[5] * mz + t[1];
                    const float z = R[6] * mx + R[7] * my + R[8] * mz + t[2];
                    const float limx = L.fov_clamp * 0.5f * (float)vd.W / fx;
                    const float limy = L.fov_clamp * 0.5f * (float)vd.H / fy;
                    const float iz = 1.f / z, iz2 = iz * iz;
                    const float ur = x * iz, wr = y * iz;
                    const bool u_in = ur >= -limx && ur <= limx, w_in = wr >= -limy && wr <= limy;
                    const float u = fminf(fmaxf(ur, -limx), limx), w = fminf(fmaxf(wr, -limy), limy);
                    const float J00 = fx * iz, J02 = -fx * u * iz, J11 = fy * iz, J12 = -fy * w * iz;
                    float T[6];
                    T[0] = J00 * R[0] + J02 * R[6]; T[1] = J00 * R[1] + J02 * R[7]; T[2] = J00 * R[2] + J02 * R[8];
                    T[3] = J11 * R[3] + J12 * R[6]; T[4] = J11 * R[4] + J12 * R[7]; T[5] = J11 * R[5] + J12 * R[8];
                    float TS[6];   // T Sigma
                    TS[0] = T[0] * S00 + T[1] * S01 + T[2] * S02;
                    TS[1] = T[0] * S01 + T[1] * S11 + T[2] * S12;
                    TS[2] = T[0] * S02 + T[1] * S12 + T[2] * S22;
                    TS[3] = T[3] * S00 + T[4] * S01 + T[5] * S02;
                    TS[4] = T[3] * S01 + T[4] * S11 + T[5] * S12;
                    TS[5] = T[3] * S02 + T[4] * S12 + T[5] * S22;

                    go += gop;

                    // colour -> SH and view direction
                    const float Cx = -(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]);
                    const float Cy = -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]);
                    const float Cz = -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]);
                    const float dxv = mx - Cx, dyv = my - Cy, dzv = mz - Cz;
                    const float idl = rsqrtf(dxv * dxv + dyv * dyv + dzv * dzv);
                    const float d0 = dxv * idl, d1 = dyv * idl, d2 = dzv * idl;
                    float graw[3];
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) graw[ch] = (clamp_bits >> ch) & 1 ? 0.f : grgb[ch];
                    float gC3[3] = {0.f, 0.f, 0.f};
                    if (DEG > 0 || GAUSS) {
                        float Yb[16];
                        sh_basis<DEG>(d0, d1, d2, Yb);
                        float gY[16];
#pragma unroll
                        for (int k = 0; k < K; ++k) gY[k] = 0.f;
                        if (TMA) {
#pragma unroll
                            for (int j = 0; j < 12; ++j) {
                                const float4 q4 = j < 8 ? S[0].shA[swz128(r, j)] : S[0].shB[swz64(r, j - 8)];
                                const float fv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e) gY[(4 * j + e) / 3] += fv[e] * graw[(4 * j + e) % 3];
                            }
                        } else if (DEG == 1 || DEG == 3) {
                            // 3K floats = 3K/4 float4 (rows are 16-byte aligned for these degrees)
                            const float4 *f4 = reinterpret_cast<const float4 *>(f);
#pragma unroll
                            for (int j = 0; j < 3 * K / 4; ++j) {
                                const float4 q4 = __ldg(f4 + j);
                                const float fv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e) gY[(4 * j + e) / 3] += fv[e] * graw[(4 * j + e) % 3];
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < K; ++k)
                                gY[k] = __ldg(f + 3 * k) * graw[0] + __ldg(f + 3 * k + 1) * graw[1] +
                                        __ldg(f + 3 * k + 2) * graw[2];
                        }
                        if (GAUSS && TMA) {
#pragma unroll
                            for (int j = 0; j < 12; ++j) {
                                float4 &gq = j < 8 ? S[0].gA[swz128(r, j)] : S[0].gB[swz64(r, j - 8)];
                                float4 t = gq;
                                t.x += Yb[(4 * j) / 3] * graw[(4 * j) % 3];
                                t.y += Yb[(4 * j + 1) / 3] * graw[(4 * j + 1) % 3];
                                t.z += Yb[(4 * j + 2) / 3] * graw[(4 * j + 2) % 3];
                                t.w += Yb[(4 * j + 3) / 3] * graw[(4 * j + 3) % 3];
                                gq = t;
                            }
                        } else if (GAUSS) {
#pragma unroll
                            for (int k = 0; k < K; ++k) {
                                gf[3 * k] += Yb[k] * graw[0];
                                gf[3 * k + 1] += Yb[k] * graw[1];
                                gf[3 * k + 2] += Yb[k] * graw[2];
                            }
                        }
                        if (DEG > 0) {
                            float gdx, gdy, gdz;
                            sh_basis_vjp<DEG>(d0, d1, d2, gY, gdx, gdy, gdz);
                            const float dg = d0 * gdx + d1 * gdy + d2 * gdz;
                            const float gdir0 = (gdx - d0 * dg) * idl, gdir1 = (gdy - d1 * dg) * idl,
                                        gdir2 = (gdz - d2 * dg) * idl;
                            gm[0] += gdir0; gm[1] += gdir1; gm[2] += gdir2;
                            gC3[0] = -gdir0; gC3[1] = -gdir1; gC3[2] = -gdir2;
                        }
                    }
                    // C = -R^T t: dL/dR[a][b] += -t_a gC_b, dL/dt_a += -sum_b R[a][b] gC_b
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) {
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) pg[3 * aa + bb] += -t[aa] * gC3[bb];
                        pg[9 + aa] += -(R[3 * aa] * gC3[0] + R[3 * aa + 1] * gC3[1] + R[3 * aa + 2] * gC3[2]);
                    }

                    // grad2d carries dL/d(a, b, c) of the dilated covariance directly
                    const float P00 = gsa, P01 = 0.5f * gsb, P11 = gsc;   // symmetric full-matrix gradient
                    // dL/dT = 2 P T Sigma
                    float GT[6];
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        GT[cc] = 2.f * (P00 * TS[cc] + P01 * TS[3 + cc]);
                        GT[3 + cc] = 2.f * (P01 * TS[cc] + P11 * TS[3 + cc]);
                    }
                    if (GAUSS) {
                        // dL/dSigma = T^T P T
                        float PT[6];
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) {
                            PT[cc] = P00 * T[cc] + P01 * T[3 + cc];
                            PT[3 + cc] = P01 * T[cc] + P11 * T[3 + cc];
                        }
                        GS00 += T[0] * PT[0] + T[3] * PT[3];
                        GS01 += T[0] * PT[1] + T[3] * PT[4];
                        GS02 += T[0] * PT[2] + T[3] * PT[5];
                        GS11 += T[1] * PT[1] + T[4] * PT[4];
                        GS12 += T[1] * PT[2] + T[4] * PT[5];
                        GS22 += T[2] * PT[2] + T[5] * PT[5];
                    }
                    // T = J R: dL/dJ = GT R^T, dL/dR += J^T GT
                    const float GJ00 = GT[0] * R[0] + GT[1] * R[1] + GT[2] * R[2];
                    const float GJ02 = GT[0] * R[6] + GT[1] * R[7] + GT[2] * R[8];
                    const float GJ11 = GT[3] * R[3] + GT[4] * R[4] + GT[5] * R[5];
                    const float GJ12 = GT[3] * R[6] + GT[4] * R[7] + GT[5] * R[8];
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        pg[cc] += J00 * GT[cc];
                        pg[3 + cc] += J11 * GT[3 + cc];
                        pg[6 + cc] += J02 * GT[cc] + J12 * GT[3 + cc];
                    }
                    float gmc0 = 0.f, gmc1 = 0.f, gmc2 = 0.f;
                    gmc2 += GJ00 * (-fx * iz2) + GJ02 * (fx * u * iz2) + GJ11 * (-fy * iz2) + GJ12 * (fy * w * iz2);
                    const float gu = GJ02 * (-fx * iz), gw = GJ12 * (-fy * iz);
                    if (u_in) { gmc0 += gu * iz; gmc2 += -gu * x * iz2; }
                    if (w_in) { gmc1 += gw * iz; gmc2 += -gw * y * iz2; }
                    gmc0 += gx * fx * iz;
                    gmc2 += -gx * fx * x * iz2;
                    gmc1 += gy * fy * iz;
                    gmc2 += -gy * fy * y * iz2;
                    // m = R mu + t
                    gm[0] += R[0] * gmc0 + R[3] * gmc1 + R[6] * gmc2;
                    gm[1] += R[1] * gmc0 + R[4] * gmc1 + R[7] * gmc2;
                    gm[2] += R[2] * gmc0 + R[5] * gmc1 + R[8] * gmc2;
                    const float gmc[3] = {gmc0, gmc1, gmc2};
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) {
                        pg[3 * aa] += gmc[aa] * mx;
                        pg[3 * aa + 1] += gmc[aa] * my;
                        pg[3 * aa + 2] += gmc[aa] * mz;
                        pg[9 + aa] += gmc[aa];
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int cc = 0; cc < 12; ++cc) {
                    float val = pg[cc];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                    pg[cc] = val;
                }
                if (lane == 0) {
#pragma unroll
                    for (int cc = 0; cc < 12; ++cc) s_pose[(wid * nv + v) * 12 + cc] += pg[cc];
                }
            }
        }

        // (with accumulation a Gaussian without a gradient has nothing to add)
        if (valid && GAUSS && (loaded || !L.accumulate)) {
            // Sigma = M M^T: dL/dM = 2 GS M (GS symmetric)
            const float GSf[9] = {GS00, GS01, GS02, GS01, GS11, GS12, GS02, GS12, GS22};
            float gs[3] = {0.f, 0.f, 0.f}, GRq[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    const float GM = 2.f * (GSf[3 * r] * M[cc] + GSf[3 * r + 1] * M[3 + cc] + GSf[3 * r + 2] * M[6 + cc]);
                    gs[cc] += GM * Rq[3 * r + cc];
                    GRq[3 * r + cc] = GM * sc[cc];
                }
            const bool acc = L.accumulate;
            put(g_log_scales + 3 * i, gs[0] * sc[0], acc);
            put(g_log_scales + 3 * i + 1, gs[1] * sc[1], acc);
            put(g_log_scales + 3 * i + 2, gs[2] * sc[2], acc);
            // rotation of (w,x,y,z) -> quaternion gradient
            const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
            const float gw = 2.f * (-z * GRq[1] + y * GRq[2] + z * GRq[3] - x * GRq[5] - y * GRq[6] + x * GRq[7]);
            const float gxq = 2.f * (y * GRq[1] + z * GRq[2] + y * GRq[3] - 2.f * x * GRq[4] - w * GRq[5] +
                                     z * GRq[6] + w * GRq[7] - 2.f * x * GRq[8]);
            const float gyq = 2.f * (-2.f * y * GRq[0] + x * GRq[1] + w * GRq[2] + x * GRq[3] + z * GRq[5] -
                                     w * GRq[6] + z * GRq[7] - 2.f * y * GRq[8]);
            const float gzq = 2.f * (-2.f * z * GRq[0] - w * GRq[1] + x * GRq[2] + w * GRq[3] - 2.f * z * GRq[4] +
                                     y * GRq[5] + x * GRq[6] + y * GRq[7]);
            const float dq = gw * w + gxq * x + gyq * y + gzq * z;
            const float iq = 1.f / qlen;
            float4 gq = make_float4((gw - w * dq) * iq, (gxq - x * dq) * iq, (gyq - y * dq) * iq, (gzq - z * dq) * iq);
            if (acc) {
                const float4 o = reinterpret_cast<const float4 *>(g_quats)[i];
                gq = make_float4(o.x + gq.x, o.y + gq.y, o.z + gq.z, o.w + gq.w);
            }
            reinterpret_cast<float4 *>(g_quats)[i] = gq;
            put(g_means + 3 * i, gm[0], acc);
            put(g_means + 3 * i + 1, gm[1], acc);
            put(g_means + 3 * i + 2, gm[2], acc);
            put(g_logits + i, go * opac * (1.f - opac), acc);
        }
        if constexpr (GAUSS && TMA) {
            if (full) {
                // the block's SH-coefficient gradient rows leave as two boxes
                fence_async_smem();
                __syncthreads();
                if (threadIdx.x == 0) {
                    tma_store_2d(&tm_gA, S[0].gA, 0, row0);
                    tma_store_2d(&tm_gB, S[0].gB, 32, row0);
                    bulk_commit();
                }
            } else {
                if (valid) {
                    float4 *dst = reinterpret_cast<float4 *>(g_sh + 48LL * i);
#pragma unroll
                    for (int c = 0; c < 8; ++c) dst[c] = S[0].gA[swz128(r, c)];
#pragma unroll
                    for (int c = 0; c < 4; ++c) dst[8 + c] = S[0].gB[swz64(r, c)];
                }
                __syncthreads();
            }
        } else if constexpr (GAUSS) {
            // the block's SH-coefficient gradients: row r goes to Gaussian s_row[r]
            __syncthreads();
            for (int e = threadIdx.x; e < PB_THREADS * 3 * K; e += PB_THREADS) {
                const int rr = e / (3 * K), c = e % (3 * K);
                const long long row = s_row[rr];
                if (row >= 0) put(g_sh + row * 3 * K + c, s_gf[rr * GP + c], L.accumulate);
            }
            __syncthreads();
        } else if constexpr (TMA) {
            __syncthreads();   // the staged SH rows are free for the next iteration
        }
    }
    if (TMA && GAUSS && threadIdx.x == 0) bulk_wait_read_all();
    __syncthreads();
    for (int e = threadIdx.x; e < nv * 12; e += PB_THREADS) {
        const int v = e / 12, cc = e % 12;
        float acc = 0.f;
#pragma unroll
        for (int ww = 0; ww < PB_WARPS; ++ww) acc += s_pose[(ww * nv + v) * 12 + cc];
        pose_partials[((long long)v * gridDim.x + blockIdx.x) * 12 + cc] = acc;
    }
}

int pose_blocks(long long n) {
    long long b = (n + PB_THREADS - 1) / PB_THREADS;
    const long long cap = 4LL * num_sms();   // one wave of resident blocks
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

int launch_project_bwd(const Launch &L, int deg, const gs_gaussians *g, const float *viewmats, const float *intr,
                       const float *proj, const float *grad2d, const gs_grads *out, int want_gauss, int nblk,
                       int32_t *status, cudaStream_t st) {
    const float4 *p = reinterpret_cast<const float4 *>(proj);
    const float4 *g2 = reinterpret_cast<const float4 *>(grad2d);
    const size_t dyn = (size_t)PB_WARPS * L.n_views * 12 * sizeof(float);
    CUtensorMap ma, mb, ga, gb, m2;
    memset(&ma, 0, sizeof ma); memset(&mb, 0, sizeof mb); memset(&ga, 0, sizeof ga); memset(&gb, 0, sizeof gb);
    memset(&m2, 0, sizeof m2);
    // one-view calls run the chain over the Gaussians with a nonzero 2D
    // gradient only (see COMPACT); each block zeroes its range's rows first
    const bool compact = L.n_views == 1;
    // several views, degree 3 with 16-byte aligned SH rows and gradient rows:
    // the staged path, unless the configuration turns tensor copies off. The
    // pose-only backward reads SH rows only for Gaussians with a nonzero 2D
    // gradient, which the per-thread path does (measured faster there: 46 vs
    // 63 us at 1M Gaussians)
    bool tma = !compact && want_gauss && deg == 3 && L.use_tma && ((uintptr_t)g->sh & 15u) == 0 &&
               g->n < 0x7fffffffLL &&
               encode_tmap_2d(&ma, g->sh, 48, (uint64_t)g->n, 192, 32, PB_THREADS, CU_TENSOR_MAP_SWIZZLE_128B) &&
               encode_tmap_2d(&mb, g->sh, 48, (uint64_t)g->n, 192, 16, PB_THREADS, CU_TENSOR_MAP_SWIZZLE_64B);
    if (tma)
        tma = L.n_slots < 0x7fffffffLL &&
              encode_tmap_2d(&m2, grad2d, 12, (uint64_t)L.n_slots, 48, 12, PB_THREADS, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (tma && want_gauss)
        tma = ((uintptr_t)out->sh & 15u) == 0 &&
              encode_tmap_2d(&ga, out->sh, 48, (uint64_t)g->n, 192, 32, PB_THREADS, CU_TENSOR_MAP_SWIZZLE_128B) &&
              encode_tmap_2d(&gb, out->sh, 48, (uint64_t)g->n, 192, 16, PB_THREADS, CU_TENSOR_MAP_SWIZZLE_64B);
#define GS_PB(D, G, T, Z)                                                                                          \
    k_project_bwd<D, G, T, Z><<<nblk, PB_THREADS, dyn, st>>>(                                                      \
        L, g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, viewmats, intr, p, g2, out->means,        \
        out->log_scales, out->quats, out->opacity_logits, out->sh, out->pose_partials, ma, mb, ga, gb, m2, status)
    if (want_gauss) {
        switch (deg) {
        case 0: if (compact) GS_PB(0, true, false, true); else GS_PB(0, true, false, false); break;
        case 1: if (compact) GS_PB(1, true, false, true); else GS_PB(1, true, false, false); break;
        case 2: if (compact) GS_PB(2, true, false, true); else GS_PB(2, true, false, false); break;
        case 3:
            if (compact) GS_PB(3, true, false, true);
            else if (tma) GS_PB(3, true, true, false);
            else GS_PB(3, true, false, false);
            break;
        default: return GS_ERR_UNSUPPORTED;
        }
    } else {
        // the pose-only backward reads a Gaussian's parameters only in its
        // contributing views already (per-thread path)
        switch (deg) {
        case 0: if (compact) GS_PB(0, false, false, true); else GS_PB(0, false, false, false); break;
        case 1: if (compact) GS_PB(1, false, false, true); else GS_PB(1, false, false, false); break;
        case 2: if (compact) GS_PB(2, false, false, true); else GS_PB(2, false, false, false); break;
        case 3: if (compact) GS_PB(3, false, false, true); else GS_PB(3, false, false, false); break;
        default: return GS_ERR_UNSUPPORTED;
        }
    }
#undef GS_PB
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// pose partials -> dL/d(R,t) and the left-twist gradient, fixed order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_pose_reduce(const float *__restrict__ partials, int nblk,
                                                     const float *__restrict__ viewmats, float *__restrict__ out_rt,
                                                     float *__restrict__ out_twist) {
    __shared__ float s[12][256];
    const int v = blockIdx.x;
    float acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = 0.f;
    for (int b = threadIdx.x; b < nblk; b += 256)
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] += partials[((long long)v * nblk + b) * 12 + c];
#pragma unroll
    for (int c = 0; c < 12; ++c) s[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int c = 0; c < 12; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float g[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            g[c] = s[c][0];
            out_rt[12 * v + c] = g[c];
        }
        if (out_twist) {
            const float *R = viewmats + 12 * v, *t = viewmats + 12 * v + 9;
            // M = dL/dR R^T + dL/dt t^T
            float Mm[9];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    Mm[3 * a + b] = g[3 * a] * R[3 * b] + g[3 * a + 1] * R[3 * b + 1] + g[3 * a + 2] * R[3 * b + 2] +
                                    g[9 + a] * t[b];
            out_twist[6 * v + 0] = g[9];
            out_twist[6 * v + 1] = g[10];
            out_twist[6 * v + 2] = g[11];
            out_twist[6 * v + 3] = Mm[7] - Mm[5];
            out_twist[6 * v + 4] = Mm[2] - Mm[6];
            out_twist[6 * v + 5] = Mm[3] - Mm[1];
        }
    }
}

int launch_pose_reduce(int n_views, const float *partials, int nblk, const float *viewmats, float *out_rt,
                       float *out_twist, cudaStream_t st) {
    k_pose_reduce<<<n_views, 256, 0, st>>>(partials, nblk, viewmats, out_rt, out_twist);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// mean L1 loss and its gradient
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_l1(const float4 *__restrict__ img, const float4 *__restrict__ tgt,
                                            long long n4, const float *__restrict__ img1,
                                            const float *__restrict__ tgt1, long long n, float inv_n,
                                            float4 *__restrict__ grad4, float *__restrict__ grad1,
                                            float *__restrict__ loss) {
    __shared__ float s_w[8];
    float acc = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 a = img[i], b = tgt[i];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        grad4[i] = make_float4(d0 > 0.f ? inv_n : (d0 < 0.f ? -inv_n : 0.f), d1 > 0.f ? inv_n : (d1 < 0.f ? -inv_n : 0.f),
                               d2 > 0.f ? inv_n : (d2 < 0.f ? -inv_n : 0.f), d3 > 0.f ? inv_n : (d3 < 0.f ? -inv_n : 0.f));
    }
    for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const float d = img1[i] - tgt1[i];
        acc += fabsf(d);
        grad1[i] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        atomicAdd(loss, t * inv_n);
    }
}

int launch_l1(const float *image, const float *target, long long n, float *loss, float *grad, cudaStream_t st) {
    if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return GS_ERR_CUDA;
    if (n == 0) return GS_OK;
    const bool al = ((uintptr_t)image % 16 == 0) && ((uintptr_t)target % 16 == 0) && ((uintptr_t)grad % 16 == 0);
    const long long n4 = al ? n / 4 : 0;
    long long blocks = (n + 1023) / 1024;
    if (blocks > 8LL * num_sms()) blocks = 8LL * num_sms();
    // grad4 and grad1 view the same buffer but address disjoint ranges (the
    // float4 body [0, 4 n4) and the scalar tail [4 n4, n)), as do img/img1
    // and tgt/tgt1, so the restrict qualifiers hold
    k_l1<<<(int)blocks, 256, 0, st>>>(reinterpret_cast<const float4 *>(image), reinterpret_cast<const float4 *>(target),
                                      n4, image, target, n, 1.f / (float)n, reinterpret_cast<float4 *>(grad), grad,
                                      loss);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gsk
