// Front-to-back alpha compositing (forward) and its recompute-T backward.
//
// Section 3.1: a pixel's colour is the alpha blend of the depth-sorted
// Gaussians covering it, c_p = sum_i c_i alpha_i T_i + T_final bg with
// T_i = prod_{j<i} (1 - alpha_j). Per Gaussian and pixel:
//   alpha = min(alpha_max, o exp(-1/2 d^T conic d)), skipped if the exponent
//   is > 0 or alpha < alpha_min, and (pixel gate) if |dx| or |dy| > radius;
//   the Gaussian that would bring T (1 - alpha) below t_min is not composited
//   and the pixel stops.
//
// Both kernels are persistent: blocks pull tiles from an atomic queue over
// tile_order (largest tiles first). Each thread owns two pixels and each warp
// an 8x8-pixel patch of the tile; a tile's instances are staged through
// shared memory in batches (the number per thread chosen at launch: by
// default two in the forward, one in the backward), and a warp skips every
// staged Gaussian that cannot reach its patch.
//
// The backward does not store or replay transmittance: it walks the same list
// front to back with bit-identical arithmetic (explicit-rounding intrinsics,
// so forward and backward take the same decisions), and gets the colour of
// everything behind Gaussian i from the forward image,
//   S_i = sum_{j>i} c_j alpha_j T_j + T_final bg = image - sum_{j<=i} c_j alpha_j T_j,
// so that dL/dalpha_i = T_i (c_i . g) - (S_i . g) / (1 - alpha_i).
// Per-Gaussian gradients (mean2D, 2D covariance, opacity, colour) are summed over a
// warp through a shared-memory transpose: a warp writes the 9 values of up to
// three consecutive visits as rows of a per-warp buffer (one column per lane),
// then 27 lanes each add one row with 16-byte loads; then over the block in
// shared memory, and into the per-slot grad2d record with one vector atomic
// per float4.
// Both kernels run a thread's two pixels through packed float2 arithmetic
// (f32x2 fma/mul/add, one instruction for both), branch-free: a pixel that
// does not composite a Gaussian contributes zeros.
#include "gs_common.cuh"

namespace gsk {


// Staged instance: xy = mean relative to the block origin and the reach
// half-extents (ext_x, ext_y <= radius, so the test |dx| <= ext_x, |dy| <=
// ext_y implies the radius gate and rejects only pixels whose alpha is below
// alpha_min anyway); con = quadratic-form coefficients and opacity; rgb =
// colour and the slot.
//
// The exponent -1/2 d^T conic d is evaluated as the sum of two non-negative
// terms, -1/2 [A u^2 + dy^2 / c] with u = dx - (b/c) dy and A = c / det (the
// conditional x|y and marginal y parts of the 2D Gaussian with covariance
// (a, b, c)). The expanded form A dx^2 + 2B dx dy + C dy^2 cancels badly for
// elongated Gaussians far along their long axis (a factor ~100 in float32);
// this one does not, at the same five operations per pixel.
__device__ __forceinline__ void stage(const float4 *__restrict__ proj, unsigned int slot, float ox, float oy,
                                      float4 &xy, float4 &con, float4 &rgb) {
    const float4 r0 = proj[4ull * slot];
    const float4 r1 = proj[4ull * slot + 1];
    const float4 r2 = proj[4ull * slot + 2];
    const float4 r3 = proj[4ull * slot + 3];
    xy = make_float4(__fadd_rn(__fsub_rn(r0.x, ox), r3.x), __fadd_rn(__fsub_rn(r0.y, oy), r3.y), r0.z, r0.w);
    con = r1;   // the conic in the staged form, written by the projection
    rgb = make_float4(r2.x, r2.y, r2.z, __uint_as_float(slot));
}

// alpha of a staged Gaussian at a pixel (the forward and the backward share
// this arithmetic and so take identical decisions): with dx = pcx - x,
// dy = pcy - y (block-relative pixel centre minus mean),
//   gate   |dx| <= ext_x and |dy| <= ext_y (the column test is shared by a
//          thread's two pixels, which lie in one column),
//   u = dx + beta dy, p2 = Ah u^2 + Dh dy^2 (base 2; never positive: Ah, Dh < 0
//          for every staged, positive-definite conic, so no guard),
//   G = 2^p2, alpha = min(alpha_max, o G) ("clamped" if o G > alpha_max),
//   skipped if alpha < alpha_min.

// Packed pair arithmetic (sm_100+ f32x2): a thread's two pixels run through
// one instruction stream, lane .x = pixel (px, py0), lane .y = pixel
// (px, py0 + 4). Each lane of a packed operation is the IEEE-rounded scalar
// operation, so the backward reproduces the forward's scalar alpha and
// transmittance bit for bit.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct TileInfo {
    int view;
    int px, py0;      // this thread's pixels: (px, py0) and (px, py0 + 4)
    float ox, oy;     // origin of the enclosing 32x32-pixel block
    float pcx, pcy0;  // pixel centres relative to the block origin (second pixel: pcy0 + 4)
    float tbx, tby;   // tile origin relative to the block origin
    bool in0, in1;    // pixels inside the image
};

// Pixels: warp w covers the 8x8 patch (w % (TW/8), w / (TW/8)) of the tile;
// lane l owns column l & 7 and rows (l >> 3) and (l >> 3) + 4 of the patch.
// Positions are relative to the enclosing 32x32-pixel block (every supported
// tile nests in one), so a pixel's arithmetic is the same for every tile
// shape and the image is bit-identical across shapes.
template <int TW, int TH>
__device__ __forceinline__ TileInfo tile_info(const Launch &L, int tile) {
    TileInfo ti;
    ti.view = view_of_tile(L, tile);
    const ViewDesc &vd = L.v[ti.view];
    const int lt = tile - vd.tile_base;
    const int tx = lt % vd.Gx, ty = lt / vd.Gx;
    const int w = (int)threadIdx.x >> 5, l = (int)threadIdx.x & 31;
    ti.px = tx * TW + (w % (TW / 8)) * 8 + (l & 7);
    ti.py0 = ty * TH + (w / (TW / 8)) * 8 + (l >> 3);
    const int bx = (tx * TW) & ~31, by = (ty * TH) & ~31;
    ti.ox = (float)bx;
    ti.oy = (float)by;
    ti.pcx = (float)(ti.px - bx) + 0.5f;
    ti.pcy0 = (float)(ti.py0 - by) + 0.5f;
    ti.tbx = (float)(tx * TW - bx);
    ti.tby = (float)(ty * TH - by);
    ti.in0 = ti.px < vd.W && ti.py0 < vd.H;
    ti.in1 = ti.px < vd.W && ti.py0 + 4 < vd.H;
    return ti;
}

// Bit w set if the staged Gaussian may reach warp w's 8x8 patch. Two
// conservative tests (the per-pixel test still decides exactly):
//  * the reach box |dx| <= ext_x, |dy| <= ext_y overlaps the patch (box
//    enlarged by 1e-3 px against float rounding);
//  * the exponent can reach log2(alpha_min / o) somewhere in the patch: with
//    u = dx + beta dy, the base-2 exponent Ah u^2 + Dh dy^2 (Ah, Dh < 0) is at
//    most Ah umin^2 + Dh dymin^2, where umin and dymin are the smallest |u|
//    and |dy| over the patch (u ranges over the patch's dx interval shifted
//    by beta times its dy interval). A 1e-3 margin keeps the test safe.
template <int TW, int TH>
__device__ __forceinline__ unsigned int warp_mask(const float4 &xy, const float4 &con, float alpha_min, float tbx,
                                                  float tby) {
    constexpr int WX = TW / 8, WY = TH / 8;
    const float ex = xy.z + 1e-3f, ey = xy.w + 1e-3f;
    const float lim = __log2f(alpha_min / con.w) - 1e-3f;
    float dxlo[WX], dylo[WY], bmin[WY], bmax[WY], dy2[WY];
#pragma unroll
    for (int c = 0; c < WX; ++c) dxlo[c] = tbx + (float)(c * 8) + 0.5f - xy.x;
#pragma unroll
    for (int r = 0; r < WY; ++r) {
        dylo[r] = tby + (float)(r * 8) + 0.5f - xy.y;
        const float b0 = con.y * dylo[r], b1 = con.y * (dylo[r] + 7.f);
        bmin[r] = fminf(b0, b1);
        bmax[r] = fmaxf(b0, b1);
        const float dm = fmaxf(0.f, fmaxf(dylo[r], -(dylo[r] + 7.f)));
        dy2[r] = con.z * dm * dm;
    }
    unsigned int m = 0;
#pragma unroll
    for (int w = 0; w < WX * WY; ++w) {
        const int c = w % WX, r = w / WX;
        const bool box = dxlo[c] <= ex && dxlo[c] + 7.f >= -ex && dylo[r] <= ey && dylo[r] + 7.f >= -ey;
        const float ulo = dxlo[c] + bmin[r], uhi = dxlo[c] + 7.f + bmax[r];
        const float um = fmaxf(0.f, fmaxf(ulo, -uhi));
        const bool reach = con.x * um * um + dy2[r] >= lim;
        m |= (unsigned int)(box && reach) << w;
    }
    return m;
}

// add a thread's pair counts to the 64-bit counters at counters + at (one atomic per warp)
__device__ __forceinline__ void count_pairs(int *counters, int at, unsigned int n_eval, unsigned int n_comp) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
        n_comp += __shfl_xor_sync(0xffffffffu, n_comp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *c = reinterpret_cast<unsigned long long *>(counters + at);
        atomicAdd(c, (unsigned long long)n_eval);
        atomicAdd(c + 1, (unsigned long long)n_comp);
    }
}

// Stage instances [b0, min(b0 + per BS, end)) of a tile: per (1, 2 or 4)
// per thread, the batch size chosen at launch.
template <int TW, int TH>
__device__ __forceinline__ void stage_batch(const Launch &L, const float4 *__restrict__ proj,
                                            const unsigned int *__restrict__ ids, int b0, int end, int per,
                                            const TileInfo &ti, float4 *s_xy, float4 *s_con, float4 *s_rgb,
                                            unsigned int *s_mask) {
    constexpr int BS = TW * TH / 2;
    for (int h = 0; h < per; ++h) {
        const int k = threadIdx.x + h * BS;
        if (b0 + k < end) {
            stage(proj, ids[b0 + k], ti.ox, ti.oy, s_xy[k], s_con[k], s_rgb[k]);
            s_mask[k] = warp_mask<TW, TH>(s_xy[k], s_con[k], L.alpha_min, ti.tbx, ti.tby);
        }
    }
}

// Shared-memory bytes of one staged Gaussian: position, conic and colour
// (3 x 16 B) and the warp mask; the backward adds the conic's natural-log
// terms (8 B) and the per-Gaussian gradient sums (9 floats).
constexpr int FWD_STAGE_BYTES = 52;
constexpr int BWD_STAGE_BYTES = 96;
// The backward's per-warp reduction buffer: RED_SLOTS visits x 9 values as
// rows of 32 lane columns, row pitch RED_PITCH floats (16-byte aligned rows;
// the 4-float pad puts the 8 lanes of a quarter-warp reading 16 bytes of 8
// different rows on 8 disjoint groups of 4 banks).
constexpr int RED_SLOTS = 3;
constexpr int RED_PITCH = 36;
constexpr int RED_WARP_FLOATS = RED_SLOTS * 9 * RED_PITCH;

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2) k_render_fwd(const Launch L, const float4 *__restrict__ proj,
                                                            const int2 *__restrict__ ranges,
                                                            const unsigned int *__restrict__ ids,
                                                            const int *__restrict__ order, int *__restrict__ counters,
                                                            float *__restrict__ image, int *__restrict__ last_contrib,
                                                            int *__restrict__ tile_work) {
    // the staged batch (L.fwd_batch Gaussians per thread) in dynamic shared memory
    constexpr int BS = TW * TH / 2;
    const int NB = L.fwd_batch * BS;
    extern __shared__ float4 s_dyn[];
    float4 *s_xy = s_dyn, *s_con = s_xy + NB, *s_rgb = s_con + NB;
    unsigned int *s_mask = reinterpret_cast<unsigned int *>(s_rgb + NB);
    __shared__ int s_item, s_end;
    // the backward's accumulators that follow (zeroed by a programmatic
    // dependent) may be cleared on SMs this kernel leaves in its tail
    launch_dependents();
    const bool abort = counters[CNT_ABORT] != 0;
    const unsigned int wbit = 1u << (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    int prev_tile = -1;   // (thread 0) the tile whose replay length s_end holds
    if (threadIdx.x == 0) s_end = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counters + CNT_Q_FWD, 1);
        __syncthreads();
        const int item = s_item;
        if (tile_work && threadIdx.x == 0) {
            // every warp has added the previous tile's length before the barrier
            if (prev_tile >= 0) tile_work[prev_tile] = s_end;
            s_end = 0;
        }
        __syncthreads();
        if (item >= L.n_tiles) break;
        const int tile = order[item];
        const TileInfo ti = tile_info<TW, TH>(L, tile);
        const int2 r = abort ? make_int2(0, 0) : ranges[tile];
        // lane .x = pixel (px, py0), lane .y = pixel (px, py0 + 4)
        float2 T = f2(1.f), CR = f2(0.f), CG = f2(0.f), CB = f2(0.f);
        // per pixel the alpha threshold it still composites at: alpha_min,
        // or +inf once the pixel has stopped (or lies outside the image), so
        // that the alpha test also excludes stopped pixels
        const float amin = L.alpha_min, INF = __int_as_float(0x7f800000);
        float am0 = ti.in0 ? amin : INF, am1 = ti.in1 ? amin : INF;
        int end0 = r.x, end1 = r.x;   // one past the last composited instance
        const float2 PCY = make_float2(ti.pcy0, ti.pcy0 + 4.f);
        for (int b0 = r.x; b0 < r.y; b0 += NB) {
            if (__syncthreads_count(am0 == INF && am1 == INF) == BS) break;
            stage_batch<TW, TH>(L, proj, ids, b0, r.y, L.fwd_batch, ti, s_xy, s_con, s_rgb, s_mask);
            __syncthreads();
            const int nb = min(NB, r.y - b0);
            // the warp walks only the staged Gaussians that may reach its patch:
            // 32 masks per ballot, then the set bits in order
            for (int k0 = 0; k0 < nb; k0 += 32) {
                if (__all_sync(0xffffffffu, am0 == INF && am1 == INF)) break;
                unsigned int hits = __ballot_sync(0xffffffffu, k0 + lane < nb && (s_mask[k0 + lane] & wbit));
                while (hits) {
                    const int k = k0 + __ffs(hits) - 1;
                    hits &= hits - 1;
                    const float4 xy = s_xy[k], con = s_con[k];
                    const float dx = __fsub_rn(ti.pcx, xy.x);
                    const bool col = fabsf(dx) <= xy.z;   // the column gate, shared by both pixels
                    const float2 dy = __fadd2_rn(PCY, f2(-xy.y));
                    const float2 u = __ffma2_rn(f2(con.y), dy, f2(dx));
                    const float2 p2 = __ffma2_rn(f2(con.x), __fmul2_rn(u, u), __fmul2_rn(f2(con.z), __fmul2_rn(dy, dy)));
                    const float2 oG = __fmul2_rn(f2(con.w), make_float2(ex2_approx(p2.x), ex2_approx(p2.y)));
                    const float a0 = fminf(oG.x, L.alpha_max), a1 = fminf(oG.y, L.alpha_max);
                    const bool ok0 = col && fabsf(dy.x) <= xy.w && a0 >= am0;
                    const bool ok1 = col && fabsf(dy.y) <= xy.w && a1 >= am1;
                    if (!__any_sync(0xffffffffu, ok0 || ok1)) continue;
                    // the Gaussian that would bring T below t_min is not composited
                    // and the pixel stops; otherwise C += c alpha T, T *= 1 - alpha
                    const float2 Tn = __fmul2_rn(T, __fadd2_rn(f2(1.f), make_float2(-a0, -a1)));
                    const bool st0 = ok0 && Tn.x < L.t_min, st1 = ok1 && Tn.y < L.t_min;
                    const bool cp0 = ok0 && !st0, cp1 = ok1 && !st1;
                    am0 = st0 ? INF : am0;
                    am1 = st1 ? INF : am1;
                    end0 = cp0 ? b0 + k + 1 : end0;
                    end1 = cp1 ? b0 + k + 1 : end1;
                    // weight and transmittance through the composited alpha (alpha, or 0
                    // for a pixel that does not composite: T (1 - 0) is T bit for bit)
                    const float2 ac = make_float2(cp0 ? a0 : 0.f, cp1 ? a1 : 0.f);
                    const float2 w = __fmul2_rn(ac, T);
                    T = __fmul2_rn(T, __fadd2_rn(f2(1.f), make_float2(-ac.x, -ac.y)));
                    const float4 c = s_rgb[k];
                    CR = __ffma2_rn(f2(c.x), w, CR);
                    CG = __ffma2_rn(f2(c.y), w, CG);
                    CB = __ffma2_rn(f2(c.z), w, CB);
                }
            }
        }
        const float T0 = T.x, T1 = T.y, C00 = CR.x, C01 = CG.x, C02 = CB.x, C10 = CR.y, C11 = CG.y, C12 = CB.y;
        const ViewDesc &vd = L.v[ti.view];
        const long long hw = (long long)vd.W * vd.H;
        if (ti.in0) {
            const long long o = vd.pix_base + (long long)ti.py0 * vd.W + ti.px;
            image[o] = abort ? 0.f : __fmaf_rn(T0, L.bg[0], C00);
            image[o + hw] = abort ? 0.f : __fmaf_rn(T0, L.bg[1], C01);
            image[o + 2 * hw] = abort ? 0.f : __fmaf_rn(T0, L.bg[2], C02);
            if (last_contrib) last_contrib[vd.pix_base / 3 + (long long)ti.py0 * vd.W + ti.px] = end0;
        }
        if (ti.in1) {
            const long long o = vd.pix_base + (long long)(ti.py0 + 4) * vd.W + ti.px;
            image[o] = abort ? 0.f : __fmaf_rn(T1, L.bg[0], C10);
            image[o + hw] = abort ? 0.f : __fmaf_rn(T1, L.bg[1], C11);
            image[o + 2 * hw] = abort ? 0.f : __fmaf_rn(T1, L.bg[2], C12);
            if (last_contrib) last_contrib[vd.pix_base / 3 + (long long)(ti.py0 + 4) * vd.W + ti.px] = end1;
        }
        if (tile_work) {
            // the backward's replay length of this tile: its pixels' largest
            // end (written by thread 0 after the next item's barrier)
            const int e = __reduce_max_sync(0xffffffffu, max(end0, end1) - r.x);
            if (lane == 0) atomicMax(&s_end, e);
            prev_tile = tile;
        }
    }
}

// With LAST, each pixel's replay ends at the position after its last
// composited Gaussian, which the forward recorded in last_contrib: no
// Gaussian before that position stops the pixel (the stop comes after the
// last composited one), so every Gaussian that passes the alpha test there
// is composited, and the warp and the block stop at their pixels' largest
// end instead of walking on to saturation or the end of the list.
template <int TW, int TH, bool COUNT, bool LAST>
__global__ void __launch_bounds__(TW * TH / 2, 1024 / (TW * TH / 2)) k_render_bwd(const Launch L, const float4 *__restrict__ proj,
                                                            const int2 *__restrict__ ranges,
                                                            const unsigned int *__restrict__ ids,
                                                            const int *__restrict__ order, int *__restrict__ counters,
                                                            const float *__restrict__ image,
                                                            const float *__restrict__ dL_dimage,
                                                            const int *__restrict__ last_contrib,
                                                            float4 *__restrict__ grad2d,
                                                            const float *__restrict__ l1_target,
                                                            float *__restrict__ l1_loss, float l1_inv_n) {
    // dynamic shared memory: the per-warp reduction buffers, then the staged
    // batch (L.bwd_batch Gaussians per thread): positions, conics, colours,
    // the conic's A and D (natural-log units), the per-Gaussian gradient sums
    // (pitch 9, odd: no bank conflicts) and warp masks
    constexpr int BS = TW * TH / 2;
    const int NB = L.bwd_batch * BS;
    extern __shared__ float4 s_dyn[];
    float *s_red = reinterpret_cast<float *>(s_dyn);
    float4 *s_xy = s_dyn + (BS / 32) * RED_WARP_FLOATS / 4, *s_con = s_xy + NB, *s_rgb = s_con + NB;
    float2 *s_ad = reinterpret_cast<float2 *>(s_rgb + NB);
    float *s_g = reinterpret_cast<float *>(s_ad + NB);
    unsigned int *s_mask = reinterpret_cast<unsigned int *>(s_g + 9 * NB);
    __shared__ int s_item;
    __shared__ float s_l1[BS / 32];
    // the projection backward that follows (launched as a programmatic
    // dependent) may start its blocks on SMs this kernel leaves in its tail:
    // it zeroes its gradient rows there, then waits for this grid to finish
    launch_dependents();
    if (counters[CNT_ABORT]) return;
    const int lane = threadIdx.x & 31;
    const unsigned int wbit = 1u << (threadIdx.x >> 5);
    // this warp's buffer: row 9 s + j holds value j of the warp's pending
    // visit s (s < RED_SLOTS), column l that of lane l
    float *rb = s_red + (threadIdx.x >> 5) * RED_WARP_FLOATS;
    // at a flush, lane 9 s + j (j < 9) adds row 9 s + j: value j of pending
    // visit s, whose staged index lane s holds
    const int red_j = lane % 9, red_s = lane / 9;
    const float4 *red_row = reinterpret_cast<const float4 *>(rb + lane * RED_PITCH);
    for (int k = threadIdx.x; k < NB; k += BS)
        for (int c = 0; c < 9; ++c) s_g[9 * k + c] = 0.f;
    float l1_sum = 0.f;   // with l1_target: this thread's sum of |image - target|
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counters + CNT_Q_BWD, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= L.n_tiles) break;
        const int tile = order[item];
        const TileInfo ti = tile_info<TW, TH>(L, tile);
        const int2 r = ranges[tile];
        const ViewDesc &vd = L.v[ti.view];
        const long long hw = (long long)vd.W * vd.H;
        // per pixel: upstream gradient g (one pair per channel), -image.g, and
        // the running colour dotted with g (the colour behind a Gaussian enters
        // dL/dalpha only as S.g = image.g - C.g). With l1_target, g is the mean
        // L1 loss's gradient sign(image - target) / count, formed here (the
        // value gs_l1_loss writes, bit for bit) instead of read
        float gg[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, ig[2] = {0.f, 0.f};
        bool done0 = !ti.in0, done1 = !ti.in1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!(h ? ti.in1 : ti.in0)) continue;
            const long long o = vd.pix_base + (long long)(ti.py0 + 4 * h) * vd.W + ti.px;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float im = image[o + ch * hw];
                float g;
                if (l1_target) {
                    const float d = im - l1_target[o + ch * hw];
                    l1_sum += fabsf(d);
                    g = d > 0.f ? l1_inv_n : (d < 0.f ? -l1_inv_n : 0.f);
                } else {
                    g = dL_dimage[o + ch * hw];
                }
                gg[h][ch] = g;
                ig[h] = fmaf(im, g, ig[h]);
            }
        }
        done0 = done0 || (gg[0][0] == 0.f && gg[0][1] == 0.f && gg[0][2] == 0.f);
        done1 = done1 || (gg[1][0] == 0.f && gg[1][1] == 0.f && gg[1][2] == 0.f);
        // LAST: the end of each pixel's replay (the tile start for a pixel that
        // needs none), and the later of the two
        int end0 = r.x, end1 = r.x;
        if (LAST) {
            if (!done0) end0 = last_contrib[vd.pix_base / 3 + (long long)ti.py0 * vd.W + ti.px];
            if (!done1) end1 = last_contrib[vd.pix_base / 3 + (long long)(ti.py0 + 4) * vd.W + ti.px];
        }
        const int endm = max(end0, end1);
        const float2 GR = make_float2(gg[0][0], gg[1][0]), GG = make_float2(gg[0][1], gg[1][1]),
                     GB = make_float2(gg[0][2], gg[1][2]), NIG = make_float2(-ig[0], -ig[1]);
        const float2 PCY = make_float2(ti.pcy0, ti.pcy0 + 4.f);
        float2 T = f2(1.f), CG = f2(0.f);
        unsigned int n_eval = 0, n_comp = 0;
        // the warp's pending visits (warp-uniform) and, in lane s, the staged
        // index of pending visit s
        int npend = 0, kpend = 0;
        // add the pending visits' rows to their Gaussians' sums in s_g (each
        // row over the 32 lanes: two f32x2 chains over 8 16-byte loads, then
        // the two lanes of the pair)
        auto flush = [&]() {
            __syncwarp();
            const int kk = __shfl_sync(0xffffffffu, kpend, red_s);
            if (lane < 9 * npend) {
                float4 v = red_row[0];
                float2 sa = make_float2(v.x, v.y), sb = make_float2(v.z, v.w);
#pragma unroll
                for (int i = 1; i < 8; ++i) {
                    v = red_row[i];
                    sa = __fadd2_rn(sa, make_float2(v.x, v.y));
                    sb = __fadd2_rn(sb, make_float2(v.z, v.w));
                }
                sa = __fadd2_rn(sa, sb);
                atomicAdd(&s_g[9 * kk + red_j], sa.x + sa.y);
            }
            npend = 0;
            __syncwarp();   // the buffer is free for the next visits
        };
        for (int b0 = r.x; b0 < r.y; b0 += NB) {
            if (__syncthreads_count(LAST ? b0 >= endm : done0 && done1) == BS) break;
            // LAST: the pixels' ends relative to this batch
            const int e0 = end0 - b0, e1 = end1 - b0;
            stage_batch<TW, TH>(L, proj, ids, b0, r.y, L.bwd_batch, ti, s_xy, s_con, s_rgb, s_mask);
            for (int h = 0; h < L.bwd_batch; ++h) {
                const int k = threadIdx.x + h * BS;
                if (b0 + k < r.y)
                    s_ad[k] = make_float2(s_con[k].x * (-2.f * LN2), s_con[k].z * (-2.f * LN2));
            }
            __syncthreads();
            const int nb = min(NB, r.y - b0);
            for (int k0 = 0; k0 < nb; k0 += 32) {
                // the warp's pixels have all stopped
                if (__all_sync(0xffffffffu, LAST ? b0 + k0 >= endm : done0 && done1)) break;
                // only the staged Gaussians that may reach this warp's patch, in order
                unsigned int hits = __ballot_sync(0xffffffffu, k0 + lane < nb && (s_mask[k0 + lane] & wbit));
                while (hits) {
                    const int k = k0 + __ffs(hits) - 1;
                    hits &= hits - 1;
                    const float4 xy = s_xy[k], con = s_con[k];
                    // both pixels' alphas, the forward's arithmetic and decisions
                    const float dx = __fsub_rn(ti.pcx, xy.x);
                    const bool col = fabsf(dx) <= xy.z;   // the column gate, shared by both pixels
                    const float2 dy = __fadd2_rn(PCY, f2(-xy.y));
                    const float2 u = __ffma2_rn(f2(con.y), dy, f2(dx));
                    const float2 p2 = __ffma2_rn(f2(con.x), __fmul2_rn(u, u), __fmul2_rn(f2(con.z), __fmul2_rn(dy, dy)));
                    const float2 G = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
                    const float2 oG = __fmul2_rn(f2(con.w), G);
                    const float a0 = fminf(oG.x, L.alpha_max), a1 = fminf(oG.y, L.alpha_max);
                    const bool live0 = LAST ? k < e0 : !done0, live1 = LAST ? k < e1 : !done1;
                    const bool ev0 = col && live0 && fabsf(dy.x) <= xy.w, ev1 = col && live1 && fabsf(dy.y) <= xy.w;
                    const bool ok0 = ev0 && a0 >= L.alpha_min, ok1 = ev1 && a1 >= L.alpha_min;
                    if (COUNT) n_eval += (unsigned int)ev0 + (unsigned int)ev1;
                    if (!__any_sync(0xffffffffu, ok0 || ok1)) continue;
                    // transmittance: the pixel stops before a Gaussian that would
                    // bring T below t_min; otherwise the Gaussian is composited
                    // (with LAST no such Gaussian comes before the pixel's end).
                    // ac = the composited alpha (alpha, or 0 for a pixel that does not
                    // composite, whose T (1 - 0) is T bit for bit); oma = 1 - ac
                    bool cp0, cp1;
                    float2 ac, oma, Tn;
                    if constexpr (LAST) {
                        cp0 = ok0;
                        cp1 = ok1;
                        ac = make_float2(cp0 ? a0 : 0.f, cp1 ? a1 : 0.f);
                        oma = __fadd2_rn(f2(1.f), make_float2(-ac.x, -ac.y));
                        Tn = __fmul2_rn(T, oma);
                    } else {
                        const float2 om = __fadd2_rn(f2(1.f), make_float2(-a0, -a1));
                        const float2 Tt = __fmul2_rn(T, om);
                        const bool st0 = ok0 && Tt.x < L.t_min, st1 = ok1 && Tt.y < L.t_min;
                        cp0 = ok0 && !st0;
                        cp1 = ok1 && !st1;
                        done0 = done0 || st0;
                        done1 = done1 || st1;
                        ac = make_float2(cp0 ? a0 : 0.f, cp1 ? a1 : 0.f);
                        oma = om;   // (enters only terms that are zero where nothing is composited)
                        Tn = make_float2(cp0 ? Tt.x : T.x, cp1 ? Tt.y : T.y);
                    }
                    if (COUNT) n_comp += (unsigned int)cp0 + (unsigned int)cp1;
                    // gradients; a pixel that does not composite contributes zeros
                    // (its weight and its alpha factors are zero)
                    const float4 c = s_rgb[k];
                    const float2 ad = s_ad[k];
                    const float2 w = __fmul2_rn(ac, T);
                    const float2 Told = T;
                    T = Tn;
                    const float2 g6 = __fmul2_rn(w, GR), g7 = __fmul2_rn(w, GG), g8 = __fmul2_rn(w, GB);
                    // c.g, and C.g accumulated through this Gaussian; S.g = image.g - C.g,
                    // dL/dalpha = T (c.g) - (S.g) / (1 - alpha) (1 - alpha >= 0.01, so
                    // the approximate reciprocal's few-ulp error is far inside the
                    // gradient tolerance)
                    const float2 cgk = __ffma2_rn(f2(c.z), GB, __ffma2_rn(f2(c.y), GG, __fmul2_rn(f2(c.x), GR)));
                    CG = __ffma2_rn(w, cgk, CG);
                    const float2 q = __fmul2_rn(__fadd2_rn(CG, NIG), make_float2(rcp_approx(oma.x), rcp_approx(oma.y)));
                    const float2 dla = __ffma2_rn(Told, cgk, q);
                    // alpha = o G unless clamped; G = exp(power), power = -1/2 d^T Q d,
                    // Q the conic, d = pixel - mean. With v = Q d = (A u, A beta u + D dy)
                    // from the staged form, d power / d mean = v and d power / d Sigma' =
                    // v v^T / 2, i.e. (v0^2/2, v0 v1, v1^2/2) for (a, b, c); summing these
                    // well-scaled terms avoids the ill-conditioned conic -> covariance
                    // conversion of summed conic gradients. The halves of the (a) and (c)
                    // sums are applied once, at the flush. Gu = G where the pixel composites
                    // an unclamped alpha, else 0; d alpha / d power = o Gu.
                    const bool un0 = cp0 && oG.x <= L.alpha_max, un1 = cp1 && oG.y <= L.alpha_max;
                    const float2 g5 = __fmul2_rn(dla, make_float2(un0 ? G.x : 0.f, un1 ? G.y : 0.f));
                    const float2 dp = __fmul2_rn(f2(con.w), g5);
                    const float2 v0 = __fmul2_rn(f2(ad.x), u);
                    const float2 v1 = __ffma2_rn(v0, f2(con.y), __fmul2_rn(f2(ad.y), dy));
                    const float2 g0 = __fmul2_rn(dp, v0), g1 = __fmul2_rn(dp, v1);
                    const float2 g2 = __fmul2_rn(g0, v0), g3 = __fmul2_rn(g0, v1), g4 = __fmul2_rn(g1, v1);
                    if (__any_sync(0xffffffffu, cp0 || cp1)) {
                        // gradient of this thread's pixels w.r.t. (x, y, a, b, c, o, r, g, b),
                        // as column `lane` of the next pending visit's rows
                        float *wr = rb + npend * (9 * RED_PITCH) + lane;
                        wr[0 * RED_PITCH] = g0.x + g0.y;
                        wr[1 * RED_PITCH] = g1.x + g1.y;
                        wr[2 * RED_PITCH] = g2.x + g2.y;
                        wr[3 * RED_PITCH] = g3.x + g3.y;
                        wr[4 * RED_PITCH] = g4.x + g4.y;
                        wr[5 * RED_PITCH] = g5.x + g5.y;
                        wr[6 * RED_PITCH] = g6.x + g6.y;
                        wr[7 * RED_PITCH] = g7.x + g7.y;
                        wr[8 * RED_PITCH] = g8.x + g8.y;
                        kpend = lane == npend ? k : kpend;
                        if (++npend == RED_SLOTS) flush();
                    }
                }
            }
            if (npend) flush();   // (warp-uniform) before the batch's sums leave
            __syncthreads();
            // flush this batch's per-Gaussian sums
            for (int h = 0; h < L.bwd_batch; ++h) {
                const int k = threadIdx.x + h * BS;
                if (k < nb) {
                    const float *sg = s_g + 9 * k;
                    const float a0 = sg[0], a1 = sg[1], a2 = 0.5f * sg[2], a3 = sg[3];
                    const float a4 = 0.5f * sg[4];
                    const float a5 = sg[5], a6 = sg[6], a7 = sg[7], a8 = sg[8];
                    if (a0 != 0.f || a1 != 0.f || a2 != 0.f || a3 != 0.f || a4 != 0.f || a5 != 0.f || a6 != 0.f ||
                        a7 != 0.f || a8 != 0.f) {
                        const unsigned int slot = __float_as_uint(s_rgb[k].w);
                        float4 *dst = grad2d + 3ull * slot;
                        atomicAdd(dst, make_float4(a0, a1, a2, a3));
                        atomicAdd(dst + 1, make_float4(a4, a5, a6, a7));
                        atomicAdd(dst + 2, make_float4(a8, 0.f, 0.f, 0.f));
                    }
#pragma unroll
                    for (int cc = 0; cc < 9; ++cc) s_g[9 * k + cc] = 0.f;
                }
            }
        }
        if (COUNT) count_pairs(counters, 12, n_eval, n_comp);
    }
    if (l1_loss) {
        // the block's part of the loss: one atomic per block (the loss's last
        // bits depend on their order)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l1_sum += __shfl_xor_sync(0xffffffffu, l1_sum, o);
        if (lane == 0) s_l1[threadIdx.x >> 5] = l1_sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < BS / 32; ++w) t += s_l1[w];
            atomicAdd(l1_loss, t * l1_inv_n);
        }
    }
}

// Zero the raster backward's accumulators (the 2D gradients, and the L1 loss
// when given) as a programmatic dependent of the kernel ahead on the stream
// (in a step, the raster forward): nothing here touches what that kernel
// reads or writes, so the stores run on the SMs it leaves in its tail; the
// wait at the end keeps the stream's order for the kernels after this one.
__global__ void __launch_bounds__(256) k_zero_accumulators(float4 *__restrict__ p, long long n4,
                                                           float *__restrict__ loss) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n4; i += (long long)gridDim.x * 256) p[i] = z;
    if (loss && blockIdx.x == 0 && threadIdx.x == 0) *loss = 0.f;
    grid_dependency_wait();
}

int launch_zero_accumulators(float *grad2d, long long n_floats, float *loss, cudaStream_t st) {
    // (n_floats: 12 per slot, a whole number of float4; grad2d 16-byte aligned)
    const long long n4 = n_floats / 4;
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.gridDim = dim3((unsigned)max(1LL, min((long long)num_sms() * 8, (n4 + 255) / 256)));
    lc.blockDim = dim3(256);
    lc.stream = st;
    lc.attrs = at;
    lc.numAttrs = 1;
    if (cudaLaunchKernelEx(&lc, k_zero_accumulators, reinterpret_cast<float4 *>(grad2d), n4, loss) != cudaSuccess)
        return GS_ERR_CUDA;
    return GS_OK;
}

// Resident blocks per SM of a raster kernel at the launch's block and
// dynamic shared-memory size (cached per batch size; the attribute that
// allows more than 48 KB of dynamic shared memory is set on first use).
template <typename K>
static int raster_blocks_per_sm(K kernel, int threads, size_t smem, int batch, int *cache) {
    if (!cache[batch]) {
        int n = 0;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
            cudaGetLastError();   // the launch itself reports a size that cannot run
            n = 1;
        }
        cache[batch] = n;
    }
    return cache[batch];
}

// Few tiles per SM: the tail of a largest-first queue then decides a raster
// kernel's length, and the backward orders its tiles by replay length.
static bool order_by_work(const Launch &L, const gs_bins *b) {
    return b->last_contrib && L.n_tiles > 0 && L.n_tiles < 16LL * num_sms();
}
// where the forward records the replay lengths: the caller's kept record,
// else tile_scratch (this call only)
static int *work_record(const gs_bins *b) { return b->tile_work ? b->tile_work : b->tile_scratch; }

// The work order of a raster kernel: the tiles by decreasing predicted work,
// so that the longest start first and the persistent blocks finish together
// (ordered by instance count, the blocks of the 32x32 backward on the
// 1M-Gaussian view were busy 86 % of the kernel's time on average, the
// busiest 99 %). The prediction is a recorded replay length, or with
// `ranges` given and nothing recorded (<= 0) the tile's instance count. One
// block; 1024 buckets of the prediction, 32 per octave; order within a bucket
// is unspecified (no result depends on the order).
__device__ __forceinline__ int work_bucket(int w) {
    if (w <= 0) return 0;
    const int e = 31 - __clz(w);
    return min(1023, e * 32 + ((w >> max(0, e - 5)) & 31));
}
__global__ void __launch_bounds__(1024) k_order_by_work(const int *__restrict__ work,
                                                       const int2 *__restrict__ ranges, int n_tiles,
                                                       int *__restrict__ order) {
    __shared__ int s_cnt[1024];
    __shared__ int s_part[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    auto predicted = [&](int t) {
        const int w = work[t];
        if (w > 0 || !ranges) return w;
        const int2 r = ranges[t];
        return r.y - r.x;
    };
    s_cnt[tid] = 0;
    __syncthreads();
    for (int t = tid; t < n_tiles; t += 1024) atomicAdd(&s_cnt[work_bucket(predicted(t))], 1);
    __syncthreads();
    // exclusive scan over the buckets from the longest down: thread i owns
    // bucket 1023 - i
    const int c = s_cnt[1023 - tid];
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_part[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = s_part[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        s_part[lane] = wi - w;
    }
    __syncthreads();
    s_cnt[1023 - tid] = s_part[wid] + incl - c;   // the bucket's first position
    __syncthreads();
    for (int t = tid; t < n_tiles; t += 1024) order[atomicAdd(&s_cnt[work_bucket(predicted(t))], 1)] = t;
}

template <int TW, int TH>
static int launch_fwd_t(const Launch &L, const float *proj, const gs_bins *b, float *image, cudaStream_t st) {
    static int blocks_per_sm[5];
    const size_t smem = (size_t)FWD_STAGE_BYTES * L.fwd_batch * (TW * TH / 2);
    const int grid = min(num_sms() * raster_blocks_per_sm(k_render_fwd<TW, TH>, TW * TH / 2, smem, L.fwd_batch,
                                                          blocks_per_sm),
                         max(1, L.n_tiles));
    // every call walks all tiles again: reset this kernel's work-queue head
    if (cudaMemsetAsync(b->counters + CNT_Q_FWD, 0, sizeof(int), st) != cudaSuccess) return GS_ERR_CUDA;
    // with the last-contrib record and few tiles per SM, also each tile's
    // replay length for the backward's work order: into the kept work record
    // (after taking this forward's order from the previous one's lengths,
    // the instance count where none is recorded; the sort no longer needs
    // tile_order), else into tile_scratch (free after the sort)
    const bool ordered = order_by_work(L, b);
    if (ordered && b->tile_work) {
        k_order_by_work<<<1, 1024, 0, st>>>(b->tile_work, reinterpret_cast<const int2 *>(b->tile_ranges),
                                            (int)L.n_tiles, b->tile_order);
        if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    }
    k_render_fwd<TW, TH><<<grid, TW * TH / 2, smem, st>>>(L, reinterpret_cast<const float4 *>(proj),
                                                       reinterpret_cast<const int2 *>(b->tile_ranges), b->ids,
                                                       b->tile_order, b->counters, image, b->last_contrib,
                                                       ordered ? work_record(b) : nullptr);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

template <int TW, int TH, bool COUNT, bool LAST>
static int launch_bwd_c(const Launch &L, const float *proj, const gs_bins *b, const float *image,
                        const float *dL_dimage, const L1Loss &l1, float *grad2d, cudaStream_t st) {
    static int blocks_per_sm[5];
    const size_t smem = (size_t)BWD_STAGE_BYTES * L.bwd_batch * (TW * TH / 2) +
                        sizeof(float) * RED_WARP_FLOATS * (TW * TH / 64);
    const int grid = min(num_sms() * raster_blocks_per_sm(k_render_bwd<TW, TH, COUNT, LAST>, TW * TH / 2, smem,
                                                          L.bwd_batch, blocks_per_sm),
                         max(1, L.n_tiles));
    if (cudaMemsetAsync(b->counters + CNT_Q_BWD, 0, sizeof(int), st) != cudaSuccess) return GS_ERR_CUDA;
    k_render_bwd<TW, TH, COUNT, LAST><<<grid, TW * TH / 2, smem, st>>>(
        L, reinterpret_cast<const float4 *>(proj), reinterpret_cast<const int2 *>(b->tile_ranges), b->ids,
        b->tile_order, b->counters, image, dL_dimage, b->last_contrib, reinterpret_cast<float4 *>(grad2d), l1.target,
        l1.loss, l1.inv_n);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

template <int TW, int TH>
static int launch_bwd_t(const Launch &L, const float *proj, const gs_bins *b, const float *image,
                        const float *dL_dimage, const L1Loss &l1, float *grad2d, cudaStream_t st) {
    if (b->last_contrib) {
        // the forward recorded each tile's replay length
        if (order_by_work(L, b)) {
            k_order_by_work<<<1, 1024, 0, st>>>(work_record(b), nullptr, (int)L.n_tiles, b->tile_order);
            if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
        }
        return L.count_pairs ? launch_bwd_c<TW, TH, true, true>(L, proj, b, image, dL_dimage, l1, grad2d, st)
                             : launch_bwd_c<TW, TH, false, true>(L, proj, b, image, dL_dimage, l1, grad2d, st);
    }
    return L.count_pairs ? launch_bwd_c<TW, TH, true, false>(L, proj, b, image, dL_dimage, l1, grad2d, st)
                         : launch_bwd_c<TW, TH, false, false>(L, proj, b, image, dL_dimage, l1, grad2d, st);
}

int launch_render_fwd(const Launch &L, const float *proj, const gs_bins *b, float *image, cudaStream_t st) {
#define GS_CALL_FWD(TW, TH) launch_fwd_t<TW, TH>(L, proj, b, image, st)
    if (L.tw == 16 && L.th == 16) return GS_CALL_FWD(16, 16);
    if (L.tw == 8 && L.th == 8) return GS_CALL_FWD(8, 8);
    if (L.tw == 16 && L.th == 8) return GS_CALL_FWD(16, 8);
    if (L.tw == 32 && L.th == 8) return GS_CALL_FWD(32, 8);
    if (L.tw == 32 && L.th == 16) return GS_CALL_FWD(32, 16);
    if (L.tw == 32 && L.th == 32) return GS_CALL_FWD(32, 32);
    return GS_ERR_UNSUPPORTED;
#undef GS_CALL_FWD
}

int launch_render_bwd(const Launch &L, const float *proj, const gs_bins *b, const float *image,
                      const float *dL_dimage, const L1Loss &l1, float *grad2d, cudaStream_t st) {
#define GS_CALL_BWD(TW, TH) launch_bwd_t<TW, TH>(L, proj, b, image, dL_dimage, l1, grad2d, st)
    if (L.tw == 16 && L.th == 16) return GS_CALL_BWD(16, 16);
    if (L.tw == 8 && L.th == 8) return GS_CALL_BWD(8, 8);
    if (L.tw == 16 && L.th == 8) return GS_CALL_BWD(16, 8);
    if (L.tw == 32 && L.th == 8) return GS_CALL_BWD(32, 8);
    if (L.tw == 32 && L.th == 16) return GS_CALL_BWD(32, 16);
    if (L.tw == 32 && L.th == 32) return GS_CALL_BWD(32, 32);
    return GS_ERR_UNSUPPORTED;
#undef GS_CALL_BWD
}

}  // namespace gsk
