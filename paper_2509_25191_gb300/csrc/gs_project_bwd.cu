// Backward of the projection: per-slot 2D gradients -> raw Gaussian
// parameters and camera poses.
//
// Three schemes, chosen per call, with the same chain (view_term) and the
// same per-Gaussian end (gauss_epilogue):
//  * k_project_bwd, one thread per Gaussian (fixed grid, grid-stride),
//    looping over the views of its scene: the pose-only backward, and, as
//    COMPACT, the one-view call, which runs the chain only for the Gaussians
//    with a nonzero 2D gradient, listed per block;
//  * k_project_bwd_views, several views with Gaussian gradients: per block
//    and window of views, the chains run either by owner lanes or over
//    per-view lists of the Gaussians with a gradient, whichever takes fewer
//    warp runs.
// A Gaussian's gradients are summed over its views in ascending order and
// written once (overwritten, or added to the caller's values when the
// configuration accumulates); the SH-coefficient gradients leave from shared
// memory, 16 bytes per store. Each view's pose
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
#include "gs_common.cuh"

namespace gsk {

constexpr int PB_THREADS = 128;   // 128 registers: 4 blocks per SM, no spills

// a parameter gradient: written (overwrite) or added to the caller's value
__device__ __forceinline__ void put(float *p, float v, bool acc) { *p = acc ? *p + v : v; }
constexpr int PB_WARPS = PB_THREADS / 32;


// The block's SH-coefficient gradient rows from shared memory (row r, pitch
// 3K + 1, to Gaussian rows[r], none if negative), written or added: 16 bytes
// per store where the rows are whole, 16-byte aligned float4s (degrees 1 and
// 3 with an aligned array), else one float per store. Whole block.
template <int K>
__device__ __forceinline__ void write_sh_rows(const float *s_gf, const long long *rows, float *__restrict__ g_sh,
                                              bool acc) {
    constexpr int GP = 3 * K + 1;
    if constexpr ((3 * K) % 4 == 0) {
        if (((uintptr_t)g_sh & 15u) == 0) {
            constexpr int C4 = 3 * K / 4;
            for (int e = threadIdx.x; e < PB_THREADS * C4; e += PB_THREADS) {
                const int rr = e / C4, c = 4 * (e % C4);
                const long long row = rows[rr];
                if (row < 0) continue;
                const float *src = s_gf + rr * GP + c;
                float4 v4 = make_float4(src[0], src[1], src[2], src[3]);
                float4 *dst = reinterpret_cast<float4 *>(g_sh + row * 3 * K + c);
                if (acc) {
                    const float4 o = *dst;
                    v4 = make_float4(o.x + v4.x, o.y + v4.y, o.z + v4.z, o.w + v4.w);
                }
                *dst = v4;
            }
            return;
        }
    }
    for (int e = threadIdx.x; e < PB_THREADS * 3 * K; e += PB_THREADS) {
        const int rr = e / (3 * K), c = e % (3 * K);
        const long long row = rows[rr];
        if (row >= 0) put(g_sh + row * 3 * K + c, s_gf[rr * GP + c], acc);
    }
}

// One (Gaussian, view) term of the chain, for a Gaussian with a nonzero
// 2D-gradient row (ga4, gb4, gc4) in view v at slot `slot`: adds to the
// Gaussian's sums (gm, go, GS.., and its SH-coefficient gradients in gf) and
// to the view's pose partial pg. The mean and the 3D covariance Sigma come
// from the caller, the SH row is f. Every Gaussian's sums take its views in
// ascending order.
template <int DEG, bool GAUSS>
__device__ __forceinline__ void view_term(const Launch &L, int v, long long slot, const float4 &ga4,
                                          const float4 &gb4, const float4 &gc4, const float4 *__restrict__ proj,
                                          const float *__restrict__ viewmats, const float *__restrict__ intr,
                                          float mx, float my, float mz, float S00, float S01, float S02, float S11,
                                          float S12, float S22, const float *__restrict__ f, float *gf,
                                          float (&gm)[3], float &go, float &GS00, float &GS01, float &GS02,
                                          float &GS11, float &GS12, float &GS22, float (&pg)[12]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
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
        if (DEG == 1 || DEG == 3) {
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
        if (GAUSS) {
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

// The end of the chain for Gaussian i from its sums over views: the 3D
// covariance gradient GS (symmetric) through Sigma = M M^T, M = R(q) diag(s),
// to the log-scales and the (normalised) quaternion, and the mean and
// opacity-logit gradients; written, or added to the caller's values.
__device__ __forceinline__ void gauss_epilogue(long long i, bool acc, const float (&M)[9], const float (&Rq)[9],
                                               const float (&sc)[3], const float (&qn)[4], float qlen, float opac,
                                               const float (&gm)[3], float go, float GS00, float GS01, float GS02,
                                               float GS11, float GS12, float GS22, float *__restrict__ g_means,
                                               float *__restrict__ g_log_scales, float *__restrict__ g_quats,
                                               float *__restrict__ g_logits) {
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

// COMPACT (one-view calls): most Gaussians of a dense scene get no 2D
// gradient in one view (they are hidden behind saturated pixels), and a
// thread per Gaussian left most lanes idle. Instead each block takes a
// contiguous range of Gaussians, finds those with a nonzero 2D-gradient row
// (PB_SUB at a time, listed in shared memory in an order fixed by their
// indices) and runs the chain over the list with full warps. A block's
// parameter-gradient rows are zeroed by the block, coalesced, before
// anything else (launched as a programmatic dependent of the raster backward,
// while that kernel's last blocks still run), and the listed Gaussians' rows
// written again after a barrier (accumulating, the others are left as they
// are). The pose partials stay
// per block over a fixed range, so the pose gradient is deterministic.
// Several views take k_project_bwd_views, which compacts per view.
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

template <int DEG, bool GAUSS, bool COMPACT>
__global__ void __launch_bounds__(PB_THREADS, 4) k_project_bwd(
    const Launch L, const float *__restrict__ means, const float *__restrict__ log_scales,
    const float *__restrict__ quats, const float *__restrict__ logits, const float *__restrict__ sh,
    const float *__restrict__ viewmats, const float *__restrict__ intr, const float4 *__restrict__ proj,
    const float4 *__restrict__ grad2d, float *__restrict__ g_means, float *__restrict__ g_log_scales,
    float *__restrict__ g_quats, float *__restrict__ g_logits, float *__restrict__ g_sh,
    float *__restrict__ pose_partials) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int GP = 3 * K + 1;   // odd row pitch: conflict-free column access
    // per-warp pose partials [PB_WARPS][n_views][12] (dynamic: sized by the launch)
    extern __shared__ float s_pose[];
    // per-thread SH-coefficient gradients, summed over views here and written
    // out by the whole block with coalesced stores
    __shared__ float s_gf[GAUSS ? PB_THREADS * GP : 1];
    __shared__ long long s_row[GAUSS ? PB_THREADS : 1];
    __shared__ int s_list[COMPACT ? PB_SUB : 1];   // offsets from the range's current start
    __shared__ int s_wsum[PB_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nv = L.n_views;
    for (int i = threadIdx.x; i < PB_WARPS * nv * 12; i += PB_THREADS) s_pose[i] = 0.f;
    __syncthreads();

    const long long stride = (long long)gridDim.x * PB_THREADS;
    // COMPACT: this block's range [c_next, c_end), the current list of c_cnt
    // offsets from c_at, and how far it has been taken
    long long c_next = 0, c_end = 0, c_at = 0;
    int c_cnt = 0, c_pos = 0;
    if constexpr (COMPACT) {
        const long long per = (L.n_threads + gridDim.x - 1) / gridDim.x;
        c_next = min((long long)L.n_threads, (long long)blockIdx.x * per);
        c_end = min((long long)L.n_threads, c_next + per);
        if (GAUSS && !L.accumulate && c_next < c_end) {
            // this block's rows, zero (one view: its Gaussians are contiguous);
            // the kernel ahead does not touch them, so this runs before the
            // wait below (launched with overlap_prev: on SMs the raster
            // backward has left). The listed Gaussians' rows are written again
            // after later barriers.
            const int sc = scene_of_thread(L, c_next);
            zero_rows<K>(L.s[sc].g_begin + (c_next - L.s[sc].thread_base), c_end - c_next, g_means, g_log_scales,
                         g_quats, g_logits, g_sh);
        }
    }
    // the 2D gradients and everything else below come from the kernels ahead
    grid_dependency_wait();
    for (long long base = (long long)blockIdx.x * PB_THREADS;; base += stride) {
        long long gid;
        bool valid;
        if constexpr (COMPACT) {
            while (c_pos >= c_cnt && c_next < c_end) {   // (uniform over the block)
                const long long g1 = min(c_end, c_next + PB_SUB);
                c_cnt = compact_range(L, grad2d, c_next, g1, s_list, s_wsum);
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

        float mx = 0.f, my = 0.f, mz = 0.f, sc[3] = {0.f, 0.f, 0.f}, qn[4] = {1.f, 0.f, 0.f, 0.f}, qlen = 1.f;
        float Rq[9], M[9], S00 = 0, S01 = 0, S02 = 0, S11 = 0, S12 = 0, S22 = 0, opac = 0.f;
        bool loaded = false;
        // SH coefficients are read per view where needed (L1-resident), not
        // held in registers
        const float *f = sh + (long long)3 * K * (valid ? i : 0);

        // accumulators over views
        float gm[3] = {0.f, 0.f, 0.f}, go = 0.f;
        float GS00 = 0, GS01 = 0, GS02 = 0, GS11 = 0, GS12 = 0, GS22 = 0;   // full-matrix entries, symmetric
        float *gf = s_gf + (GAUSS ? threadIdx.x * GP : 0);
        if (GAUSS) {
#pragma unroll
            for (int k = 0; k < 3 * K; ++k) gf[k] = 0.f;
            s_row[threadIdx.x] = valid ? i : -1;
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
                const float4 ga4 = grad2d[3 * slot], gb4 = grad2d[3 * slot + 1], gc4 = grad2d[3 * slot + 2];
                contrib = ga4.x != 0.f || ga4.y != 0.f || ga4.z != 0.f || ga4.w != 0.f || gb4.x != 0.f ||
                          gb4.y != 0.f || gb4.z != 0.f || gb4.w != 0.f || gc4.x != 0.f;
                if (contrib)
                    view_term<DEG, GAUSS>(L, v, slot, ga4, gb4, gc4, proj, viewmats, intr, mx, my, mz, S00, S01, S02,
                                          S11, S12, S22, f, gf, gm, go, GS00, GS01, GS02, GS11, GS12, GS22, pg);
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
        if (valid && GAUSS && (loaded || !L.accumulate))
            gauss_epilogue(i, L.accumulate, M, Rq, sc, qn, qlen, opac, gm, go, GS00, GS01, GS02, GS11, GS12, GS22,
                           g_means, g_log_scales, g_quats, g_logits);
        if constexpr (GAUSS) {
            // the block's SH-coefficient gradients: row r goes to Gaussian s_row[r]
            __syncthreads();
            write_sh_rows<K>(s_gf, s_row, g_sh, L.accumulate);
            __syncthreads();
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nv * 12; e += PB_THREADS) {
        const int v = e / 12, cc = e % 12;
        float acc = 0.f;
#pragma unroll
        for (int ww = 0; ww < PB_WARPS; ++ww) acc += s_pose[(ww * nv + v) * 12 + cc];
        pose_partials[((long long)v * gridDim.x + blockIdx.x) * 12 + cc] = acc;
    }
}

// Several views, compacted per view. A thread per Gaussian looping over its
// views ran the chain for a view whenever one of its warp's 32 Gaussians had
// a 2D gradient there, with the other lanes idle (on a 16-view batch most
// Gaussians are seen in every view but reach the image in few). Here a block
// sets up its 128 Gaussians (parameters, mean and Sigma into shared memory,
// sums zeroed), and for each view lists the Gaussians with a nonzero
// 2D-gradient row there and runs the chain over the list with full warps,
// each term added to its Gaussian's sums in shared memory. A Gaussian's sums
// take its views in ascending order (as in k_project_bwd), so its gradients
// are the same bit for bit; the pose partial of a view is summed per warp
// over the list (fixed by the Gaussians' indices), then per block.
constexpr int PB_LIST_VIEW_COST = 3;   // a view's listing and barriers, in chain runs of a warp (measured: 1-4)
template <int DEG>
__global__ void __launch_bounds__(PB_THREADS, 4) k_project_bwd_views(
    const Launch L, const float *__restrict__ means, const float *__restrict__ log_scales,
    const float *__restrict__ quats, const float *__restrict__ logits, const float *__restrict__ sh,
    const float *__restrict__ viewmats, const float *__restrict__ intr, const float4 *__restrict__ proj,
    const float4 *__restrict__ grad2d, float *__restrict__ g_means, float *__restrict__ g_log_scales,
    float *__restrict__ g_quats, float *__restrict__ g_logits, float *__restrict__ g_sh,
    float *__restrict__ pose_partials) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int GP = 3 * K + 1;   // odd row pitch: conflict-free column access
    constexpr int NA = 10;          // sums per Gaussian: mean (3), opacity, Sigma (6)
    extern __shared__ float s_pose[];   // [PB_WARPS][n_views][12]
    __shared__ float s_gf[PB_THREADS * GP];
    __shared__ float s_acc[PB_THREADS * NA];
    __shared__ float s_ms[PB_THREADS * 9];   // mean, Sigma (S00 S01 S02 S11 S12 S22)
    __shared__ long long s_row[PB_THREADS];
    __shared__ int s_list[PB_THREADS];
    __shared__ int s_wsum[PB_WARPS];
    __shared__ int s_vr[2];
    __shared__ unsigned long long s_vany;   // views of the current window with a gradient somewhere in the block
    __shared__ int s_vcnt[64];              // per view of the window: Gaussians of the block with a gradient
    __shared__ int s_owner_runs;            // chain runs of the owner-lane way
    __shared__ bool s_lists;                // run the window by per-view lists
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nv = L.n_views;
    for (int e = threadIdx.x; e < PB_WARPS * nv * 12; e += PB_THREADS) s_pose[e] = 0.f;
    if (threadIdx.x == 0) {
        s_vany = 0ull;
        s_owner_runs = 0;
    }
    if (threadIdx.x < 64) s_vcnt[threadIdx.x] = 0;
    const long long stride = (long long)gridDim.x * PB_THREADS;
    for (long long base = (long long)blockIdx.x * PB_THREADS; base < L.n_threads; base += stride) {
        const long long gid = base + threadIdx.x;
        const bool valid = gid < L.n_threads;
        const int s = valid ? scene_of_thread(L, gid) : 0;
        const long long li = valid ? gid - L.s[s].thread_base : 0;
        const long long i = L.s[s].g_begin + li;
        const int vb = valid ? L.s[s].v_begin : 0x7fffffff, ve = valid ? L.s[s].v_end : 0;
        if (threadIdx.x == 0) {
            s_vr[0] = 0x7fffffff;
            s_vr[1] = 0;
        }
        // this Gaussian's activations (the owner thread keeps them for the end)
        float l3[3] = {0.f, 0.f, 0.f}, lg = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
        float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
        if (valid) {
            mx = means[3 * i]; my = means[3 * i + 1]; mz = means[3 * i + 2];
#pragma unroll
            for (int a = 0; a < 3; ++a) l3[a] = log_scales[3 * i + a];
            q = reinterpret_cast<const float4 *>(quats)[i];
            lg = logits[i];
        }
        float sc[3], qn[4], Rq[9], M[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) sc[a] = valid ? expf(l3[a]) : 0.f;
        const float qlen = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        {
            const float iq = 1.f / qlen;
            qn[0] = q.x * iq; qn[1] = q.y * iq; qn[2] = q.z * iq; qn[3] = q.w * iq;
        }
        const float opac = valid ? 1.f / (1.f + expf(-lg)) : 0.f;
        quat_rot(qn[0], qn[1], qn[2], qn[3], Rq);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) M[3 * a + b] = Rq[3 * a + b] * sc[b];
        {
            float *ms = s_ms + threadIdx.x * 9;
            ms[0] = mx; ms[1] = my; ms[2] = mz;
            ms[3] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
            ms[4] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
            ms[5] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
            ms[6] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
            ms[7] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
            ms[8] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) s_acc[threadIdx.x * NA + a] = 0.f;
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) s_gf[threadIdx.x * GP + k] = 0.f;
        s_row[threadIdx.x] = valid ? i : -1;
        __syncthreads();   // (s_vr and s_vany initialised)
        {
            const int wvb = __reduce_min_sync(0xffffffffu, vb), wve = __reduce_max_sync(0xffffffffu, ve);
            if (lane == 0) {
                atomicMin(&s_vr[0], wvb);
                atomicMax(&s_vr[1], wve);
            }
        }
        __syncthreads();
        const int bvb = s_vr[0], bve = s_vr[1];
        // views in windows of 64: first every view's 2D-gradient row of this
        // Gaussian (all loads in flight together) into a bit mask, then the
        // views where some Gaussian of the block has a gradient, one by one
        for (int w0 = bvb; w0 < bve; w0 += 64) {
            const int w1 = min(bve, w0 + 64);
            unsigned long long vmask = 0ull;
#pragma unroll 4
            for (int v = max(w0, vb); v < min(w1, ve); ++v) {
                const long long slot = L.v[v].slot_base + li;
                const float4 a4 = grad2d[3 * slot], b4 = grad2d[3 * slot + 1];
                const float c0 = reinterpret_cast<const float *>(grad2d)[12 * slot + 8];
                const bool c = a4.x != 0.f || a4.y != 0.f || a4.z != 0.f || a4.w != 0.f || b4.x != 0.f || b4.y != 0.f ||
                               b4.z != 0.f || b4.w != 0.f || c0 != 0.f;
                vmask |= (unsigned long long)c << (v - w0);
            }
            // the views where some lane of this warp has a gradient, and per
            // view the block's count: the cost of the two ways to run this
            // window's chains, in chain runs of a warp (owner lanes: one per
            // (warp, view) with a gradient; lists: ceil(count / 32) per view
            // plus PB_LIST_VIEW_COST for the view's listing and barriers)
            const unsigned long long wm = (unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned int)vmask) |
                                          ((unsigned long long)__reduce_or_sync(0xffffffffu,
                                                                                (unsigned int)(vmask >> 32)) << 32);
            if (lane == 0) {
                atomicOr(&s_vany, wm);
                atomicAdd(&s_owner_runs, __popcll(wm));
            }
            for (unsigned long long b = wm; b;) {
                const int j = __ffsll((long long)b) - 1;
                b &= b - 1;
                const int cnt = __popc(__ballot_sync(0xffffffffu, (vmask >> j) & 1ull));
                if (lane == 0) atomicAdd(&s_vcnt[j], cnt);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int list_runs = 0;
                for (unsigned long long b = s_vany; b;) {
                    const int j = __ffsll((long long)b) - 1;
                    b &= b - 1;
                    list_runs += (s_vcnt[j] + 31) / 32 + PB_LIST_VIEW_COST;
                }
                s_lists = list_runs < s_owner_runs;
            }
            __syncthreads();
            unsigned long long todo = s_vany;
            const bool lists = s_lists;
            __syncthreads();   // read by every thread before they are cleared for the next window
            if (threadIdx.x == 0) {
                s_vany = 0ull;
                s_owner_runs = 0;
            }
            if (threadIdx.x < 64) s_vcnt[threadIdx.x] = 0;
            __syncthreads();   // cleared before any warp adds the next window's
            if (!lists) {
                // owner lanes: each warp walks the views where one of its lanes
                // has a gradient, in ascending order, the other lanes idle (no
                // list, no block barrier per view: cheaper where gradients are sparse)
                const float *ms = s_ms + threadIdx.x * 9;
                float *acc = s_acc + threadIdx.x * NA;
                float gm[3] = {acc[0], acc[1], acc[2]}, go = acc[3];
                float GS00 = acc[4], GS01 = acc[5], GS02 = acc[6], GS11 = acc[7], GS12 = acc[8], GS22 = acc[9];
                for (unsigned long long b = wm; b;) {
                    const int j = __ffsll((long long)b) - 1;
                    b &= b - 1;
                    const int v = w0 + j;
                    float pg[12];
#pragma unroll
                    for (int cc = 0; cc < 12; ++cc) pg[cc] = 0.f;
                    if ((vmask >> j) & 1ull) {
                        const long long slot = L.v[v].slot_base + li;
                        const float4 ga4 = grad2d[3 * slot], gb4 = grad2d[3 * slot + 1], gc4 = grad2d[3 * slot + 2];
                        view_term<DEG, true>(L, v, slot, ga4, gb4, gc4, proj, viewmats, intr, ms[0], ms[1], ms[2],
                                             ms[3], ms[4], ms[5], ms[6], ms[7], ms[8], sh + 3LL * K * i,
                                             s_gf + threadIdx.x * GP, gm, go, GS00, GS01, GS02, GS11, GS12, GS22, pg);
                    }
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
                acc[0] = gm[0]; acc[1] = gm[1]; acc[2] = gm[2]; acc[3] = go;
                acc[4] = GS00; acc[5] = GS01; acc[6] = GS02; acc[7] = GS11; acc[8] = GS12; acc[9] = GS22;
                todo = 0ull;
            }
            while (todo) {
                const int v = w0 + __ffsll((long long)todo) - 1;
                todo &= todo - 1;
                const bool c = (vmask >> (v - w0)) & 1ull;
                const unsigned int bal = __ballot_sync(0xffffffffu, c);
                if (lane == 0) s_wsum[wid] = __popc(bal);
                __syncthreads();
                int at = __popc(bal & ((1u << lane) - 1u)), total = 0;
#pragma unroll
                for (int w = 0; w < PB_WARPS; ++w) {
                    if (w < wid) at += s_wsum[w];
                    total += s_wsum[w];
                }
                if (c) s_list[at] = threadIdx.x;
                __syncthreads();
                // the list, one Gaussian per thread (threads past it idle)
                float pg[12];
#pragma unroll
                for (int cc = 0; cc < 12; ++cc) pg[cc] = 0.f;
                const bool has = (int)threadIdx.x < total;
                if (has) {
                    const int rr = s_list[threadIdx.x];
                    const long long g2 = base + rr;
                    const int s2 = scene_of_thread(L, g2);
                    const long long li2 = g2 - L.s[s2].thread_base;
                    const long long i2 = L.s[s2].g_begin + li2;
                    const long long slot = L.v[v].slot_base + li2;
                    const float4 ga4 = grad2d[3 * slot], gb4 = grad2d[3 * slot + 1], gc4 = grad2d[3 * slot + 2];
                    const float *ms = s_ms + rr * 9;
                    float *acc = s_acc + rr * NA;
                    float gm[3] = {acc[0], acc[1], acc[2]}, go = acc[3];
                    float GS00 = acc[4], GS01 = acc[5], GS02 = acc[6], GS11 = acc[7], GS12 = acc[8], GS22 = acc[9];
                    view_term<DEG, true>(L, v, slot, ga4, gb4, gc4, proj, viewmats, intr, ms[0], ms[1], ms[2], ms[3],
                                             ms[4], ms[5], ms[6], ms[7], ms[8], sh + 3LL * K * i2, s_gf + rr * GP, gm,
                                             go, GS00, GS01, GS02, GS11, GS12, GS22, pg);
                    acc[0] = gm[0]; acc[1] = gm[1]; acc[2] = gm[2]; acc[3] = go;
                    acc[4] = GS00; acc[5] = GS01; acc[6] = GS02; acc[7] = GS11; acc[8] = GS12; acc[9] = GS22;
                }
                if (__any_sync(0xffffffffu, has)) {
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
                __syncthreads();   // the sums are updated and the list is free for the next view
            }
        }
        if (valid) {
            const float *acc = s_acc + threadIdx.x * NA;
            const float gm[3] = {acc[0], acc[1], acc[2]};
            gauss_epilogue(i, L.accumulate, M, Rq, sc, qn, qlen, opac, gm, acc[3], acc[4], acc[5], acc[6], acc[7],
                           acc[8], acc[9], g_means, g_log_scales, g_quats, g_logits);
        }
        // the block's SH-coefficient gradients: row r goes to Gaussian s_row[r]
        __syncthreads();   // (owner lanes end without a barrier)
        write_sh_rows<K>(s_gf, s_row, g_sh, L.accumulate);
        __syncthreads();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nv * 12; e += PB_THREADS) {
        const int v = e / 12, cc = e % 12;
        float a = 0.f;
#pragma unroll
        for (int ww = 0; ww < PB_WARPS; ++ww) a += s_pose[(ww * nv + v) * 12 + cc];
        pose_partials[((long long)v * gridDim.x + blockIdx.x) * 12 + cc] = a;
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
    (void)status;   // (no bounded wait on this path)
    // one-view calls run the chain over the Gaussians with a nonzero 2D
    // gradient only (see COMPACT); each block zeroes its range's rows first
    const bool compact = L.n_views == 1;
#define GS_PB(D, G, Z)                                                                                             \
    k_project_bwd<D, G, Z><<<nblk, PB_THREADS, dyn, st>>>(                                                         \
        L, g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, viewmats, intr, p, g2, out->means,        \
        out->log_scales, out->quats, out->opacity_logits, out->sh, out->pose_partials)
    // one-view calls with parameter gradients and overlap_prev: a programmatic
    // dependent of the kernel ahead (the raster backward in a step), so that
    // each block zeroes its rows while that kernel's tail still runs
#define GS_PB_EARLY(D)                                                                                             \
    do {                                                                                                           \
        cudaLaunchConfig_t lc = {};                                                                                \
        cudaLaunchAttribute at[1];                                                                                 \
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                                            \
        at[0].val.programmaticStreamSerializationAllowed = 1;                                                     \
        lc.gridDim = dim3(nblk);                                                                                   \
        lc.blockDim = dim3(PB_THREADS);                                                                            \
        lc.dynamicSmemBytes = dyn;                                                                                 \
        lc.stream = st;                                                                                            \
        lc.attrs = at;                                                                                             \
        lc.numAttrs = 1;                                                                                           \
        if (cudaLaunchKernelEx(&lc, k_project_bwd<D, true, true>, L, g->means, g->log_scales, g->quats,           \
                               g->opacity_logits, g->sh, viewmats, intr, p, g2, out->means, out->log_scales,      \
                               out->quats, out->opacity_logits, out->sh, out->pose_partials) != cudaSuccess)      \
            return GS_ERR_CUDA;                                                                                    \
    } while (0)
    // (the per-view pose partials of up to GS_MAX_VIEWS views take the
    // several-view kernel to the default 48 KB of shared memory per block)
#define GS_PBV(D)                                                                                                  \
    do {                                                                                                           \
        static bool big_smem = false;                                                                              \
        if (!big_smem) {                                                                                           \
            if (cudaFuncSetAttribute(k_project_bwd_views<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                     (int)(PB_WARPS * GS_MAX_VIEWS * 12 * sizeof(float))) != cudaSuccess)          \
                return GS_ERR_CUDA;                                                                                \
            big_smem = true;                                                                                       \
        }                                                                                                          \
        k_project_bwd_views<D><<<nblk, PB_THREADS, dyn, st>>>(                                                     \
            L, g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, viewmats, intr, p, g2, out->means,    \
            out->log_scales, out->quats, out->opacity_logits, out->sh, out->pose_partials);                       \
    } while (0)
    if (want_gauss && !compact) {
        switch (deg) {
        case 0: GS_PBV(0); break;
        case 1: GS_PBV(1); break;
        case 2: GS_PBV(2); break;
        case 3: GS_PBV(3); break;
        default: return GS_ERR_UNSUPPORTED;
        }
    } else if (want_gauss && L.overlap_prev) {
        switch (deg) {
        case 0: GS_PB_EARLY(0); break;
        case 1: GS_PB_EARLY(1); break;
        case 2: GS_PB_EARLY(2); break;
        case 3: GS_PB_EARLY(3); break;
        default: return GS_ERR_UNSUPPORTED;
        }
    } else if (want_gauss) {
        switch (deg) {
        case 0: GS_PB(0, true, true); break;
        case 1: GS_PB(1, true, true); break;
        case 2: GS_PB(2, true, true); break;
        case 3: GS_PB(3, true, true); break;
        default: return GS_ERR_UNSUPPORTED;
        }
    } else {
        // the pose-only backward reads a Gaussian's parameters only in its
        // contributing views already (per-thread path)
        switch (deg) {
        case 0: if (compact) GS_PB(0, false, true); else GS_PB(0, false, false); break;
        case 1: if (compact) GS_PB(1, false, true); else GS_PB(1, false, false); break;
        case 2: if (compact) GS_PB(2, false, true); else GS_PB(2, false, false); break;
        case 3: if (compact) GS_PB(3, false, true); else GS_PB(3, false, false); break;
        default: return GS_ERR_UNSUPPORTED;
        }
    }
#undef GS_PB
#undef GS_PB_EARLY
#undef GS_PBV
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
