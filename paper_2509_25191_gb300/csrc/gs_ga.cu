// Camera global alignment (Section 3.3): candidate pairs by viewing angle,
// epipolar distances of keypoint matches under the current cameras, the
// weighted loss of Eq. 2 with its gradient to every camera's intrinsics and
// extrinsics, and the histogram-PDF weights (Eq. 3) and median order
// statistics (Eq. 4) of the initial distances.
//
// The per-iteration work is k_ga_pairs (one block per image pair, 20 bytes
// per match streamed once with four loads in flight per thread, HBM-bound)
// followed by the tiny k_ga_total and k_ga_cams. The
// distance is evaluated in normalised coordinates, s = x^'^T E x^ with
// x^ = K_i^-1 x, x^' = K_j^-1 x', which is x'^T F x without forming F, and
// the gradient is accumulated per pair as G^ = sum_k a^_k x^_k^T with
// a^ = K_j^-1 de/dl (l = F x): dL/dE = G^/W, and the intrinsics' gradients
// follow from E^T G^ and E G^^T without cancellation between K entries.
#include <climits>

#include "gs_common.cuh"

namespace gsk {

constexpr int GA_THREADS = 128;
constexpr int GA_CAM_THREADS = 128;
constexpr int GA_SEL_THREADS = 1024;
constexpr int GA_RADIX_BINS = 2048;

struct GaCam {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
};

__device__ __forceinline__ void ga_load_cam(const float *intr, const float *vm, int n, GaCam &c) {
    c.fx = intr[4 * n + 0];
    c.fy = intr[4 * n + 1];
    c.cx = intr[4 * n + 2];
    c.cy = intr[4 * n + 3];
#pragma unroll
    for (int k = 0; k < 9; ++k) c.R[k] = vm[12 * n + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) c.t[k] = vm[12 * n + 9 + k];
}

// R = R_j R_i^T, t = t_j - R t_i, E = [t]x R.
__device__ __forceinline__ void ga_relative(const GaCam &a, const GaCam &b, float R[9], float t[3], float E[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            R[3 * r + c] = b.R[3 * r + 0] * a.R[3 * c + 0] + b.R[3 * r + 1] * a.R[3 * c + 1] +
                           b.R[3 * r + 2] * a.R[3 * c + 2];
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = b.t[r] - (R[3 * r] * a.t[0] + R[3 * r + 1] * a.t[1] + R[3 * r + 2] * a.t[2]);
    // rows of [t]x: (0, -t2, t1), (t2, 0, -t0), (-t1, t0, 0)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        E[c] = -t[2] * R[3 + c] + t[1] * R[6 + c];
        E[3 + c] = t[2] * R[c] - t[0] * R[6 + c];
        E[6 + c] = -t[1] * R[c] + t[0] * R[3 + c];
    }
}

template <int NV>
__device__ __forceinline__ void warp_sum(float (&v)[NV]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// ---------------------------------------------------------------------------
// Per pair: distances, sum w e, sum w and G^ (9 values).
// ---------------------------------------------------------------------------
struct GaPairGeom {
    float E[9];
    float cxi, cyi, cxj, cyj, rfi, rgi, rfj, rgj;
};

// One match: e = |x^'.m| / |(m0/fx_j, m1/fy_j)| with m = E x^, and its
// contribution to sum w e, sum w and G^ = sum a^ x^^T.
template <bool WRITE_DIST>
__device__ __forceinline__ void ga_match(const GaPairGeom &g, float4 q, float w, float *acc, float *dist_k) {
    const float x0 = (q.x - g.cxi) * g.rfi, x1 = (q.y - g.cyi) * g.rgi;
    const float y0 = (q.z - g.cxj) * g.rfj, y1 = (q.w - g.cyj) * g.rgj;
    const float m0 = fmaf(g.E[0], x0, fmaf(g.E[1], x1, g.E[2]));
    const float m1 = fmaf(g.E[3], x0, fmaf(g.E[4], x1, g.E[5]));
    const float m2 = fmaf(g.E[6], x0, fmaf(g.E[7], x1, g.E[8]));
    const float s = fmaf(y0, m0, fmaf(y1, m1, m2));
    const float l0 = m0 * g.rfj, l1 = m1 * g.rgj;
    const float n2 = fmaf(l0, l0, l1 * l1);
    float e = 0.f;
    if (n2 > 0.f && n2 < INFINITY) {
        const float rn = rsqrtf(n2);
        const float as = fabsf(s);
        e = as * rn;
        const float c1 = s > 0.f ? w * rn : (s < 0.f ? -w * rn : 0.f);
        const float c2 = w * as * rn * rn * rn;
        const float h0 = c1 * y0 - c2 * l0 * g.rfj;
        const float h1 = c1 * y1 - c2 * l1 * g.rgj;
        const float h2 = c1;
        acc[2] = fmaf(h0, x0, acc[2]);
        acc[3] = fmaf(h0, x1, acc[3]);
        acc[4] += h0;
        acc[5] = fmaf(h1, x0, acc[5]);
        acc[6] = fmaf(h1, x1, acc[6]);
        acc[7] += h1;
        acc[8] = fmaf(h2, x0, acc[8]);
        acc[9] = fmaf(h2, x1, acc[9]);
        acc[10] += h2;
    }
    if (WRITE_DIST) *dist_k = e;
    acc[0] = fmaf(w, e, acc[0]);
    acc[1] += w;
}

constexpr int GA_UNROLL = 4;
template <bool WRITE_DIST>
__global__ void __launch_bounds__(GA_THREADS) k_ga_pairs(const gs_ga_problem P, float *__restrict__ dist,
                                                         float *__restrict__ pair_sums, int32_t *status) {
    __shared__ float s_red[GA_THREADS / 32][11];
    const float4 *__restrict__ M4 = reinterpret_cast<const float4 *>(P.matches);
    const float *__restrict__ Wt = P.weights;
    for (long long m = blockIdx.x; m < P.n_pairs; m += gridDim.x) {
        const int ci = P.pairs[2 * m], cj = P.pairs[2 * m + 1];
        const long long a = P.match_offsets[m], b = P.match_offsets[m + 1];
        if (ci < 0 || ci >= P.n_cams || cj < 0 || cj >= P.n_cams || a < 0 || a > b || b > P.n_matches) {
            // malformed pair (block-uniform): contributes nothing, reported
            if (threadIdx.x < GS_GA_PAIR_FLOATS) pair_sums[m * GS_GA_PAIR_FLOATS + threadIdx.x] = 0.f;
            if (threadIdx.x == 0 && status) {
                status[0] = GS_ERR_ARG;
                status[1] = (int32_t)m;
                status[2] = 0;
            }
            continue;
        }
        GaCam A, B;
        ga_load_cam(P.intrinsics, P.viewmats, ci, A);
        ga_load_cam(P.intrinsics, P.viewmats, cj, B);
        GaPairGeom g;
        float R[9], t[3];
        ga_relative(A, B, R, t, g.E);
        g.cxi = A.cx;
        g.cyi = A.cy;
        g.cxj = B.cx;
        g.cyj = B.cy;
        g.rfi = 1.f / A.fx;
        g.rgi = 1.f / A.fy;
        g.rfj = 1.f / B.fx;
        g.rgj = 1.f / B.fy;
        float acc[11];
#pragma unroll
        for (int k = 0; k < 11; ++k) acc[k] = 0.f;
        long long k = a + threadIdx.x;
        // GA_UNROLL matches in flight per thread: all loads first, then the math
        for (; k + (GA_UNROLL - 1) * GA_THREADS < b; k += GA_UNROLL * GA_THREADS) {
            float4 q[GA_UNROLL];
            float w[GA_UNROLL];
#pragma unroll
            for (int u = 0; u < GA_UNROLL; ++u) {
                q[u] = __ldcs(M4 + k + u * GA_THREADS);
                w[u] = Wt ? __ldcs(Wt + k + u * GA_THREADS) : 1.f;
            }
#pragma unroll
            for (int u = 0; u < GA_UNROLL; ++u)
                ga_match<WRITE_DIST>(g, q[u], w[u], acc, WRITE_DIST ? dist + k + u * GA_THREADS : nullptr);
        }
        for (; k < b; k += GA_THREADS)
            ga_match<WRITE_DIST>(g, __ldcs(M4 + k), Wt ? __ldcs(Wt + k) : 1.f, acc, WRITE_DIST ? dist + k : nullptr);
        warp_sum(acc);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0)
#pragma unroll
            for (int k2 = 0; k2 < 11; ++k2) s_red[warp][k2] = acc[k2];
        __syncthreads();
        if (threadIdx.x < 11) {
            float v = 0.f;
#pragma unroll
            for (int w8 = 0; w8 < GA_THREADS / 32; ++w8) v += s_red[w8][threadIdx.x];
            // layout: G^ row-major (9), sum w e, sum w, 0
            const int slot = threadIdx.x < 2 ? 9 + threadIdx.x : threadIdx.x - 2;
            pair_sums[m * GS_GA_PAIR_FLOATS + slot] = v;
        }
        if (threadIdx.x == 11) pair_sums[m * GS_GA_PAIR_FLOATS + 11] = 0.f;
        __syncthreads();
    }
}

// Block-wide fixed-order sum of NV values (blockDim.x = GA_CAM_THREADS).
template <int NV>
__device__ __forceinline__ void block_sum_cam(float (&v)[NV], float (*s_red)[NV]) {
    warp_sum(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) s_red[warp][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < GA_CAM_THREADS / 32; ++w) s += s_red[w][k];
        v[k] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Totals over all pairs in a fixed order (one block): the loss
// sum w e / sum w, and 1 / sum w for the camera gradients (stored in the pad
// slot of pair 0's partial sums).
// ---------------------------------------------------------------------------
constexpr int GA_TOTAL_THREADS = 1024;

__global__ void __launch_bounds__(GA_TOTAL_THREADS) k_ga_total(long long n_pairs, float *pair_sums, float *loss) {
    __shared__ float s_we[GA_TOTAL_THREADS / 32], s_w[GA_TOTAL_THREADS / 32];
    float we = 0.f, w = 0.f;
    for (long long m = threadIdx.x; m < n_pairs; m += GA_TOTAL_THREADS) {
        we += pair_sums[m * GS_GA_PAIR_FLOATS + 9];
        w += pair_sums[m * GS_GA_PAIR_FLOATS + 10];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        we += __shfl_xor_sync(0xffffffffu, we, o);
        w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_we[threadIdx.x >> 5] = we;
        s_w[threadIdx.x >> 5] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int k = 0; k < GA_TOTAL_THREADS / 32; ++k) {
            a += s_we[k];
            b += s_w[k];
        }
        const float inv = b > 0.f ? 1.f / b : 0.f;
        loss[0] = a * inv;
        if (n_pairs > 0) pair_sums[GS_GA_PAIR_FLOATS - 1] = inv;
    }
}

// ---------------------------------------------------------------------------
// Per camera: chain every incident pair's G^ to (fx, fy, cx, cy, R, t),
// reduce in a fixed order and divide by W = sum of all weights.
// ---------------------------------------------------------------------------
struct GaStepArgs {
    const float *intr0, *vm0;
    float *res, *m, *v, *d_res;
    const int32_t *step;
    float lr, eps;
    float b1, b2, omb1, omb2;   // beta and 1 - beta (formed in double on the host)
    float lnb1, lnb2;           // ln beta (double on the host)
    int focal;
};

__device__ void ga_residual_step(const GaStepArgs &S, int c, const float gI[4], const float gV[12]);

template <bool STEP>
__global__ void __launch_bounds__(GA_CAM_THREADS) k_ga_cams(const gs_ga_problem P, const float *__restrict__ pair_sums,
                                                            const int32_t *__restrict__ cam_offsets,
                                                            const int32_t *__restrict__ cam_pairs, float *loss,
                                                            float *d_intr, float *d_vm, const GaStepArgs S) {
    __shared__ float s_red16[GA_CAM_THREADS / 32][16];
    // 1 / sum of all weights, left by k_ga_total in the pad slot of row 0
    const float invW = P.n_pairs > 0 ? pair_sums[GS_GA_PAIR_FLOATS - 1] : 0.f;
    const int c = blockIdx.x;
    float g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = 0.f;
    const bool lists = cam_offsets && cam_pairs;
    const long long e_beg = lists ? (long long)max(0, cam_offsets[c]) : 0;
    const long long e_end = lists ? min((long long)cam_offsets[c + 1], (long long)(2 * P.n_pairs)) : 0;
    for (long long e = e_beg + threadIdx.x; e < e_end; e += GA_CAM_THREADS) {
        const int code = cam_pairs[e];
        const long long m = code >> 1;
        if (code < 0 || m >= P.n_pairs) continue;
        const bool second = code & 1;
        const int ci = P.pairs[2 * m], cj = P.pairs[2 * m + 1];
        if (ci < 0 || ci >= P.n_cams || cj < 0 || cj >= P.n_cams || (second ? cj : ci) != c) continue;
        GaCam A, B;
        ga_load_cam(P.intrinsics, P.viewmats, ci, A);
        ga_load_cam(P.intrinsics, P.viewmats, cj, B);
        float R[9], t[3], E[9], G[9];
        ga_relative(A, B, R, t, E);
#pragma unroll
        for (int k = 0; k < 9; ++k) G[k] = pair_sums[m * GS_GA_PAIR_FLOATS + k];
        // dL/dR_rel = [t]x^T G = -[t]x G ; M = G R^T ; dL/dt_rel from M
        float GR[9], Mt[9];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            GR[cc] = -(-t[2] * G[3 + cc] + t[1] * G[6 + cc]);
            GR[3 + cc] = -(t[2] * G[cc] - t[0] * G[6 + cc]);
            GR[6 + cc] = -(-t[1] * G[cc] + t[0] * G[3 + cc]);
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                Mt[3 * r + cc] = G[3 * r] * R[3 * cc] + G[3 * r + 1] * R[3 * cc + 1] + G[3 * r + 2] * R[3 * cc + 2];
        const float Gt[3] = {Mt[7] - Mt[5], Mt[2] - Mt[6], Mt[3] - Mt[1]};
        // the translation t_rel = t_j - R t_i also depends on R: G_R' = G_R - G_t t_i^T
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) GR[3 * r + cc] -= Gt[r] * A.t[cc];
        if (!second) {
            // intrinsics of the first camera: Q = E^T G^
            const float q00 = E[0] * G[0] + E[3] * G[3] + E[6] * G[6];
            const float q02 = E[0] * G[2] + E[3] * G[5] + E[6] * G[8];
            const float q11 = E[1] * G[1] + E[4] * G[4] + E[7] * G[7];
            const float q12 = E[1] * G[2] + E[4] * G[5] + E[7] * G[8];
            g[0] -= q00 / A.fx;
            g[1] -= q11 / A.fy;
            g[2] -= q02 / A.fx;
            g[3] -= q12 / A.fy;
            // dL/dR_i = G_R'^T R_j ; dL/dt_i = -R^T G_t
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    g[4 + 3 * r + cc] += GR[r] * B.R[cc] + GR[3 + r] * B.R[3 + cc] + GR[6 + r] * B.R[6 + cc];
#pragma unroll
            for (int r = 0; r < 3; ++r) g[13 + r] -= R[r] * Gt[0] + R[3 + r] * Gt[1] + R[6 + r] * Gt[2];
        } else {
            // intrinsics of the second camera: Q = E G^^T
            const float q00 = E[0] * G[0] + E[1] * G[1] + E[2] * G[2];
            const float q02 = E[0] * G[6] + E[1] * G[7] + E[2] * G[8];
            const float q11 = E[3] * G[3] + E[4] * G[4] + E[5] * G[5];
            const float q12 = E[3] * G[6] + E[4] * G[7] + E[5] * G[8];
            g[0] -= q00 / B.fx;
            g[1] -= q11 / B.fy;
            g[2] -= q02 / B.fx;
            g[3] -= q12 / B.fy;
            // dL/dR_j = G_R' R_i ; dL/dt_j = G_t
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    g[4 + 3 * r + cc] += GR[3 * r] * A.R[cc] + GR[3 * r + 1] * A.R[3 + cc] + GR[3 * r + 2] * A.R[6 + cc];
#pragma unroll
            for (int r = 0; r < 3; ++r) g[13 + r] += Gt[r];
        }
    }
    block_sum_cam(g, s_red16);
    if (STEP) {
        if (threadIdx.x == 0) {
            float gI[4], gV[12];
#pragma unroll
            for (int k = 0; k < 4; ++k) gI[k] = g[k] * invW;
#pragma unroll
            for (int k = 0; k < 12; ++k) gV[k] = g[4 + k] * invW;
            ga_residual_step(S, c, gI, gV);
        }
        return;
    }
    if (threadIdx.x < 4) d_intr[4 * c + threadIdx.x] = g[threadIdx.x] * invW;
    else if (threadIdx.x < 16) d_vm[12 * c + threadIdx.x - 4] = g[threadIdx.x] * invW;
}

// ---------------------------------------------------------------------------
// Residual parametrisation of the cameras and its backward (fused step).
// ---------------------------------------------------------------------------
struct Rot6 {
    float b1[3], b2[3], b3[3], a2[3];
    float n1, nu, s;
};

__device__ __forceinline__ void rot6_fwd(const float *a, Rot6 &r) {
    r.n1 = sqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.b1[k] = a[k] / r.n1;
#pragma unroll
    for (int k = 0; k < 3; ++k) r.a2[k] = a[3 + k];
    r.s = r.b1[0] * r.a2[0] + r.b1[1] * r.a2[1] + r.b1[2] * r.a2[2];
    float u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = r.a2[k] - r.s * r.b1[k];
    r.nu = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.b2[k] = u[k] / r.nu;
    r.b3[0] = r.b1[1] * r.b2[2] - r.b1[2] * r.b2[1];
    r.b3[1] = r.b1[2] * r.b2[0] - r.b1[0] * r.b2[2];
    r.b3[2] = r.b1[0] * r.b2[1] - r.b1[1] * r.b2[0];
}

__global__ void k_ga_apply(const GaStepArgs S, int n, float *intr, float *vm, int32_t *step) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) step[0] += 1;
    if (c >= n) return;
    const float *res = S.res + 10 * c;
    Rot6 r;
    rot6_fwd(res, r);
    const float *R0 = S.vm0 + 12 * c;
    // R = dR R0 with dR = [b1 b2 b3] (columns): dR[i][k] = b_k[i]
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            vm[12 * c + 3 * i + j] = r.b1[i] * R0[j] + r.b2[i] * R0[3 + j] + r.b3[i] * R0[6 + j];
#pragma unroll
    for (int k = 0; k < 3; ++k) vm[12 * c + 9 + k] = R0[9 + k] + res[6 + k];
    const float sc = S.focal ? expf(res[9]) : 1.f;
    intr[4 * c + 0] = S.intr0[4 * c + 0] * sc;
    intr[4 * c + 1] = S.intr0[4 * c + 1] * sc;
    intr[4 * c + 2] = S.intr0[4 * c + 2];
    intr[4 * c + 3] = S.intr0[4 * c + 3];
}

__device__ void ga_residual_step(const GaStepArgs &S, int c, const float gI[4], const float gV[12]) {
    float *res = S.res + 10 * c;
    Rot6 r;
    rot6_fwd(res, r);
    const float *R0 = S.vm0 + 12 * c;
    // G_dR = G_R' R0^T; its columns are the gradients of b1, b2, b3
    float g1[3], g2[3], g3[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g1[i] = gV[3 * i] * R0[0] + gV[3 * i + 1] * R0[1] + gV[3 * i + 2] * R0[2];
        g2[i] = gV[3 * i] * R0[3] + gV[3 * i + 1] * R0[4] + gV[3 * i + 2] * R0[5];
        g3[i] = gV[3 * i] * R0[6] + gV[3 * i + 1] * R0[7] + gV[3 * i + 2] * R0[8];
    }
    // b3 = b1 x b2
    g1[0] += r.b2[1] * g3[2] - r.b2[2] * g3[1];
    g1[1] += r.b2[2] * g3[0] - r.b2[0] * g3[2];
    g1[2] += r.b2[0] * g3[1] - r.b2[1] * g3[0];
    g2[0] += g3[1] * r.b1[2] - g3[2] * r.b1[1];
    g2[1] += g3[2] * r.b1[0] - g3[0] * r.b1[2];
    g2[2] += g3[0] * r.b1[1] - g3[1] * r.b1[0];
    // b2 = u / |u|
    const float d2 = r.b2[0] * g2[0] + r.b2[1] * g2[1] + r.b2[2] * g2[2];
    float gu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) gu[k] = (g2[k] - r.b2[k] * d2) / r.nu;
    // u = a2 - (b1.a2) b1
    const float bgu = r.b1[0] * gu[0] + r.b1[1] * gu[1] + r.b1[2] * gu[2];
    float g[10];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g[3 + k] = gu[k] - bgu * r.b1[k];
        g1[k] += -r.s * gu[k] - bgu * r.a2[k];
    }
    // b1 = a1 / |a1|
    const float d1 = r.b1[0] * g1[0] + r.b1[1] * g1[1] + r.b1[2] * g1[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = (g1[k] - r.b1[k] * d1) / r.n1;
#pragma unroll
    for (int k = 0; k < 3; ++k) g[6 + k] = gV[9 + k];
    if (S.focal) {
        const float sc = expf(res[9]);
        g[9] = gI[0] * (S.intr0[4 * c] * sc) + gI[1] * (S.intr0[4 * c + 1] * sc);
    } else {
        g[9] = 0.f;
    }
    if (S.d_res)
#pragma unroll
        for (int k = 0; k < 10; ++k) S.d_res[10 * c + k] = g[k];
    // Adam with the bias correction of the incremented step
    // 1 - beta^t = -expm1(t ln beta): accurate in float for every t (no
    // cancellation at small t), and no FP64 on the device
    const float t = (float)S.step[0];
    const float ibc1 = -1.f / expm1f(t * S.lnb1);
    const float ibc2 = -1.f / expm1f(t * S.lnb2);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        float m = S.m[10 * c + k], v = S.v[10 * c + k];
        m = S.b1 * m + S.omb1 * g[k];
        v = S.b2 * v + S.omb2 * g[k] * g[k];
        S.m[10 * c + k] = m;
        S.v[10 * c + k] = v;
        res[k] -= S.lr * (m * ibc1) / (sqrtf(v * ibc2) + S.eps);
    }
}

// ---------------------------------------------------------------------------
// Candidate pairs: one block; warps own rows i; pass 1 counts, a block scan
// gives row offsets, pass 2 writes in row-major order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool ga_pair_pass(const float *vm, int i, int j, float cos_thr) {
    const float *a = vm + 12 * i + 6, *b = vm + 12 * j + 6;
    const float d = __fadd_rn(__fadd_rn(__fmul_rn(a[0], b[0]), __fmul_rn(a[1], b[1])), __fmul_rn(a[2], b[2]));
    return d > cos_thr;
}

__global__ void __launch_bounds__(GA_SEL_THREADS) k_ga_select(const float *__restrict__ vm, int n, float cos_thr,
                                                              int32_t *pairs, long long capacity,
                                                              long long *n_out, int32_t *status) {
    extern __shared__ long long s_rows[];   // [n + 1] row counts, then offsets
    __shared__ long long s_part[GA_SEL_THREADS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = GA_SEL_THREADS / 32;
    for (int i = warp; i < n; i += nw) {
        long long cnt = 0;
        for (int j0 = i + 1; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const bool f = j < n && ga_pair_pass(vm, i, j, cos_thr);
            cnt += __popc(__ballot_sync(0xffffffffu, f));
        }
        if (lane == 0) s_rows[i] = cnt;
    }
    __syncthreads();
    // exclusive scan over n rows: contiguous segments per thread
    const int seg = (n + GA_SEL_THREADS - 1) / GA_SEL_THREADS;
    const int lo = min(n, (int)threadIdx.x * seg), hi = min(n, lo + seg);
    long long sum = 0;
    for (int r = lo; r < hi; ++r) sum += s_rows[r];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int k = 0; k < GA_SEL_THREADS; ++k) {
            const long long v = s_part[k];
            s_part[k] = run;
            run += v;
        }
        s_rows[n] = run;
    }
    __syncthreads();
    long long run = s_part[threadIdx.x];
    for (int r = lo; r < hi; ++r) {
        const long long v = s_rows[r];
        s_rows[r] = run;
        run += v;
    }
    __syncthreads();
    const long long total = s_rows[n];
    if (threadIdx.x == 0) {
        n_out[0] = total;
        if (total > capacity && status) {
            status[0] = GS_ERR_CAPACITY;
            status[1] = (int32_t)(total & 0xffffffff);
            status[2] = (int32_t)(total >> 32);
        }
    }
    if (total > capacity) return;
    for (int i = warp; i < n; i += nw) {
        long long off = s_rows[i];
        for (int j0 = i + 1; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const bool f = j < n && ga_pair_pass(vm, i, j, cos_thr);
            const unsigned mask = __ballot_sync(0xffffffffu, f);
            if (f) {
                const long long p = off + __popc(mask & ((1u << lane) - 1u));
                pairs[2 * p] = i;
                pairs[2 * p + 1] = j;
            }
            off += __popc(mask);
        }
    }
}

// ---------------------------------------------------------------------------
// Incidence lists: one block counts, scans and fills (shared atomics), then
// one block per camera sorts its list so that the order is fixed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GA_SEL_THREADS) k_ga_inc_build(const int32_t *__restrict__ pairs, long long n_pairs,
                                                                 int n, int32_t *cam_offsets, int32_t *cam_pairs,
                                                                 int32_t *status) {
    extern __shared__ int s_cnt[];   // [n + 1]
    __shared__ int s_part[GA_SEL_THREADS];
    for (int c = threadIdx.x; c <= n; c += GA_SEL_THREADS) s_cnt[c] = 0;
    __syncthreads();
    for (long long m = threadIdx.x; m < n_pairs; m += GA_SEL_THREADS) {
        const int i = pairs[2 * m], j = pairs[2 * m + 1];
        if (i < 0 || i >= n || j < 0 || j >= n) {   // left out, reported
            if (status) {
                status[0] = GS_ERR_ARG;
                status[1] = (int32_t)m;
                status[2] = 0;
            }
            continue;
        }
        atomicAdd(&s_cnt[i], 1);
        atomicAdd(&s_cnt[j], 1);
    }
    __syncthreads();
    const int seg = (n + GA_SEL_THREADS - 1) / GA_SEL_THREADS;
    const int lo = min(n, (int)threadIdx.x * seg), hi = min(n, lo + seg);
    int sum = 0;
    for (int r = lo; r < hi; ++r) sum += s_cnt[r];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < GA_SEL_THREADS; ++k) {
            const int v = s_part[k];
            s_part[k] = run;
            run += v;
        }
        s_cnt[n] = run;
        cam_offsets[n] = run;
    }
    __syncthreads();
    int run = s_part[threadIdx.x];
    for (int r = lo; r < hi; ++r) {
        const int v = s_cnt[r];
        s_cnt[r] = run;
        cam_offsets[r] = run;
        run += v;
    }
    __syncthreads();
    for (long long m = threadIdx.x; m < n_pairs; m += GA_SEL_THREADS) {
        const int i = pairs[2 * m], j = pairs[2 * m + 1];
        if (i < 0 || i >= n || j < 0 || j >= n) continue;
        cam_pairs[atomicAdd(&s_cnt[i], 1)] = (int32_t)(2 * m);
        cam_pairs[atomicAdd(&s_cnt[j], 1)] = (int32_t)(2 * m + 1);
    }
}

__global__ void __launch_bounds__(GA_SEL_THREADS) k_ga_inc_sort(const int32_t *__restrict__ cam_offsets,
                                                                int32_t *cam_pairs, int32_t *status) {
    __shared__ int s_key[GS_GA_MAX_CAMS];
    const int c = blockIdx.x;
    const int a = cam_offsets[c], len = cam_offsets[c + 1] - a;
    if (len <= 1) return;
    if (len > GS_GA_MAX_CAMS) {
        if (threadIdx.x == 0 && status) {
            status[0] = GS_ERR_ARG;
            status[1] = c;
            status[2] = 0;
        }
        return;
    }
    int np2 = 1;
    while (np2 < len) np2 <<= 1;
    for (int k = threadIdx.x; k < np2; k += GA_SEL_THREADS) s_key[k] = k < len ? cam_pairs[a + k] : INT_MAX;
    __syncthreads();
    for (int size = 2; size <= np2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < np2; k += GA_SEL_THREADS) {
                const int o = k ^ stride;
                if (o > k) {
                    const bool up = (k & size) == 0;
                    const int x = s_key[k], y = s_key[o];
                    if ((x > y) == up) {
                        s_key[k] = y;
                        s_key[o] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < len; k += GA_SEL_THREADS) cam_pairs[a + k] = s_key[k];
}

// ---------------------------------------------------------------------------
// Weights (Eq. 3) and median order statistics (Eq. 4).
// scratch words: [0] max bits, [1] radix prefix, [2] rank, [8..8+2048) radix
// histogram, [8+2048..) per-bin weight table (floats).
// ---------------------------------------------------------------------------
constexpr int GA_W_HIST = 8;
constexpr int GA_W_TABLE = 8 + GA_RADIX_BINS;

__global__ void __launch_bounds__(256) k_ga_max(const float *__restrict__ e, long long n, uint32_t *scratch) {
    uint32_t mx = 0;
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n; k += (long long)gridDim.x * 256)
        mx = max(mx, __float_as_uint(e[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&scratch[0], mx);
}

__device__ __forceinline__ int ga_bin(float e, float inv, int nb, bool any) {
    if (!any) return 0;
    return max(0, min(nb - 1, (int)floorf(__fmul_rn(e, inv))));
}

__global__ void __launch_bounds__(256) k_ga_hist(const float *__restrict__ e, long long n, int nb,
                                                 const uint32_t *__restrict__ scratch, uint32_t *counts) {
    extern __shared__ uint32_t s_h[];
    for (int b = threadIdx.x; b < nb; b += 256) s_h[b] = 0;
    __syncthreads();
    const float emax = __uint_as_float(scratch[0]);
    const bool any = emax > 0.f;
    const float inv = any ? __fdiv_rn((float)nb, emax) : 0.f;
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n; k += (long long)gridDim.x * 256)
        atomicAdd(&s_h[ga_bin(e[k], inv, nb, any)], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += 256)
        if (s_h[b]) atomicAdd(&counts[b], s_h[b]);
}

__global__ void __launch_bounds__(256) k_ga_table(const uint32_t *__restrict__ counts, int nb, long long n,
                                                  double alpha, uint32_t *scratch) {
    __shared__ double s_part[256];
    double s2 = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) s2 += (double)counts[b] * (double)counts[b];
    s_part[threadIdx.x] = s2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_part[threadIdx.x] += s_part[threadIdx.x + o];
        __syncthreads();
    }
    const double S2 = s_part[0];
    float *table = reinterpret_cast<float *>(scratch + GA_W_TABLE);
    for (int b = threadIdx.x; b < nb; b += 256)
        table[b] = counts[b] ? (float)pow((double)n * (double)counts[b] / S2, alpha) : 0.f;
}

__global__ void __launch_bounds__(256) k_ga_gather(const float *__restrict__ e, long long n, int nb,
                                                   const uint32_t *__restrict__ scratch, float *w) {
    const float emax = __uint_as_float(scratch[0]);
    const bool any = emax > 0.f;
    const float inv = any ? __fdiv_rn((float)nb, emax) : 0.f;
    const float *table = reinterpret_cast<const float *>(scratch + GA_W_TABLE);
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n; k += (long long)gridDim.x * 256)
        w[k] = table[ga_bin(e[k], inv, nb, any)];
}

// Radix select of the rank-th smallest key (float bits of e >= 0): three
// digit passes of 11, 11 and 10 bits from the top.
__global__ void __launch_bounds__(256) k_ga_radix_hist(const float *__restrict__ e, long long n, int shift, int bits,
                                                       uint32_t pmask, uint32_t *scratch) {
    __shared__ uint32_t s_h[GA_RADIX_BINS];
    for (int b = threadIdx.x; b < GA_RADIX_BINS; b += 256) s_h[b] = 0;
    __syncthreads();
    const uint32_t prefix = scratch[1];
    const uint32_t dmask = (1u << bits) - 1u;
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < n; k += (long long)gridDim.x * 256) {
        const uint32_t key = __float_as_uint(e[k]);
        if ((key & pmask) == prefix) atomicAdd(&s_h[(key >> shift) & dmask], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < GA_RADIX_BINS; b += 256)
        if (s_h[b]) atomicAdd(&scratch[GA_W_HIST + b], s_h[b]);
}

__global__ void k_ga_radix_init(uint32_t *scratch, uint32_t rank) {
    scratch[1] = 0u;
    scratch[2] = rank;
}

// One warp: find the digit holding the rank, extend the prefix, subtract the
// keys below it from the rank, clear the histogram for the next pass.
__global__ void k_ga_radix_pick(int shift, int bits, uint32_t *scratch, float *stats_out) {
    const int lane = threadIdx.x;
    const int nbins = 1 << bits, per = nbins / 32;
    uint32_t *h = scratch + GA_W_HIST;
    uint32_t rank = scratch[2];
    uint32_t local = 0;
    for (int k = 0; k < per; ++k) local += h[lane * per + k];
    // inclusive scan across lanes
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - local;
    const bool mine = rank >= excl && rank < incl;
    if (mine) {
        uint32_t r = rank - excl;
        int d = lane * per;
        while (r >= h[d]) {
            r -= h[d];
            ++d;
        }
        const uint32_t prefix = scratch[1] | ((uint32_t)d << shift);
        scratch[1] = prefix;
        scratch[2] = r;
        if (stats_out) *stats_out = __uint_as_float(prefix);
    }
    __syncwarp();
    for (int k = lane; k < nbins; k += 32) h[k] = 0;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// One block per pair (the hardware scheduler balances pairs of unequal size).
static unsigned ga_pairs_grid(long long n_pairs) {
    return (unsigned)(n_pairs < (1LL << 30) ? n_pairs : (1LL << 30));
}

int launch_ga_select(const float *vm, int n, float cos_thr, int32_t *pairs, long long capacity, long long *n_out,
                     int32_t *status, cudaStream_t st) {
    const size_t smem = sizeof(long long) * (size_t)(n + 1);
    if (smem > 48 * 1024)
        if (cudaFuncSetAttribute(k_ga_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GS_ERR_CUDA;
    k_ga_select<<<1, GA_SEL_THREADS, smem, st>>>(vm, n, cos_thr, pairs, capacity, n_out, status);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_ga_incidence(const int32_t *pairs, long long n_pairs, int n, int32_t *cam_offsets, int32_t *cam_pairs,
                        int32_t *status, cudaStream_t st) {
    const size_t smem = sizeof(int) * (size_t)(n + 1);
    k_ga_inc_build<<<1, GA_SEL_THREADS, smem, st>>>(pairs, n_pairs, n, cam_offsets, cam_pairs, status);
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    k_ga_inc_sort<<<n, GA_SEL_THREADS, 0, st>>>(cam_offsets, cam_pairs, status);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_ga_epipolar(const gs_ga_problem &P, float *dist, float *pair_sums, const int32_t *cam_offsets,
                       const int32_t *cam_pairs, float *loss, float *d_intr, float *d_vm, int32_t *status,
                       cudaStream_t st) {
    if (P.n_pairs > 0) {
        const unsigned grid = ga_pairs_grid(P.n_pairs);
        if (dist) k_ga_pairs<true><<<grid, GA_THREADS, 0, st>>>(P, dist, pair_sums, status);
        else k_ga_pairs<false><<<grid, GA_THREADS, 0, st>>>(P, dist, pair_sums, status);
        if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    }
    k_ga_total<<<1, GA_TOTAL_THREADS, 0, st>>>(P.n_pairs, pair_sums, loss);
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    if (d_intr && d_vm)
        k_ga_cams<false><<<P.n_cams, GA_CAM_THREADS, 0, st>>>(P, pair_sums, cam_offsets, cam_pairs, loss, d_intr,
                                                               d_vm, GaStepArgs{});
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_ga_step(const gs_ga_state &s, const gs_ga_problem &P, float *pair_sums, const int32_t *cam_offsets,
                   const int32_t *cam_pairs, float *loss, float *d_res, int32_t *status, cudaStream_t st) {
    GaStepArgs S;
    S.intr0 = s.intrinsics0;
    S.vm0 = s.viewmats0;
    S.res = s.residuals;
    S.m = s.exp_avg;
    S.v = s.exp_avg_sq;
    S.d_res = d_res;
    S.step = s.step;
    S.lr = s.lr;
    S.eps = (float)s.eps;
    S.b1 = (float)s.beta1;
    S.b2 = (float)s.beta2;
    S.omb1 = (float)(1.0 - s.beta1);
    S.omb2 = (float)(1.0 - s.beta2);
    S.lnb1 = (float)log(s.beta1);
    S.lnb2 = (float)log(s.beta2);
    S.focal = s.optimise_focal;
    k_ga_apply<<<(s.n_cams + 127) / 128, 128, 0, st>>>(S, s.n_cams, s.intrinsics, s.viewmats, s.step);
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    if (P.n_pairs > 0) {
        k_ga_pairs<false><<<ga_pairs_grid(P.n_pairs), GA_THREADS, 0, st>>>(P, nullptr, pair_sums, status);
        if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    }
    k_ga_total<<<1, GA_TOTAL_THREADS, 0, st>>>(P.n_pairs, pair_sums, loss);
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    k_ga_cams<true><<<P.n_cams, GA_CAM_THREADS, 0, st>>>(P, pair_sums, cam_offsets, cam_pairs, loss, nullptr,
                                                          nullptr, S);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int launch_ga_weights(const float *e, long long n, int nb, double alpha, uint32_t *counts, float *w, float *stats,
                      uint32_t *scratch, cudaStream_t st) {
    const size_t words = (size_t)GA_W_TABLE + (size_t)nb;
    if (cudaMemsetAsync(scratch, 0, words * 4, st) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(stats, 0, 4 * sizeof(float), st) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(counts, 0, (size_t)nb * 4, st) != cudaSuccess) return GS_ERR_CUDA;
    if (n == 0) return GS_OK;
    const int grid = 4 * num_sms();
    k_ga_max<<<grid, 256, 0, st>>>(e, n, scratch);
    const size_t smem = (size_t)nb * 4;
    if (smem > 48 * 1024)
        if (cudaFuncSetAttribute(k_ga_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GS_ERR_CUDA;
    k_ga_hist<<<2 * num_sms(), 256, smem, st>>>(e, n, nb, scratch, counts);
    k_ga_table<<<1, 256, 0, st>>>(counts, nb, n, alpha, scratch);
    k_ga_gather<<<grid, 256, 0, st>>>(e, n, nb, scratch, w);
    if (cudaMemcpyAsync(stats, scratch, 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return GS_ERR_CUDA;
    // median order statistics: ranks (n-1)/2 and n/2
    const long long ranks[2] = {(n - 1) / 2, n / 2};
    const int shifts[3] = {21, 10, 0}, bits[3] = {11, 11, 10};
    for (int r = 0; r < 2; ++r) {
        k_ga_radix_init<<<1, 1, 0, st>>>(scratch, (uint32_t)ranks[r]);
        uint32_t pmask = 0;
        for (int p = 0; p < 3; ++p) {
            k_ga_radix_hist<<<grid, 256, 0, st>>>(e, n, shifts[p], bits[p], pmask, scratch);
            k_ga_radix_pick<<<1, 32, 0, st>>>(shifts[p], bits[p], scratch, p == 2 ? stats + 1 + r : nullptr);
            pmask |= ((1u << bits[p]) - 1u) << shifts[p];
        }
    }
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gsk
