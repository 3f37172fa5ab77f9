// Projection of 3D Gaussians into every view that sees them (forward).
//
// One thread per Gaussian; the thread reads the Gaussian's raw record once
// (mean, log-scale, quaternion, opacity logit, SH) and loops over the views
// of its scene, writing one 64-byte record per (view, Gaussian) slot:
//   {x, y, ext_x, ext_y} {a, b, c, o} {r, g, b, radius} {x_lo, y_lo, depth, clamp_bits}
// with (a, b, c) the dilated 2D covariance (its inverse is the conic).
// Section 3.1: Sigma = R S S^T R^T, opacity, SH colour. EWA splatting:
// Sigma' = J W Sigma W^T J^T + dilation I, conic = inverse, radius =
// ceil(3 sqrt(lambda_max)). The camera-space mean and the pixel-space mean are
// carried as float pairs so that 1000-pixel-wide images keep ~1e-5 px
// accuracy (a plain float mean would be off by up to 1e-4 px there).
// ext_x, ext_y bound the pixels the Gaussian can reach: alpha >= alpha_min
// only inside the ellipse d^T conic d <= k, k = 2 ln(o / alpha_min), whose
// bounding box has half-extents sqrt(k Sigma'_xx), sqrt(k Sigma'_yy); they are
// clipped to the radius and enlarged by 2^-14 relative so that float32
// rounding never shrinks the region. A Gaussian with k <= 0 is culled.
#include <string.h>

#include "gs_common.cuh"

namespace gsk {

constexpr int PF_THREADS = 128;

// Staging of a block's 128 Gaussians for the degree-3 path (TMA): the SH rows
// (48 floats) arrive as a 32-float box with the 128-byte swizzle and a
// 16-float box with the 64-byte swizzle, so that each thread reads its own
// row 16 bytes at a time without bank conflicts; the 64-byte output records
// of a view leave as one 128-row box (64-byte swizzle) by a tensor store.
struct ProjStage {
    float4 shA[PF_THREADS * 8];
    float4 shB[PF_THREADS * 4];
    float4 out[PF_THREADS * 4];
    unsigned long long bar;
};

template <int DEG, bool TMA>
__global__ void __launch_bounds__(PF_THREADS) k_project_fwd(const Launch L, const float *__restrict__ means,
                                                            const float *__restrict__ log_scales,
                                                            const float *__restrict__ quats,
                                                            const float *__restrict__ logits,
                                                            const float *__restrict__ sh,
                                                            const float *__restrict__ viewmats,
                                                            const float *__restrict__ intr, float4 *__restrict__ proj,
                                                            const __grid_constant__ CUtensorMap tm_shA,
                                                            const __grid_constant__ CUtensorMap tm_shB,
                                                            const __grid_constant__ CUtensorMap tm_proj,
                                                            int *__restrict__ status) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    static_assert(!TMA || DEG == 3, "the staged path is for 48-float SH rows");
    __shared__ __align__(1024) ProjStage S[1];   // (removed by the compiler where unused)
    const long long gid0 = (long long)blockIdx.x * PF_THREADS;
    const long long gid = gid0 + threadIdx.x;
    // a block is "full" when its 128 threads are valid Gaussians of one
    // scene: then its SH rows and its records are contiguous and move as boxes
    bool full = false;
    long long li0 = 0;
    if (TMA) {
        const long long last = gid0 + PF_THREADS - 1;
        if (last < L.n_threads) {
            const int s0 = scene_of_thread(L, gid0);
            // (the swizzled boxes need a 1024-byte aligned destination)
            full = scene_of_thread(L, last) == s0 && (smem_u32(S[0].shA) & 1023u) == 0;
            li0 = gid0 - L.s[s0].thread_base;
            if (full && threadIdx.x == 0) {
                const int row = (int)(L.s[s0].g_begin + li0);
                mbar_init(&S[0].bar, 1);
                mbar_expect_tx(&S[0].bar, PF_THREADS * 48 * 4);
                tma_load_2d(S[0].shA, &tm_shA, 0, row, &S[0].bar);
                tma_load_2d(S[0].shB, &tm_shB, 32, row, &S[0].bar);
            }
            __syncthreads();
        }
    }
    if (gid >= L.n_threads) return;
    const int s = scene_of_thread(L, gid);
    const long long li = gid - L.s[s].thread_base;
    const long long i = L.s[s].g_begin + li;

    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
    const float l0 = log_scales[3 * i], l1 = log_scales[3 * i + 1], l2 = log_scales[3 * i + 2];
    const float4 q = reinterpret_cast<const float4 *>(quats)[i];
    const float lg = logits[i];
    float f[3 * K];
    if (TMA) {
        const int r = threadIdx.x;
        if (!full) {
            // a partial block stages its rows itself, in the same layout
            const float4 *src = reinterpret_cast<const float4 *>(sh + (long long)3 * K * i);
#pragma unroll
            for (int c = 0; c < 8; ++c) S[0].shA[swz128(r, c)] = src[c];
#pragma unroll
            for (int c = 0; c < 4; ++c) S[0].shB[swz64(r, c)] = src[8 + c];
        }
    } else if (DEG == 1 || DEG == 3) {
        const float4 *src = reinterpret_cast<const float4 *>(sh + (long long)3 * K * i);
#pragma unroll
        for (int k = 0; k < 3 * K / 4; ++k) {
            float4 t = src[k];
            f[4 * k] = t.x; f[4 * k + 1] = t.y; f[4 * k + 2] = t.z; f[4 * k + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) f[k] = sh[(long long)3 * K * i + k];
    }

    // activation and 3D covariance
    const float s0 = expf(l0), s1 = expf(l1), s2 = expf(l2);
    const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    const float qinv = rsqrtf(qn2);
    float Rq[9];
    quat_rot(q.x * qinv, q.y * qinv, q.z * qinv, q.w * qinv, Rq);
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        M[3 * a] = Rq[3 * a] * s0; M[3 * a + 1] = Rq[3 * a + 1] * s1; M[3 * a + 2] = Rq[3 * a + 2] * s2;
    }
    // Sigma symmetric: S00 S01 S02 S11 S12 S22
    const float S00 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    const float S01 = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    const float S02 = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    const float S11 = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    const float S12 = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    const float S22 = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    const float opac = 1.f / (1.f + expf(-lg));
    const float kext = 2.f * logf(opac / L.alpha_min);
    bool finite_in = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(S00) && isfinite(S11) &&
                     isfinite(S22) && isfinite(S01) && isfinite(S02) && isfinite(S12) && isfinite(opac) &&
                     qn2 > 0.f && kext > 0.f;

    if (TMA) {
        bool ok = true;
        if (full) ok = __syncthreads_and(mbar_wait(&S[0].bar, 0));
        if (!ok) {
            if (threadIdx.x == 0) {
                if (status) {
                    atomicCAS(status, 0, GS_ERR_TIMEOUT);
                    atomicExch(status + 1, (int)blockIdx.x);
                }
                mbar_wait(&S[0].bar, 0);   // give the copy in flight (bounded) time to land before exiting
            }
            return;
        }
    }

    for (int v = L.s[s].v_begin; v < L.s[s].v_end; ++v) {
        const ViewDesc &vd = L.v[v];
        float4 *out = proj + 4 * (vd.slot_base + li);
        const float *vm = viewmats + 12 * v;
        const float R0 = __ldg(vm + 0), R1 = __ldg(vm + 1), R2 = __ldg(vm + 2);
        const float R3 = __ldg(vm + 3), R4 = __ldg(vm + 4), R5 = __ldg(vm + 5);
        const float R6 = __ldg(vm + 6), R7 = __ldg(vm + 7), R8 = __ldg(vm + 8);
        const float t0 = __ldg(vm + 9), t1 = __ldg(vm + 10), t2 = __ldg(vm + 11);
        const float fx = __ldg(intr + 4 * v), fy = __ldg(intr + 4 * v + 1);
        const float cx = __ldg(intr + 4 * v + 2), cy = __ldg(intr + 4 * v + 3);

        const ff X = dot3_plus(R0, R1, R2, mx, my, mz, t0);
        const ff Y = dot3_plus(R3, R4, R5, mx, my, mz, t1);
        const ff Z = dot3_plus(R6, R7, R8, mx, my, mz, t2);
        const float x = X.hi, y = Y.hi, z = Z.hi;
        bool ok = finite_in && z > L.near_z;

        // Jacobian with the tangent clamp
        const float limx = L.fov_clamp * 0.5f * (float)vd.W / fx;
        const float limy = L.fov_clamp * 0.5f * (float)vd.H / fy;
        const float iz = 1.f / z;
        const float u = fminf(fmaxf(x * iz, -limx), limx);
        const float w = fminf(fmaxf(y * iz, -limy), limy);
        const float J00 = fx * iz, J02 = -fx * u * iz, J11 = fy * iz, J12 = -fy * w * iz;
        // T = J R (2x3)
        const float T00 = J00 * R0 + J02 * R6, T01 = J00 * R1 + J02 * R7, T02 = J00 * R2 + J02 * R8;
        const float T10 = J11 * R3 + J12 * R6, T11 = J11 * R4 + J12 * R7, T12 = J11 * R5 + J12 * R8;
        // Sigma' = T Sigma T^T
        const float A0 = T00 * S00 + T01 * S01 + T02 * S02;
        const float A1 = T00 * S01 + T01 * S11 + T02 * S12;
        const float A2 = T00 * S02 + T01 * S12 + T02 * S22;
        const float B0 = T10 * S00 + T11 * S01 + T12 * S02;
        const float B1 = T10 * S01 + T11 * S11 + T12 * S12;
        const float B2 = T10 * S02 + T11 * S12 + T12 * S22;
        const float ca = A0 * T00 + A1 * T01 + A2 * T02 + L.dilation;
        const float cb = A0 * T10 + A1 * T11 + A2 * T12;
        const float cc = B0 * T10 + B1 * T11 + B2 * T12 + L.dilation;
        const float det = ca * cc - cb * cb;
        ok = ok && det > 0.f;
        const float idet = 1.f / det;
        const float mid = 0.5f * (ca + cc);
        const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
        const float radius = ceilf(3.f * sqrtf(lam));

        const ff PX = project_coord(fx, X.hi, X.lo, Z.hi, Z.lo, cx);
        const ff PY = project_coord(fy, Y.hi, Y.lo, Z.hi, Z.lo, cy);
        ok = ok && !(PX.hi + radius < 0.f || PX.hi - radius > (float)vd.W || PY.hi + radius < 0.f ||
                     PY.hi - radius > (float)vd.H);

        // view-dependent colour: dir = mu - C, C = -R^T t
        const float Cx = -(R0 * t0 + R3 * t1 + R6 * t2);
        const float Cy = -(R1 * t0 + R4 * t1 + R7 * t2);
        const float Cz = -(R2 * t0 + R5 * t1 + R8 * t2);
        const float dx = mx - Cx, dy = my - Cy, dz = mz - Cz;
        const float idl = rsqrtf(dx * dx + dy * dy + dz * dz);
        float Yb[16];
        sh_basis<DEG>(dx * idl, dy * idl, dz * idl, Yb);
        float rgb[3] = {0.5f, 0.5f, 0.5f};
        if (TMA) {
            // coefficients straight from the staged rows (each channel summed in k order)
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                const float4 t = c < 8 ? S[0].shA[swz128(threadIdx.x, c)] : S[0].shB[swz64(threadIdx.x, c - 8)];
                const float fv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) rgb[(4 * c + e) % 3] += fv[e] * Yb[(4 * c + e) / 3];
            }
        } else {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
#pragma unroll
                for (int k = 0; k < K; ++k) rgb[ch] += f[3 * k + ch] * Yb[k];
        }
        int clamp_bits = 0;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            if (rgb[ch] < 0.f) { clamp_bits |= 1 << ch; rgb[ch] = 0.f; }
        ok = ok && isfinite(PX.hi) && isfinite(PY.hi) && isfinite(idet) && isfinite(ca) && isfinite(cb) &&
             isfinite(cc) && isfinite(rgb[0]) && isfinite(rgb[1]) && isfinite(rgb[2]);
        float4 rec[4];
        if (ok) {
            const float grow = 1.f + 6.103515625e-05f;   // 1 + 2^-14
            const float ex = fminf(radius, sqrtf(kext * ca) * grow);
            const float ey = fminf(radius, sqrtf(kext * cc) * grow);
            rec[0] = make_float4(PX.hi, PY.hi, ex, ey);
            // the conic in the form the rasterizer evaluates (see gs.h): with
            // det = a c - b^2 (b^2 carried exactly), A = c / det, beta = -b / c,
            // D = 1 / c, base-2 exponent Ah u^2 + Dh dy^2, u = dx + beta dy
            const ff bb = two_prod(cb, cb);
            const float cdet = __fsub_rn(__fmaf_rn(ca, cc, -bb.hi), bb.lo);
            const float A = __fdiv_rn(cc, cdet), beta = __fdiv_rn(-cb, cc), D = __fdiv_rn(1.f, cc);
            rec[1] = make_float4(__fmul_rn(A, -0.5f * LOG2E), beta, __fmul_rn(D, -0.5f * LOG2E), opac);
            rec[2] = make_float4(rgb[0], rgb[1], rgb[2], radius);
            rec[3] = make_float4(PX.lo, PY.lo, z, __int_as_float(clamp_bits));
        } else {
            rec[0] = rec[1] = rec[2] = rec[3] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (TMA && full) {
            // the previous view's store must have read the staging box first
            if (threadIdx.x == 0) bulk_wait_read_all();
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 4; ++c) S[0].out[swz64(threadIdx.x, c)] = rec[c];
            fence_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
                tma_store_2d(&tm_proj, S[0].out, 0, (int)(vd.slot_base + li0));
                bulk_commit();
            }
        } else {
            out[0] = rec[0]; out[1] = rec[1]; out[2] = rec[2]; out[3] = rec[3];
        }
    }
    if (TMA && full && threadIdx.x == 0) bulk_wait_read_all();
}

int launch_project(const Launch &L, int deg, const gs_gaussians *g, const float *viewmats, const float *intr,
                   float *proj, int32_t *status, cudaStream_t st) {
    if (L.n_threads == 0) return GS_OK;
    const long long nb = (L.n_threads + PF_THREADS - 1) / PF_THREADS;
    float4 *p = reinterpret_cast<float4 *>(proj);
    CUtensorMap ma, mb, mp;
    memset(&ma, 0, sizeof ma); memset(&mb, 0, sizeof mb); memset(&mp, 0, sizeof mp);
    // degree 3 with 16-byte aligned SH rows and int32 row coordinates: the
    // staged path; anything else reads and writes per thread (also when the
    // configuration turns tensor copies off, which the tests use to compare the two)
    const bool tma = deg == 3 && L.use_tma && ((uintptr_t)g->sh & 15u) == 0 &&
                     ((uintptr_t)proj & 15u) == 0 &&
                     L.n_slots < 0x7fffffffLL && g->n < 0x7fffffffLL &&
                     encode_tmap_2d(&ma, g->sh, 48, (uint64_t)g->n, 192, 32, PF_THREADS, CU_TENSOR_MAP_SWIZZLE_128B) &&
                     encode_tmap_2d(&mb, g->sh, 48, (uint64_t)g->n, 192, 16, PF_THREADS, CU_TENSOR_MAP_SWIZZLE_64B) &&
                     encode_tmap_2d(&mp, proj, 16, (uint64_t)L.n_slots, 64, 16, PF_THREADS, CU_TENSOR_MAP_SWIZZLE_64B);
#define GS_PF(D, T) k_project_fwd<D, T><<<nb, PF_THREADS, 0, st>>>(L, g->means, g->log_scales, g->quats, \
        g->opacity_logits, g->sh, viewmats, intr, p, ma, mb, mp, status)
    switch (deg) {
    case 0: GS_PF(0, false); break;
    case 1: GS_PF(1, false); break;
    case 2: GS_PF(2, false); break;
    case 3: if (tma) GS_PF(3, true); else GS_PF(3, false); break;
    default: return GS_ERR_UNSUPPORTED;
    }
#undef GS_PF
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gsk
