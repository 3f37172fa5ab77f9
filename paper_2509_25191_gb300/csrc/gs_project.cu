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
#include "gs_common.cuh"

namespace gsk {

template <int DEG>
__global__ void __launch_bounds__(128) k_project_fwd(const Launch L, const float *__restrict__ means,
                                                     const float *__restrict__ log_scales,
                                                     const float *__restrict__ quats,
                                                     const float *__restrict__ logits,
                                                     const float *__restrict__ sh,
                                                     const float *__restrict__ viewmats,
                                                     const float *__restrict__ intr, float4 *__restrict__ proj) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= L.n_threads) return;
    const int s = scene_of_thread(L, gid);
    const long long li = gid - L.s[s].thread_base;
    const long long i = L.s[s].g_begin + li;

    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
    const float l0 = log_scales[3 * i], l1 = log_scales[3 * i + 1], l2 = log_scales[3 * i + 2];
    const float4 q = reinterpret_cast<const float4 *>(quats)[i];
    const float lg = logits[i];
    float f[3 * K];
    if (DEG == 1 || DEG == 3) {
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
        float rgb[3];
        int clamp_bits = 0;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc += f[3 * k + ch] * Yb[k];
            if (acc < 0.f) { clamp_bits |= 1 << ch; acc = 0.f; }
            rgb[ch] = acc;
        }
        ok = ok && isfinite(PX.hi) && isfinite(PY.hi) && isfinite(idet) && isfinite(ca) && isfinite(cb) &&
             isfinite(cc) && isfinite(rgb[0]) && isfinite(rgb[1]) && isfinite(rgb[2]);
        if (ok) {
            const float grow = 1.f + 6.103515625e-05f;   // 1 + 2^-14
            const float ex = fminf(radius, sqrtf(kext * ca) * grow);
            const float ey = fminf(radius, sqrtf(kext * cc) * grow);
            out[0] = make_float4(PX.hi, PY.hi, ex, ey);
            // the conic in the form the rasterizer evaluates (see gs.h): with
            // det = a c - b^2 (b^2 carried exactly), A = c / det, beta = -b / c,
            // D = 1 / c, base-2 exponent Ah u^2 + Dh dy^2, u = dx + beta dy
            const ff bb = two_prod(cb, cb);
            const float cdet = __fsub_rn(__fmaf_rn(ca, cc, -bb.hi), bb.lo);
            const float A = __fdiv_rn(cc, cdet), beta = __fdiv_rn(-cb, cc), D = __fdiv_rn(1.f, cc);
            out[1] = make_float4(__fmul_rn(A, -0.5f * LOG2E), beta, __fmul_rn(D, -0.5f * LOG2E), opac);
            out[2] = make_float4(rgb[0], rgb[1], rgb[2], radius);
            out[3] = make_float4(PX.lo, PY.lo, z, __int_as_float(clamp_bits));
        } else {
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            out[0] = zero; out[1] = zero; out[2] = zero; out[3] = zero;
        }
    }
}

int launch_project(const Launch &L, int deg, const gs_gaussians *g, const float *viewmats, const float *intr,
                   float *proj, cudaStream_t st) {
    if (L.n_threads == 0) return GS_OK;
    const int bs = 128;
    const long long nb = (L.n_threads + bs - 1) / bs;
    float4 *p = reinterpret_cast<float4 *>(proj);
    switch (deg) {
    case 0: k_project_fwd<0><<<nb, bs, 0, st>>>(L, g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, viewmats, intr, p); break;
    case 1: k_project_fwd<1><<<nb, bs, 0, st>>>(L, g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, viewmats, intr, p); break;
    case 2: k_project_fwd<2><<<nb, bs, 0, st>>>(L, g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, viewmats, intr, p); break;
    case 3: k_project_fwd<3><<<nb, bs, 0, st>>>(L, g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, viewmats, intr, p); break;
    default: return GS_ERR_UNSUPPORTED;
    }
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gsk
