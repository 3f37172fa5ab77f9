// Fused SGLD update with an Adam direction over all parameter groups of the
// Gaussians (Eq. 1 of the paper: G <- G - lr * step(grad) + lambda_noise eps).
//
// One launch covers every group (means, log-scales, quaternions, opacity
// logits, SH coefficients, ...): the element index space is the
// concatenation of the groups, each thread updates four consecutive elements
// of one group (float4 when the group is 16-byte aligned, scalar otherwise),
// so every parameter, gradient and moment byte is read and written exactly
// once, coalesced. Exploration noise, drawn by the caller, is added to one
// group (the means).
#include "gs_common.cuh"

namespace gsk {

struct AdamGroup {
    float *p;
    const float *g;
    float *m;
    float *v;
    long long count;
    long long unit_base;   // first 4-element unit of the group
    float lr;
    int vec;               // all four arrays 16-byte aligned
};

struct AdamLaunch {
    int n_groups, noise_group;
    float b1, b2, omb1, omb2, eps, inv_bc1, inv_bc2, noise_scale;   // omb = 1 - b, formed in double
    const float *noise;
    long long n_units;
    AdamGroup gr[GS_MAX_ADAM_GROUPS];
};

__device__ __forceinline__ void adam_one(const AdamLaunch &A, float lr, float &p, float g, float &m, float &v) {
    m = A.b1 * m + A.omb1 * g;
    v = A.b2 * v + A.omb2 * g * g;
    p -= lr * (m * A.inv_bc1) / (sqrtf(v * A.inv_bc2) + A.eps);
}

__global__ void __launch_bounds__(256) k_adam_sgld(const AdamLaunch A) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < A.n_units; u += stride) {
        int k = 0;
        while (k + 1 < A.n_groups && A.gr[k + 1].unit_base <= u) ++k;
        const AdamGroup &G = A.gr[k];
        const long long j = 4 * (u - G.unit_base);
        const bool noisy = A.noise && k == A.noise_group;
        if (G.vec && j + 4 <= G.count) {
            float4 p = *reinterpret_cast<const float4 *>(G.p + j);
            const float4 g = *reinterpret_cast<const float4 *>(G.g + j);
            float4 m = *reinterpret_cast<const float4 *>(G.m + j);
            float4 v = *reinterpret_cast<const float4 *>(G.v + j);
            adam_one(A, G.lr, p.x, g.x, m.x, v.x);
            adam_one(A, G.lr, p.y, g.y, m.y, v.y);
            adam_one(A, G.lr, p.z, g.z, m.z, v.z);
            adam_one(A, G.lr, p.w, g.w, m.w, v.w);
            if (noisy) {
                p.x += A.noise_scale * A.noise[j];
                p.y += A.noise_scale * A.noise[j + 1];
                p.z += A.noise_scale * A.noise[j + 2];
                p.w += A.noise_scale * A.noise[j + 3];
            }
            *reinterpret_cast<float4 *>(G.p + j) = p;
            *reinterpret_cast<float4 *>(G.m + j) = m;
            *reinterpret_cast<float4 *>(G.v + j) = v;
        } else {
            for (long long e = j; e < j + 4 && e < G.count; ++e) {
                float p = G.p[e], m = G.m[e], v = G.v[e];
                adam_one(A, G.lr, p, G.g[e], m, v);
                if (noisy) p += A.noise_scale * A.noise[e];
                G.p[e] = p;
                G.m[e] = m;
                G.v[e] = v;
            }
        }
    }
}

int launch_adam_sgld(const gs_adam_group *groups, int n_groups, int step, double beta1, double beta2, double eps,
                     const float *noise, float noise_scale, int noise_group, cudaStream_t st) {
    AdamLaunch A;
    A.n_groups = n_groups;
    A.noise_group = noise_group;
    A.b1 = (float)beta1;
    A.b2 = (float)beta2;
    A.omb1 = (float)(1.0 - beta1);   // 1 - 0.999f in float would be off by 1e-5
    A.omb2 = (float)(1.0 - beta2);
    A.eps = (float)eps;
    A.inv_bc1 = (float)(1.0 / (1.0 - pow(beta1, step)));
    A.inv_bc2 = (float)(1.0 / (1.0 - pow(beta2, step)));
    A.noise = noise;
    A.noise_scale = noise_scale;
    long long units = 0;
    for (int k = 0; k < n_groups; ++k) {
        const gs_adam_group &g = groups[k];
        AdamGroup &d = A.gr[k];
        d.p = g.param;
        d.g = g.grad;
        d.m = g.exp_avg;
        d.v = g.exp_avg_sq;
        d.count = g.count;
        d.lr = g.lr;
        d.unit_base = units;
        d.vec = (((uintptr_t)g.param | (uintptr_t)g.grad | (uintptr_t)g.exp_avg | (uintptr_t)g.exp_avg_sq) & 15u) == 0;
        units += (g.count + 3) / 4;
    }
    A.n_units = units;
    if (units == 0) return GS_OK;
    long long blocks = (units + 255) / 256;
    if (blocks > 8LL * num_sms()) blocks = 8LL * num_sms();
    k_adam_sgld<<<(int)blocks, 256, 0, st>>>(A);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gsk
