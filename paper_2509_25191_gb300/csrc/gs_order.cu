// Spatial (Morton) codes of the Gaussian means, for callers that keep their
// Gaussians in a spatial order (refreshed between densification steps of a
// training run). The order changes no result of the rasterizer (the image
// and every gradient are permutation-invariant for distinct depths); it
// makes the Gaussians that project near each other neighbours in memory, so
// binning blocks write longer runs per tile and the projection backward's
// warps agree on which Gaussians carry a gradient.
//
// Code of mean m in the box [lo, hi]: each coordinate quantised to 21 bits,
// q = min(2^21 - 1, floor((m - lo) / (hi - lo) * 2^21)) (0 below lo), and the
// bits interleaved as x0 y0 z0 x1 y1 z1 ... (bit 3b + a holds bit b of axis
// a). Non-finite means get the largest code.
#include "gs_common.cuh"

namespace gsk {

__device__ __forceinline__ unsigned long long spread21(unsigned int v) {
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ unsigned int quant21(float m, float lo, float scale) {
    const float t = (m - lo) * scale;
    if (!(t > 0.f)) return 0u;
    return t >= 2097151.f ? 2097151u : (unsigned int)t;
}

__global__ void __launch_bounds__(256) k_morton(const float *__restrict__ means, long long n, float lx, float ly,
                                                float lz, float sx, float sy, float sz,
                                                unsigned long long *__restrict__ codes) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float x = means[3 * i], y = means[3 * i + 1], z = means[3 * i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
        codes[i] = ~0ull;
        return;
    }
    codes[i] = spread21(quant21(x, lx, sx)) | (spread21(quant21(y, ly, sy)) << 1) |
               (spread21(quant21(z, lz, sz)) << 2);
}

}  // namespace gsk

extern "C" int gs_spatial_codes(const float *means, int64_t n, const float *box, uint64_t *codes, void *stream) {
    using namespace gsk;
    if (n < 0 || !box || (n > 0 && (!means || !codes))) return GS_ERR_ARG;
    float s[3];
    for (int a = 0; a < 3; ++a) {
        const float ext = box[3 + a] - box[a];
        if (!(ext >= 0.f) || !isfinite(box[a]) || !isfinite(box[3 + a])) return GS_ERR_ARG;
        s[a] = ext > 0.f ? 2097152.f / ext : 0.f;
    }
    if (n == 0) return GS_OK;
    const long long blocks = (n + 255) / 256;
    k_morton<<<(unsigned int)blocks, 256, 0, (cudaStream_t)stream>>>(
        means, n, box[0], box[1], box[2], s[0], s[1], s[2], reinterpret_cast<unsigned long long *>(codes));
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
