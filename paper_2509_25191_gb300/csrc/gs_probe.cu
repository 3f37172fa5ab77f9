// Throughput probes of the arithmetic pipes the raster kernels are bound by:
// scalar FP32 fused multiply-add, packed f32x2 fused multiply-add (one
// instruction for two lanes' worth of FMAs) and the ex2.approx special-
// function instruction. Each thread runs 8 independent dependency chains
// (enough to cover the pipes' latency at full occupancy) for `iters`
// iterations; the chains' results are written out so nothing is dropped.
// The caller times the launch with events; operations per launch =
// grid x block x iters x 8 (x 2 lanes for the packed form).
#include "gs_common.cuh"

namespace gsk {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(int iters, float a, float b, float *out) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma2(int iters, float a, float b, float *out) {
    float2 x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 2e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ex2(int iters, float a, float b, float *out) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = -(float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = -ex2_approx(x[c]);   // stays in (-1, 0]: no overflow
    }
    float s = a * b;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

}  // namespace gsk

extern "C" int gs_probe_blocks(void) { return 8 * gsk::num_sms(); }

extern "C" int gs_peak_probe(int kind, int iters, float *out, void *stream) {
    using namespace gsk;
    if (kind < 0 || kind > 2 || iters < 1 || !out) return GS_ERR_ARG;
    const int grid = 8 * num_sms();
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
    case 0: k_probe_fma<<<grid, PROBE_THREADS, 0, st>>>(iters, 0.999f, 1e-4f, out); break;
    case 1: k_probe_fma2<<<grid, PROBE_THREADS, 0, st>>>(iters, 0.999f, 1e-4f, out); break;
    default: k_probe_ex2<<<grid, PROBE_THREADS, 0, st>>>(iters, 1.f, 0.f, out); break;
    }
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
