// Photometric loss with D-SSIM (Section 3.1): L = (1 - lambda) mean|x - y|
// + lambda (1 - mean SSIM(x, y)), SSIM from local statistics under an 11x11
// Gaussian window (sigma 1.5) with zero padding, per channel of every view,
// and its gradient with respect to the rendered image x.
//
// One kernel does the forward and the backward for a 32x32 output tile and
// all three channels: it stages x and y with a 10-pixel halo in shared
// memory, blurs x, y, x^2, y^2, xy (separable: a horizontal then a vertical
// 11-tap pass) over the tile plus a 5-pixel halo, forms SSIM and the three
// per-pixel derivative fields a = dS/dmu_x, b = dS/dE[x^2], c = dS/dE[xy]
// there, blurs those over the tile, and writes
//   dL/dx = (1 - lambda) sign(x - y) / n - lambda / n (G a + 2 x G b + y G c).
// Every pass keeps a run of outputs per thread in registers so that each
// staged value is read from shared memory once per run, not once per tap.
#include "gs_common.cuh"

namespace gsk {

constexpr int SS_T = 32;                 // output tile (square)
constexpr int SS_R = 5;                  // window radius
constexpr int SS_S1 = SS_T + 2 * SS_R;   // 42: tile + halo where SSIM is formed
constexpr int SS_IN = SS_T + 4 * SS_R;   // 52: staged input
constexpr int SS_THREADS = 256;
constexpr float SS_C1 = 0.0001f, SS_C2 = 0.0009f;

struct SsimLaunch {
    int n_views;
    int tiles_x[GS_MAX_VIEWS], tiles_y[GS_MAX_VIEWS];
    int W[GS_MAX_VIEWS], H[GS_MAX_VIEWS];
    long long tile_base[GS_MAX_VIEWS + 1];
    long long pix_base[GS_MAX_VIEWS];
    float g[2 * SS_R + 1];
    float lambda, inv_n;
};

struct SsimSmem {
    float x[SS_IN][SS_IN];
    float y[SS_IN][SS_IN];
    union {
        float h1[5][SS_IN][SS_S1];   // horizontal blurs of x, y, x^2, y^2, xy
        float h2[3][SS_S1][SS_T];    // horizontal blurs of a, b, c
    } u;
    float abc[3][SS_S1][SS_S1];
    float red[2][SS_THREADS / 32];
};

__global__ void __launch_bounds__(SS_THREADS, 2) k_l1_dssim(const SsimLaunch L, const float *__restrict__ image,
                                                            const float *__restrict__ target, float *__restrict__ grad,
                                                            float *loss) {
    extern __shared__ __align__(16) unsigned char ss_raw[];
    SsimSmem &sm = *reinterpret_cast<SsimSmem *>(ss_raw);
    const long long tile = blockIdx.x;
    int v = 0;
    while (v + 1 < L.n_views && L.tile_base[v + 1] <= tile) ++v;
    const int lt = (int)(tile - L.tile_base[v]);
    const int W = L.W[v], H = L.H[v];
    const int ox = (lt % L.tiles_x[v]) * SS_T, oy = (lt / L.tiles_x[v]) * SS_T;
    const int tid = threadIdx.x;
    float g[2 * SS_R + 1];
#pragma unroll
    for (int k = 0; k <= 2 * SS_R; ++k) g[k] = L.g[k];
    float acc_s = 0.f, acc_l1 = 0.f;

    for (int ch = 0; ch < 3; ++ch) {
        const float *X = image + L.pix_base[v] + (long long)ch * W * H;
        const float *Y = target + L.pix_base[v] + (long long)ch * W * H;
        float *G = grad + L.pix_base[v] + (long long)ch * W * H;
        // stage x, y with a 10-pixel halo (0 outside the image)
        for (int i = tid; i < SS_IN * SS_IN; i += SS_THREADS) {
            const int r = i / SS_IN, c = i % SS_IN;
            const int gy = oy - 2 * SS_R + r, gx = ox - 2 * SS_R + c;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            sm.x[r][c] = in ? X[(long long)gy * W + gx] : 0.f;
            sm.y[r][c] = in ? Y[(long long)gy * W + gx] : 0.f;
        }
        __syncthreads();
        // horizontal pass: 52 rows x 42 columns, runs of 7 columns per thread
        constexpr int RUN1 = 7;
        for (int i = tid; i < SS_IN * (SS_S1 / RUN1); i += SS_THREADS) {
            const int r = i / (SS_S1 / RUN1), c0 = (i % (SS_S1 / RUN1)) * RUN1;
            float a[5][RUN1];
#pragma unroll
            for (int q = 0; q < 5; ++q)
#pragma unroll
                for (int j = 0; j < RUN1; ++j) a[q][j] = 0.f;
#pragma unroll
            for (int k = 0; k < RUN1 + 2 * SS_R; ++k) {
                const float xv = sm.x[r][c0 + k], yv = sm.y[r][c0 + k];
                const float xx = xv * xv, yy = yv * yv, xy = xv * yv;
#pragma unroll
                for (int j = 0; j < RUN1; ++j) {
                    const int t = k - j;
                    if (t >= 0 && t <= 2 * SS_R) {
                        a[0][j] = fmaf(g[t], xv, a[0][j]);
                        a[1][j] = fmaf(g[t], yv, a[1][j]);
                        a[2][j] = fmaf(g[t], xx, a[2][j]);
                        a[3][j] = fmaf(g[t], yy, a[3][j]);
                        a[4][j] = fmaf(g[t], xy, a[4][j]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 5; ++q)
#pragma unroll
                for (int j = 0; j < RUN1; ++j) sm.u.h1[q][r][c0 + j] = a[q][j];
        }
        __syncthreads();
        // vertical pass over the 42x42 region, runs of 7 rows: SSIM and a, b, c
        for (int i = tid; i < SS_S1 * (SS_S1 / RUN1); i += SS_THREADS) {
            const int c = i % SS_S1, r0 = (i / SS_S1) * RUN1;
            float a[5][RUN1];
#pragma unroll
            for (int q = 0; q < 5; ++q)
#pragma unroll
                for (int j = 0; j < RUN1; ++j) a[q][j] = 0.f;
#pragma unroll
            for (int k = 0; k < RUN1 + 2 * SS_R; ++k) {
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const float hv = sm.u.h1[q][r0 + k][c];
#pragma unroll
                    for (int j = 0; j < RUN1; ++j) {
                        const int t = k - j;
                        if (t >= 0 && t <= 2 * SS_R) a[q][j] = fmaf(g[t], hv, a[q][j]);
                    }
                }
            }
            const int gx = ox - SS_R + c;
#pragma unroll
            for (int j = 0; j < RUN1; ++j) {
                const int r = r0 + j;
                const int gy = oy - SS_R + r;
                float da = 0.f, db = 0.f, dc = 0.f;
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const float mx = a[0][j], my = a[1][j];
                    const float sxx = a[2][j] - mx * mx, syy = a[3][j] - my * my, sxy = a[4][j] - mx * my;
                    const float l1 = 2.f * mx * my + SS_C1, l2 = 2.f * sxy + SS_C2;
                    const float d1 = mx * mx + my * my + SS_C1, d2 = sxx + syy + SS_C2;
                    const float rd1 = 1.f / d1, rd2 = 1.f / d2, rq = rd1 * rd2;
                    const float S = l1 * l2 * rq;
                    // dS/dmu_x with E[x^2] and E[xy] held fixed, written without
                    // dividing by l1 or l2 (l2 = 2 s_xy + C2 can be ~0):
                    // S (2 my / l1 - 2 my / l2) = 2 my (l2 - l1) / (d1 d2)
                    da = 2.f * my * (l2 - l1) * rq + 2.f * mx * S * (rd2 - rd1);
                    db = -S * rd2;
                    dc = 2.f * l1 * rq;
                    if (r >= SS_R && r < SS_R + SS_T && c >= SS_R && c < SS_R + SS_T) acc_s += S;
                }
                sm.abc[0][r][c] = da;
                sm.abc[1][r][c] = db;
                sm.abc[2][r][c] = dc;
            }
        }
        __syncthreads();
        // horizontal pass of a, b, c: 42 rows x 32 columns, runs of 4
        constexpr int RUN2 = 4;
        for (int i = tid; i < SS_S1 * (SS_T / RUN2); i += SS_THREADS) {
            const int r = i / (SS_T / RUN2), c0 = (i % (SS_T / RUN2)) * RUN2;
            float a[3][RUN2];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int j = 0; j < RUN2; ++j) a[q][j] = 0.f;
#pragma unroll
            for (int k = 0; k < RUN2 + 2 * SS_R; ++k) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float hv = sm.abc[q][r][c0 + k];
#pragma unroll
                    for (int j = 0; j < RUN2; ++j) {
                        const int t = k - j;
                        if (t >= 0 && t <= 2 * SS_R) a[q][j] = fmaf(g[t], hv, a[q][j]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int j = 0; j < RUN2; ++j) sm.u.h2[q][r][c0 + j] = a[q][j];
        }
        __syncthreads();
        // vertical pass to the 32x32 tile, runs of 4 rows; write the gradient
        for (int i = tid; i < SS_T * (SS_T / RUN2); i += SS_THREADS) {
            const int c = i % SS_T, r0 = (i / SS_T) * RUN2;
            float a[3][RUN2];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int j = 0; j < RUN2; ++j) a[q][j] = 0.f;
#pragma unroll
            for (int k = 0; k < RUN2 + 2 * SS_R; ++k) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float hv = sm.u.h2[q][r0 + k][c];
#pragma unroll
                    for (int j = 0; j < RUN2; ++j) {
                        const int t = k - j;
                        if (t >= 0 && t <= 2 * SS_R) a[q][j] = fmaf(g[t], hv, a[q][j]);
                    }
                }
            }
            const int gx = ox + c;
#pragma unroll
            for (int j = 0; j < RUN2; ++j) {
                const int gy = oy + r0 + j;
                if (gy < H && gx < W) {
                    const float xv = sm.x[2 * SS_R + r0 + j][2 * SS_R + c], yv = sm.y[2 * SS_R + r0 + j][2 * SS_R + c];
                    const float d = xv - yv;
                    acc_l1 += fabsf(d);
                    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                    const float gs = a[0][j] + 2.f * xv * a[1][j] + yv * a[2][j];
                    G[(long long)gy * W + gx] = L.inv_n * ((1.f - L.lambda) * sg - L.lambda * gs);
                }
            }
        }
        __syncthreads();
    }
    // block sums of SSIM and |x - y| over the tile (fixed order), one atomic each
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_s += __shfl_xor_sync(0xffffffffu, acc_s, o);
        acc_l1 += __shfl_xor_sync(0xffffffffu, acc_l1, o);
    }
    if ((tid & 31) == 0) {
        sm.red[0][tid >> 5] = acc_s;
        sm.red[1][tid >> 5] = acc_l1;
    }
    __syncthreads();
    if (tid == 0) {
        float s = 0.f, l = 0.f;
        for (int w = 0; w < SS_THREADS / 32; ++w) {
            s += sm.red[0][w];
            l += sm.red[1][w];
        }
        atomicAdd(&loss[1], l * L.inv_n);
        atomicAdd(&loss[2], s * L.inv_n);
    }
}

// loss = {total, mean L1, 1 - mean SSIM} from the accumulated means
__global__ void k_l1_dssim_final(float *loss, float lambda) {
    const float l1 = loss[1], dssim = 1.f - loss[2];
    loss[2] = dssim;
    loss[0] = (1.f - lambda) * l1 + lambda * dssim;
}

int launch_l1_dssim(const int *W, const int *H, int n_views, const float *image, const float *target, float lambda,
                    float *loss, float *grad, cudaStream_t st) {
    SsimLaunch L{};
    L.n_views = n_views;
    long long tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        L.W[v] = W[v];
        L.H[v] = H[v];
        L.tiles_x[v] = (W[v] + SS_T - 1) / SS_T;
        L.tiles_y[v] = (H[v] + SS_T - 1) / SS_T;
        L.tile_base[v] = tiles;
        L.pix_base[v] = pix;
        tiles += (long long)L.tiles_x[v] * L.tiles_y[v];
        pix += 3LL * W[v] * H[v];
    }
    L.tile_base[n_views] = tiles;
    double gs[2 * SS_R + 1], tot = 0.0;
    for (int k = 0; k <= 2 * SS_R; ++k) {
        const double d = k - SS_R;
        gs[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
        tot += gs[k];
    }
    for (int k = 0; k <= 2 * SS_R; ++k) L.g[k] = (float)(gs[k] / tot);
    L.lambda = lambda;
    L.inv_n = pix > 0 ? (float)(1.0 / (double)pix) : 0.f;
    if (cudaMemsetAsync(loss, 0, 3 * sizeof(float), st) != cudaSuccess) return GS_ERR_CUDA;
    if (tiles > 0) {
        const size_t smem = sizeof(SsimSmem);
        if (cudaFuncSetAttribute(k_l1_dssim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GS_ERR_CUDA;
        k_l1_dssim<<<(unsigned)tiles, SS_THREADS, smem, st>>>(L, image, target, grad, loss);
        if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    }
    k_l1_dssim_final<<<1, 1, 0, st>>>(loss, lambda);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace gsk
