// extern "C" entry points of libgsplat_gb300.so (declared in include/gs.h):
// host-side argument checks, the per-call launch description, and dispatch
// to the kernels. No allocation; the one synchronising call is
// gs_status_read.
#include <math.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "gs_common.cuh"

namespace gsk {

// A named NVTX range around each entry point that enqueues work, so that a
// profiler's timeline shows which library call launched which kernels (the
// header-only NVTX library does nothing unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define GS_TRACE() gsk::NvtxRange gs_trace_range_(__func__)

int launch_project(const Launch &L, int deg, const gs_gaussians *g, const float *viewmats, const float *intr,
                   float *proj, int32_t *status, cudaStream_t st);
int launch_bin_sort(const Launch &L, const float *proj, const gs_bins *b, int32_t *status, cudaStream_t st);
int launch_render_fwd(const Launch &L, const float *proj, const gs_bins *b, float *image, cudaStream_t st);
int launch_render_bwd(const Launch &L, const float *proj, const gs_bins *b, const float *image,
                      const float *dL_dimage, const L1Loss &l1, float *grad2d, cudaStream_t st);
int launch_zero_accumulators(float *grad2d, long long n_floats, float *loss, cudaStream_t st);
int launch_project_bwd(const Launch &L, int deg, const gs_gaussians *g, const float *viewmats, const float *intr,
                       const float *proj, const float *grad2d, const gs_grads *out, int want_gauss, int nblk,
                       int32_t *status, cudaStream_t st);
int launch_pose_reduce(int n_views, const float *partials, int nblk, const float *viewmats, float *out_rt,
                       float *out_twist, cudaStream_t st);
int launch_l1(const float *image, const float *target, long long n, float *loss, float *grad, cudaStream_t st);
int launch_adam_sgld(const gs_adam_group *groups, int n_groups, int step, double beta1, double beta2, double eps,
                     const float *noise, float noise_scale, int noise_group, cudaStream_t st);
int pose_blocks(long long n);
int launch_ga_select(const float *vm, int n, float cos_thr, int32_t *pairs, long long capacity, long long *n_out,
                     int32_t *status, cudaStream_t st);
int launch_ga_incidence(const int32_t *pairs, long long n_pairs, int n, int32_t *cam_offsets, int32_t *cam_pairs,
                        int32_t *status, cudaStream_t st);
int launch_ga_epipolar(const gs_ga_problem &P, float *dist, float *pair_sums, const int32_t *cam_offsets,
                       const int32_t *cam_pairs, float *loss, float *d_intr, float *d_vm, int32_t *status,
                       cudaStream_t st);
int launch_ga_weights(const float *e, long long n, int nb, double alpha, uint32_t *counts, float *w, float *stats,
                      uint32_t *scratch, cudaStream_t st);
int launch_l1_dssim(const int *W, const int *H, int n_views, const float *image, const float *target, float lambda,
                    float *loss, float *grad, cudaStream_t st);
int launch_ga_step(const gs_ga_state &s, const gs_ga_problem &P, float *pair_sums, const int32_t *cam_offsets,
                   const int32_t *cam_pairs, float *loss, float *d_res, int32_t *status, cudaStream_t st);

int num_sms() {
    static int cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

// cuTensorMapEncodeTiled, fetched from the CUDA driver once (the library links
// only the static CUDA runtime)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

bool encode_tmap_2d(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
                    uint32_t box_inner, uint32_t box_rows, CUtensorMapSwizzle swizzle) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn || rows == 0 || rows > 0x7fffffffULL) return false;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool tile_supported(int tw, int th) {
    return (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 16 && th == 8) || (tw == 32 && th == 8) ||
           (tw == 32 && th == 16) || (tw == 32 && th == 32);
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Validate views/config and fill the launch description.
static int build_launch(const gs_views *vw, const gs_config *cfg, Launch &L) {
    if (!vw || !cfg) return GS_ERR_ARG;
    const int V = vw->n_views;
    if (V < 1 || V > GS_MAX_VIEWS) return GS_ERR_ARG;
    if (!vw->width || !vw->height || !vw->gauss_begin || !vw->gauss_count) return GS_ERR_ARG;
    if (!tile_supported(cfg->tile_w, cfg->tile_h) || !cfg->pixel_gate) return GS_ERR_UNSUPPORTED;
    memset(&L, 0, sizeof L);
    L.n_views = V;
    L.tw = cfg->tile_w;
    L.th = cfg->tile_h;
    L.pixel_gate = cfg->pixel_gate ? 1 : 0;
    L.near_z = cfg->near_z;
    L.dilation = cfg->dilation;
    L.alpha_min = cfg->alpha_min;
    L.alpha_max = cfg->alpha_max;
    L.t_min = cfg->t_min;
    L.fov_clamp = cfg->fov_clamp;
    L.bg[0] = cfg->bg[0]; L.bg[1] = cfg->bg[1]; L.bg[2] = cfg->bg[2];
    L.count_pairs = cfg->count_pairs != 0;
    L.accumulate = cfg->accumulate_grads != 0;
    L.use_tma = cfg->use_tma != 0;
    L.fwd_batch = cfg->fwd_batch;
    L.bwd_batch = cfg->bwd_batch;
    L.overlap_prev = cfg->overlap_prev != 0;
    if (!(L.fwd_batch == 1 || L.fwd_batch == 2 || L.fwd_batch == 4) || !(L.bwd_batch == 1 || L.bwd_batch == 2))
        return GS_ERR_UNSUPPORTED;
    if (!(L.alpha_max > 0.f && L.alpha_max < 1.f) || !(L.t_min > 0.f)) return GS_ERR_ARG;
    long long slot = 0, pix = 0, tiles = 0;
    for (int v = 0; v < V; ++v) {
        const int W = vw->width[v], H = vw->height[v];
        const long long gb = vw->gauss_begin[v], gc = vw->gauss_count[v];
        if (W < 1 || H < 1 || W > 65536 || H > 65536 || gb < 0 || gc < 0 || gc > 0x7fffffffLL) return GS_ERR_ARG;
        ViewDesc &d = L.v[v];
        d.W = W; d.H = H;
        d.Gx = (W + L.tw - 1) / L.tw;
        d.Gy = (H + L.th - 1) / L.th;
        d.tile_base = (int)tiles;
        d.g_count = (int)gc;
        d.g_begin = gb;
        d.slot_base = slot;
        d.pix_base = pix;
        slot += gc;
        pix += 3LL * W * H;
        tiles += (long long)d.Gx * d.Gy;
        if (tiles > 0x7fffffffLL) return GS_ERR_ARG;
        // scene groups: runs of views with the same Gaussian range
        if (v > 0 && gb == vw->gauss_begin[v - 1] && gc == vw->gauss_count[v - 1]) {
            L.s[L.n_scenes - 1].v_end = v + 1;
        } else {
            SceneDesc &s = L.s[L.n_scenes++];
            s.g_begin = gb; s.g_count = (int)gc; s.v_begin = v; s.v_end = v + 1;
        }
    }
    if (slot > 0xffffffffLL) return GS_ERR_ARG;   // slots are 32-bit in the sort keys
    // scene groups must not overlap (each Gaussian is handled by one thread)
    for (int a = 0; a < L.n_scenes; ++a)
        for (int b = a + 1; b < L.n_scenes; ++b) {
            const SceneDesc &x = L.s[a], &y = L.s[b];
            if (x.g_begin < y.g_begin + y.g_count && y.g_begin < x.g_begin + x.g_count) return GS_ERR_ARG;
        }
    long long thr = 0;
    for (int a = 0; a < L.n_scenes; ++a) {
        L.s[a].thread_base = thr;
        thr += L.s[a].g_count;
    }
    L.n_threads = thr;
    L.n_slots = slot;
    L.n_tiles = (int)tiles;
    return GS_OK;
}

static int check_gaussians(const gs_gaussians *g, const gs_views *vw) {
    if (!g || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) return g && (g->sh_degree > 3) ? GS_ERR_UNSUPPORTED : GS_ERR_ARG;
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh)) return GS_ERR_ARG;
    if (g->n > 0 && !aligned16(g->quats)) return GS_ERR_ARG;
    if (g->n > 0 && (g->sh_degree == 1 || g->sh_degree == 3) && !aligned16(g->sh)) return GS_ERR_ARG;
    for (int v = 0; v < vw->n_views; ++v)
        if (vw->gauss_begin[v] + vw->gauss_count[v] > g->n) return GS_ERR_ARG;
    return GS_OK;
}

}  // namespace gsk

using namespace gsk;

extern "C" {

void gs_config_default(gs_config *cfg) {
    if (!cfg) return;
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->pixel_gate = 1;
    cfg->near_z = 0.2f;
    cfg->dilation = 0.3f;
    cfg->alpha_min = 1.0f / 255.0f;
    cfg->alpha_max = 0.99f;
    cfg->t_min = 1e-4f;
    cfg->fov_clamp = 1.3f;
    cfg->bg[0] = cfg->bg[1] = cfg->bg[2] = 0.0f;
    cfg->count_pairs = 0;
    cfg->accumulate_grads = 0;
    cfg->use_tma = 1;
    cfg->fwd_batch = 2;
    cfg->bwd_batch = 1;
    cfg->overlap_prev = 0;
}

int64_t gs_num_slots(const gs_views *vw) {
    if (!vw || vw->n_views < 1) return 0;
    int64_t s = 0;
    for (int v = 0; v < vw->n_views; ++v) s += vw->gauss_count[v];
    return s;
}

int64_t gs_slot_base(const gs_views *vw, int v) {
    int64_t s = 0;
    for (int u = 0; u < v; ++u) s += vw->gauss_count[u];
    return s;
}

int64_t gs_num_tiles(const gs_views *vw, const gs_config *cfg) {
    if (!vw || !cfg || cfg->tile_w < 1 || cfg->tile_h < 1) return 0;
    int64_t t = 0;
    for (int v = 0; v < vw->n_views; ++v)
        t += (int64_t)((vw->width[v] + cfg->tile_w - 1) / cfg->tile_w) * ((vw->height[v] + cfg->tile_h - 1) / cfg->tile_h);
    return t;
}

int64_t gs_tile_base(const gs_views *vw, const gs_config *cfg, int v) {
    int64_t t = 0;
    for (int u = 0; u < v; ++u)
        t += (int64_t)((vw->width[u] + cfg->tile_w - 1) / cfg->tile_w) * ((vw->height[u] + cfg->tile_h - 1) / cfg->tile_h);
    return t;
}

int64_t gs_num_image_floats(const gs_views *vw) {
    if (!vw) return 0;
    int64_t p = 0;
    for (int v = 0; v < vw->n_views; ++v) p += 3LL * vw->width[v] * vw->height[v];
    return p;
}

int64_t gs_pixel_base(const gs_views *vw, int v) {
    int64_t p = 0;
    for (int u = 0; u < v; ++u) p += 3LL * vw->width[u] * vw->height[u];
    return p;
}

int gs_pose_blocks(int64_t n) { return pose_blocks(n); }

// Pieces of the step workspace, in this order, each at a 256-byte boundary.
static size_t ws_layout(const gs_views *vw, const gs_config *cfg, int64_t n, int64_t cap, size_t off[11]) {
    if (!vw || !cfg || vw->n_views < 1 || vw->n_views > GS_MAX_VIEWS || !vw->width || !vw->height ||
        !vw->gauss_count || n < 0 || cap < 0 || cfg->tile_w < 1 || cfg->tile_h < 1)
        return 0;
    const int64_t T = gs_num_tiles(vw, cfg), P = gs_num_slots(vw), px = gs_num_image_floats(vw) / 3;
    const int64_t c = cap > 0 ? cap : 1;
    const size_t sizes[11] = {
        sizeof(int32_t) * 2 * (size_t)(T > 0 ? T : 1),           // tile_ranges
        sizeof(uint64_t) * (size_t)c,                            // keys
        sizeof(uint32_t) * (size_t)c,                            // ids
        sizeof(uint64_t) * (size_t)c,                            // keys_tmp
        sizeof(int32_t) * (size_t)(T > 0 ? T : 1),               // tile_order
        sizeof(int32_t) * 5 * (size_t)(T > 0 ? T : 1),           // tile_scratch
        sizeof(int32_t) * GS_NUM_COUNTERS,                       // counters
        sizeof(int32_t) * (size_t)(px > 0 ? px : 1),             // last_contrib
        sizeof(int32_t) * (size_t)(T > 0 ? T : 1),               // tile_work
        sizeof(float) * GS_GRAD2D_FLOATS * (size_t)(P > 0 ? P : 1),                      // grad2d
        sizeof(float) * 12 * (size_t)vw->n_views * (size_t)pose_blocks(n)};              // pose_partials
    size_t at = 0;
    for (int k = 0; k < 11; ++k) {
        off[k] = at;
        at += (sizes[k] + 255) & ~(size_t)255;
    }
    return at;
}

size_t gs_workspace_size(const gs_views *vw, const gs_config *cfg, int64_t n_gaussians, int64_t capacity) {
    size_t off[11];
    return ws_layout(vw, cfg, n_gaussians, capacity, off);
}

int gs_workspace_carve(const gs_views *vw, const gs_config *cfg, int64_t n_gaussians, int64_t capacity, void *ws,
                       size_t ws_bytes, gs_bins *bins, gs_grads *grads) {
    size_t off[11];
    const size_t need = ws_layout(vw, cfg, n_gaussians, capacity, off);
    if (!need || !ws || ws_bytes < need || ((uintptr_t)ws & 255u) || !bins || !grads) return GS_ERR_ARG;
    char *b = static_cast<char *>(ws);
    bins->capacity = capacity;
    bins->tile_ranges = reinterpret_cast<int32_t *>(b + off[0]);
    bins->keys = reinterpret_cast<uint64_t *>(b + off[1]);
    bins->ids = reinterpret_cast<uint32_t *>(b + off[2]);
    bins->keys_tmp = reinterpret_cast<uint64_t *>(b + off[3]);
    bins->tile_order = reinterpret_cast<int32_t *>(b + off[4]);
    bins->tile_scratch = reinterpret_cast<int32_t *>(b + off[5]);
    bins->counters = reinterpret_cast<int32_t *>(b + off[6]);
    bins->last_contrib = reinterpret_cast<int32_t *>(b + off[7]);
    bins->tile_work = reinterpret_cast<int32_t *>(b + off[8]);
    grads->grad2d = reinterpret_cast<float *>(b + off[9]);
    grads->pose_partials = reinterpret_cast<float *>(b + off[10]);
    return GS_OK;
}

int gs_status_read(const int32_t *status, int32_t *host_status, void *stream) {
    GS_TRACE();
    if (!status || !host_status) return GS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(host_status, status, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GS_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int gs_project(const gs_gaussians *g, const gs_views *vw, const gs_config *cfg, float *proj, int32_t *status,
               void *stream) {
    GS_TRACE();
    Launch L;
    int rc = build_launch(vw, cfg, L);
    if (rc) return rc;
    if ((rc = check_gaussians(g, vw))) return rc;
    if (!vw->viewmats || !vw->intrinsics || (L.n_slots > 0 && !proj)) return GS_ERR_ARG;
    if (!aligned16(proj)) return GS_ERR_ARG;
    return launch_project(L, g->sh_degree, g, vw->viewmats, vw->intrinsics, proj, status, (cudaStream_t)stream);
}

int gs_bin_sort(const gs_views *vw, const gs_config *cfg, const float *proj, const gs_bins *b, int32_t *status,
                void *stream) {
    GS_TRACE();
    Launch L;
    int rc = build_launch(vw, cfg, L);
    if (rc) return rc;
    if (!b || !proj || !b->tile_ranges || !b->tile_order || !b->tile_scratch || !b->counters) return GS_ERR_ARG;
    if (b->capacity < 0) return GS_ERR_ARG;
    if (b->capacity > 0 && (!b->keys || !b->ids || !b->keys_tmp)) return GS_ERR_ARG;
    if (!aligned16(proj) || !aligned16(b->tile_ranges)) return GS_ERR_ARG;
    return launch_bin_sort(L, proj, b, status, (cudaStream_t)stream);
}

int gs_render_fwd(const gs_views *vw, const gs_config *cfg, const float *proj, const gs_bins *b, float *image,
                  int32_t *status, void *stream) {
    GS_TRACE();
    (void)status;
    Launch L;
    int rc = build_launch(vw, cfg, L);
    if (rc) return rc;
    if (!b || !proj || !image || !b->tile_ranges || !b->tile_order || !b->counters || !b->ids) return GS_ERR_ARG;
    return launch_render_fwd(L, proj, b, image, (cudaStream_t)stream);
}

int gs_rasterize_bwd(const gs_views *vw, const gs_config *cfg, const float *proj, const gs_bins *b,
                     const float *image, const float *dL_dimage, float *grad2d, int32_t *status,
                     void *stream) {
    GS_TRACE();
    Launch L;
    int rc = build_launch(vw, cfg, L);
    if (rc) return rc;
    if (!b || !proj || !image || !dL_dimage || !grad2d || !b->tile_ranges || !b->tile_order || !b->counters ||
        !b->ids)
        return GS_ERR_ARG;
    if (!aligned16(grad2d)) return GS_ERR_ARG;
    (void)status;   // the raster backward reports nothing on the device
    cudaStream_t st = (cudaStream_t)stream;
    if (L.overlap_prev) {
        if ((rc = launch_zero_accumulators(grad2d, (long long)GS_GRAD2D_FLOATS * L.n_slots, nullptr, st))) return rc;
    } else if (cudaMemsetAsync(grad2d, 0, sizeof(float) * GS_GRAD2D_FLOATS * (size_t)L.n_slots, st) != cudaSuccess) {
        return GS_ERR_CUDA;
    }
    return launch_render_bwd(L, proj, b, image, dL_dimage, L1Loss{}, grad2d, st);
}

int gs_rasterize_bwd_l1(const gs_views *vw, const gs_config *cfg, const float *proj, const gs_bins *b,
                        const float *image, const float *target, float *loss, float *grad2d, int32_t *status,
                        void *stream) {
    GS_TRACE();
    Launch L;
    int rc = build_launch(vw, cfg, L);
    if (rc) return rc;
    if (!b || !proj || !image || !target || !loss || !grad2d || !b->tile_ranges || !b->tile_order ||
        !b->counters || !b->ids)
        return GS_ERR_ARG;
    if (!aligned16(grad2d)) return GS_ERR_ARG;
    (void)status;   // the raster backward reports nothing on the device
    const int64_t count = gs_num_image_floats(vw);
    if (count < 1) return GS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (L.overlap_prev) {
        if ((rc = launch_zero_accumulators(grad2d, (long long)GS_GRAD2D_FLOATS * L.n_slots, loss, st))) return rc;
    } else if (cudaMemsetAsync(grad2d, 0, sizeof(float) * GS_GRAD2D_FLOATS * (size_t)L.n_slots, st) != cudaSuccess ||
               cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) {
        return GS_ERR_CUDA;
    }
    L1Loss l1;
    l1.target = target;
    l1.loss = loss;
    l1.inv_n = 1.f / (float)count;
    return launch_render_bwd(L, proj, b, image, nullptr, l1, grad2d, st);
}

int gs_project_bwd(const gs_gaussians *g, const gs_views *vw, const gs_config *cfg, const float *proj,
                   const float *grad2d, const gs_grads *out, int want_gaussian_grads, int32_t *status,
                   void *stream) {
    GS_TRACE();
    Launch L;
    int rc = build_launch(vw, cfg, L);
    if (rc) return rc;
    if ((rc = check_gaussians(g, vw))) return rc;
    if (!proj || !grad2d || !out || !out->pose_partials || !vw->viewmats || !vw->intrinsics) return GS_ERR_ARG;
    if (want_gaussian_grads && g->n > 0 &&
        (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh))
        return GS_ERR_ARG;
    if (!aligned16(grad2d) || (want_gaussian_grads && g->n > 0 && !aligned16(out->quats))) return GS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (want_gaussian_grads && !L.accumulate) {
        // Gaussians outside every view's range still get (zero) gradients
        long long covered = 0;
        for (int a = 0; a < L.n_scenes; ++a) covered += L.s[a].g_count;
        if (covered != g->n && g->n > 0) {
            const int K = (g->sh_degree + 1) * (g->sh_degree + 1);
            const size_t n = (size_t)g->n;
            if (cudaMemsetAsync(out->means, 0, sizeof(float) * 3 * n, st) ||
                cudaMemsetAsync(out->log_scales, 0, sizeof(float) * 3 * n, st) ||
                cudaMemsetAsync(out->quats, 0, sizeof(float) * 4 * n, st) ||
                cudaMemsetAsync(out->opacity_logits, 0, sizeof(float) * n, st) ||
                cudaMemsetAsync(out->sh, 0, sizeof(float) * 3 * K * n, st))
                return GS_ERR_CUDA;
        }
    }
    return launch_project_bwd(L, g->sh_degree, g, vw->viewmats, vw->intrinsics, proj, grad2d, out,
                              want_gaussian_grads, pose_blocks(g->n), status, st);
}

int gs_render_bwd(const gs_gaussians *g, const gs_views *vw, const gs_config *cfg, const float *proj,
                  const gs_bins *b, const float *image, const float *dL_dimage, const gs_grads *out,
                  int want_gaussian_grads, int32_t *status, void *stream) {
    GS_TRACE();
    if (!out) return GS_ERR_ARG;
    int rc = check_gaussians(g, vw);
    if (rc) return rc;
    rc = gs_rasterize_bwd(vw, cfg, proj, b, image, dL_dimage, out->grad2d, status, stream);
    if (rc) return rc;
    return gs_project_bwd(g, vw, cfg, proj, out->grad2d, out, want_gaussian_grads, status, stream);
}

int gs_pose_grad(const gs_views *vw, const float *pose_partials, int n_blocks, float *dL_dviewmat,
                 float *dL_dtwist, void *stream) {
    GS_TRACE();
    if (!vw || vw->n_views < 1 || vw->n_views > GS_MAX_VIEWS || !pose_partials || !dL_dviewmat || n_blocks < 1 ||
        !vw->viewmats)
        return GS_ERR_ARG;
    return launch_pose_reduce(vw->n_views, pose_partials, n_blocks, vw->viewmats, dL_dviewmat, dL_dtwist,
                              (cudaStream_t)stream);
}

int gs_l1_loss(const float *image, const float *target, int64_t count, float *loss, float *dL_dimage,
               void *stream) {
    GS_TRACE();
    if (count < 0 || !loss || (count > 0 && (!image || !target || !dL_dimage))) return GS_ERR_ARG;
    return launch_l1(image, target, count, loss, dL_dimage, (cudaStream_t)stream);
}

int gs_sgld_adam_step(const gs_adam_group *groups, int n_groups, int step, double beta1, double beta2, double eps,
                      const float *noise, float noise_scale, int noise_group, void *stream) {
    GS_TRACE();
    if (!groups || n_groups < 1 || n_groups > GS_MAX_ADAM_GROUPS || step < 1) return GS_ERR_ARG;
    if (!(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps >= 0.0)) return GS_ERR_ARG;
    for (int k = 0; k < n_groups; ++k) {
        const gs_adam_group &g = groups[k];
        if (g.count < 0 || (g.count > 0 && (!g.param || !g.grad || !g.exp_avg || !g.exp_avg_sq))) return GS_ERR_ARG;
    }
    if (noise && (noise_group < 0 || noise_group >= n_groups)) return GS_ERR_ARG;
    return launch_adam_sgld(groups, n_groups, step, beta1, beta2, eps, noise, noise_scale, noise_group,
                            (cudaStream_t)stream);
}

int gs_l1_dssim_loss(const gs_views *views, const float *image, const float *target, float lambda, float *loss,
                     float *dL_dimage, void *stream) {
    GS_TRACE();
    if (!views || views->n_views < 1 || views->n_views > GS_MAX_VIEWS || !views->width || !views->height ||
        !image || !target || !loss || !dL_dimage || !(lambda >= 0.f && lambda <= 1.f))
        return GS_ERR_ARG;
    for (int v = 0; v < views->n_views; ++v)
        if (views->width[v] < 1 || views->height[v] < 1 || (long long)views->width[v] * views->height[v] > (1LL << 40))
            return GS_ERR_ARG;
    return launch_l1_dssim(views->width, views->height, views->n_views, image, target, lambda, loss, dL_dimage,
                           (cudaStream_t)stream);
}

int gs_ga_select_pairs(const float *viewmats, int n_cams, double max_angle_deg, int32_t *pairs, int64_t capacity,
                       int64_t *n_pairs_out, int32_t *status, void *stream) {
    GS_TRACE();
    if (!viewmats || n_cams < 1 || n_cams > GS_GA_MAX_CAMS || capacity < 0 || (capacity > 0 && !pairs) ||
        !n_pairs_out || !(max_angle_deg > 0.0 && max_angle_deg <= 180.0))
        return GS_ERR_ARG;
    const float cos_thr = (float)cos(max_angle_deg * (M_PI / 180.0));
    return launch_ga_select(viewmats, n_cams, cos_thr, pairs, capacity, (long long *)n_pairs_out, status,
                            (cudaStream_t)stream);
}

int gs_ga_incidence(const int32_t *pairs, int64_t n_pairs, int n_cams, int32_t *cam_offsets, int32_t *cam_pairs,
                    int32_t *status, void *stream) {
    GS_TRACE();
    if (n_cams < 1 || n_cams > GS_GA_MAX_CAMS || n_pairs < 0 || 2 * n_pairs > 0x7fffffffLL || !cam_offsets ||
        (n_pairs > 0 && (!pairs || !cam_pairs)))
        return GS_ERR_ARG;
    return launch_ga_incidence(pairs, n_pairs, n_cams, cam_offsets, cam_pairs, status, (cudaStream_t)stream);
}

int gs_ga_epipolar(const gs_ga_problem *p, float *dist, float *pair_sums, const int32_t *cam_offsets,
                   const int32_t *cam_pairs, float *loss, float *d_intrinsics, float *d_viewmats, int32_t *status,
                   void *stream) {
    GS_TRACE();
    if (!p || p->n_cams < 1 || p->n_cams > GS_GA_MAX_CAMS || !p->intrinsics || !p->viewmats || p->n_pairs < 0 ||
        p->n_matches < 0 || !loss || 2 * p->n_pairs > 0x7fffffffLL)
        return GS_ERR_ARG;
    if (p->n_pairs > 0 && (!p->pairs || !p->match_offsets || !pair_sums)) return GS_ERR_ARG;
    if (p->n_matches > 0 && (!p->matches || ((uintptr_t)p->matches & 15))) return GS_ERR_ARG;
    const bool grads = d_intrinsics || d_viewmats;
    if (grads && (!d_intrinsics || !d_viewmats || (p->n_pairs > 0 && (!cam_offsets || !cam_pairs))))
        return GS_ERR_ARG;
    return launch_ga_epipolar(*p, dist, pair_sums, cam_offsets, cam_pairs, loss, d_intrinsics, d_viewmats, status,
                              (cudaStream_t)stream);
}

int gs_ga_step(const gs_ga_state *s, const gs_ga_problem *p, float *pair_sums, const int32_t *cam_offsets,
               const int32_t *cam_pairs, float *loss, float *d_residuals, int32_t *status, void *stream) {
    GS_TRACE();
    if (!s || !p || s->n_cams != p->n_cams || !s->intrinsics0 || !s->viewmats0 || !s->residuals || !s->exp_avg ||
        !s->exp_avg_sq || !s->step || !s->intrinsics || !s->viewmats || p->intrinsics != s->intrinsics ||
        p->viewmats != s->viewmats)
        return GS_ERR_ARG;
    if (!(s->beta1 > 0.0 && s->beta1 < 1.0 && s->beta2 > 0.0 && s->beta2 < 1.0 && s->eps >= 0.0)) return GS_ERR_ARG;
    if (p->n_cams < 1 || p->n_cams > GS_GA_MAX_CAMS || p->n_pairs < 0 || p->n_matches < 0 || !loss ||
        2 * p->n_pairs > 0x7fffffffLL)
        return GS_ERR_ARG;
    if (p->n_pairs > 0 && (!p->pairs || !p->match_offsets || !pair_sums || !cam_offsets || !cam_pairs))
        return GS_ERR_ARG;
    if (p->n_matches > 0 && (!p->matches || ((uintptr_t)p->matches & 15))) return GS_ERR_ARG;
    return launch_ga_step(*s, *p, pair_sums, cam_offsets, cam_pairs, loss, d_residuals, status,
                          (cudaStream_t)stream);
}

size_t gs_ga_weights_scratch_bytes(int n_bins) {
    if (n_bins < 1 || n_bins > GS_GA_MAX_BINS) return 0;
    return (size_t)(8 + 2048 + n_bins) * 4;
}

int gs_ga_weights(const float *dist, int64_t n, int n_bins, double alpha, uint32_t *counts, float *weights,
                  float *stats, void *scratch, void *stream) {
    GS_TRACE();
    if (n < 0 || n > 0xffffffffLL || n_bins < 1 || n_bins > GS_GA_MAX_BINS || !(alpha >= 0.0) || !counts ||
        !stats || !scratch || (n > 0 && (!dist || !weights)))
        return GS_ERR_ARG;
    return launch_ga_weights(dist, n, n_bins, alpha, counts, weights, stats, (uint32_t *)scratch,
                             (cudaStream_t)stream);
}

const char *gs_error_string(int code) {
    switch (code) {
    case GS_OK: return "ok";
    case GS_ERR_ARG: return "invalid argument";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_CAPACITY: return "instance capacity exceeded";
    case GS_ERR_UNSUPPORTED: return "unsupported configuration";
    case GS_ERR_OVERFLOW: return "more than 2^31-1 tile instances";
    case GS_ERR_TOO_LARGE: return "pose partials exceed the fixed scratch of the allocation-free entry point";
    case GS_ERR_TIMEOUT: return "a bounded wait for an asynchronous copy ran out";
    default: return "unknown status";
    }
}

int gs_version(void) { return 1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free projection backward (gs_project_bwd_noalloc): the pose
// partials live in this file-scope device array instead of a caller buffer.
// ---------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) float g_noalloc_pose[GS_NOALLOC_POSE_FLOATS];

namespace {
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[64];   // device address of g_noalloc_pose found by the last uncaptured call, per device

// Host code cannot use the array's name as a device address; its address is
// looked up with the device current. An uncaptured call looks it up every
// time (the module, and with it the array, may have moved if the context was
// destroyed and created again); a call whose stream is being captured cannot
// load modules, so it uses the address the last uncaptured call found.
int noalloc_scratch(cudaStream_t st, float **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GS_ERR_CUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_pose) != cudaSuccess || !p) return GS_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    } else if (!g_noalloc_ptr[dev]) {
        return GS_ERR_CUDA;   // no uncaptured call on this device yet
    }
    *out = g_noalloc_ptr[dev];
    return GS_OK;
}
}  // namespace

extern "C" int gs_project_bwd_noalloc(const gs_gaussians *g, const gs_views *vw, const gs_config *cfg,
                                      const float *proj, const float *grad2d, const gs_grads *grads,
                                      int want_gaussian_grads, float *dL_dviewmat, float *dL_dtwist,
                                      int32_t *status, void *stream) {
    GS_TRACE();
    Launch L;
    int rc = build_launch(vw, cfg, L);
    if (rc) return rc;
    if ((rc = check_gaussians(g, vw))) return rc;
    if (!proj || !grad2d || !grads || !dL_dviewmat || !vw->viewmats || !vw->intrinsics) return GS_ERR_ARG;
    if (want_gaussian_grads && g->n > 0 &&
        (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits || !grads->sh))
        return GS_ERR_ARG;
    if (!aligned16(grad2d) || (want_gaussian_grads && g->n > 0 && !aligned16(grads->quats))) return GS_ERR_ARG;
    const int nblk = pose_blocks(g->n);
    if ((long long)L.n_views * nblk * 12 > (long long)GS_NOALLOC_POSE_FLOATS) return GS_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)stream;
    float *scratch = nullptr;
    if ((rc = noalloc_scratch(st, &scratch))) return rc;
    if (want_gaussian_grads && !L.accumulate) {
        long long covered = 0;
        for (int a = 0; a < L.n_scenes; ++a) covered += L.s[a].g_count;
        if (covered != g->n && g->n > 0) {
            const int K = (g->sh_degree + 1) * (g->sh_degree + 1);
            const size_t n = (size_t)g->n;
            if (cudaMemsetAsync(grads->means, 0, sizeof(float) * 3 * n, st) ||
                cudaMemsetAsync(grads->log_scales, 0, sizeof(float) * 3 * n, st) ||
                cudaMemsetAsync(grads->quats, 0, sizeof(float) * 4 * n, st) ||
                cudaMemsetAsync(grads->opacity_logits, 0, sizeof(float) * n, st) ||
                cudaMemsetAsync(grads->sh, 0, sizeof(float) * 3 * K * n, st))
                return GS_ERR_CUDA;
        }
    }
    gs_grads out = *grads;
    out.pose_partials = scratch;   // every partial the reduction reads is written first
    rc = launch_project_bwd(L, g->sh_degree, g, vw->viewmats, vw->intrinsics, proj, grad2d, &out,
                            want_gaussian_grads, nblk, status, st);
    if (rc) return rc;
    return launch_pose_reduce(L.n_views, scratch, nblk, vw->viewmats, dL_dviewmat, dL_dtwist, st);
}

// ---------------------------------------------------------------------------
// Check of the bounded wait (gs_check_bounded_wait): one thread arms an
// mbarrier for 16 bytes of a copy that is never issued and waits on it with
// the projection kernels' bounded wait, which must give up and report.
// ---------------------------------------------------------------------------
namespace gsk {
__global__ void k_wait_check(int32_t *status) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16);   // the one arrival, with 16 bytes outstanding that nothing delivers
    if (!mbar_wait(&bar, 0)) {
        atomicCAS(status, 0, GS_ERR_TIMEOUT);
        atomicExch(status + 1, 0);
    }
}
}  // namespace gsk

extern "C" int gs_check_bounded_wait(int32_t *status, void *stream) {
    GS_TRACE();
    if (!status) return GS_ERR_ARG;
    gsk::k_wait_check<<<1, 32, 0, (cudaStream_t)stream>>>(status);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
