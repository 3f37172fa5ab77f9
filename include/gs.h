/*
 * gs.h -- C ABI of libgsplat_gb300.so: a differentiable tile-based 3D Gaussian
 * Splatting rasterizer with camera-pose gradients for NVIDIA GB300 (sm_103a).
 *
 * Paper anchors (arXiv 2509.25191, "VGGT-X"):
 *   Section 3.1 -- Gaussians with mean, covariance R S S^T R^T, opacity and
 *                  degree-3 SH colour; pixel colours by alpha blending;
 *                  training by photometric loss.
 *   Section 3.4 -- joint optimisation of per-view residual poses (translation
 *                  and 6D rotation) with the Gaussians, which needs the
 *                  gradient of the rendered images w.r.t. each camera pose.
 *   The rasterizer itself is cited, not specified, by the paper; the EWA
 *   projection Sigma' = J W Sigma W^T J^T + 0.3 I, the alpha clamp 0.99, the
 *   1/255 cutoff and the stop before T < 1e-4 are the readings this library
 *   implements (defaults of gs_config).
 *
 * Conventions for every entry point
 *   - All functions return int: GS_OK (0) or a gs_status code. No exception
 *     or abort crosses the ABI. gs_error_string() names a code.
 *   - Buffers marked DEVICE are device pointers owned by the caller; the
 *     library never allocates or frees, and only gs_status_read waits for
 *     the device. Buffers marked HOST are read during the call only.
 *   - Work is enqueued on the caller's stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream). Given the same host arguments,
 *     the enqueued work is the same on every call, so a call sequence can be
 *     captured into a CUDA graph and replayed with new DEVICE contents.
 *   - Host-side argument errors return GS_ERR_ARG before anything is
 *     enqueued; a failed launch returns GS_ERR_CUDA. Conditions found on the
 *     device (instance capacity exceeded) are written to the caller's DEVICE
 *     status word int32[4] = {code, detail_lo, detail_hi, 0}; the caller reads
 *     it at a point of its choosing (gs_status_read). Kernels never trap; the
 *     only waits are the forward projection's bounded waits for its own
 *     tensor copies (GS_ERR_TIMEOUT if one runs out; gs_check_bounded_wait
 *     makes one run out on purpose, for tests of this path). When the status
 *     word is non-zero after a call, that call's outputs are undefined.
 *   - The enqueued work depends only on the arguments: no environment
 *     variable or global setting steers it (gs_config.use_tma selects the
 *     forward projection's staging).
 *   - float32 everywhere. Quaternions are (w,x,y,z). Cameras are
 *     world->camera rigid transforms with OpenCV axes (x right, y down,
 *     z forward); a pixel (u,v) has its centre at (u+0.5, v+0.5).
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_MAX_VIEWS 64        /* views per call */
#define GS_RECORD_FLOATS 16    /* floats per projected record */
#define GS_GRAD2D_FLOATS 12    /* floats per 2D-gradient record */
#define GS_POSE_FLOATS 12      /* dL/dR (row-major) then dL/dt */

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_ARG = 1,          /* invalid argument (host check) */
    GS_ERR_CUDA = 2,         /* a CUDA call or launch failed */
    GS_ERR_CAPACITY = 3,     /* device: instance capacity too small; detail = instances needed */
    GS_ERR_UNSUPPORTED = 4,  /* configuration not compiled in (tile shape, SH degree) */
    GS_ERR_OVERFLOW = 5,     /* device: more than 2^31-1 tile instances */
    GS_ERR_TOO_LARGE = 6,    /* exceeds the fixed scratch of gs_project_bwd_noalloc */
    GS_ERR_TIMEOUT = 7       /* device: a bounded wait for an asynchronous copy ran out */
} gs_status;

/* Rasterizer settings. gs_config_default() fills the defaults in brackets. */
typedef struct gs_config {
    int tile_w, tile_h;   /* tile in pixels [16,16]; supported: 16x16, 8x8, 16x8, 32x8, 32x16, 32x32 */
    int pixel_gate;       /* [1] evaluate a Gaussian at a pixel only if |dx|,|dy| <= radius
                             (the only supported value: it makes images tile-size invariant) */
    float near_z;         /* [0.2] cull if camera-space z <= near_z */
    float dilation;       /* [0.3] added to the 2D covariance diagonal (pixels^2) */
    float alpha_min;      /* [1/255] skip contributions with alpha below this */
    float alpha_max;      /* [0.99] clamp alpha to this */
    float t_min;          /* [1e-4] stop before transmittance would fall below this */
    float fov_clamp;      /* [1.3] clamp x/z, y/z to +-fov_clamp*tan(half fov) inside J */
    float bg[3];          /* [0,0,0] background colour */
    int count_pairs;      /* [0] if nonzero, the raster backward also counts the pixel-Gaussian pairs it
                             evaluates and composites into bins->counters (diagnostics; costs time) */
    int accumulate_grads; /* [0] 0: the backward overwrites the raw-parameter gradients (gs_grads.means ..
                             .sh); nonzero: it adds to them (+=), so gradients of several calls (views,
                             losses) sum in the caller's buffers, which the caller zeroes first */
    int use_tma;          /* [1] nonzero: the forward projection stages degree-3 SH rows and records by
                             tensor copies where the layout allows; 0: per-thread loads and stores. The
                             results are the same bit for bit. */
    int fwd_batch;        /* [2] Gaussians each thread stages per shared-memory batch in gs_render_fwd:
                             1, 2 or 4 (a batch is fwd_batch x tile_w x tile_h / 2 Gaussians) */
    int bwd_batch;        /* [1] the same for gs_rasterize_bwd: 1 or 2. Neither changes the image; the
                             2D gradients change only in the order of their float additions. */
    int overlap_prev;     /* [0] nonzero: gs_rasterize_bwd(_l1) and the one-view gs_project_bwd with
                             parameter gradients are launched as programmatic dependents of the kernel
                             ahead of them on the stream, and zero their accumulators (the 2D gradients
                             and the L1 loss; the parameter-gradient rows) while that kernel's last
                             blocks still run, waiting for it before anything else. The caller
                             guarantees that the kernel ahead neither reads nor writes those outputs
                             (true in a step: gs_render_fwd, then gs_rasterize_bwd_l1, then
                             gs_project_bwd); 0: every kernel starts after the work ahead of it. */
} gs_config;

/* Gaussians (all DEVICE, float32, contiguous). Several scenes may be
 * concatenated; each view names the range it sees (gs_views). */
typedef struct gs_gaussians {
    int64_t n;                   /* total Gaussians */
    int sh_degree;               /* 0..3; K = (sh_degree+1)^2 */
    const float *means;          /* [n,3] */
    const float *log_scales;     /* [n,3]; scale = exp */
    const float *quats;          /* [n,4] (w,x,y,z), need not be unit */
    const float *opacity_logits; /* [n]; opacity = sigmoid */
    const float *sh;             /* [n,K,3], coefficient l*l+l+m, channel last */
} gs_gaussians;

/* Views rendered by one call. Views that see the same Gaussian range must be
 * contiguous; ranges of different groups must not overlap. */
typedef struct gs_views {
    int n_views;                 /* V, 1..GS_MAX_VIEWS */
    const float *viewmats;       /* DEVICE [V,12]: R row-major (9) then t (3), world->camera */
    const float *intrinsics;     /* DEVICE [V,4]: fx, fy, cx, cy (pixels) */
    const int32_t *width;        /* HOST [V] */
    const int32_t *height;       /* HOST [V] */
    const int64_t *gauss_begin;  /* HOST [V] first Gaussian the view sees */
    const int64_t *gauss_count;  /* HOST [V] number of Gaussians the view sees */
} gs_views;

/* Tile lists produced by gs_bin_sort (all DEVICE, caller-allocated with the
 * sizes from the layout queries below). */
typedef struct gs_bins {
    int64_t capacity;     /* instance capacity of keys/ids/keys_tmp */
    int32_t *tile_ranges; /* [T,2] start,end of each tile's instances; tiles of view v
                             start at gs_tile_base(v), tile (tx,ty) at +ty*Gx+tx */
    uint64_t *keys;       /* [capacity] (float32 depth bits << 32) | slot, ascending per tile */
    uint32_t *ids;        /* [capacity] slot of each instance, same order as keys */
    uint64_t *keys_tmp;   /* [capacity] scratch for tiles too large for on-chip sorting */
    int32_t *tile_order;  /* [T] work order: tiles by decreasing instance count */
    int32_t *tile_scratch;/* [5T] scratch (per-tile counters, then the runs of large tiles that
                             are sorted in pieces) */
    int32_t *counters;    /* [GS_NUM_COUNTERS] scratch; counters[0] = instances after the call;
                             int64 at counters+8: pixel-Gaussian pairs evaluated by gs_render_fwd,
                             +10: composited by it, +12/+14: the same for gs_rasterize_bwd */
    int32_t *last_contrib;/* optional [sum_v H_v W_v] (NULL = not kept): per pixel (view v's pixel
                             (u, y) at gs_pixel_base(v)/3 + y W_v + u), one past the instance index
                             (into keys/ids) of the last Gaussian gs_render_fwd composited there (the
                             tile's start if none). gs_render_fwd writes it; gs_rasterize_bwd, given the
                             same bins, then stops each pixel there instead of replaying its list to
                             the end. 4 bytes per pixel: an index, not a stored transmittance. */
    int32_t *tile_work;   /* optional [T] (NULL = none), used with last_contrib when the call has fewer
                             than 16 tiles per SM: per tile, the replay length of the last gs_render_fwd
                             on these bins (the largest last-contributor offset of its pixels). Kept
                             across calls: gs_render_fwd takes its tiles longest first by these values
                             (a value <= 0 counts as the tile's instance count) and overwrites them;
                             gs_rasterize_bwd takes its tiles in the same way. Only the order in which
                             the persistent blocks take the tiles depends on it, never a result, so any
                             contents are safe (zero it once for a count-ordered first call). */
} gs_bins;
#define GS_NUM_COUNTERS 16

/* Gradient outputs of gs_render_bwd (all DEVICE). The parameter gradients are
 * overwritten, or accumulated (+=) when gs_config.accumulate_grads is set.
 * grad2d and pose_partials are caller-owned scratch that also remain
 * readable after the call. */
typedef struct gs_grads {
    float *means;          /* [n,3] */
    float *log_scales;     /* [n,3] */
    float *quats;          /* [n,4] */
    float *opacity_logits; /* [n] */
    float *sh;             /* [n,K,3] */
    float *grad2d;         /* [P,12] per slot: dL/d(x, y, a, b | c, o, r, g | b_col, -, -, -): mean,
                              dilated 2D covariance (a, b, c; b the off-diagonal value), opacity,
                              colour */
    float *pose_partials;  /* [V, gs_pose_blocks(n), 12] */
} gs_grads;

/* ---------------- layout queries (host, pure) ---------------- */

void gs_config_default(gs_config *cfg);
/* P: number of projected records (slots). Slot of Gaussian i in view v is
 * gs_slot_base(v) + (i - gauss_begin[v]). */
int64_t gs_num_slots(const gs_views *views);
int64_t gs_slot_base(const gs_views *views, int v);
/* T: total tiles over all views; ceil(W/tile_w)*ceil(H/tile_h) per view. */
int64_t gs_num_tiles(const gs_views *views, const gs_config *cfg);
int64_t gs_tile_base(const gs_views *views, const gs_config *cfg, int v);
/* Image floats: sum_v 3*H_v*W_v; view v is [3,H_v,W_v] at float offset
 * gs_pixel_base(v) (= 3 * sum_{u<v} H_u*W_u). */
int64_t gs_num_image_floats(const gs_views *views);
int64_t gs_pixel_base(const gs_views *views, int v);
/* Blocks of the projection-backward grid for n Gaussians (pose partials). */
int gs_pose_blocks(int64_t n);

/* One caller buffer for every scratch array of a forward + backward step over
 * these views: the tile lists of gs_bins (tile_ranges, keys, ids, keys_tmp,
 * tile_order, tile_scratch, counters, last_contrib, tile_work for `capacity` tile
 * instances) and the backward's grad2d [P,12] and pose_partials [V,
 * gs_pose_blocks(n_gaussians), 12]. gs_workspace_size returns its size in
 * bytes (0 for invalid arguments); gs_workspace_carve fills bins (all of its
 * fields) and grads->grad2d, grads->pose_partials with 256-byte aligned
 * pieces of ws (DEVICE, ws_bytes >= gs_workspace_size(...), 256-byte
 * aligned); the parameter-gradient pointers of grads are left as they are.
 * Both are host arithmetic only (nothing is enqueued or touched on the
 * device). The instance count of a step is known after gs_bin_sort
 * (counters[0]; GS_ERR_CAPACITY in the status word if capacity was too
 * small). */
size_t gs_workspace_size(const gs_views *views, const gs_config *cfg, int64_t n_gaussians, int64_t capacity);
int gs_workspace_carve(const gs_views *views, const gs_config *cfg, int64_t n_gaussians, int64_t capacity,
                       void *ws, size_t ws_bytes, gs_bins *bins, gs_grads *grads);

/* Copy the DEVICE status word int32[4] to host_status (HOST int32[4]) once
 * the work enqueued on `stream` so far has finished: the one entry point
 * that synchronises (the caller's chosen sync point; not capturable). Returns
 * GS_ERR_CUDA if the copy or the wait fails; host_status[0] is then the
 * status code the kernels left (GS_OK, GS_ERR_CAPACITY with the needed
 * instance count in host_status[1..2], GS_ERR_OVERFLOW or GS_ERR_TIMEOUT). */
int gs_status_read(const int32_t *status, int32_t *host_status, void *stream);

/* ---------------- the rasterizer ---------------- */

/* Project every Gaussian into every view that sees it (Section 3.1
 * primitive; EWA splatting). Per slot p, proj[16p..16p+15] =
 *   {x, y, ext_x, ext_y} mean in pixels (high part) and the half-extents of
 *                       the pixels the Gaussian can reach: min(radius,
 *                       sqrt(k Sigma'_xx)) (and yy) with k = 2 ln(o /
 *                       alpha_min), the bounding box of the ellipse where
 *                       alpha >= alpha_min (culled if k <= 0),
 *   {Ah, beta, Dh, o}   the conic (inverse of the dilated 2D covariance
 *                       Sigma' = [[a, b], [b, c]]) in the form the raster
 *                       kernels evaluate, and the opacity: with det =
 *                       a c - b^2, A = c / det, beta = -b / c, D = 1 / c,
 *                       Ah = -A / (2 ln 2), Dh = -D / (2 ln 2), the Gaussian
 *                       at offset (dx, dy) from the mean is
 *                       2^(Ah u^2 + Dh dy^2) with u = dx + beta dy,
 *   {r, g, b, radius}   colour (SH evaluated, +0.5, clamped at 0) and the
 *                       integer radius ceil(3 sqrt(lambda_max)) (0 = culled),
 *   {x_lo, y_lo, depth, clamp_bits}  low parts of the mean (x + x_lo is the
 *                       position to ~1e-5 px), camera z, bit c set if colour
 *                       channel c was clamped.
 * Culled records are all zero.
 * proj: DEVICE [P,16], 16-byte aligned. status: DEVICE int32[4] or NULL;
 * with cfg->use_tma the degree-3 path stages each block's SH rows and
 * records with tensor copies, and if a bounded wait for one runs out (a copy
 * that never lands) it sets status = {GS_ERR_TIMEOUT, block} and leaves that
 * block's records unwritten. */
int gs_project(const gs_gaussians *g, const gs_views *views, const gs_config *cfg,
               float *proj, int32_t *status, void *stream);

/* Bin the projected records into tiles and sort each tile by (depth, slot).
 * A record with radius > 0 touches the tiles [floor((x-ext_x)/tw),
 * floor((x+ext_x)/tw)] x [floor((y-ext_y)/th), floor((y+ext_y)/th)], clipped
 * to the view's grid, computed in float32. If the instance count
 * exceeds bins->capacity, status = {GS_ERR_CAPACITY, needed} and the lists
 * are left unsorted; counters[0] holds the count either way (a call with
 * capacity 0 is a pure count). */
int gs_bin_sort(const gs_views *views, const gs_config *cfg, const float *proj,
                const gs_bins *bins, int32_t *status, void *stream);

/* Composite every pixel front to back (Section 3.1 alpha blending) and
 * write image: DEVICE [sum_v 3 H_v W_v] (view layout as gs_pixel_base), and
 * bins->last_contrib if it is set. If a capacity error is pending in
 * counters, images are filled with zeros. */
int gs_render_fwd(const gs_views *views, const gs_config *cfg, const float *proj,
                  const gs_bins *bins, float *image, int32_t *status, void *stream);

/* Backward of gs_project + gs_render_fwd for the upstream gradient
 * dL_dimage (same layout as image). image must be the forward's output for
 * the same inputs (transmittance is recomputed, not stored; the colour
 * behind each Gaussian is taken from the image).
 * Writes grads->grad2d (zeroed by the call), the raw-parameter gradients
 * (unless want_gaussian_grads == 0) and grads->pose_partials. */
int gs_render_bwd(const gs_gaussians *g, const gs_views *views, const gs_config *cfg,
                  const float *proj, const gs_bins *bins, const float *image,
                  const float *dL_dimage, const gs_grads *grads, int want_gaussian_grads,
                  int32_t *status, void *stream);

/* The two stages of gs_render_bwd, callable separately (same arguments and
 * semantics as there). gs_rasterize_bwd zeroes grad2d [P,12] and adds the
 * per-slot 2D gradients (layout as gs_grads.grad2d); if bins->last_contrib is
 * set it must hold what gs_render_fwd wrote for this image with these bins,
 * and each pixel's replay ends at its last composited Gaussian (the result is
 * the same as without it). gs_project_bwd chains grad2d to the raw
 * parameters (overwritten, or added with cfg->accumulate_grads; a
 * Gaussian's terms are summed over its views in ascending order, then
 * written or added once) and the pose partials (always overwritten). With
 * one view it runs the chain only for the Gaussians with a nonzero 2D
 * gradient and writes zeros for the others (accumulating, leaves them as
 * they are); with cfg->overlap_prev that one-view call with parameter
 * gradients zeroes those rows in the tail of the kernel ahead (see
 * gs_config.overlap_prev). With several views it
 * runs the chains per block either by each Gaussian's thread or over
 * per-view lists of the Gaussians with a gradient, whichever takes fewer
 * warp runs (the pose partials' grouping follows that choice and is
 * deterministic). */
int gs_rasterize_bwd(const gs_views *views, const gs_config *cfg, const float *proj, const gs_bins *bins,
                     const float *image, const float *dL_dimage, float *grad2d, int32_t *status,
                     void *stream);
int gs_project_bwd(const gs_gaussians *g, const gs_views *views, const gs_config *cfg, const float *proj,
                   const float *grad2d, const gs_grads *grads, int want_gaussian_grads, int32_t *status,
                   void *stream);

/* gs_rasterize_bwd for the mean L1 photometric loss (Section 3.1 photometric
 * supervision), with the loss folded in: the upstream gradient of each image
 * value is sign(image - target) / count, count = gs_num_image_floats(views)
 * (0 where they are equal; the value gs_l1_loss writes, bit for bit),
 * formed in the kernel from image and target (DEVICE, same layout as image)
 * instead of read from a dL_dimage buffer, which is neither needed nor
 * written. loss DEVICE [1] is overwritten with mean |image - target| (block
 * partials added with atomics, so its last bits depend on their order).
 * grad2d as in gs_rasterize_bwd. Same errors as gs_rasterize_bwd; GS_ERR_ARG
 * also for a NULL target or loss. */
int gs_rasterize_bwd_l1(const gs_views *views, const gs_config *cfg, const float *proj, const gs_bins *bins,
                        const float *image, const float *target, float *loss, float *grad2d, int32_t *status,
                        void *stream);

/* Reduce pose partials (Section 3.4 pose residuals): dL_dviewmat DEVICE
 * [V,12] = dL/dR (row-major) then dL/dt; dL_dtwist DEVICE [V,6] (may be NULL)
 * = gradient w.r.t. a left twist (rho, phi), T <- exp(xi^) T:
 * M = dL/dR R^T + dL/dt t^T (3x3, 1-based indices below),
 * dL/dphi = (M32 - M23, M13 - M31, M21 - M12), dL/drho = dL/dt.
 * Summation order is fixed (deterministic). */
int gs_pose_grad(const gs_views *views, const float *pose_partials, int n_blocks,
                 float *dL_dviewmat, float *dL_dtwist, void *stream);

/* Mean L1 photometric loss (Section 3.1 photometric supervision) and its
 * gradient: loss DEVICE [1] = mean |image - target| (overwritten; block
 * partials are added with atomics, so its last bits depend on their order),
 * dL_dimage DEVICE [count] = sign(image - target) / count (deterministic). */
int gs_l1_loss(const float *image, const float *target, int64_t count, float *loss,
               float *dL_dimage, void *stream);

/* SGLD update with an Adam direction (paper Eq. 1, the MCMC-3DGS update the
 * method trains with): for every group,
 *   m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
 *   p <- p - lr * (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps),
 * and, for group noise_group only, p <- p + noise_scale * noise (the
 * exploration term lambda_noise * eps; noise is drawn by the caller, DEVICE
 * [count of that group], or NULL for none). All arrays DEVICE float32,
 * updated in place; step >= 1 counts Adam steps; beta1, beta2, eps are
 * doubles so that 1 - beta is formed exactly before rounding. One launch for
 * all groups (at most GS_MAX_ADAM_GROUPS). */
#define GS_MAX_ADAM_GROUPS 8
typedef struct gs_adam_group {
    float *param;
    const float *grad;
    float *exp_avg;
    float *exp_avg_sq;
    int64_t count;
    float lr;
} gs_adam_group;
int gs_sgld_adam_step(const gs_adam_group *groups, int n_groups, int step, double beta1, double beta2, double eps,
                      const float *noise, float noise_scale, int noise_group, void *stream);

/* Photometric loss with D-SSIM (Section 3.1: a weighted sum of an L1 and a
 * D-SSIM term; weighting and SSIM settings of the cited 3DGS training):
 *   L = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y)),
 * SSIM per channel of every view from local statistics under an 11x11
 * Gaussian window (sigma 1.5, normalised) as a same-size correlation with
 * zero padding, C1 = 0.01^2, C2 = 0.03^2, both means over all values of all
 * views. image, target: DEVICE, views concatenated, each [3,H,W] (the layout
 * of gs_render_fwd; only views->n_views, width, height are read). loss:
 * DEVICE [3] = {L, mean L1, 1 - mean SSIM} (overwritten); dL_dimage: DEVICE,
 * same layout (overwritten). 0 <= lambda <= 1. One fused forward+backward
 * kernel over 32x32 tiles; the loss sums use atomics (the gradient is
 * deterministic, the last bits of the loss are not). */
int gs_l1_dssim_loss(const gs_views *views, const float *image, const float *target, float lambda, float *loss,
                     float *dL_dimage, void *stream);

/* ------------------------------------------------------------------------
 * Camera global alignment (paper Section 3.3, Eqs. 2-4).
 *
 * Cameras n = 0..n_cams-1: intrinsics (fx, fy, cx, cy) and world-to-camera
 * extrinsics (R row-major, t) as in gs_views. A pair (i, j) holds keypoint
 * matches (x, y, x', y'): x in image i, x' in image j, in pixels. With
 * R_ij = R_j R_i^T, t_ij = t_j - R_ij t_i and F = K_j^-T [t_ij]x R_ij K_i^-1
 * (Eq. 2) a match's epipolar distance is e = |x'^T F x| / ||(F x)_{1,2}||,
 * the distance of x' to the epipolar line of x in pixels (0, with no
 * gradient, where the line is undefined). The loss is
 * L = sum_k w_k e_k / sum_k w_k over all matches of all pairs (Eq. 2).
 * ---------------------------------------------------------------------- */
#define GS_GA_MAX_CAMS 8192
#define GS_GA_PAIR_FLOATS 12   /* per-pair partial sums */
#define GS_GA_MAX_BINS 16384

typedef struct gs_ga_problem {
    int n_cams;
    const float *intrinsics;        /* DEVICE [n_cams,4] fx, fy, cx, cy */
    const float *viewmats;          /* DEVICE [n_cams,12] R row-major, t */
    int64_t n_pairs;
    const int32_t *pairs;           /* DEVICE [n_pairs,2] (i, j), i != j, no pair listed twice */
    const int64_t *match_offsets;   /* DEVICE [n_pairs+1]: pair m owns matches offsets[m]..offsets[m+1]-1 */
    int64_t n_matches;
    const float *matches;           /* DEVICE [n_matches,4] (x, y, x', y'), 16-byte aligned */
    const float *weights;           /* DEVICE [n_matches] w_k, or NULL for all 1 */
} gs_ga_problem;

/* Candidate pairs (Section 3.3; threshold 30 degrees in Section 4.1): every
 * (i, j), i < j, whose viewing directions (third rows of R_i and R_j) are
 * less than max_angle_deg apart, i.e. d_i . d_j > cos(max_angle_deg) with
 * the dot product rounded to float32 after each operation and the cosine
 * formed in double, then rounded. Pairs are written in row-major order
 * (ascending i, then j) to pairs (DEVICE int32 [capacity,2]); the number
 * found goes to n_pairs_out (DEVICE int64 [1]). If it exceeds capacity,
 * status = {GS_ERR_CAPACITY, count} and no pair is written. One block;
 * n_cams <= GS_GA_MAX_CAMS. */
int gs_ga_select_pairs(const float *viewmats, int n_cams, double max_angle_deg, int32_t *pairs, int64_t capacity,
                       int64_t *n_pairs_out, int32_t *status, void *stream);

/* Camera -> pair incidence lists for the gradient reduction: cam_offsets
 * (DEVICE int32 [n_cams+1]) and cam_pairs (DEVICE int32 [2*n_pairs]), the
 * entries of camera n being cam_pairs[cam_offsets[n]..cam_offsets[n+1]-1]
 * = 2*m + (1 if n is the pair's second camera), sorted ascending (the
 * reduction order is fixed, so gradients are bit-reproducible). A camera in
 * more than GS_GA_MAX_CAMS pairs sets status = {GS_ERR_ARG, camera}. */
int gs_ga_incidence(const int32_t *pairs, int64_t n_pairs, int n_cams, int32_t *cam_offsets, int32_t *cam_pairs,
                    int32_t *status, void *stream);

/* Epipolar distances, loss and camera gradients (Eq. 2). dist (DEVICE
 * [n_matches]) receives every e_k, or NULL. pair_sums is caller scratch
 * (DEVICE float [n_pairs, GS_GA_PAIR_FLOATS]). loss (DEVICE [1]) receives L
 * (0 if the weights sum to 0). If d_intrinsics (DEVICE [n_cams,4]) and
 * d_viewmats (DEVICE [n_cams,12]) are both non-NULL they are overwritten
 * with dL/d(fx, fy, cx, cy) and dL/d(R, t) of every camera (zero for a
 * camera in no pair); that needs the incidence lists of gs_ga_incidence.
 * The distances are computed in float32 in normalised coordinates
 * (K^-1 x), the gradient sums in float32 per pair and reduced per camera in
 * a fixed order. A pair whose camera index or match range is out of
 * bounds contributes nothing and sets status = {GS_ERR_ARG, pair} (status
 * may be NULL). No allocation, no synchronisation: capturable. */
int gs_ga_epipolar(const gs_ga_problem *p, float *dist, float *pair_sums, const int32_t *cam_offsets,
                   const int32_t *cam_pairs, float *loss, float *d_intrinsics, float *d_viewmats, int32_t *status,
                   void *stream);

/* One whole global-alignment iteration on the device (three launches, no
 * host work, capturable): the cameras from per-camera residuals, the Eq. 2
 * loss and camera gradients (as gs_ga_epipolar), the gradients chained to
 * the residuals and one Adam step on them. The residuals of camera n,
 * residuals[10n..10n+9], are a 6D rotation residual (a1, a2: dR has columns
 * b1 = a1/|a1|, b2 = normalised a2 - (b1.a2) b1, b3 = b1 x b2), a
 * translation residual dt and a log-focal residual df (Section 3.4's pose
 * residual plus a focal scale): R = dR R0, t = t0 + dt, (fx, fy) = (fx0,
 * fy0) exp(df), principal point fixed (df stays 0 unless optimise_focal).
 * The call increments *step (DEVICE int32, 0 before the first call), writes
 * the cameras it used to intrinsics / viewmats (which p->intrinsics and
 * p->viewmats must point at), the loss at those cameras, dL/d(residuals) to
 * d_residuals (DEVICE [n,10], or NULL), and updates residuals, exp_avg and
 * exp_avg_sq in place with Adam (bias-corrected with the incremented step,
 * 1 - beta formed in double, 1 - beta^t as -expm1(t ln beta) in float;
 * 0 < beta < 1): p <- p - lr m^ / (sqrt(v^) + eps). */
typedef struct gs_ga_state {
    int n_cams;
    const float *intrinsics0;   /* DEVICE [n_cams,4] */
    const float *viewmats0;     /* DEVICE [n_cams,12] */
    float *residuals;           /* DEVICE [n_cams,10]; identity (1,0,0, 0,1,0, 0,0,0, 0) */
    float *exp_avg;             /* DEVICE [n_cams,10] */
    float *exp_avg_sq;          /* DEVICE [n_cams,10] */
    int32_t *step;              /* DEVICE [1] */
    float *intrinsics;          /* DEVICE [n_cams,4], written */
    float *viewmats;            /* DEVICE [n_cams,12], written */
    float lr;
    double beta1, beta2, eps;
    int optimise_focal;
} gs_ga_state;
int gs_ga_step(const gs_ga_state *s, const gs_ga_problem *p, float *pair_sums, const int32_t *cam_offsets,
               const int32_t *cam_pairs, float *loss, float *d_residuals, int32_t *status, void *stream);

/* Adaptive weights (Eq. 3) and the median (Eq. 4) of n distances dist
 * (DEVICE, finite, >= 0): a histogram with n_bins equal bins on
 * [0, max e], bin b = min(n_bins - 1, floor(e * (n_bins / max e))) with the
 * quotient and the product rounded to float32 (all in bin 0 if max e is 0);
 * counts (DEVICE uint32 [n_bins]) receives it; weights (DEVICE [n]) gets
 * w_k = (f(e_k) / mean_k f(e_k))^alpha with f the histogram density, which
 * equals (n c_b / sum_b c_b^2)^alpha (formed in double per bin); stats
 * (DEVICE float [4]) = {max e, lower middle, upper middle order statistic
 * (equal for odd n; the median is their mean), 0}. scratch: DEVICE, at
 * least gs_ga_weights_scratch_bytes(n_bins) bytes. 1 <= n_bins <=
 * GS_GA_MAX_BINS, alpha >= 0; n = 0 writes stats = 0 and nothing else. */
size_t gs_ga_weights_scratch_bytes(int n_bins);
int gs_ga_weights(const float *dist, int64_t n, int n_bins, double alpha, uint32_t *counts, float *weights,
                  float *stats, void *scratch, void *stream);

/* Allocation-free variant of gs_project_bwd followed by gs_pose_grad (the
 * paper has no counterpart: this exists for callers, not for the method).
 *
 * Some callers cannot hand the library a scratch buffer: code that runs
 * under a memory planner or inside another runtime that owns every device
 * allocation (a plugin host, an inference server or graph executor that
 * forbids cudaMalloc after start-up) has no way to allocate the per-block
 * pose partials that gs_project_bwd needs. This entry point takes the same
 * inputs and the same parameter-gradient outputs as gs_project_bwd, and
 * writes the reduced pose gradients like gs_pose_grad (dL_dviewmat [V,12],
 * dL_dtwist [V,6] or NULL); grads->grad2d and grads->pose_partials are
 * ignored. It calls no cudaMalloc/cudaFree and no allocating library
 * routine.
 *
 * Its scratch is a file-scope static device array of GS_NOALLOC_POSE_FLOATS
 * floats (3 MB) that every GPU which loads the library keeps until the
 * process exits. The pose partials of one call need V * gs_pose_blocks(n) *
 * 12 floats; a call beyond that returns GS_ERR_TOO_LARGE before enqueuing
 * anything. Every call shares the one array and leaves its contents behind
 * (each call overwrites all the partials it reads, so nothing needs
 * clearing; the outputs of a call that sets the status word are
 * undefined): calls that overlap on
 * the GPU (other streams, other host threads on the same device) race and
 * must be serialised by the caller. An uncaptured call looks up the array's
 * device address with the current device's context (so a context that was
 * destroyed and created again is followed); a call made while its stream is
 * being captured uses the address the last uncaptured call on that device
 * found, so make one uncaptured call on each device before any capture. */
#define GS_NOALLOC_MAX_BLOCKS 1024
#define GS_NOALLOC_POSE_FLOATS (GS_MAX_VIEWS * GS_NOALLOC_MAX_BLOCKS * 12)
int gs_project_bwd_noalloc(const gs_gaussians *g, const gs_views *views, const gs_config *cfg, const float *proj,
                           const float *grad2d, const gs_grads *grads, int want_gaussian_grads,
                           float *dL_dviewmat, float *dL_dtwist, int32_t *status, void *stream);

/* Check of the device-side failure path: enqueues one thread that arms a
 * copy barrier (PTX mbarrier with 16 transaction bytes) for a copy that is
 * never issued and waits on it with the same bounded wait the projection
 * kernels use. The wait gives up after about one second and the thread sets
 * status = {GS_ERR_TIMEOUT, 0} (DEVICE int32[4]; the caller zeroes it before
 * the call and reads it after synchronising); nothing faults or traps, and
 * the context stays usable. Returns GS_ERR_ARG for a NULL status. */
int gs_check_bounded_wait(int32_t *status, void *stream);

/* Spatial (Morton) codes of the means (data layout; no result of the
 * rasterizer depends on the order of the Gaussians, for distinct depths).
 * A training loop that keeps its Gaussians sorted by these codes, refreshed
 * between densification steps, makes Gaussians that project near each other
 * neighbours in memory: binning writes longer runs per tile and the
 * projection backward's warps agree on which Gaussians carry a gradient.
 * codes DEVICE uint64 [n]: each coordinate of means (DEVICE [n,3]) quantised
 * to 21 bits in box (HOST float [6] = lo x, y, z, hi x, y, z) as
 * min(2^21 - 1, floor((m - lo) / (hi - lo) 2^21)) (0 below lo), bits
 * interleaved x0 y0 z0 x1 y1 z1 ...; a non-finite mean gets UINT64_MAX. */
int gs_spatial_codes(const float *means, int64_t n, const float *box, uint64_t *codes, void *stream);

/* Arithmetic-throughput probes (measurement only; the paper has no
 * counterpart): the raster kernels are bound by FP32 and special-function
 * issue rather than by memory, so their roofline needs these pipes' measured
 * rates. kind 0 = scalar FP32 fused multiply-add, 1 = packed f32x2 fused
 * multiply-add, 2 = ex2.approx. One launch of gs_probe_blocks() blocks of 256
 * threads, each thread running 8 independent chains of `iters` operations;
 * out: DEVICE float [gs_probe_blocks() * 256] (overwritten). The caller
 * times the launch: operations = blocks x 256 x 8 x iters (x 2 for kind 1;
 * an FMA is 2 FLOPs). */
int gs_probe_blocks(void);
int gs_peak_probe(int kind, int iters, float *out, void *stream);

const char *gs_error_string(int code);
int gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
