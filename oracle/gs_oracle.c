/*
 * gs_oracle.c -- plain, slow FP64 reference of the differentiable 3D Gaussian
 * Splatting rasterizer with camera-pose gradients.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links or calls this
 * file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do. It shares no code, header, table or constant with the CUDA
 * library.
 *
 * What it computes (paper: Section 3.1 "Preliminary" for the primitive and
 * alpha blending; Section 3.4 for the per-view pose residuals whose gradient
 * is needed; the EWA splatting formula and the compositing thresholds are the
 * readings listed with the design notes):
 *
 *   Gaussian i: mean mu, log-scale l (s = exp l), quaternion q (normalised),
 *   opacity logit (o = sigmoid), SH coefficients f[k][ch], k < (d+1)^2.
 *   Sigma = R(q) S S^T R(q)^T, S = diag(s).
 *   View v (world->camera R_v, t_v, pinhole fx, fy, cx, cy):
 *     m = R_v mu + t_v; culled if m_z <= near.
 *     J = [[fx/z, 0, -fx u/z], [0, fy/z, -fy w/z]], u = clamp(x/z), w = clamp(y/z)
 *         to +-1.3 tan(half field of view) (J only).
 *     Sigma' = J R_v Sigma R_v^T J^T + dilation I.
 *     conic = inverse(Sigma'), radius = ceil(3 sqrt(lambda_max)) with the
 *     eigenvalue floor max(0.1, mid^2 - det) under the root.
 *     mean2D = (fx x/z + cx, fy y/z + cy); pixel (u,v) has centre (u+.5, v+.5).
 *     colour = max(0, sum_k f_k Y_k(dir) + 0.5), dir = normalise(mu - C_v),
 *     C_v = -R_v^T t_v, real SH with the Condon-Shortley phase.
 *   A Gaussian of opacity o can give alpha >= alpha_min only inside the
 *   ellipse d^T conic d <= k, k = 2 ln(o / alpha_min) (culled if k <= 0);
 *   the half-extents of that ellipse's bounding box, min(radius,
 *   sqrt(k Sigma'_xx)) and min(radius, sqrt(k Sigma'_yy)), bound the tiles
 *   it can touch. Binning is done in float32 (bit-exact contract with the
 *   GPU) from those extents, sorting by (float32 depth, index). Compositing per pixel, front to back, over the
 *   Gaussians whose tile rectangle holds the pixel's tile and whose square
 *   |dx|,|dy| <= radius holds the pixel centre:
 *     alpha = min(alpha_max, o exp(-1/2 d^T conic d)); skipped if the
 *     exponent is > 0 or alpha < alpha_min; the Gaussian that would bring
 *     T (1 - alpha) below t_min is not composited and the pixel stops.
 *     C = sum c_i alpha_i T_i + T_final bg.
 *   Backward: exact chain rule of all of the above, in FP64, including the
 *   view's rotation and translation.
 */
#define _USE_MATH_DEFINES
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double near_z;     /* cull if camera z <= near_z */
    double dilation;   /* added to the 2D covariance diagonal */
    double alpha_min;  /* drop alpha below this */
    double alpha_max;  /* clamp alpha to this */
    double t_min;      /* stop when transmittance would fall below this */
    double fov_clamp;  /* tangent clamp factor for J */
    double bg[3];      /* background colour */
    int pixel_gate;    /* 1: also require |dx|,|dy| <= radius per pixel */
    /* margins used to flag pixels whose FP32 result may legitimately differ */
    double eps_gate;   /* pixels */
    double eps_alpha;  /* relative */
    double eps_t;      /* relative */
    double eps_depth;  /* relative */
    double eps_clamp;  /* relative */
} or_params;

typedef struct {
    double R[9];       /* world->camera rotation, row-major */
    double t[3];
    double fx, fy, cx, cy;
    int W, H;
} or_cam;

/* pixel flag bits */
enum {
    OR_FLAG_GATE = 1,    /* a pixel centre within eps of a gate edge */
    OR_FLAG_ALPHA = 2,   /* some o*G within eps of alpha_min */
    OR_FLAG_T = 4,       /* T (1 - alpha) within eps of t_min */
    OR_FLAG_DEPTH = 8,   /* two composited depths within eps */
    OR_FLAG_CLAMP = 16,  /* some o*G within eps of alpha_max (gradient only) */
    OR_FLAG_RADIUS = 32  /* a Gaussian whose 3 sqrt(lambda) sits within eps of an integer */
};

/* ------------------------------------------------------------------------ */
/* real spherical harmonics, degree <= 3, derived from the Legendre          */
/* polynomials: Y_lm = K_lm (-1)^m P_l^(m)(z) Re/Im((x+iy)^|m|)              */
/* K_l0 = sqrt((2l+1)/(4 pi)), K_lm = sqrt(2) sqrt((2l+1)/(4 pi)             */
/*        (l-|m|)!/(l+|m|)!); cos-type (Re) for m > 0, sin-type (Im) m < 0.  */
/* ------------------------------------------------------------------------ */

static double factorial(int k)
{
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
}

/* coefficients of P_l(z) = sum_k c[k] z^k, via Bonnet's recursion
 * (l+1) P_{l+1} = (2l+1) z P_l - l P_{l-1}. */
static void legendre_poly(int l, double c[8])
{
    double p0[8] = {1}, p1[8] = {0, 1}, p2[8];
    memset(c, 0, 8 * sizeof(double));
    if (l == 0) { c[0] = 1; return; }
    for (int n = 1; n < l; ++n) {
        memset(p2, 0, sizeof p2);
        for (int k = 0; k < 7; ++k) p2[k + 1] += (2.0 * n + 1.0) * p1[k] / (n + 1.0);
        for (int k = 0; k < 8; ++k) p2[k] -= n * p0[k] / (n + 1.0);
        memcpy(p0, p1, sizeof p0);
        memcpy(p1, p2, sizeof p1);
    }
    memcpy(c, p1, sizeof p1);
}

/* m-th derivative of sum c[k] z^k, evaluated at z */
static double poly_deriv(const double c[8], int m, double z)
{
    double r = 0.0;
    for (int k = m; k < 8; ++k) {
        if (c[k] == 0.0) continue;
        r += c[k] * factorial(k) / factorial(k - m) * pow(z, k - m);
    }
    return r;
}

/* Y[k], k = l*l + l + m, and dY[k*3 + j] = dY_k / dd_j of the polynomial
 * form above (any extension off the sphere gives the same gradient once the
 * direction normalisation is applied). */
void or_sh_basis(int degree, const double *d, double *Y, double *dY)
{
    double x = d[0], y = d[1], z = d[2];
    /* re[m] + i im[m] = (x + i y)^m */
    double re[5], im[5];
    re[0] = 1.0; im[0] = 0.0;
    for (int m = 1; m < 5; ++m) {
        re[m] = re[m - 1] * x - im[m - 1] * y;
        im[m] = re[m - 1] * y + im[m - 1] * x;
    }
    for (int l = 0; l <= degree; ++l) {
        double c[8];
        legendre_poly(l, c);
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            if (am) K *= sqrt(2.0);
            double sgn = (am % 2) ? -1.0 : 1.0;
            double P = poly_deriv(c, am, z), dP = poly_deriv(c, am + 1, z);
            double F, dFx, dFy;
            if (m > 0) {
                F = re[am];
                dFx = am * re[am - 1];
                dFy = -am * im[am - 1];
            } else if (m < 0) {
                F = im[am];
                dFx = am * im[am - 1];
                dFy = am * re[am - 1];
            } else {
                F = 1.0; dFx = 0.0; dFy = 0.0;
            }
            int k = l * l + l + m;
            Y[k] = K * sgn * P * F;
            if (dY) {
                dY[k * 3 + 0] = K * sgn * P * dFx;
                dY[k * 3 + 1] = K * sgn * P * dFy;
                dY[k * 3 + 2] = K * sgn * dP * F;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* small linear algebra                                                     */
/* ------------------------------------------------------------------------ */

/* rotation of the unit quaternion q = (w, x, y, z) */
static void quat_to_rot(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* g_q[j] = sum_ab G[a][b] dR[a][b]/dq_j for the map above */
static void quat_to_rot_vjp(const double *q, const double *G, double *gq)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    const double dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const double dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const double dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const double dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int k = 0; k < 9; ++k) {
        s0 += G[k] * dw[k]; s1 += G[k] * dx[k]; s2 += G[k] * dy[k]; s3 += G[k] * dz[k];
    }
    gq[0] = s0; gq[1] = s1; gq[2] = s2; gq[3] = s3;
}

/* ------------------------------------------------------------------------ */
/* projection of one Gaussian into one view                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int valid;
    double mc[3];
    double px, py, depth;
    double s[3], qn[4], qlen, Rq[9], M[9], Sig[9];
    double u, w; int u_in, w_in;
    double J[6], T[6], cov[3], det, conic[3], lam, r_real, ext[2];
    int radius;
    double o;
    double dir[3], dlen, d[3], Y[16], dY[48];
    double rgb_raw[3], rgb[3];
    int clamped[3];
} or_fwd;

static int finite3(const double *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

static void project_one(const double *mean, const double *ls, const double *quat, double logit,
                        const double *sh, int deg, const or_cam *cam, const or_params *P, or_fwd *f)
{
    memset(f, 0, sizeof *f);
    if (!finite3(mean) || !finite3(ls) || !isfinite(quat[0]) || !finite3(quat + 1) || !isfinite(logit))
        return;
    const double *R = cam->R;
    for (int a = 0; a < 3; ++a)
        f->mc[a] = R[3 * a] * mean[0] + R[3 * a + 1] * mean[1] + R[3 * a + 2] * mean[2] + cam->t[a];
    double x = f->mc[0], y = f->mc[1], z = f->mc[2];
    if (!(z > P->near_z)) return;

    /* Sigma = Rq diag(s^2) Rq^T */
    for (int a = 0; a < 3; ++a) f->s[a] = exp(ls[a]);
    f->qlen = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    if (!(f->qlen > 0)) return;
    for (int a = 0; a < 4; ++a) f->qn[a] = quat[a] / f->qlen;
    quat_to_rot(f->qn, f->Rq);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) f->M[3 * a + b] = f->Rq[3 * a + b] * f->s[b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += f->M[3 * a + k] * f->M[3 * b + k];
            f->Sig[3 * a + b] = acc;
        }

    /* Jacobian of the perspective map with the tangent clamp */
    double limx = P->fov_clamp * (0.5 * cam->W / cam->fx);
    double limy = P->fov_clamp * (0.5 * cam->H / cam->fy);
    f->u = x / z; f->u_in = 1;
    if (f->u < -limx) { f->u = -limx; f->u_in = 0; }
    if (f->u > limx) { f->u = limx; f->u_in = 0; }
    f->w = y / z; f->w_in = 1;
    if (f->w < -limy) { f->w = -limy; f->w_in = 0; }
    if (f->w > limy) { f->w = limy; f->w_in = 0; }
    f->J[0] = cam->fx / z; f->J[1] = 0; f->J[2] = -cam->fx * f->u / z;
    f->J[3] = 0; f->J[4] = cam->fy / z; f->J[5] = -cam->fy * f->w / z;
    /* T = J R_v (2x3) */
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += f->J[3 * a + k] * R[3 * k + b];
            f->T[3 * a + b] = acc;
        }
    /* Sigma' = T Sigma T^T */
    double TS[6];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += f->T[3 * a + k] * f->Sig[3 * k + b];
            TS[3 * a + b] = acc;
        }
    double s00 = 0, s01 = 0, s11 = 0;
    for (int k = 0; k < 3; ++k) {
        s00 += TS[k] * f->T[k];
        s01 += TS[k] * f->T[3 + k];
        s11 += TS[3 + k] * f->T[3 + k];
    }
    f->cov[0] = s00 + P->dilation;
    f->cov[1] = s01;
    f->cov[2] = s11 + P->dilation;
    f->det = f->cov[0] * f->cov[2] - f->cov[1] * f->cov[1];
    if (!(f->det > 0)) return;
    f->conic[0] = f->cov[2] / f->det;
    f->conic[1] = -f->cov[1] / f->det;
    f->conic[2] = f->cov[0] / f->det;
    double mid = 0.5 * (f->cov[0] + f->cov[2]);
    double disc = mid * mid - f->det;
    if (disc < 0.1) disc = 0.1;
    f->lam = mid + sqrt(disc);
    f->r_real = 3.0 * sqrt(f->lam);
    f->radius = (int)ceil(f->r_real);

    f->px = cam->fx * x / z + cam->cx;
    f->py = cam->fy * y / z + cam->cy;
    f->depth = z;
    double r = f->radius;
    /* off-screen cull (independent of the tile size): the square of half-side
     * r around the mean misses the image rectangle [0,W]x[0,H] */
    if (f->px + r < 0 || f->px - r > cam->W || f->py + r < 0 || f->py - r > cam->H) return;

    f->o = 1.0 / (1.0 + exp(-logit));
    /* bounding box of the region where alpha can reach alpha_min */
    double k = 2.0 * log(f->o / P->alpha_min);
    if (!(k > 0)) return;
    f->ext[0] = fmin(r, sqrt(k * f->cov[0]));
    f->ext[1] = fmin(r, sqrt(k * f->cov[2]));

    /* view-dependent colour */
    double C[3];
    for (int b = 0; b < 3; ++b) C[b] = -(R[b] * cam->t[0] + R[3 + b] * cam->t[1] + R[6 + b] * cam->t[2]);
    for (int a = 0; a < 3; ++a) f->dir[a] = mean[a] - C[a];
    f->dlen = sqrt(f->dir[0] * f->dir[0] + f->dir[1] * f->dir[1] + f->dir[2] * f->dir[2]);
    for (int a = 0; a < 3; ++a) f->d[a] = f->dir[a] / f->dlen;
    int K = (deg + 1) * (deg + 1);
    or_sh_basis(deg, f->d, f->Y, f->dY);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += sh[3 * k + ch] * f->Y[k];
        f->rgb_raw[ch] = acc;
        f->clamped[ch] = acc < 0;
        f->rgb[ch] = acc < 0 ? 0.0 : acc;
    }
    if (!isfinite(f->px) || !isfinite(f->py) || !finite3(f->conic) || !finite3(f->rgb)) return;
    f->valid = 1;
}

/* Project n Gaussians (FP64 inputs) into one view. Outputs per Gaussian:
 * xy[2], depth, conic[3], cov[3] (dilated), opacity, rgb[3], radius (0 =
 * culled), r_real = 3 sqrt(lambda_max), clamped[3], ext[2] (tile extents). */
void or_project(int64_t n, int deg, const double *means, const double *log_scales, const double *quats,
                const double *logits, const double *sh, const or_cam *cam, const or_params *P,
                double *xy, double *depth, double *conic, double *cov, double *opac, double *rgb,
                int32_t *radius, double *r_real, int32_t *clamped, double *ext)
{
    int K = (deg + 1) * (deg + 1);
    for (int64_t i = 0; i < n; ++i) {
        or_fwd f;
        project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i], sh + 3 * K * i, deg, cam, P, &f);
        xy[2 * i] = f.px; xy[2 * i + 1] = f.py; depth[i] = f.depth;
        for (int a = 0; a < 3; ++a) {
            conic[3 * i + a] = f.conic[a];
            cov[3 * i + a] = f.cov[a];
            rgb[3 * i + a] = f.rgb[a];
            clamped[3 * i + a] = f.clamped[a];
        }
        opac[i] = f.o;
        ext[2 * i] = f.valid ? f.ext[0] : 0.0;
        ext[2 * i + 1] = f.valid ? f.ext[1] : 0.0;
        radius[i] = f.valid ? f.radius : 0;
        r_real[i] = f.valid ? f.r_real : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* binning in float32                                                       */
/* ------------------------------------------------------------------------ */

static void rect_f32(float x, float y, float ex, float ey, int TW, int TH, int Gx, int Gy,
                     int *x0, int *x1, int *y0, int *y1)
{
    float tw = (float)TW, th = (float)TH;
    float a0 = floorf((x - ex) / tw), a1 = floorf((x + ex) / tw) + 1.0f;
    float b0 = floorf((y - ey) / th), b1 = floorf((y + ey) / th) + 1.0f;
    a0 = a0 < 0.0f ? 0.0f : (a0 > (float)Gx ? (float)Gx : a0);
    a1 = a1 < 0.0f ? 0.0f : (a1 > (float)Gx ? (float)Gx : a1);
    b0 = b0 < 0.0f ? 0.0f : (b0 > (float)Gy ? (float)Gy : b0);
    b1 = b1 < 0.0f ? 0.0f : (b1 > (float)Gy ? (float)Gy : b1);
    *x0 = (int)a0; *x1 = (int)a1; *y0 = (int)b0; *y1 = (int)b1;
}

/* Count tile instances of n projected Gaussians of one view. r == 0 means
 * culled; ext[2i], ext[2i+1] are the half-extents of the tile rectangle.
 * Writes counts[Gx*Gy] (tile id ty*Gx + tx); returns the total. */
int64_t or_bin_count(int64_t n, const float *x, const float *y, const int32_t *r, const float *ext, int W, int H,
                     int TW, int TH, int32_t *counts)
{
    int Gx = (W + TW - 1) / TW, Gy = (H + TH - 1) / TH;
    memset(counts, 0, sizeof(int32_t) * (size_t)Gx * Gy);
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (r[i] <= 0) continue;
        int x0, x1, y0, y1;
        rect_f32(x[i], y[i], ext[2 * i], ext[2 * i + 1], TW, TH, Gx, Gy, &x0, &x1, &y0, &y1);
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) { counts[ty * Gx + tx]++; total++; }
    }
    return total;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Fill the per-tile lists: ranges[2*tile] = [start, end) in tile-id order,
 * keys[j] = (float32 bits of depth << 32) | index, ascending within a tile,
 * ids[j] = index. Arrays must hold the total from or_bin_count. */
void or_bin_fill(int64_t n, const float *x, const float *y, const int32_t *r, const float *ext,
                 const float *depth, int W, int H, int TW, int TH, int64_t *ranges, uint64_t *keys, int32_t *ids)
{
    int Gx = (W + TW - 1) / TW, Gy = (H + TH - 1) / TH;
    int64_t G = (int64_t)Gx * Gy;
    int32_t *counts = (int32_t *)calloc((size_t)G, sizeof(int32_t));
    int64_t *fill = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    or_bin_count(n, x, y, r, ext, W, H, TW, TH, counts);
    int64_t acc = 0;
    for (int64_t t = 0; t < G; ++t) {
        ranges[2 * t] = acc;
        acc += counts[t];
        ranges[2 * t + 1] = acc;
        fill[t] = ranges[2 * t];
    }
    for (int64_t i = 0; i < n; ++i) {
        if (r[i] <= 0) continue;
        int x0, x1, y0, y1;
        rect_f32(x[i], y[i], ext[2 * i], ext[2 * i + 1], TW, TH, Gx, Gy, &x0, &x1, &y0, &y1);
        uint32_t bits;
        memcpy(&bits, &depth[i], 4);
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) {
                int64_t t = (int64_t)ty * Gx + tx;
                keys[fill[t]++] = ((uint64_t)bits << 32) | (uint32_t)i;
            }
    }
    for (int64_t t = 0; t < G; ++t) {
        int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
        qsort(keys + s, (size_t)(e - s), sizeof(uint64_t), cmp_u64);
        for (int64_t j = s; j < e; ++j) ids[j] = (int32_t)(keys[j] & 0xffffffffu);
    }
    free(counts);
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* compositing                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t id;
    double alpha, G, T, dx, dy;
    int clamped;
} or_hit;

/* Walk one pixel's list front to back. Returns the number of composited
 * Gaussians written to hits (capacity cap); *T_out = final transmittance,
 * C[3] the colour without background, *flags the margin bits. */
static int composite_pixel(int px, int py, int64_t s, int64_t e, const int32_t *ids, const double *xy,
                           const double *conic, const double *opac, const double *rgb, const int32_t *radius,
                           const double *r_real, const double *depth, const or_params *P,
                           or_hit *hits, double *C, double *T_out, int *flags)
{
    double pcx = px + 0.5, pcy = py + 0.5;
    double T = 1.0;
    int nh = 0;
    double last_depth = -1.0;
    C[0] = C[1] = C[2] = 0.0;
    *flags = 0;
    for (int64_t j = s; j < e; ++j) {
        int32_t g = ids[j];
        double dx = pcx - xy[2 * g], dy = pcy - xy[2 * g + 1];
        double r = radius[g];
        double adx = fabs(dx), ady = fabs(dy);
        if (r_real) {
            /* a float32 radius may round to the neighbouring integer: flag the
             * pixels whose gate would flip with r - 1 or r + 1 */
            double fr = r_real[g] - floor(r_real[g]);
            double dmax = adx > ady ? adx : ady;
            if ((fr < P->eps_gate || fr > 1.0 - P->eps_gate) && dmax > r - 1.0 && dmax <= r + 1.0)
                *flags |= OR_FLAG_RADIUS;
        }
        if (P->pixel_gate) {
            if ((fabs(adx - r) < P->eps_gate && ady <= r + P->eps_gate) ||
                (fabs(ady - r) < P->eps_gate && adx <= r + P->eps_gate)) *flags |= OR_FLAG_GATE;
            if (adx > r || ady > r) continue;
        }
        double A = conic[3 * g], B = conic[3 * g + 1], Cc = conic[3 * g + 2];
        double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
        if (power > 0) continue;
        double G = exp(power);
        double oG = opac[g] * G;
        if (fabs(oG - P->alpha_min) < P->eps_alpha * P->alpha_min) *flags |= OR_FLAG_ALPHA;
        if (fabs(oG - P->alpha_max) < P->eps_clamp * P->alpha_max) *flags |= OR_FLAG_CLAMP;
        int clamped = oG > P->alpha_max;
        double alpha = clamped ? P->alpha_max : oG;
        if (alpha < P->alpha_min) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - P->t_min) < P->eps_t * P->t_min) *flags |= OR_FLAG_T;
        if (Tn < P->t_min) break;
        if (last_depth >= 0 && fabs(depth[g] - last_depth) <= P->eps_depth * depth[g]) *flags |= OR_FLAG_DEPTH;
        last_depth = depth[g];
        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
        if (hits) {
            hits[nh].id = g; hits[nh].alpha = alpha; hits[nh].G = G; hits[nh].T = T;
            hits[nh].dx = dx; hits[nh].dy = dy; hits[nh].clamped = clamped;
        }
        nh++;
        T = Tn;
    }
    *T_out = T;
    return nh;
}

/* Render one view. Tile lists (ranges over tiles ty*Gx+tx, ids) come from
 * or_bin_fill (possibly built with enlarged radii so that every Gaussian a
 * float32 computation might list is present; the gate below uses radius).
 * img is [3,H,W]; T_final, n_contrib and flags are [H,W]. If mask is not
 * NULL, only pixels with mask[py*W+px] != 0 are computed. */
void or_render(const double *xy, const double *conic, const double *opac, const double *rgb,
               const int32_t *radius, const double *r_real, const double *depth,
               int W, int H, int TW, int TH, const int64_t *ranges, const int32_t *ids,
               const or_params *P, const uint8_t *mask, double *img, double *T_final, int32_t *n_contrib,
               int32_t *flags)
{
    int Gx = (W + TW - 1) / TW;
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            if (mask && !mask[(int64_t)py * W + px]) continue;
            int64_t t = (int64_t)(py / TH) * Gx + px / TW;
            double C[3], T;
            int fl;
            int nh = composite_pixel(px, py, ranges[2 * t], ranges[2 * t + 1], ids, xy, conic, opac, rgb,
                                     radius, r_real, depth, P, NULL, C, &T, &fl);
            int64_t p = (int64_t)py * W + px;
            for (int ch = 0; ch < 3; ++ch) img[(int64_t)ch * W * H + p] = C[ch] + T * P->bg[ch];
            T_final[p] = T;
            n_contrib[p] = nh;
            flags[p] = fl;
        }
}

/* Backward of or_render for upstream dL/dimg [3,H,W]. Accumulates into
 * g2d[n,9] = dL/d(x, y, A, B, C, opacity, r, g, b) per Gaussian. Pixels with
 * dL/dimg == 0 in all channels are skipped. */
void or_render_bwd(int64_t n, const double *xy, const double *conic, const double *opac, const double *rgb,
                   const int32_t *radius, const double *depth, int W, int H, int TW, int TH,
                   const int64_t *ranges, const int32_t *ids, const or_params *P,
                   const double *dL_dimg, double *g2d)
{
    int Gx = (W + TW - 1) / TW;
    int64_t cap = 0;
    for (int64_t t = 0; t < (int64_t)Gx * ((H + TH - 1) / TH); ++t) {
        int64_t len = ranges[2 * t + 1] - ranges[2 * t];
        if (len > cap) cap = len;
    }
    or_hit *hits = (or_hit *)malloc(sizeof(or_hit) * (size_t)(cap > 0 ? cap : 1));
    (void)n;
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int64_t p = (int64_t)py * W + px;
            double g[3];
            for (int ch = 0; ch < 3; ++ch) g[ch] = dL_dimg[(int64_t)ch * W * H + p];
            if (g[0] == 0 && g[1] == 0 && g[2] == 0) continue;
            int64_t t = (int64_t)(py / TH) * Gx + px / TW;
            double C[3], T_final;
            int fl;
            int nh = composite_pixel(px, py, ranges[2 * t], ranges[2 * t + 1], ids, xy, conic, opac, rgb,
                                     radius, NULL, depth, P, hits, C, &T_final, &fl);
            /* S = sum over later Gaussians of c alpha T, plus T_final bg */
            double S[3];
            for (int ch = 0; ch < 3; ++ch) S[ch] = T_final * P->bg[ch];
            for (int k = nh - 1; k >= 0; --k) {
                const or_hit *h = &hits[k];
                int gi = h->id;
                const double *c = rgb + 3 * gi;
                double dL_dalpha = 0;
                for (int ch = 0; ch < 3; ++ch) {
                    g2d[9 * gi + 6 + ch] += h->alpha * h->T * g[ch];
                    dL_dalpha += g[ch] * (c[ch] * h->T - S[ch] / (1.0 - h->alpha));
                }
                for (int ch = 0; ch < 3; ++ch) S[ch] += c[ch] * h->alpha * h->T;
                if (h->clamped) continue;
                double o = opac[gi];
                double A = conic[3 * gi], B = conic[3 * gi + 1], Cc = conic[3 * gi + 2];
                g2d[9 * gi + 5] += dL_dalpha * h->G;
                double dL_dpow = dL_dalpha * o * h->G;
                /* power = -1/2 (A dx^2 + 2 B dx dy + C dy^2), dx = pc - x */
                g2d[9 * gi + 0] += dL_dpow * (A * h->dx + B * h->dy);
                g2d[9 * gi + 1] += dL_dpow * (B * h->dx + Cc * h->dy);
                g2d[9 * gi + 2] += dL_dpow * (-0.5 * h->dx * h->dx);
                g2d[9 * gi + 3] += dL_dpow * (-h->dx * h->dy);
                g2d[9 * gi + 4] += dL_dpow * (-0.5 * h->dy * h->dy);
            }
        }
    free(hits);
}

/* ------------------------------------------------------------------------ */
/* projection backward                                                      */
/* ------------------------------------------------------------------------ */

/* Chain g2d[n,9] (w.r.t. x, y, A, B, C, opacity, r, g, b) of one view to the
 * raw parameters (accumulated into g_means[n,3], g_log_scales[n,3],
 * g_quats[n,4], g_logits[n], g_sh[n,K,3]) and to the view's rotation and
 * translation (accumulated into gR[9], gt[3]). */
void or_project_bwd(int64_t n, int deg, const double *means, const double *log_scales, const double *quats,
                    const double *logits, const double *sh, const or_cam *cam, const or_params *P,
                    const double *g2d, double *g_means, double *g_log_scales, double *g_quats,
                    double *g_logits, double *g_sh, double *gR, double *gt)
{
    int K = (deg + 1) * (deg + 1);
    const double *R = cam->R;
    for (int64_t i = 0; i < n; ++i) {
        const double *g = g2d + 9 * i;
        int any = 0;
        for (int a = 0; a < 9; ++a) any |= g[a] != 0.0;
        if (!any) continue;
        or_fwd f;
        const double *shi = sh + 3 * K * i;
        project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i], shi, deg, cam, P, &f);
        if (!f.valid) continue;
        double x = f.mc[0], y = f.mc[1], z = f.mc[2];
        double gmc[3] = {0, 0, 0};
        double *gm = g_means + 3 * i;

        /* opacity */
        g_logits[i] += g[5] * f.o * (1.0 - f.o);

        /* colour -> SH coefficients and view direction */
        double graw[3], gY[16] = {0}, gd[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) graw[ch] = f.clamped[ch] ? 0.0 : g[6 + ch];
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) {
                g_sh[3 * K * i + 3 * k + ch] += f.Y[k] * graw[ch];
                gY[k] += shi[3 * k + ch] * graw[ch];
            }
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < 3; ++j) gd[j] += gY[k] * f.dY[3 * k + j];
        double dgd = f.d[0] * gd[0] + f.d[1] * gd[1] + f.d[2] * gd[2];
        double gdir[3], gC[3];
        for (int a = 0; a < 3; ++a) {
            gdir[a] = (gd[a] - f.d[a] * dgd) / f.dlen;
            gm[a] += gdir[a];
            gC[a] = -gdir[a];
        }
        /* C = -R^T t */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                gR[3 * a + b] += -cam->t[a] * gC[b];
                gt[a] += -R[3 * a + b] * gC[b];
            }

        /* conic -> dilated covariance (a, b, c); b is the off-diagonal value */
        double a = f.cov[0], b = f.cov[1], c = f.cov[2], det2 = f.det * f.det;
        double gA = g[2], gB = g[3], gCc = g[4];
        double ga = (-c * c * gA + b * c * gB - b * b * gCc) / det2;
        double gb = (2 * b * c * gA - (a * c + b * b) * gB + 2 * a * b * gCc) / det2;
        double gc = (-b * b * gA + a * b * gB - a * a * gCc) / det2;
        /* Sigma' = T Sigma T^T, full-matrix gradient Gp (symmetric) */
        double Gp[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
        double GT[6], GS[9], TS[6];
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += f.T[3 * r + k] * f.Sig[3 * k + cc];
                TS[3 * r + cc] = acc;
            }
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 3; ++cc)
                GT[3 * r + cc] = 2.0 * (Gp[2 * r] * TS[cc] + Gp[2 * r + 1] * TS[3 + cc]);
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double acc = 0;
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) acc += f.T[3 * p + r] * Gp[2 * p + q] * f.T[3 * q + cc];
                GS[3 * r + cc] = acc;
            }
        /* T = J R_v */
        double GJ[6];
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += GT[3 * r + k] * R[3 * cc + k];
                GJ[3 * r + cc] = acc;
            }
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc)
                gR[3 * r + cc] += f.J[r] * GT[cc] + f.J[3 + r] * GT[3 + cc];
        /* J entries */
        double fx = cam->fx, fy = cam->fy, z2 = z * z;
        gmc[2] += GJ[0] * (-fx / z2) + GJ[2] * (fx * f.u / z2) + GJ[4] * (-fy / z2) + GJ[5] * (fy * f.w / z2);
        double gu = GJ[2] * (-fx / z), gw = GJ[5] * (-fy / z);
        if (f.u_in) { gmc[0] += gu / z; gmc[2] += -gu * x / z2; }
        if (f.w_in) { gmc[1] += gw / z; gmc[2] += -gw * y / z2; }
        /* mean2D */
        gmc[0] += g[0] * fx / z;
        gmc[2] += -g[0] * fx * x / z2;
        gmc[1] += g[1] * fy / z;
        gmc[2] += -g[1] * fy * y / z2;
        /* camera-space mean m = R_v mu + t_v */
        for (int r = 0; r < 3; ++r) {
            gt[r] += gmc[r];
            for (int cc = 0; cc < 3; ++cc) {
                gm[cc] += R[3 * r + cc] * gmc[r];
                gR[3 * r + cc] += gmc[r] * means[3 * i + cc];
            }
        }
        /* Sigma = M M^T, M = Rq diag(s) */
        double GM[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += (GS[3 * r + k] + GS[3 * k + r]) * f.M[3 * k + cc];
                GM[3 * r + cc] = acc;
            }
        double GRq[9];
        for (int cc = 0; cc < 3; ++cc) {
            double gs = 0;
            for (int r = 0; r < 3; ++r) {
                gs += GM[3 * r + cc] * f.Rq[3 * r + cc];
                GRq[3 * r + cc] = GM[3 * r + cc] * f.s[cc];
            }
            g_log_scales[3 * i + cc] += gs * f.s[cc];
        }
        double gqn[4];
        quat_to_rot_vjp(f.qn, GRq, gqn);
        double dq = gqn[0] * f.qn[0] + gqn[1] * f.qn[1] + gqn[2] * f.qn[2] + gqn[3] * f.qn[3];
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] += (gqn[k] - f.qn[k] * dq) / f.qlen;
    }
}

/* Gradient w.r.t. a left twist xi = (rho, phi) of the pose, T <- exp(xi^) T:
 * M = dL/dR R^T + dL/dt t^T; dL/dphi = (M32 - M23, M13 - M31, M21 - M12),
 * dL/drho = dL/dt. */
void or_pose_twist(const double *R, const double *t, const double *gR, const double *gt, double *twist)
{
    double M[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = gt[a] * t[b];
            for (int k = 0; k < 3; ++k) acc += gR[3 * a + k] * R[3 * b + k];
            M[3 * a + b] = acc;
        }
    twist[0] = gt[0]; twist[1] = gt[1]; twist[2] = gt[2];
    twist[3] = M[7] - M[5];
    twist[4] = M[2] - M[6];
    twist[5] = M[3] - M[1];
}

/* ------------------------------------------------------------------------ */
/* Threaded variants, for timing the oracle on all host cores (the tests    */
/* check them against the single-threaded functions above): the same       */
/* per-Gaussian or per-pixel work split over threads -- Gaussians in        */
/* contiguous chunks, pixels by interleaved rows of tiles -- with partial   */
/* sums combined in thread order.                                          */
/* ------------------------------------------------------------------------ */
#include <pthread.h>

#define OR_MAX_THREADS 256

typedef struct {
    int tid, nth;
    int64_t n;
    int deg;
    const double *means, *log_scales, *quats, *logits, *sh;
    const or_cam *cam;
    const or_params *P;
    /* projection outputs */
    double *xy, *depth, *conic, *cov, *opac, *rgb, *r_real, *ext;
    int32_t *radius, *clamped;
    /* projection backward */
    const double *g2d;
    double *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh, gR[9], gt[3];
    /* rendering */
    const double *cxy, *cconic, *copac, *crgb, *cr_real, *cdepth;
    const int32_t *cradius, *ids;
    const int64_t *ranges;
    int W, H, TW, TH;
    const uint8_t *mask;
    double *img, *T_final;
    int32_t *n_contrib, *flags;
    const double *dL_dimg;
    double *g2d_out;
} or_job;

static void chunk(int64_t n, int tid, int nth, int64_t *b, int64_t *e)
{
    *b = n * tid / nth;
    *e = n * (tid + 1) / nth;
}

static void *project_worker(void *arg)
{
    or_job *j = (or_job *)arg;
    int K = (j->deg + 1) * (j->deg + 1);
    int64_t b, e;
    chunk(j->n, j->tid, j->nth, &b, &e);
    or_project(e - b, j->deg, j->means + 3 * b, j->log_scales + 3 * b, j->quats + 4 * b, j->logits + b,
               j->sh + 3 * K * b, j->cam, j->P, j->xy + 2 * b, j->depth + b, j->conic + 3 * b, j->cov + 3 * b,
               j->opac + b, j->rgb + 3 * b, j->radius + b, j->r_real + b, j->clamped + 3 * b, j->ext + 2 * b);
    return NULL;
}

static void *project_bwd_worker(void *arg)
{
    or_job *j = (or_job *)arg;
    int K = (j->deg + 1) * (j->deg + 1);
    int64_t b, e;
    chunk(j->n, j->tid, j->nth, &b, &e);
    for (int a = 0; a < 9; ++a) j->gR[a] = 0.0;
    for (int a = 0; a < 3; ++a) j->gt[a] = 0.0;
    or_project_bwd(e - b, j->deg, j->means + 3 * b, j->log_scales + 3 * b, j->quats + 4 * b, j->logits + b,
                   j->sh + 3 * K * b, j->cam, j->P, j->g2d + 9 * b, j->g_means + 3 * b, j->g_log_scales + 3 * b,
                   j->g_quats + 4 * b, j->g_logits + b, j->g_sh + 3 * K * b, j->gR, j->gt);
    return NULL;
}

static void *render_worker(void *arg)
{
    or_job *j = (or_job *)arg;
    int Gx = (j->W + j->TW - 1) / j->TW, Gy = (j->H + j->TH - 1) / j->TH;
    for (int ty = j->tid; ty < Gy; ty += j->nth)
        for (int py = ty * j->TH; py < (ty + 1) * j->TH && py < j->H; ++py)
            for (int px = 0; px < j->W; ++px) {
                if (j->mask && !j->mask[(int64_t)py * j->W + px]) continue;
                int64_t t = (int64_t)(py / j->TH) * Gx + px / j->TW;
                double C[3], T;
                int fl;
                int nh = composite_pixel(px, py, j->ranges[2 * t], j->ranges[2 * t + 1], j->ids, j->cxy, j->cconic,
                                         j->copac, j->crgb, j->cradius, j->cr_real, j->cdepth, j->P, NULL, C, &T,
                                         &fl);
                int64_t p = (int64_t)py * j->W + px;
                for (int ch = 0; ch < 3; ++ch) j->img[(int64_t)ch * j->W * j->H + p] = C[ch] + T * j->P->bg[ch];
                j->T_final[p] = T;
                j->n_contrib[p] = nh;
                j->flags[p] = fl;
            }
    return NULL;
}

/* one thread's pixels (interleaved rows of tiles) of or_render_bwd, into
 * its own g2d_out */
static void *render_bwd_worker(void *arg)
{
    or_job *j = (or_job *)arg;
    int Gx = (j->W + j->TW - 1) / j->TW, Gy = (j->H + j->TH - 1) / j->TH;
    /* a copy of the image gradient that is zero outside this thread's rows:
     * or_render_bwd skips pixels whose upstream gradient is zero */
    int64_t WH = (int64_t)j->W * j->H;
    double *up = (double *)calloc((size_t)(3 * WH), sizeof(double));
    if (!up) return (void *)1;
    for (int ty = j->tid; ty < Gy; ty += j->nth)
        for (int py = ty * j->TH; py < (ty + 1) * j->TH && py < j->H; ++py)
            for (int ch = 0; ch < 3; ++ch)
                memcpy(up + ch * WH + (int64_t)py * j->W, j->dL_dimg + ch * WH + (int64_t)py * j->W,
                       sizeof(double) * (size_t)j->W);
    (void)Gx;
    or_render_bwd(j->n, j->cxy, j->cconic, j->copac, j->crgb, j->cradius, j->cdepth, j->W, j->H, j->TW, j->TH,
                  j->ranges, j->ids, j->P, up, j->g2d_out);
    free(up);
    return NULL;
}

static int run_jobs(or_job *jobs, int nth, void *(*fn)(void *))
{
    pthread_t th[OR_MAX_THREADS];
    int started = 0, rc = 0;
    for (int t = 1; t < nth; ++t) {
        if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) break;
        started = t;
    }
    for (int t = started + 1; t < nth; ++t) fn(&jobs[t]);   /* threads that could not start run here */
    if (fn(&jobs[0])) rc = 1;
    for (int t = 1; t <= started; ++t) {
        void *r = NULL;
        pthread_join(th[t], &r);
        if (r) rc = 1;
    }
    return rc;
}

static int clamp_threads(int nth) { return nth < 1 ? 1 : (nth > OR_MAX_THREADS ? OR_MAX_THREADS : nth); }

void or_project_mt(int64_t n, int deg, const double *means, const double *log_scales, const double *quats,
                   const double *logits, const double *sh, const or_cam *cam, const or_params *P, double *xy,
                   double *depth, double *conic, double *cov, double *opac, double *rgb, int32_t *radius,
                   double *r_real, int32_t *clamped, double *ext, int nth)
{
    nth = clamp_threads(nth);
    or_job jobs[OR_MAX_THREADS];
    for (int t = 0; t < nth; ++t) {
        or_job *j = &jobs[t];
        memset(j, 0, sizeof *j);
        j->tid = t; j->nth = nth; j->n = n; j->deg = deg;
        j->means = means; j->log_scales = log_scales; j->quats = quats; j->logits = logits; j->sh = sh;
        j->cam = cam; j->P = P;
        j->xy = xy; j->depth = depth; j->conic = conic; j->cov = cov; j->opac = opac; j->rgb = rgb;
        j->radius = radius; j->r_real = r_real; j->clamped = clamped; j->ext = ext;
    }
    run_jobs(jobs, nth, project_worker);
}

void or_project_bwd_mt(int64_t n, int deg, const double *means, const double *log_scales, const double *quats,
                       const double *logits, const double *sh, const or_cam *cam, const or_params *P,
                       const double *g2d, double *g_means, double *g_log_scales, double *g_quats, double *g_logits,
                       double *g_sh, double *gR, double *gt, int nth)
{
    nth = clamp_threads(nth);
    or_job jobs[OR_MAX_THREADS];
    for (int t = 0; t < nth; ++t) {
        or_job *j = &jobs[t];
        memset(j, 0, sizeof *j);
        j->tid = t; j->nth = nth; j->n = n; j->deg = deg;
        j->means = means; j->log_scales = log_scales; j->quats = quats; j->logits = logits; j->sh = sh;
        j->cam = cam; j->P = P; j->g2d = g2d;
        j->g_means = g_means; j->g_log_scales = g_log_scales; j->g_quats = g_quats; j->g_logits = g_logits;
        j->g_sh = g_sh;
    }
    run_jobs(jobs, nth, project_bwd_worker);
    for (int t = 0; t < nth; ++t) {
        for (int a = 0; a < 9; ++a) gR[a] += jobs[t].gR[a];
        for (int a = 0; a < 3; ++a) gt[a] += jobs[t].gt[a];
    }
}

void or_render_mt(const double *xy, const double *conic, const double *opac, const double *rgb,
                  const int32_t *radius, const double *r_real, const double *depth, int W, int H, int TW, int TH,
                  const int64_t *ranges, const int32_t *ids, const or_params *P, const uint8_t *mask, double *img,
                  double *T_final, int32_t *n_contrib, int32_t *flags, int nth)
{
    nth = clamp_threads(nth);
    or_job jobs[OR_MAX_THREADS];
    for (int t = 0; t < nth; ++t) {
        or_job *j = &jobs[t];
        memset(j, 0, sizeof *j);
        j->tid = t; j->nth = nth; j->P = P;
        j->cxy = xy; j->cconic = conic; j->copac = opac; j->crgb = rgb; j->cradius = radius; j->cr_real = r_real;
        j->cdepth = depth; j->W = W; j->H = H; j->TW = TW; j->TH = TH; j->ranges = ranges; j->ids = ids;
        j->mask = mask; j->img = img; j->T_final = T_final; j->n_contrib = n_contrib; j->flags = flags;
    }
    run_jobs(jobs, nth, render_worker);
}

/* returns 0, or 1 if a thread could not allocate its scratch (g2d is then
 * incomplete) */
int or_render_bwd_mt(int64_t n, const double *xy, const double *conic, const double *opac, const double *rgb,
                     const int32_t *radius, const double *depth, int W, int H, int TW, int TH,
                     const int64_t *ranges, const int32_t *ids, const or_params *P, const double *dL_dimg,
                     double *g2d, int nth)
{
    nth = clamp_threads(nth);
    or_job jobs[OR_MAX_THREADS];
    double *part = (double *)calloc((size_t)nth * (size_t)(9 * (n > 0 ? n : 1)), sizeof(double));
    if (!part) return 1;
    for (int t = 0; t < nth; ++t) {
        or_job *j = &jobs[t];
        memset(j, 0, sizeof *j);
        j->tid = t; j->nth = nth; j->n = n; j->P = P;
        j->cxy = xy; j->cconic = conic; j->copac = opac; j->crgb = rgb; j->cradius = radius; j->cdepth = depth;
        j->W = W; j->H = H; j->TW = TW; j->TH = TH; j->ranges = ranges; j->ids = ids; j->dL_dimg = dL_dimg;
        j->g2d_out = part + (size_t)t * (size_t)(9 * n);
    }
    int rc = run_jobs(jobs, nth, render_bwd_worker);
    for (int t = 0; t < nth; ++t)
        for (int64_t k = 0; k < 9 * n; ++k) g2d[k] += part[(size_t)t * (size_t)(9 * n) + (size_t)k];
    free(part);
    return rc;
}
