// Internal definitions shared by the CUDA sources of libgsplat_gb300.
#pragma once

#include <cuda.h>   // CUtensorMap and its enums (types only: the encoder is fetched from the CUDA driver at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gsk {

// ---------------------------------------------------------------------------
// launch description, passed by value as a kernel parameter (views and scene
// groups of one call; host-built, so a captured graph bakes it in)
// ---------------------------------------------------------------------------
struct ViewDesc {
    int W, H, Gx, Gy;
    int tile_base;        // first global tile id of the view
    int g_count;          // Gaussians the view sees
    long long slot_base;  // first projected slot of the view
    long long g_begin;    // first Gaussian the view sees
    long long pix_base;   // float offset of the view's [3,H,W] image
};

struct SceneDesc {        // a run of views that see the same Gaussian range
    long long g_begin;
    long long thread_base;  // first thread of the group in a per-Gaussian grid
    int g_count;
    int v_begin, v_end;
};

struct Launch {
    int n_views, n_scenes;
    int tw, th;
    long long n_slots;      // P
    long long n_threads;    // sum of scene sizes (per-Gaussian grids)
    int n_tiles;            // T
    int pixel_gate;
    int count_pairs;        // the raster backward also counts pixel-Gaussian pairs
    int accumulate;         // the projection backward adds to the parameter gradients
    int use_tma;            // the projection kernels may stage through tensor copies
    int fwd_batch, bwd_batch;   // Gaussians staged per thread per shared-memory batch
    int overlap_prev;           // zero the backward's accumulators in the tail of the kernel ahead
    float near_z, dilation, alpha_min, alpha_max, t_min, fov_clamp;
    float bg[3];
    ViewDesc v[GS_MAX_VIEWS];
    SceneDesc s[GS_MAX_VIEWS];
};

// The mean L1 loss folded into the raster backward: with target set, the
// upstream gradient of each image value is sign(image - target) * inv_n and
// the loss inv_n * sum |image - target| is added to *loss.
struct L1Loss {
    const float *target = nullptr;
    float *loss = nullptr;
    float inv_n = 0.f;
};

// counters[] slots
enum {
    CNT_INSTANCES = 0,   // total tile instances
    CNT_ABORT = 1,       // nonzero: capacity exceeded, skip the rest
    CNT_Q_FWD = 2,       // work queue heads
    CNT_Q_BWD = 3,
    CNT_Q_SORT = 4,
    CNT_RUN_RES = 5,     // runs of split large tiles listed for the sort
    CNT_MAX_TILE = 6,    // largest per-tile count
    CNT_Q_SPLIT = 7      // queue head of the large-tile split
};

// ---------------------------------------------------------------------------
// lookups (binary search over ascending bases)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int view_of_slot(const Launch &L, long long slot) {
    int lo = 0, hi = L.n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (L.v[mid].slot_base <= slot) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int view_of_tile(const Launch &L, int tile) {
    int lo = 0, hi = L.n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (L.v[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int scene_of_thread(const Launch &L, long long gid) {
    int lo = 0, hi = L.n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (L.s[mid].thread_base <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// arithmetic helpers (explicit rounding: these never get contracted, so the
// forward and the backward replay take bit-identical decisions)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float LOG2E = 1.4426950408889634f;
constexpr float LN2 = 0.69314718055994531f;

struct ff { float hi, lo; };   // unevaluated sum hi + lo

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// r0*a + r1*b + r2*c + t with a float-pair result (error ~1e-14 relative)
__device__ __forceinline__ ff dot3_plus(float r0, float r1, float r2, float a, float b, float c, float t) {
    ff p0 = two_prod(r0, a), p1 = two_prod(r1, b), p2 = two_prod(r2, c);
    ff s = two_sum(p0.hi, p1.hi);
    float lo = __fadd_rn(__fadd_rn(p0.lo, p1.lo), s.lo);
    ff s2 = two_sum(s.hi, p2.hi);
    lo = __fadd_rn(lo, __fadd_rn(p2.lo, s2.lo));
    ff s3 = two_sum(s2.hi, t);
    lo = __fadd_rn(lo, s3.lo);
    return two_sum(s3.hi, lo);
}

// f * (xh + xl) / (zh + zl) + c as a float pair
__device__ __forceinline__ ff project_coord(float f, float xh, float xl, float zh, float zl, float c) {
    float q0 = __fdiv_rn(xh, zh);
    float e = __fmaf_rn(-q0, zh, xh);                       // exact xh - q0 zh
    float r = __fsub_rn(__fadd_rn(e, xl), __fmul_rn(q0, zl));
    float q1 = __fdiv_rn(r, zh);
    ff p = two_prod(f, q0);
    float plo = __fmaf_rn(f, q1, p.lo);
    ff s = two_sum(p.hi, c);
    return two_sum(s.hi, __fadd_rn(s.lo, plo));
}

// Tile rectangle [x0,x1) x [y0,y1) of a record, in float32 exactly as the
// bit-exact binning contract states: floor((x -+ ex)/tile) (+1 for the end),
// same in y with ey, clamped to the grid. inv_tw = 1/tw is exact (tw a
// power of two).
__device__ __forceinline__ void tile_rect(float x, float y, float ex, float ey, float inv_tw, float inv_th,
                                          int Gx, int Gy, int &x0, int &x1, int &y0, int &y1) {
    float a0 = floorf(__fmul_rn(__fsub_rn(x, ex), inv_tw));
    float a1 = __fadd_rn(floorf(__fmul_rn(__fadd_rn(x, ex), inv_tw)), 1.0f);
    float b0 = floorf(__fmul_rn(__fsub_rn(y, ey), inv_th));
    float b1 = __fadd_rn(floorf(__fmul_rn(__fadd_rn(y, ey), inv_th)), 1.0f);
    x0 = (int)fminf(fmaxf(a0, 0.0f), (float)Gx);
    x1 = (int)fminf(fmaxf(a1, 0.0f), (float)Gx);
    y0 = (int)fminf(fmaxf(b0, 0.0f), (float)Gy);
    y1 = (int)fminf(fmaxf(b1, 0.0f), (float)Gy);
}

// ---------------------------------------------------------------------------
// real spherical harmonics up to degree 3 (Condon-Shortley phase), as
// homogeneous polynomials of the unit direction. Constants are the
// normalisations sqrt((2l+1)/(4pi) (l-|m|)!/(l+|m|)!) (x sqrt2 for m != 0)
// times the polynomial factors of P_l^|m|:
//   l=0: 1/(2 sqrt(pi))
//   l=1: sqrt(3/(4pi)) {-y, z, -x}
//   l=2: sqrt(15/(4pi)) {xy, -yz, -xz}, sqrt(5/(16pi)) (2z^2-x^2-y^2),
//        sqrt(15/(16pi)) (x^2-y^2)
//   l=3: sqrt(35/(32pi)) {-y(3x^2-y^2), -x(x^2-3y^2)}, sqrt(105/(4pi)) xyz,
//        sqrt(21/(32pi)) {-y(4z^2-x^2-y^2), -x(4z^2-x^2-y^2)},
//        sqrt(7/(16pi)) z(2z^2-3x^2-3y^2), sqrt(105/(16pi)) z(x^2-y^2)
// ---------------------------------------------------------------------------
#define GS_SH_C0 0.28209479177387814f
#define GS_SH_C1 0.48860251190291992f
#define GS_SH_C2A 1.0925484305920792f
#define GS_SH_C20 0.31539156525252005f
#define GS_SH_C22 0.54627421529603959f
#define GS_SH_C33 0.59004358992664352f
#define GS_SH_C32A 2.8906114426405538f
#define GS_SH_C31 0.45704579946446572f
#define GS_SH_C30 0.37317633259011540f
#define GS_SH_C32 1.4453057213202769f

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    Y[0] = GS_SH_C0;
    if (DEG >= 1) {
        Y[1] = -GS_SH_C1 * y;
        Y[2] = GS_SH_C1 * z;
        Y[3] = -GS_SH_C1 * x;
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = GS_SH_C2A * x * y;
        Y[5] = -GS_SH_C2A * y * z;
        Y[6] = GS_SH_C20 * (2.f * zz - xx - yy);
        Y[7] = -GS_SH_C2A * x * z;
        Y[8] = GS_SH_C22 * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -GS_SH_C33 * y * (3.f * xx - yy);
            Y[10] = GS_SH_C32A * x * y * z;
            Y[11] = -GS_SH_C31 * y * (4.f * zz - xx - yy);
            Y[12] = GS_SH_C30 * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -GS_SH_C31 * x * (4.f * zz - xx - yy);
            Y[14] = GS_SH_C32 * z * (xx - yy);
            Y[15] = -GS_SH_C33 * x * (xx - 3.f * yy);
        }
    }
}

// g_d = sum_k gY[k] * grad(Y_k) of the polynomials above (unprojected)
template <int DEG>
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float *gY, float &gx, float &gy,
                                             float &gz) {
    gx = gy = gz = 0.f;
    if (DEG >= 1) {
        gy += -GS_SH_C1 * gY[1];
        gz += GS_SH_C1 * gY[2];
        gx += -GS_SH_C1 * gY[3];
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        gx += GS_SH_C2A * y * gY[4];
        gy += GS_SH_C2A * x * gY[4];
        gy += -GS_SH_C2A * z * gY[5];
        gz += -GS_SH_C2A * y * gY[5];
        gx += -2.f * GS_SH_C20 * x * gY[6];
        gy += -2.f * GS_SH_C20 * y * gY[6];
        gz += 4.f * GS_SH_C20 * z * gY[6];
        gx += -GS_SH_C2A * z * gY[7];
        gz += -GS_SH_C2A * x * gY[7];
        gx += 2.f * GS_SH_C22 * x * gY[8];
        gy += -2.f * GS_SH_C22 * y * gY[8];
        if (DEG >= 3) {
            gx += -6.f * GS_SH_C33 * x * y * gY[9];
            gy += -GS_SH_C33 * (3.f * xx - 3.f * yy) * gY[9];
            gx += GS_SH_C32A * y * z * gY[10];
            gy += GS_SH_C32A * x * z * gY[10];
            gz += GS_SH_C32A * x * y * gY[10];
            gx += 2.f * GS_SH_C31 * x * y * gY[11];
            gy += -GS_SH_C31 * (4.f * zz - xx - 3.f * yy) * gY[11];
            gz += -8.f * GS_SH_C31 * y * z * gY[11];
            gx += -6.f * GS_SH_C30 * x * z * gY[12];
            gy += -6.f * GS_SH_C30 * y * z * gY[12];
            gz += GS_SH_C30 * (6.f * zz - 3.f * xx - 3.f * yy) * gY[12];
            gx += -GS_SH_C31 * (4.f * zz - 3.f * xx - yy) * gY[13];
            gy += 2.f * GS_SH_C31 * x * y * gY[13];
            gz += -8.f * GS_SH_C31 * x * z * gY[13];
            gx += 2.f * GS_SH_C32 * x * z * gY[14];
            gy += -2.f * GS_SH_C32 * y * z * gY[14];
            gz += GS_SH_C32 * (xx - yy) * gY[14];
            gx += -GS_SH_C33 * (3.f * xx - 3.f * yy) * gY[15];
            gy += 6.f * GS_SH_C33 * x * y * gY[15];
        }
    }
}

// rotation of a unit quaternion (w,x,y,z), row-major
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float *R) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// ---------------------------------------------------------------------------
// asynchronous bulk copies (TMA) with an mbarrier, PTX ISA "cp.async.bulk"
// and "mbarrier". Every wait is bounded: it gives up after 2^20 polls of
// mbarrier.try_wait or once GS_WAIT_LIMIT_NS of the global nanosecond timer
// have passed, whichever comes first (a poll may suspend the thread for a
// system-dependent time, so the timer bounds the wait's duration), and a
// copy that never lands ends in an error status instead of a hang.
// ---------------------------------------------------------------------------
constexpr unsigned long long GS_WAIT_LIMIT_NS = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start before the kernel ahead of it in the stream has
// finished, once every block of that kernel has signalled (or exited).
// launch_dependents signals from this block; grid_dependency_wait returns
// once the kernel ahead has completed and its memory is visible (at once for
// a kernel launched without the attribute).
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true once the barrier's phase `parity` has completed; false if the bounded
// number of polls ran out first
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 0) {   // the timer is read only while the copy is late
            const unsigned long long t = global_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > GS_WAIT_LIMIT_NS) return false;
        }
    }
    return false;
}

// 2D tiled load of the box at (x, y) (x in elements, a multiple of 16 bytes)
// into shared memory, completing on bar
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 2D tiled store of a shared-memory box to (x, y) (x = 0 here; rows outside
// the tensor are not written), tracked by the issuing thread's bulk group
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of all committed bulk stores have been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// make this thread's generic shared-memory writes visible to bulk copies
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared (cp.async, cached in L2 only),
// tracked per thread; cp_async_wait_all makes this thread's copies visible
// to this thread
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// 16-byte chunk c of row r of a box staged with the 128-byte swizzle (rows
// of 128 bytes) or the 64-byte swizzle (rows of 64 bytes): the hardware XORs
// the chunk index with address bits 7..9 (7..8), so a thread reading chunk c
// of its own row hits a different bank group than its neighbours
__device__ __forceinline__ int swz128(int r, int c) { return r * 8 + (c ^ (r & 7)); }
__device__ __forceinline__ int swz64(int r, int c) { return r * 4 + (c ^ ((r >> 1) & 3)); }

// ---------------------------------------------------------------------------
// host-side launch helpers (defined in gs_api.cu)
// ---------------------------------------------------------------------------
int num_sms();
// encode a 2D float32 tensor map: `rows` rows of `inner` floats, `row_bytes`
// apart, box = box_inner x box_rows, with the given swizzle; false if the
// driver's encoder is unavailable or rejects the description
bool encode_tmap_2d(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
                    uint32_t box_inner, uint32_t box_rows, CUtensorMapSwizzle swizzle);

}  // namespace gsk
