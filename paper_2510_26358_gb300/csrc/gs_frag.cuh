// Types, constants and per-fragment arithmetic of the rasterisers: the
// record layout, the per-view table, the renderer constants and the device
// functions that the forward and the backward must evaluate bit-identically.
// (Everything the raster kernels are built from besides gs_raster.cu itself.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------

constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;  // pair depth key of an invisible pair
constexpr int kRecF4 = 3;                     // float4 per projected record
constexpr int kGrad = 10;                     // floats per image-space gradient record
// image-space gradient components (same order as the oracle's)
enum { G_U = 0, G_V, G_QA, G_QB, G_QC, G_LNO, G_R, G_G, G_B, G_Z };

// sqrt(log2(e)/2): scales the Cholesky factor of Sigma'^-1 so that
// log2(alpha) = log2(o) - (t1^2 + t2^2)
constexpr float kCholScale = 0.84932180028801904272f;
// 2 ln 2 = 1/kCholScale^2: converts scaled factors back to natural units
constexpr float kTwoLn2 = 1.38629436111989061883f;
constexpr float kLog2e = 1.44269504088896340736f;

constexpr int kSortThreads = 256;
constexpr int kProjThreads = 256;
constexpr int kOrderBuckets = 64;     // list-length buckets of the raster work order
constexpr int kOrderShift = 5;        // bucket = min(63, length >> 5)
constexpr int kOrderBlocks = 64;      // blocks of the two work-order kernels

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------

struct ViewInfo {
    int32_t W, H, ntx, nty;
    int32_t pix_off, tile_off, pair_off, g0;
    int32_t ng, submap, k_in_submap, pad;
};

// Constants every kernel needs, passed by value.
struct Consts {
    float near_z, dilation, alpha_min, alpha_max, t_min, jac_clamp;
    float ext_rel_pad, ext_abs_pad;
    float log2_alpha_min;   // log2(alpha_min)
    float ln_alpha_min;     // ln(alpha_min)
    int32_t tile_w, tile_h;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two floats in one 64-bit register, for the packed single-precision
// arithmetic of sm_100 and later: one add / sub / mul / fma instruction works
// both halves, each rounded exactly as the scalar instruction rounds it (no
// flush to zero, like the scalar code built without -ftz).
struct f2 {
    unsigned long long v;
};

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2 f2_bcast(float x) { return f2_pack(x, x); }
__device__ __forceinline__ void f2_unpack(f2 a, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ float f2_lo(f2 a) {
    float lo, hi;
    f2_unpack(a, lo, hi);
    return lo;
}
__device__ __forceinline__ float f2_hi(f2 a) {
    float lo, hi;
    f2_unpack(a, lo, hi);
    return hi;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
// a * b + c with one rounding per half
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}

// Staged copy of one projected record, as the rasterisers keep it in shared
// memory: a = (U, V, k1, k2) with U, V the integer pixel of the mean and
// k1 = l11 hx + l12 hy, k2 = l22 hy; b = (l11, l12, l22, log2 o) the scaled
// Cholesky factor of Sigma'^-1; c = (r, g, b, z).
__device__ __forceinline__ void stage_record(const float4 r0, const float4 r1, float4 &a, float4 &b) {
    // r0 = (U, V, hx, hy), r1 = (l11, l12, l22, log2o)
    a.x = r0.x;
    a.y = r0.y;
    a.z = __fmaf_rn(r1.x, r0.z, __fmul_rn(r1.y, r0.w));
    a.w = __fmul_rn(r1.z, r0.w);
    b = r1;
}

// log2 of the unclamped alpha of a staged Gaussian at integer pixel (px, py):
// d = (px - U + hx, py - V + hy), t1 = l11 dx + l12 dy, t2 = l22 dy,
// e = log2 o - t1^2 - t2^2, evaluated as
//   column part (shared by the pixels of one column):  dxi = px - U,
//                                                      u1 = l11 dxi + k1
//   pixel part:   dyi = py - V,  t1 = l12 dyi + u1,  t2 = l22 dyi + k2,
//                 e = log2 o - t1^2 - t2^2
// with exact integer offsets dxi, dyi.  Both passes call these functions, so
// the backward recomputes exactly the forward's alpha and decisions, for any
// tile size and any number of pixels per thread.
__device__ __forceinline__ void frag_column(const float4 a, const float4 b, float pxf, float &dxi, float &u1) {
    dxi = __fsub_rn(pxf, a.x);
    u1 = __fmaf_rn(b.x, dxi, a.z);
}

__device__ __forceinline__ float frag_pixel(const float4 a, const float4 b, float u1, float pyf, float &t1,
                                            float &t2, float &dyi) {
    dyi = __fsub_rn(pyf, a.y);
    t1 = __fmaf_rn(b.y, dyi, u1);
    t2 = __fmaf_rn(b.z, dyi, a.w);
    return __fmaf_rn(-t1, t1, __fmaf_rn(-t2, t2, b.w));
}

__device__ __forceinline__ int view_of_tile(const ViewInfo *views, int n_views, int tile) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__host__ __device__ inline void chunk_range(uint64_t n, int b, int nblocks, int tile, uint32_t &lo,
                                            uint32_t &hi) {
    uint64_t per = (n + nblocks - 1) / nblocks;
    per = (per + tile - 1) / tile * tile;
    uint64_t l = (uint64_t)b * per;
    if (l > n) l = n;
    uint64_t h = l + per;
    if (h > n) h = n;
    lo = (uint32_t)l;
    hi = (uint32_t)h;
}

}  // namespace gs
