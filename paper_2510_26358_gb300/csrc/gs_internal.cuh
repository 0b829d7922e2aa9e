// Internal declarations of libgsraster: workspace layout, per-view tables,
// launch helpers and the per-fragment arithmetic that the forward and the
// backward rasteriser must evaluate bit-identically.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gs.h"

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

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------

struct ViewInfo {
    int32_t W, H, ntx, nty;
    int32_t pix_off, tile_off, pair_off, g0;
    int32_t ng, submap, k_in_submap, pad;
};

struct SubmapInfo {
    int32_t g0, ng, nviews, block0;  // block0: first projection-backward block
    int32_t nblocks, pad0, pad1, pad2;
};

// Device-resident counters and flags (one per workspace).
struct DevState {
    uint32_t n_vis;             // visible pairs after compaction
    uint32_t n_inst;            // instances in the lists (0 after an overflow)
    unsigned long long n_inst_needed;
    uint32_t flags;             // kFlagCapacity
    uint32_t fwd_counter;       // persistent-raster work queues
    uint32_t bwd_counter;
    float depth_scale;          // lambda_L / |Omega| of the last gs_depth_loss
    uint32_t depth_valid;
    uint32_t pad[7];
};
constexpr uint32_t kFlagCapacity = 1u;

// Constants every kernel needs, passed by value.
struct Consts {
    float near_z, dilation, alpha_min, alpha_max, t_min, jac_clamp;
    float ext_rel_pad, ext_abs_pad;
    float log2_alpha_min;   // log2(alpha_min)
    float ln_alpha_min;     // ln(alpha_min)
    int32_t tile_w, tile_h;
};

}  // namespace gs

// The workspace (opaque to C callers).
struct gs_workspace {
    int32_t n_views = 0, n_submaps = 0, sh_degree = 0, device = 0, num_sms = 0;
    gs_config cfg{};
    gs::Consts consts{};
    int64_t n = 0, n_pairs = 0, n_tiles = 0, n_pix = 0, inst_cap = 0;
    int32_t tile_bits = 0, sort_blocks = 0, proj_blocks = 0, max_views_per_submap = 0;
    int32_t raster_grid_fwd = 0, raster_grid_bwd = 0, raster_grid_fwd_var = 0, raster_grid_bwd_var = 0;
    size_t bytes = 0;
    int64_t kernel_launches = 0;  // kernels enqueued by this workspace so far
    std::vector<gs::ViewInfo> views_h;
    std::vector<gs::SubmapInfo> subs_h;
    std::vector<int32_t> sub_views_h;  // [n_submaps][max_views_per_submap]
    // device tables
    gs::ViewInfo *views = nullptr;
    gs::SubmapInfo *subs = nullptr;
    int32_t *sub_views = nullptr;
    // per-pair buffers
    float4 *rec = nullptr;         // [n_pairs][3]
    uint32_t *pkey = nullptr;      // [n_pairs]
    short4 *rect = nullptr;        // [n_pairs]
    float *g2d = nullptr;          // [n_pairs][10]
    uint32_t *vis_key = nullptr, *vis_pair = nullptr, *vis_key_alt = nullptr, *vis_pair_alt = nullptr;
    uint32_t *ioff = nullptr;      // [n_pairs]
    // per-instance buffers
    uint32_t *inst_tile = nullptr, *inst_val = nullptr, *inst_tile_alt = nullptr, *inst_val_alt = nullptr;
    // per-tile / per-pixel
    uint2 *ranges = nullptr;       // [n_tiles]
    uint32_t *tile_order = nullptr; // [n_tiles] tiles by decreasing list length (raster work order)
    uint32_t *tile_buckets = nullptr; // [2][kOrderBuckets] histogram and cursors for tile_order
    uint32_t *last = nullptr;      // [n_pix]
    float *tfin = nullptr;         // [n_pix]
    float4 *vstat = nullptr;       // [n_pix] depth (mean, var, 1/W, 0) of the variance forward
    // scratch
    uint32_t *hist = nullptr;      // [256][sort_blocks]
    uint32_t *part = nullptr;      // [sort_blocks + 1]
    uint32_t *digit_tot = nullptr; // [256] digit totals of the current radix pass
    float *pose_part = nullptr;    // [proj_blocks][max_views_per_submap][6]
    double *red_part = nullptr;    // [2][sort_blocks] loss partials
    gs::DevState *st = nullptr;
    // host-side order checks
    bool projected = false, binned = false, rendered = false, rendered_var = false;
    // optional per-stage timing (events recorded around each kernel group)
    bool profiling = false;
    cudaEvent_t ev[2 * GS_NUM_STAGES] = {};
    bool ev_used[GS_NUM_STAGES] = {};
};

namespace gs {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------

void set_last_error(const std::string &msg);
gs_status check_launch(const char *what);

// Brackets the kernels of one stage with timing events when profiling is on.
struct StageTimer {
    gs_workspace *ws;
    int id;
    cudaStream_t s;
    StageTimer(gs_workspace *w, int stage, cudaStream_t st) : ws(w), id(stage), s(st) {
        if (ws->profiling) cudaEventRecord(ws->ev[2 * id], s);
    }
    ~StageTimer() {
        if (ws->profiling) {
            cudaEventRecord(ws->ev[2 * id + 1], s);
            ws->ev_used[id] = true;
        }
    }
};

// ---------------------------------------------------------------------------
// stage launchers (one translation unit each)
// ---------------------------------------------------------------------------

gs_status launch_project_fwd(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams,
                             cudaStream_t s);
gs_status launch_project_bwd(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams,
                             const gs_grads *out, cudaStream_t s);
gs_status launch_bin_sort(gs_workspace *ws, cudaStream_t s);
// mean == nullptr: plain forward; otherwise also the depth mean and variance
gs_status launch_raster_fwd(gs_workspace *ws, float *rgb, float *depth, float *alpha, float *mean,
                            float *var, cudaStream_t s);
gs_status launch_raster_bwd(gs_workspace *ws, const float *dL_drgb, const float *dL_ddepth,
                            const float *dL_dalpha, bool var, const float *dL_dmean,
                            const float *dL_dvar, cudaStream_t s);
// mode 0, 1: gs_depth_loss on `depth`; mode 2: the rendered-variance KL on
// (`depth` = mean, var), gradients to mean (dL_ddepth) and var
gs_status launch_depth_loss(gs_workspace *ws, int mode, const float *depth, const float *alpha,
                            const float *var, const float *lidar, int64_t n_pts, float *loss,
                            float *dL_ddepth, float *dL_dvar, cudaStream_t s);
gs_status launch_image_l1(gs_workspace *ws, const float *rgb, const float *target, float *loss,
                          float *dL_drgb, cudaStream_t s);
// occupancy-derived persistent grid sizes for the rasterisers
gs_status raster_configure(gs_workspace *ws);
gs_status sort_configure();

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
