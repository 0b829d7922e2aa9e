// Internal declarations of libgsraster: workspace layout, device state and
// the stage launchers.  The types and per-fragment arithmetic the kernels are
// built from live in gs_frag.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gs.h"
#include "gs_frag.cuh"

namespace gs {

// Threads and Gaussians of one projection-backward block (a chunk of one
// submap).  Both backward kernels are bound by memory latency; many small
// blocks keep the most loads in flight (500k orchard, both kernels: 256 x
// 1024 -> 0.114 ms, 256 x 512 -> 0.096 ms, 128 x 256 -> 0.090 ms,
// 128 x 128 -> 0.100 ms).
constexpr int kProjBwdThreads = 128;
constexpr int kProjBwdChunk = 256;

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
    uint32_t done_l1, done_depth;  // finished blocks of the loss reductions (the last one finishes)
    uint32_t pad[5];
    unsigned long long frag_count[4];  // gs_workspace_fragment_counts
};
constexpr uint32_t kFlagCapacity = 1u;
constexpr int kEmitWindow = 1024;      // output slots per emission window
constexpr uint32_t kFlagTimeout = 2u;  // a bounded device wait (TMA) gave up

}  // namespace gs

// The workspace (opaque to C callers).
struct gs_workspace {
    int32_t n_views = 0, n_submaps = 0, sh_degree = 0, device = 0, num_sms = 0;
    gs_config cfg{};
    gs::Consts consts{};
    int64_t n = 0, n_pairs = 0, n_tiles = 0, n_pix = 0, inst_cap = 0;
    int32_t tile_bits = 0, sort_blocks = 0, proj_blocks = 0, max_views_per_submap = 0;
    int32_t wide_blocks = 0;  // blocks of the compaction and of the depth sort (short, latency-bound chains)
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
    float4 *gdir = nullptr;        // [n_pairs] colour gradient w.r.t. the view direction
    uint32_t *vis_key = nullptr, *vis_pair = nullptr, *vis_key_alt = nullptr, *vis_pair_alt = nullptr;
    uint32_t *ioff = nullptr;      // [n_pairs]
    uint32_t *win_pair = nullptr;  // [inst_cap / kEmitWindow + 1] owner of each emission window's first slot
    // per-instance buffers
    uint32_t *inst_tile = nullptr, *inst_val = nullptr, *inst_tile_alt = nullptr, *inst_val_alt = nullptr;
    // per-tile / per-pixel
    uint2 *ranges = nullptr;       // [n_tiles]
    uint32_t *tile_order = nullptr; // [n_tiles] tiles by decreasing list length (raster work order)
    uint32_t *order_tot = nullptr;  // [kOrderBuckets] work-order bucket totals
    uint32_t *order_base = nullptr; // [kOrderBlocks][kOrderBuckets] each block's base inside each bucket
    uint32_t *last = nullptr;      // [n_pix]
    float *tfin = nullptr;         // [n_pix]
    float4 *vstat = nullptr;       // [n_pix] depth (mean, var, 1/W, 0) of the variance forward
    // scratch
    uint32_t *hist = nullptr;      // [256][hist_cols]
    int32_t hist_cols = 0;         // max(2 sort_blocks, wide_blocks): the most blocks a radix pass may run
    uint32_t *part = nullptr;      // [max(sort_blocks, wide_blocks) + 1]
    uint32_t *digit_tot = nullptr; // [256] digit totals of the current radix pass
    float *pose_part = nullptr;    // [proj_blocks][max_views_per_submap][6]
    double *red_part = nullptr;    // [2][sort_blocks] loss partials
    int64_t n_ssim_tiles = 0;      // 32x16 SSIM tiles over all channel planes
    float *ssim_d = nullptr;       // [3][3 n_pix] SSIM partials for the backward
    double *ssim_part = nullptr;   // [n_ssim_tiles] per-tile sums of the SSIM map
    gs::DevState *st = nullptr;
    // host-side order checks
    bool projected = false, binned = false, rendered = false, rendered_var = false;
    bool g2d_clear = false;  // the last projection cleared g2d and no backward has run since
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
gs_status launch_image_l1_u8(gs_workspace *ws, const float *rgb, const uint8_t *target, float *loss,
                             float *dL_drgb, cudaStream_t s);
gs_status launch_image_l1(gs_workspace *ws, const float *rgb, const float *target, float *loss,
                          float *dL_drgb, cudaStream_t s);
// Eq. (6): (1 - lambda) L1 + lambda (1 - SSIM); loss[0..2] = total, L1, 1 - SSIM
gs_status launch_image_loss(gs_workspace *ws, const float *rgb, const float *target, float lambda,
                            float *loss, float *dL_drgb, cudaStream_t s);
// SSIM map sums into ws->ssim_part; with dL_drgb, adds grad_scale * dSSIM/dx
gs_status launch_ssim(gs_workspace *ws, const float *rgb, const float *target, float grad_scale,
                      float *dL_drgb, cudaStream_t s);
int64_t ssim_tiles(const std::vector<ViewInfo> &views);
// occupancy-derived persistent grid sizes for the rasterisers
gs_status raster_configure(gs_workspace *ws);
gs_status sort_configure();

}  // namespace gs
