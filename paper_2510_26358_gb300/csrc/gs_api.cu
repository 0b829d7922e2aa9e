// C ABI of libgsraster: argument checks, workspace allocation and the
// ordering of the stage launches.  See include/gs.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "gs_internal.cuh"

namespace gs {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

gs_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

namespace {

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

gs_status fail(gs_status s, const std::string &msg) {
    set_last_error(msg);
    return s;
}

template <class Tp>
gs_status alloc(gs_workspace *ws, Tp *&p, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(Tp);
    cudaError_t e = cudaMalloc((void **)&p, bytes);
    if (e != cudaSuccess) {
        p = nullptr;
        return fail(GS_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ws->bytes += bytes;
    return GS_OK;
}

gs_status check_config(const gs_config *c) {
    bool tile_ok = (c->tile_w == 8 && c->tile_h == 8) || (c->tile_w == 16 && c->tile_h == 16) ||
                   (c->tile_w == 16 && c->tile_h == 32) || (c->tile_w == 32 && c->tile_h == 16);
    if (!tile_ok) return fail(GS_ERR_INVALID_ARG, "tile size must be 8x8, 16x16, 16x32 or 32x16");
    if (c->batch_depth < 32 || c->batch_depth > 256 || c->batch_depth % 32)
        return fail(GS_ERR_INVALID_ARG, "batch_depth must be a multiple of 32 in [32, 256]");
    if (c->depth_mode != 0 && c->depth_mode != 1) return fail(GS_ERR_INVALID_ARG, "depth_mode must be 0 or 1");
    if (!(c->near_z > 0.f) || !(c->dilation >= 0.f) || !(c->alpha_min > 0.f) ||
        !(c->alpha_max > c->alpha_min) || !(c->alpha_max < 1.f) || !(c->t_min > 0.f) ||
        !(c->t_min < 1.f) || !(c->jac_clamp > 0.f) || !(c->ext_rel_pad >= 0.f) ||
        !(c->ext_abs_pad >= 0.f) || !(c->sigma_L > 0.f) || !(c->sigma_U > 0.f) || !std::isfinite(c->lambda_L))
        return fail(GS_ERR_INVALID_ARG, "renderer constant out of range");
    return GS_OK;
}

gs_status check_gaussians(const gs_workspace *ws, const gs_gaussians *g) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n != ws->n) return fail(GS_ERR_INVALID_ARG, "gaussians.n differs from the workspace's submap total");
    if (ws->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail(GS_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
    return GS_OK;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

void gs_config_default(gs_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->batch_depth = 256;
    cfg->depth_mode = 0;
    cfg->near_z = 0.2f;
    cfg->dilation = 0.3f;
    cfg->alpha_min = 1.f / 255.f;
    cfg->alpha_max = 0.99f;
    cfg->t_min = 1e-4f;
    cfg->jac_clamp = 1.3f;
    cfg->ext_rel_pad = 1e-3f;
    cfg->ext_abs_pad = 1e-2f;
    cfg->sigma_L = 0.05f;
    cfg->sigma_U = 0.05f;
    cfg->lambda_L = 1.f;
}

gs_status gs_workspace_set_profiling(gs_workspace *ws, int32_t on) {
    if (!ws) return fail(GS_ERR_INVALID_ARG, "NULL workspace");
    if (on && !ws->ev[0]) {
        for (cudaEvent_t &e : ws->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return fail(GS_ERR_CUDA, std::string("event: ") + cudaGetErrorString(r));
        }
    }
    ws->profiling = on != 0;
    for (bool &u : ws->ev_used) u = false;
    return GS_OK;
}

gs_status gs_workspace_stage_ms(gs_workspace *ws, float *ms, int32_t n) {
    if (!ws || !ms || n < 0) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    for (int i = 0; i < n && i < GS_NUM_STAGES; ++i) {
        ms[i] = -1.f;
        if (!ws->ev_used[i]) continue;
        cudaError_t r = cudaEventSynchronize(ws->ev[2 * i + 1]);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&ms[i], ws->ev[2 * i], ws->ev[2 * i + 1]);
        if (r != cudaSuccess) return fail(GS_ERR_CUDA, std::string("stage timing: ") + cudaGetErrorString(r));
    }
    return GS_OK;
}

const char *gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_CAPACITY: return "instance capacity exceeded";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_STATE: return "call out of order";
        case GS_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    }
    return "unknown status";
}

const char *gs_last_error(void) { return g_last_error.c_str(); }

void gs_workspace_destroy(gs_workspace *ws) {
    if (!ws) return;
    void *ptrs[] = {ws->views, ws->subs, ws->sub_views, ws->rec, ws->pkey, ws->rect, ws->g2d, ws->gdir,
                    ws->vis_key, ws->vis_pair, ws->vis_key_alt, ws->vis_pair_alt, ws->ioff, ws->win_pair,
                    ws->inst_tile, ws->inst_val, ws->inst_tile_alt, ws->inst_val_alt, ws->ranges,
                    ws->tile_order, ws->order_tot, ws->order_base,
                    ws->last, ws->tfin, ws->vstat, ws->hist, ws->part, ws->digit_tot, ws->pose_part, ws->red_part, ws->ssim_d, ws->ssim_part,
                    ws->st};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : ws->ev)
        if (e) cudaEventDestroy(e);
    delete ws;
}

gs_status gs_workspace_create(const gs_camera *cams, int32_t n_views, const int64_t *submap_offsets,
                              int32_t n_submaps, int32_t sh_degree, const gs_config *cfg,
                              int64_t inst_capacity, gs_workspace **out) {
    if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cams || !submap_offsets || !cfg) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (n_views < 1 || n_views > GS_MAX_VIEWS) return fail(GS_ERR_INVALID_ARG, "n_views out of range");
    if (n_submaps < 1 || n_submaps > GS_MAX_SUBMAPS) return fail(GS_ERR_INVALID_ARG, "n_submaps out of range");
    if (sh_degree < 0 || sh_degree > 3) return fail(GS_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (inst_capacity < 1 || inst_capacity > 0x7FFFFFFFll)
        return fail(GS_ERR_INVALID_ARG, "inst_capacity must be in [1, 2^31)");
    gs_status st = check_config(cfg);
    if (st != GS_OK) return st;
    if (submap_offsets[0] != 0) return fail(GS_ERR_INVALID_ARG, "submap_offsets[0] must be 0");
    for (int s = 0; s < n_submaps; ++s)
        if (submap_offsets[s + 1] < submap_offsets[s])
            return fail(GS_ERR_INVALID_ARG, "submap_offsets must be nondecreasing");
    int64_t n = submap_offsets[n_submaps];
    if (n > 0x7FFFFFFFll) return fail(GS_ERR_INVALID_ARG, "too many Gaussians");

    gs_workspace *ws = new gs_workspace();
    ws->n_views = n_views;
    ws->n_submaps = n_submaps;
    ws->sh_degree = sh_degree;
    ws->cfg = *cfg;
    ws->n = n;
    ws->inst_cap = inst_capacity;
    cudaGetDevice(&ws->device);
    cudaDeviceGetAttribute(&ws->num_sms, cudaDevAttrMultiProcessorCount, ws->device);
    if (ws->num_sms < 1) ws->num_sms = 1;

    // tables
    std::vector<int32_t> nviews(n_submaps, 0);
    int64_t pair_off = 0, tile_off = 0, pix_off = 0;
    for (int v = 0; v < n_views; ++v) {
        const gs_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384 || c.submap < 0 ||
            c.submap >= n_submaps || c.reserved != 0) {
            delete ws;
            return fail(GS_ERR_INVALID_ARG, "camera " + std::to_string(v) + " has an invalid size or submap");
        }
        ViewInfo vi{};
        vi.W = c.width;
        vi.H = c.height;
        vi.ntx = (c.width + cfg->tile_w - 1) / cfg->tile_w;
        vi.nty = (c.height + cfg->tile_h - 1) / cfg->tile_h;
        vi.g0 = (int32_t)submap_offsets[c.submap];
        vi.ng = (int32_t)(submap_offsets[c.submap + 1] - submap_offsets[c.submap]);
        vi.submap = c.submap;
        vi.k_in_submap = nviews[c.submap]++;
        vi.pair_off = (int32_t)pair_off;
        vi.tile_off = (int32_t)tile_off;
        vi.pix_off = (int32_t)pix_off;
        pair_off += vi.ng;
        tile_off += (int64_t)vi.ntx * vi.nty;
        pix_off += (int64_t)c.width * c.height;
        if (pair_off > 0x7FFFFFFFll || 3 * pix_off > 0x7FFFFFFFll || tile_off > 0x7FFFFFFFll) {
            delete ws;
            return fail(GS_ERR_INVALID_ARG, "too many pairs, tiles or pixels");
        }
        ws->views_h.push_back(vi);
    }
    ws->n_pairs = pair_off;
    ws->n_tiles = tile_off;
    ws->n_pix = pix_off;
    // bits of the largest value n_tiles (not n_tiles - 1): the sort then
    // orders the dropped instances' kInvalidKey after every real tile id
    ws->tile_bits = 0;
    while ((1ll << ws->tile_bits) <= ws->n_tiles) ++ws->tile_bits;
    int maxv = 1;
    for (int s = 0; s < n_submaps; ++s) maxv = std::max(maxv, nviews[s]);
    ws->max_views_per_submap = maxv;
    ws->sub_views_h.assign((size_t)n_submaps * maxv, -1);
    std::vector<int32_t> fill(n_submaps, 0);
    for (int v = 0; v < n_views; ++v) {
        int s = cams[v].submap;
        ws->sub_views_h[(size_t)s * maxv + fill[s]++] = v;
    }
    int32_t blocks = 0;
    for (int s = 0; s < n_submaps; ++s) {
        SubmapInfo si{};
        si.g0 = (int32_t)submap_offsets[s];
        si.ng = (int32_t)(submap_offsets[s + 1] - submap_offsets[s]);
        si.nviews = nviews[s];
        si.block0 = blocks;
        si.nblocks = (si.ng + kProjBwdChunk - 1) / kProjBwdChunk;
        blocks += si.nblocks;
        ws->subs_h.push_back(si);
    }
    ws->proj_blocks = blocks;
    ws->sort_blocks = std::min(4 * kSortThreads, 2 * ws->num_sms);
    // the radix scan takes at most 4 kSortThreads blocks
    ws->wide_blocks = std::min(4 * kSortThreads, 6 * ws->num_sms);

    // constants
    Consts &k = ws->consts;
    k.near_z = cfg->near_z;
    k.dilation = cfg->dilation;
    k.alpha_min = cfg->alpha_min;
    k.alpha_max = cfg->alpha_max;
    k.t_min = cfg->t_min;
    k.jac_clamp = cfg->jac_clamp;
    k.ext_rel_pad = cfg->ext_rel_pad;
    k.ext_abs_pad = cfg->ext_abs_pad;
    k.log2_alpha_min = (float)std::log2((double)cfg->alpha_min);
    k.ln_alpha_min = (float)std::log((double)cfg->alpha_min);
    k.tile_w = cfg->tile_w;
    k.tile_h = cfg->tile_h;

    // device memory
    size_t P = (size_t)ws->n_pairs, I = (size_t)inst_capacity;
    gs_status r = GS_OK;
#define GS_ALLOC(ptr, cnt) \
    if (r == GS_OK) r = alloc(ws, ptr, cnt)
    GS_ALLOC(ws->views, (size_t)n_views);
    GS_ALLOC(ws->subs, (size_t)n_submaps);
    GS_ALLOC(ws->sub_views, ws->sub_views_h.size());
    GS_ALLOC(ws->rec, P * kRecF4);
    GS_ALLOC(ws->pkey, P);
    GS_ALLOC(ws->rect, P);
    GS_ALLOC(ws->g2d, P * kGrad);
    GS_ALLOC(ws->gdir, P);
    GS_ALLOC(ws->vis_key, P);
    GS_ALLOC(ws->vis_pair, P);
    GS_ALLOC(ws->vis_key_alt, P);
    GS_ALLOC(ws->vis_pair_alt, P);
    GS_ALLOC(ws->ioff, P);
    GS_ALLOC(ws->win_pair, I / kEmitWindow + 2);
    GS_ALLOC(ws->inst_tile, I);
    GS_ALLOC(ws->inst_val, I);
    GS_ALLOC(ws->inst_tile_alt, I);
    GS_ALLOC(ws->inst_val_alt, I);
    GS_ALLOC(ws->ranges, (size_t)ws->n_tiles);
    GS_ALLOC(ws->tile_order, (size_t)ws->n_tiles);
    GS_ALLOC(ws->order_tot, (size_t)kOrderBuckets);
    GS_ALLOC(ws->order_base, (size_t)kOrderBlocks * kOrderBuckets);
    GS_ALLOC(ws->last, (size_t)ws->n_pix);
    GS_ALLOC(ws->tfin, (size_t)ws->n_pix);
    GS_ALLOC(ws->vstat, (size_t)ws->n_pix);
    // the instance sort runs 2 x sort_blocks, the compaction and depth sort wide_blocks
    ws->hist_cols = std::max(2 * ws->sort_blocks, ws->wide_blocks);
    GS_ALLOC(ws->hist, (size_t)256 * ws->hist_cols);
    GS_ALLOC(ws->part, (size_t)std::max(ws->sort_blocks, ws->wide_blocks) + 1);
    GS_ALLOC(ws->digit_tot, (size_t)256);
    GS_ALLOC(ws->pose_part, (size_t)std::max(1, blocks) * maxv * 6);
    GS_ALLOC(ws->red_part, (size_t)2 * ws->sort_blocks);
    ws->n_ssim_tiles = ssim_tiles(ws->views_h);
    GS_ALLOC(ws->ssim_d, (size_t)9 * ws->n_pix);
    GS_ALLOC(ws->ssim_part, (size_t)std::max<int64_t>(1, ws->n_ssim_tiles));
    GS_ALLOC(ws->st, 1);
#undef GS_ALLOC
    if (r == GS_OK) {
        cudaError_t e = cudaMemcpy(ws->views, ws->views_h.data(), sizeof(ViewInfo) * n_views,
                                   cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ws->subs, ws->subs_h.data(), sizeof(SubmapInfo) * n_submaps, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ws->sub_views, ws->sub_views_h.data(), sizeof(int32_t) * ws->sub_views_h.size(),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(ws->st, 0, sizeof(DevState));
        if (e == cudaSuccess) e = cudaMemset(ws->ranges, 0, sizeof(uint2) * std::max<int64_t>(1, ws->n_tiles));
        if (e == cudaSuccess) e = cudaMemset(ws->last, 0, sizeof(uint32_t) * std::max<int64_t>(1, ws->n_pix));
        if (e != cudaSuccess) r = fail(GS_ERR_CUDA, std::string("workspace init: ") + cudaGetErrorString(e));
    }
    if (r == GS_OK) r = raster_configure(ws);
    if (r == GS_OK) r = sort_configure();
    if (r != GS_OK) {
        gs_workspace_destroy(ws);
        return r;
    }
    *out = ws;
    return GS_OK;
}

gs_status gs_project(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams_dev, void *stream) {
    if (!ws || !cams_dev) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_gaussians(ws, g);
    if (r != GS_OK) return r;
    r = launch_project_fwd(ws, g, cams_dev, (cudaStream_t)stream);
    if (r == GS_OK) {
        ws->projected = true;
        ws->binned = ws->rendered = ws->rendered_var = false;
    }
    return r;
}

gs_status gs_bin_sort(gs_workspace *ws, void *stream) {
    if (!ws) return fail(GS_ERR_INVALID_ARG, "NULL workspace");
    if (!ws->projected) return fail(GS_ERR_STATE, "gs_bin_sort before gs_project");
    gs_status r = launch_bin_sort(ws, (cudaStream_t)stream);
    if (r == GS_OK) ws->binned = true;
    return r;
}

gs_status gs_render_fwd(gs_workspace *ws, float *rgb, float *depth, float *alpha, void *stream) {
    if (!ws || !rgb || !depth || !alpha) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (!ws->binned) return fail(GS_ERR_STATE, "gs_render_fwd before gs_bin_sort");
    gs_status r = launch_raster_fwd(ws, rgb, depth, alpha, nullptr, nullptr, (cudaStream_t)stream);
    if (r == GS_OK) {
        ws->rendered = true;
        ws->rendered_var = false;
    }
    return r;
}

gs_status gs_render_fwd_var(gs_workspace *ws, float *rgb, float *depth, float *alpha, float *depth_mean,
                            float *depth_var, void *stream) {
    if (!ws || !rgb || !depth || !alpha || !depth_mean || !depth_var)
        return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (!ws->binned) return fail(GS_ERR_STATE, "gs_render_fwd_var before gs_bin_sort");
    gs_status r = launch_raster_fwd(ws, rgb, depth, alpha, depth_mean, depth_var, (cudaStream_t)stream);
    if (r == GS_OK) ws->rendered = ws->rendered_var = true;
    return r;
}

gs_status gs_depth_loss(gs_workspace *ws, const float *depth, const float *alpha, const float *lidar,
                        int64_t n_pts, float *loss, float *dL_ddepth, void *stream) {
    if (!ws || !depth || !alpha || !loss) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (n_pts < 0 || (n_pts > 0 && !lidar)) return fail(GS_ERR_INVALID_ARG, "bad LiDAR array");
    if (lidar && !aligned(lidar, 16)) return fail(GS_ERR_INVALID_ARG, "lidar must be 16-byte aligned");
    return launch_depth_loss(ws, ws->cfg.depth_mode, depth, alpha, nullptr, lidar, n_pts, loss, dL_ddepth,
                             nullptr, (cudaStream_t)stream);
}

gs_status gs_depth_loss_var(gs_workspace *ws, const float *alpha, const float *depth_mean, const float *depth_var,
                            const float *lidar, int64_t n_pts, float *loss, float *dL_dmean, float *dL_dvar,
                            void *stream) {
    if (!ws || !alpha || !depth_mean || !depth_var || !loss) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (n_pts < 0 || (n_pts > 0 && !lidar)) return fail(GS_ERR_INVALID_ARG, "bad LiDAR array");
    if (lidar && !aligned(lidar, 16)) return fail(GS_ERR_INVALID_ARG, "lidar must be 16-byte aligned");
    return launch_depth_loss(ws, 2, depth_mean, alpha, depth_var, lidar, n_pts, loss, dL_dmean, dL_dvar,
                             (cudaStream_t)stream);
}

gs_status gs_image_l1(gs_workspace *ws, const float *rgb, const float *target, float *loss, float *dL_drgb,
                      void *stream) {
    if (!ws || !rgb || !target || !loss) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    return launch_image_l1(ws, rgb, target, loss, dL_drgb, (cudaStream_t)stream);
}

gs_status gs_image_l1_u8(gs_workspace *ws, const float *rgb, const uint8_t *target, float *loss,
                         float *dL_drgb, void *stream) {
    if (!ws || !rgb || !target || !loss) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    return launch_image_l1_u8(ws, rgb, target, loss, dL_drgb, (cudaStream_t)stream);
}

gs_status gs_image_loss(gs_workspace *ws, const float *rgb, const float *target, float lambda, float *loss,
                        float *dL_drgb, void *stream) {
    if (!ws || !rgb || !target || !loss) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (!(lambda >= 0.f && lambda <= 1.f)) return fail(GS_ERR_INVALID_ARG, "lambda must lie in [0, 1]");
    return launch_image_loss(ws, rgb, target, lambda, loss, dL_drgb, (cudaStream_t)stream);
}

gs_status gs_render_bwd(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams_dev,
                        const float *dL_drgb, const float *dL_ddepth, const float *dL_dalpha,
                        const gs_grads *out, void *stream) {
    if (!ws || !cams_dev || !dL_drgb || !out) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_gaussians(ws, g);
    if (r != GS_OK) return r;
    if (ws->n > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh))
        return fail(GS_ERR_INVALID_ARG, "a gradient pointer is NULL");
    if ((out->overwrite != 0 && out->overwrite != 1) || out->reserved != 0)
        return fail(GS_ERR_INVALID_ARG, "gs_grads.overwrite must be 0 or 1 and reserved 0");
    if (!ws->rendered) return fail(GS_ERR_STATE, "gs_render_bwd before gs_render_fwd");
    cudaStream_t s = (cudaStream_t)stream;
    r = launch_raster_bwd(ws, dL_drgb, dL_ddepth, dL_dalpha, false, nullptr, nullptr, s);
    if (r == GS_OK) r = launch_project_bwd(ws, g, cams_dev, out, s);
    return r;
}

gs_status gs_render_bwd_var(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams_dev,
                            const float *dL_drgb, const float *dL_ddepth, const float *dL_dalpha,
                            const float *dL_dmean, const float *dL_dvar, const gs_grads *out, void *stream) {
    if (!ws || !cams_dev || !dL_drgb || !out) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    gs_status r = check_gaussians(ws, g);
    if (r != GS_OK) return r;
    if (ws->n > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh))
        return fail(GS_ERR_INVALID_ARG, "a gradient pointer is NULL");
    if ((out->overwrite != 0 && out->overwrite != 1) || out->reserved != 0)
        return fail(GS_ERR_INVALID_ARG, "gs_grads.overwrite must be 0 or 1 and reserved 0");
    if (!ws->rendered_var)
        return fail(GS_ERR_STATE, "gs_render_bwd_var needs gs_render_fwd_var as the last forward");
    cudaStream_t s = (cudaStream_t)stream;
    r = launch_raster_bwd(ws, dL_drgb, dL_ddepth, dL_dalpha, true, dL_dmean, dL_dvar, s);
    if (r == GS_OK) r = launch_project_bwd(ws, g, cams_dev, out, s);
    return r;
}

gs_status gs_workspace_status(gs_workspace *ws, void *stream, int64_t *n_instances, int64_t *n_visible) {
    if (!ws) return fail(GS_ERR_INVALID_ARG, "NULL workspace");
    DevState h{};
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(&h, ws->st, sizeof(DevState), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("status: ") + cudaGetErrorString(e));
    if (n_instances) *n_instances = (int64_t)h.n_inst_needed;
    if (n_visible) *n_visible = (int64_t)h.n_vis;
    if (h.flags & kFlagTimeout) return fail(GS_ERR_TIMEOUT, "a device-side wait for a TMA copy timed out");
    return (h.flags & kFlagCapacity) ? GS_ERR_CAPACITY : GS_OK;
}

gs_status gs_workspace_info(gs_workspace *ws, int64_t *info, int32_t n_info) {
    if (!ws || !info || n_info < 0) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    int64_t v[8] = {ws->n_pairs, ws->n_tiles, ws->n_pix,   ws->inst_cap,
                    ws->n_views, ws->n,       (int64_t)ws->bytes, ws->kernel_launches};
    for (int i = 0; i < n_info && i < 8; ++i) info[i] = v[i];
    return GS_OK;
}

gs_status gs_workspace_copy(gs_workspace *ws, int32_t which, void *dst, int64_t *bytes, void *stream) {
    if (!ws || !bytes) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    const void *src = nullptr;
    int64_t nb = 0;
    switch (which) {
        case 0: src = ws->rec; nb = ws->n_pairs * 48; break;
        case 1: src = ws->pkey; nb = ws->n_pairs * 4; break;
        case 2: src = ws->rect; nb = ws->n_pairs * 8; break;
        case 3: src = ws->inst_tile; nb = ws->inst_cap * 4; break;
        case 4: src = ws->inst_val; nb = ws->inst_cap * 4; break;
        case 5: src = ws->ranges; nb = ws->n_tiles * 8; break;
        case 6: src = ws->last; nb = ws->n_pix * 4; break;
        case 7: src = ws->tfin; nb = ws->n_pix * 4; break;
        case 8: src = ws->g2d; nb = ws->n_pairs * 40; break;
        case 9: src = ws->vstat; nb = ws->n_pix * 16; break;
        default: return fail(GS_ERR_INVALID_ARG, "unknown buffer");
    }
    if (!dst) {
        *bytes = nb;
        return GS_OK;
    }
    if (*bytes != nb) return fail(GS_ERR_INVALID_ARG, "byte count mismatch");
    if (nb == 0) return GS_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)nb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
    return GS_OK;
}

}  // extern "C"
