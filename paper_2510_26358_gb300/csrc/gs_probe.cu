// Measurement kernels: the arithmetic rates the fragment roofline is quoted
// against, and the fragment counts that turn a raster kernel's time into an
// achieved rate.  Neither runs inside the mapping step.
//
// gs_alu_probe: every thread runs `iters` rounds over eight independent
// dependency chains of one instruction kind (FP32 FMA, packed f32x2 FMA, MUFU
// ex2, MUFU rcp), so that a launch of a few blocks per SM is bound by that
// pipe's issue rate alone.  The host times the launch (CUDA events) and
// divides the operations by the time.
//
// gs_workspace_fragment_counts: after a forward, walks every pixel's list up
// to the count the forward kept (the entries the backward replays), with the
// rasterisers' own fragment functions, and counts
//   [0] (pixel, entry) pairs walked      = sum over pixels of that count,
//   [1] (pixel, entry) pairs blended     (alpha >= alpha_min among them),
//   [2] (tile, entry) pairs walked       = sum over tiles of the longest count,
//   [3] (tile, entry) pairs with a blend (any pixel of the tile blends it).
// [2] and [3] are the work units of a backward that gives a tile to one warp.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kProbeChains = 8;

template <int KIND>
__global__ void __launch_bounds__(256) k_alu_probe(int iters, float seed, float *sink) {
    const float s = seed + 1e-7f * (float)threadIdx.x;
    if (KIND == 1) {
        f2 a[kProbeChains];
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = f2_pack(s + c, s - c);
        const f2 m = f2_bcast(0.999f), b = f2_bcast(1e-3f);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) a[c] = f2_fma(a[c], m, b);
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) acc += f2_lo(a[c]) + f2_hi(a[c]);
        if (acc == 12345.f) *sink = acc;  // never true; keeps the chains live
        return;
    }
    float a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = s + 0.01f * c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            if (KIND == 0) a[c] = __fmaf_rn(a[c], 0.999f, 1e-3f);
            if (KIND == 2) a[c] = ex2_approx(-a[c]);          // stays in [0.5, 1]
            if (KIND == 3) a[c] = rcp_approx(a[c] + 1.f);     // tends to the golden ratio's inverse
                                                              // (x -> 1/x -> x would fold)
        }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc += a[c];
    if (acc == 12345.f) *sink = acc;
}

// One block per tile, one thread per pixel of the tile.
__global__ void k_count_fragments(const ViewInfo *views, int n_views, Consts c, const float4 *rec,
                                  const uint32_t *vals, const uint2 *ranges, const uint32_t *last,
                                  unsigned long long *out) {
    __shared__ uint32_t s_max;
    __shared__ unsigned long long s_cnt[2];
    const int tile = blockIdx.x;
    const int v = view_of_tile(views, n_views, tile);
    const ViewInfo vi = views[v];
    const int lt = tile - vi.tile_off;
    const int px = (lt % vi.ntx) * c.tile_w + threadIdx.x % c.tile_w;
    const int py = (lt / vi.ntx) * c.tile_h + threadIdx.x / c.tile_w;
    const bool inside = px < vi.W && py < vi.H;
    const uint32_t n = inside ? last[vi.pix_off + (int64_t)py * vi.W + px] : 0u;
    if (threadIdx.x == 0) {
        s_max = 0u;
        s_cnt[0] = s_cnt[1] = 0ull;
    }
    __syncthreads();
    atomicMax(&s_max, n);
    __syncthreads();
    const uint32_t nmax = s_max;
    const uint2 rg = ranges[tile];
    unsigned long long blended = 0ull, active = 0ull;
    for (uint32_t j = 0; j < nmax; ++j) {
        bool bl = false;
        if (j < n) {
            const uint32_t pair = vals[rg.x + j];
            float4 a, b;
            stage_record(rec[3 * (size_t)pair], rec[3 * (size_t)pair + 1], a, b);
            float dxi, u1, t1, t2, dyi;
            frag_column(a, b, (float)px, dxi, u1);
            bl = frag_pixel(a, b, u1, (float)py, t1, t2, dyi) >= c.log2_alpha_min;
        }
        blended += bl;
        active += __syncthreads_or(bl) ? 1ull : 0ull;
    }
    atomicAdd(&s_cnt[0], (unsigned long long)n);
    atomicAdd(&s_cnt[1], blended);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(out + 0, s_cnt[0]);
        atomicAdd(out + 1, s_cnt[1]);
        atomicAdd(out + 2, (unsigned long long)nmax);
        atomicAdd(out + 3, active);
    }
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_alu_probe(int32_t kind, int32_t blocks, int32_t iters, float *sink, void *stream) {
    using namespace gs;
    if (kind < 0 || kind > 3 || blocks < 1 || iters < 1 || !sink) {
        set_last_error("gs_alu_probe: kind 0..3, blocks >= 1, iters >= 1 and a sink are required");
        return GS_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const float seed = 0.5f;
    switch (kind) {
        case 0: k_alu_probe<0><<<blocks, 256, 0, s>>>(iters, seed, sink); break;
        case 1: k_alu_probe<1><<<blocks, 256, 0, s>>>(iters, seed, sink); break;
        case 2: k_alu_probe<2><<<blocks, 256, 0, s>>>(iters, seed, sink); break;
        default: k_alu_probe<3><<<blocks, 256, 0, s>>>(iters, seed, sink); break;
    }
    return check_launch("gs_alu_probe");
}

extern "C" gs_status gs_workspace_fragment_counts(gs_workspace *ws, int64_t *counts, void *stream) {
    using namespace gs;
    if (!ws || !counts) {
        set_last_error("gs_workspace_fragment_counts: NULL argument");
        return GS_ERR_INVALID_ARG;
    }
    if (!ws->rendered) {
        set_last_error("gs_workspace_fragment_counts before gs_render_fwd");
        return GS_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *dev = ws->st->frag_count;
    cudaError_t e = cudaMemsetAsync(dev, 0, 4 * sizeof(unsigned long long), s);
    if (e == cudaSuccess && ws->n_tiles > 0) {
        k_count_fragments<<<(unsigned)ws->n_tiles, ws->cfg.tile_w * ws->cfg.tile_h, 0, s>>>(
            ws->views, ws->n_views, ws->consts, ws->rec, ws->inst_val, ws->ranges, ws->last, dev);
        e = cudaGetLastError();
    }
    unsigned long long h[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, dev, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(std::string("gs_workspace_fragment_counts: ") + cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    for (int i = 0; i < 4; ++i) counts[i] = (int64_t)h[i];
    return GS_OK;
}
