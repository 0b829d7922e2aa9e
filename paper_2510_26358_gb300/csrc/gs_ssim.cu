// SSIM term of Eq. (6): the structural similarity of the rendered image and
// the target, per channel of every view, with an 11x11 Gaussian window of
// sigma 1.5 (normalised weights), zero padding outside the image and
// C1 = 0.01^2, C2 = 0.03^2.  Per pixel q, with window sums mu_x = E[x],
// mu_y = E[y], s_xx = E[x^2] - mu_x^2, s_yy = E[y^2] - mu_y^2 and
// s_xy = E[xy] - mu_x mu_y,
//   S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)).
//
// Forward: one CTA per 32x16 output tile of one channel plane stages the tile
// and its 5-pixel halo of x and y in shared memory, filters the five products
// horizontally, then vertically, and writes S's partial derivatives w.r.t.
// the three window sums that depend on x,
//   d1 = dS/dE[x],  d2 = dS/dE[x^2],  d12 = dS/dE[xy],
// plus a per-CTA sum of S (double).  Backward: the same tiling filters
// (d1, d2, d12) with the same window (the adjoint of a zero-padded symmetric
// filter is itself) and adds scale * (G*d1 + 2 x G*d2 + y G*d12) to dL/dx.
//
// Precision: E[x^2] - mu_x^2 cancels in float where the image is smooth
// (variances of 1e-5 against E[x^2] ~ 0.3, which cost 1e-4 of 1 - SSIM near
// SSIM = 1).  The forward therefore filters x' = x - c_x and y' = y - c_y
// (inside the image; the padding stays 0), with c the tile's first pixel.
// With W = sum of the window weights inside the image at the output pixel
// and M' = E[x'],
//   mu_x = M'_x + c_x W,
//   s_xx = E[x'^2] - M'_x^2 + (1 - W)(2 c_x M'_x + c_x^2 W),
//   s_xy = E[x'y'] - M'_x M'_y + (1 - W)(c_y M'_x + c_x M'_y + c_x c_y W),
// identities of the zero-padded sums whose correction vanishes in the
// interior (W = 1).
#include "gs_internal.cuh"

#include <cmath>

namespace gs {
namespace {

constexpr int TX = 32, TY = 16, R = 5, K = 2 * R + 1;
constexpr int IW = TX + 2 * R, IH = TY + 2 * R;
constexpr int NT = 256, ROWS = NT / TX;  // 8 output rows per pass, 2 passes
constexpr float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;

struct SsimArgs {
    const ViewInfo *views;
    int32_t n_views;
    const float *x, *y;  // planar images (rendered, target)
    float *dmap;         // [3][n_elem] partials, nullptr: no backward
    float *grad;         // dL/dx, accumulated
    double *part;        // [grid] per-CTA sums of S
    int64_t n_elem;
    float scale;         // gradient scale of S (backward)
    float g[K];          // window weights
};

struct PlaneTile {
    int64_t base;  // element offset of the channel plane
    int W, H, x0, y0;
};

// CTA b -> (view, channel, tile); views in order, channels in order, tiles
// row-major.  The grid holds exactly sum_v 3 ntx(v) nty(v) CTAs.
__device__ __forceinline__ PlaneTile locate(const SsimArgs &A, int b) {
    PlaneTile p{0, 0, 0, 0, 0};
    for (int v = 0; v < A.n_views; ++v) {
        const ViewInfo vi = A.views[v];
        const int ntx = (vi.W + TX - 1) / TX, nty = (vi.H + TY - 1) / TY;
        const int per_plane = ntx * nty;
        if (b < 3 * per_plane) {
            const int ch = b / per_plane, t = b % per_plane;
            p.base = 3 * (int64_t)vi.pix_off + (int64_t)ch * vi.W * vi.H;
            p.W = vi.W;
            p.H = vi.H;
            p.x0 = (t % ntx) * TX;
            p.y0 = (t / ntx) * TY;
            return p;
        }
        b -= 3 * per_plane;
    }
    return p;
}

__device__ __forceinline__ double block_sum(double v, double *sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < NT / 32; ++i) t += sm[i];
    return t;
}

__global__ void __launch_bounds__(NT) k_ssim_fwd(SsimArgs A) {
    __shared__ float sx[IH][IW], sy[IH][IW];
    __shared__ float sh[5][IH][TX];
    __shared__ double red[NT / 32];
    const PlaneTile P = locate(A, blockIdx.x);
    const float *x = A.x + P.base, *y = A.y + P.base;
    const int tid = threadIdx.x;
    // shift: the tile's first pixel, always inside the image
    const float cx = x[(int64_t)P.y0 * P.W + P.x0], cy = y[(int64_t)P.y0 * P.W + P.x0];
    for (int i = tid; i < IH * IW; i += NT) {
        const int r = i / IW, c = i % IW;
        const int gx = P.x0 - R + c, gy = P.y0 - R + r;
        const bool in = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
        const int64_t o = (int64_t)gy * P.W + gx;
        sx[r][c] = in ? x[o] - cx : 0.f;
        sy[r][c] = in ? y[o] - cy : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < IH * TX; i += NT) {
        const int r = i / TX, c = i % TX;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float u = sx[r][c + k], w = sy[r][c + k];
            const float gu = A.g[k] * u, gw = A.g[k] * w;
            a += gu;
            b += gw;
            aa = __fmaf_rn(gu, u, aa);
            bb = __fmaf_rn(gw, w, bb);
            ab = __fmaf_rn(gu, w, ab);
        }
        sh[0][r][c] = a;
        sh[1][r][c] = b;
        sh[2][r][c] = aa;
        sh[3][r][c] = bb;
        sh[4][r][c] = ab;
    }
    __syncthreads();
    const int tx = tid % TX, ty = tid / TX;
    double acc = 0.0;
#pragma unroll
    for (int pass = 0; pass < TY / ROWS; ++pass) {
        const int oy = ty + pass * ROWS;
        const int gx = P.x0 + tx, gy = P.y0 + oy;
        if (gx >= P.W || gy >= P.H) continue;
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        float wx = 0.f, wy = 0.f;  // window weight inside the image, per axis
#pragma unroll
        for (int j = 0; j < K; ++j) {
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] = __fmaf_rn(A.g[j], sh[q][oy + j][tx], m[q]);
            const int ix = gx - R + j, iy = gy - R + j;
            wx += ix >= 0 && ix < P.W ? A.g[j] : 0.f;
            wy += iy >= 0 && iy < P.H ? A.g[j] : 0.f;
        }
        const float W = wx * wy, cw = 1.f - W;
        const float px = m[0], py = m[1];  // E[x'], E[y']
        const float mx = __fmaf_rn(cx, W, px), my = __fmaf_rn(cy, W, py);
        const float sxx = (m[2] - px * px) + cw * cx * (2.f * px + cx * W);
        const float syy = (m[3] - py * py) + cw * cy * (2.f * py + cy * W);
        const float sxy = (m[4] - px * py) + cw * (cy * px + cx * py + cx * cy * W);
        const float Aa = 2.f * mx * my + C1, B = 2.f * sxy + C2;
        const float Cc = mx * mx + my * my + C1, D = sxx + syy + C2;
        const float iC = 1.f / Cc, iD = 1.f / D;
        const float S = Aa * B * iC * iD;
        acc += (double)S;
        if (A.dmap) {
            const float dsxx = -S * iD;                                       // -A B / (Cc D^2)
            const float dsxy = 2.f * Aa * iC * iD;                            // 2 A / (Cc D)
            const float dmu = 2.f * B * iD * (my * Cc - mx * Aa) * iC * iC;   // dS/dmu_x, s fixed
            const float d1 = dmu - 2.f * mx * dsxx - my * dsxy;
            const int64_t e = P.base + (int64_t)gy * P.W + gx;
            A.dmap[e] = d1;
            A.dmap[A.n_elem + e] = dsxx;
            A.dmap[2 * A.n_elem + e] = dsxy;
        }
    }
    const double t = block_sum(acc, red);
    if (tid == 0) A.part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_ssim_bwd(SsimArgs A) {
    __shared__ float sd[3][IH][IW];
    __shared__ float sh[3][IH][TX];
    const PlaneTile P = locate(A, blockIdx.x);
    const int tid = threadIdx.x;
    for (int i = tid; i < IH * IW; i += NT) {
        const int r = i / IW, c = i % IW;
        const int gx = P.x0 - R + c, gy = P.y0 - R + r;
        const bool in = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
        const int64_t e = P.base + (int64_t)gy * P.W + gx;
#pragma unroll
        for (int q = 0; q < 3; ++q) sd[q][r][c] = in ? A.dmap[q * A.n_elem + e] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < IH * TX; i += NT) {
        const int r = i / TX, c = i % TX;
        float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q) s[q] = __fmaf_rn(A.g[k], sd[q][r][c + k], s[q]);
#pragma unroll
        for (int q = 0; q < 3; ++q) sh[q][r][c] = s[q];
    }
    __syncthreads();
    const int tx = tid % TX, ty = tid / TX;
#pragma unroll
    for (int pass = 0; pass < TY / ROWS; ++pass) {
        const int oy = ty + pass * ROWS;
        const int gx = P.x0 + tx, gy = P.y0 + oy;
        if (gx >= P.W || gy >= P.H) continue;
        float f[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int q = 0; q < 3; ++q) f[q] = __fmaf_rn(A.g[j], sh[q][oy + j][tx], f[q]);
        const int64_t e = P.base + (int64_t)gy * P.W + gx;
        const float xv = A.x[e], yv = A.y[e];
        A.grad[e] += A.scale * (f[0] + 2.f * xv * f[1] + yv * f[2]);
    }
}

}  // namespace

int64_t ssim_tiles(const std::vector<ViewInfo> &views) {
    int64_t n = 0;
    for (const ViewInfo &v : views) n += 3 * (int64_t)((v.W + TX - 1) / TX) * ((v.H + TY - 1) / TY);
    return n;
}

gs_status launch_ssim(gs_workspace *ws, const float *rgb, const float *target, float grad_scale, float *dL_drgb,
                      cudaStream_t s) {
    SsimArgs A{};
    A.views = ws->views;
    A.n_views = ws->n_views;
    A.x = rgb;
    A.y = target;
    A.dmap = dL_drgb && grad_scale != 0.f ? ws->ssim_d : nullptr;
    A.grad = dL_drgb;
    A.part = ws->ssim_part;
    A.n_elem = 3 * ws->n_pix;
    A.scale = grad_scale;
    double g[K], sum = 0.0;
    for (int i = 0; i < K; ++i) {
        g[i] = std::exp(-(double)((i - R) * (i - R)) / (2.0 * 1.5 * 1.5));
        sum += g[i];
    }
    for (int i = 0; i < K; ++i) A.g[i] = (float)(g[i] / sum);
    const int grid = (int)ws->n_ssim_tiles;
    if (grid == 0) return GS_OK;
    StageTimer timer(ws, GS_STAGE_IMAGE_SSIM, s);
    ++ws->kernel_launches;
    k_ssim_fwd<<<grid, NT, 0, s>>>(A);
    gs_status r = check_launch("ssim_fwd");
    if (r != GS_OK || !dL_drgb || grad_scale == 0.f) return r;
    ++ws->kernel_launches;
    k_ssim_bwd<<<grid, NT, 0, s>>>(A);
    return check_launch("ssim_bwd");
}

}  // namespace gs
