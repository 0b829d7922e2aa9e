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
// plus a per-CTA sum of 1 - S (double).  Backward: the same tiling filters
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
//
// Views whose width is a multiple of 4 (at most kTmaViews of them) stage the
// halo tiles with TMA: one thread issues cp.async.bulk.tensor loads of a
// 48 x 42 box starting at (x0 - 8, y0 - 5) (x a multiple of 4 floats, as the
// copy requires) that complete on an mbarrier; the copy's out-of-bounds zero
// fill is the zero padding.  The wait is bounded: on time-out the kernel sets
// a flag of the workspace state and leaves the tile.  Other layouts use the
// same kernels with per-thread staging loads.
#include "gs_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

namespace gs {
namespace {

constexpr int TX = 32, TY = 32, R = 5, K = 2 * R + 1;
constexpr int IW = TX + 2 * R, IH = TY + 2 * R;
constexpr int SW = IW + 1;  // staged row stride: odd, so the blocked row reads hit distinct banks
constexpr int HW = TX + 1;  // filtered row stride
constexpr int NT = 256;
constexpr int HB = 4;                     // horizontal outputs per thread
constexpr int HITEMS = IH * (TX / HB);    // 208 row segments per tile
constexpr int VB = 4;                     // vertical outputs per thread (consecutive rows)
constexpr int SLOADS = (IH * IW + NT - 1) / NT;  // staged values per thread and map
static_assert(TY == VB * (NT / TX), "one vertical pass covers the tile");
static_assert(HITEMS <= 2 * NT, "two horizontal passes cover the tile");
constexpr float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;

struct SsimArgs {
    const ViewInfo *views;
    int32_t n_views;
    const float *x, *y;  // planar images (rendered, target)
    float *dmap;         // [3][n_elem] partials, nullptr: no backward
    float *grad;         // dL/dx, accumulated
    double *part;        // [grid] per-CTA sums of 1 - S
    int64_t n_elem;
    float scale;         // gradient scale of S (backward)
    float gsum;          // sum of the 11 weights (the in-image weight of an interior axis)
    float g[K];          // window weights
    uint32_t *flags;     // workspace state flags (TMA wait time-out)
    uint64_t wait_ns;    // limit of a TMA wait
};

struct PlaneTile {
    int64_t base;  // element offset of the channel plane
    int W, H, x0, y0;
    int v, ch;
};

// TMA path: per view, 3-D maps (x, y, channel) of the two images and a 4-D map
// (x, y, channel, partial) of the backward's three partial maps.
constexpr int kTmaViews = 8;
constexpr int BW = IW + 6;    // box width: columns x0 - 8 .. x0 + 39
constexpr int BOFF = 3;       // halo column c lives at box column c + BOFF
struct SsimTma {
    CUtensorMap x[kTmaViews], y[kTmaViews], d[kTmaViews];
};
constexpr uint64_t kTmaWaitNs = 1000000000ull;  // 1 s for a tile's copies

// CTA b -> (view, channel, tile); views in order, channels in order, tiles
// row-major.  The grid holds exactly sum_v 3 ntx(v) nty(v) CTAs.
__device__ __forceinline__ PlaneTile locate(const SsimArgs &A, int b) {
    PlaneTile p{0, 0, 0, 0, 0, 0, 0};
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
            p.v = v;
            p.ch = ch;
            return p;
        }
        b -= 3 * per_plane;
    }
    return p;
}

// Sum of the window weights whose tap lands inside [0, n) for an output at i.
__device__ __forceinline__ float inside_weight(const SsimArgs &A, int i, int n) {
    if (i >= R && i < n - R) return A.gsum;
    float w = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int t = i - R + k;
        w += t >= 0 && t < n ? A.g[k] : 0.f;
    }
    return w;
}

// Horizontal pass of the forward: row segment `item` (row r, columns
// c0..c0+HB-1) of x', y', x'^2, y'^2 and x'y' from HB + 2R staged x', y'.
__device__ __forceinline__ void horizontal_fwd(const SsimArgs &A, const float (*src)[IH][SW],
                                               float (*dst)[IH][HW], int item) {
    const int r = item / (TX / HB), c0 = (item % (TX / HB)) * HB;
    float u[HB + 2 * R], w[HB + 2 * R], uu[HB + 2 * R], ww[HB + 2 * R], uw[HB + 2 * R];
#pragma unroll
    for (int j = 0; j < HB + 2 * R; ++j) {
        u[j] = src[0][r][c0 + j];
        w[j] = src[1][r][c0 + j];
        uu[j] = u[j] * u[j];
        ww[j] = w[j] * w[j];
        uw[j] = u[j] * w[j];
    }
#pragma unroll
    for (int o = 0; o < HB; ++o) {
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            a = __fmaf_rn(A.g[k], u[o + k], a);
            b = __fmaf_rn(A.g[k], w[o + k], b);
            aa = __fmaf_rn(A.g[k], uu[o + k], aa);
            bb = __fmaf_rn(A.g[k], ww[o + k], bb);
            ab = __fmaf_rn(A.g[k], uw[o + k], ab);
        }
        dst[0][r][c0 + o] = a;
        dst[1][r][c0 + o] = b;
        dst[2][r][c0 + o] = aa;
        dst[3][r][c0 + o] = bb;
        dst[4][r][c0 + o] = ab;
    }
}

// Horizontal pass of the backward over NQ staged maps.
template <int NQ>
__device__ __forceinline__ void horizontal(const SsimArgs &A, const float (*src)[IH][SW], float (*dst)[IH][HW],
                                           int item) {
    const int r = item / (TX / HB), c0 = (item % (TX / HB)) * HB;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float v[HB + 2 * R];
#pragma unroll
        for (int j = 0; j < HB + 2 * R; ++j) v[j] = src[q][r][c0 + j];
#pragma unroll
        for (int o = 0; o < HB; ++o) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = __fmaf_rn(A.g[k], v[o + k], acc);
            dst[q][r][c0 + o] = acc;
        }
    }
}

// Vertical pass, SSIM, its partials and the tile's sum of 1 - S (shared by
// both staging paths).
__device__ __forceinline__ void ssim_epilogue(const SsimArgs &A, const PlaneTile &P, const float (*sh)[IH][HW],
                                              float cx, float cy, int lx, int ly, double *red) {
    const int gx = P.x0 + lx, oy0 = VB * ly;
    float m[VB][5];
#pragma unroll
    for (int b = 0; b < VB; ++b)
#pragma unroll
        for (int q = 0; q < 5; ++q) m[b][q] = 0.f;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        float v[K + VB - 1];
#pragma unroll
        for (int j = 0; j < K + VB - 1; ++j) v[j] = sh[q][oy0 + j][lx];
#pragma unroll
        for (int b = 0; b < VB; ++b)
#pragma unroll
            for (int k = 0; k < K; ++k) m[b][q] = __fmaf_rn(A.g[k], v[b + k], m[b][q]);
    }
    float dsum = 0.f;  // sum of 1 - S over this thread's pixels
    const float wx = inside_weight(A, gx, P.W);
#pragma unroll
    for (int b = 0; b < VB; ++b) {
        const int gy = P.y0 + oy0 + b;
        if (gx >= P.W || gy >= P.H) continue;
        const float W = wx * inside_weight(A, gy, P.H), cw = 1.f - W;
        const float px = m[b][0], py = m[b][1];  // E[x'], E[y']
        const float mx = __fmaf_rn(cx, W, px), my = __fmaf_rn(cy, W, py);
        const float sxx = (m[b][2] - px * px) + cw * cx * (2.f * px + cx * W);
        const float syy = (m[b][3] - py * py) + cw * cy * (2.f * py + cy * W);
        const float sxy = (m[b][4] - px * py) + cw * (cy * px + cx * py + cx * cy * W);
        const float Aa = 2.f * mx * my + C1, B = 2.f * sxy + C2;
        const float Cc = mx * mx + my * my + C1, D = sxx + syy + C2;
        const float iC = 1.f / Cc, iD = 1.f / D;
        const float S = Aa * B * iC * iD;
        // 1 - S as (Cc D - A B) / (Cc D): keeps its relative precision near S = 1
        dsum += __fmaf_rn(Cc, D, -Aa * B) * iC * iD;
        if (A.dmap) {
            const float dsxx = -S * iD;                                      // -A B / (Cc D^2)
            const float dsxy = 2.f * Aa * iC * iD;                           // 2 A / (Cc D)
            const float dmu = 2.f * B * iD * (my * Cc - mx * Aa) * iC * iC;  // dS/dmu_x, s fixed
            const float d1 = dmu - 2.f * mx * dsxx - my * dsxy;
            const int64_t e = P.base + (int64_t)gy * P.W + gx;
            A.dmap[e] = d1;
            A.dmap[A.n_elem + e] = dsxx;
            A.dmap[2 * A.n_elem + e] = dsxy;
        }
    }
    // warp sum in float (at most 64 terms), then the 8 warps in double
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if (lx == 0) red[ly] = (double)dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < NT / 32; ++i) t += red[i];
        A.part[blockIdx.x] = t;
    }
}

// Vertical pass of the backward and the gradient (shared by both staging paths).
// The thread's VB output values of x, y and the gradient, loaded when the
// kernel starts so that their latency hides behind the staging and the
// filters (0 outside the image; those are not written).
struct BwdOut {
    float x[VB], y[VB], g[VB];
};
__device__ __forceinline__ BwdOut ssim_bwd_prefetch(const SsimArgs &A, const PlaneTile &P, int lx, int ly) {
    BwdOut o;
    const int gx = P.x0 + lx, oy0 = VB * ly;
#pragma unroll
    for (int b = 0; b < VB; ++b) {
        const int gy = P.y0 + oy0 + b;
        const bool in = gx < P.W && gy < P.H;
        const int64_t e = P.base + (int64_t)gy * P.W + gx;
        o.x[b] = in ? A.x[e] : 0.f;
        o.y[b] = in ? A.y[e] : 0.f;
        o.g[b] = in ? A.grad[e] : 0.f;
    }
    return o;
}

__device__ __forceinline__ void ssim_bwd_epilogue(const SsimArgs &A, const PlaneTile &P, const float (*sh)[IH][HW],
                                                  int lx, int ly, const BwdOut &o) {
    const int gx = P.x0 + lx, oy0 = VB * ly;
    float f[VB][3];
#pragma unroll
    for (int b = 0; b < VB; ++b)
#pragma unroll
        for (int q = 0; q < 3; ++q) f[b][q] = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float v[K + VB - 1];
#pragma unroll
        for (int j = 0; j < K + VB - 1; ++j) v[j] = sh[q][oy0 + j][lx];
#pragma unroll
        for (int b = 0; b < VB; ++b)
#pragma unroll
            for (int k = 0; k < K; ++k) f[b][q] = __fmaf_rn(A.g[k], v[b + k], f[b][q]);
    }
#pragma unroll
    for (int b = 0; b < VB; ++b) {
        const int gy = P.y0 + oy0 + b;
        if (gx >= P.W || gy >= P.H) continue;
        const int64_t e = P.base + (int64_t)gy * P.W + gx;
        A.grad[e] = o.g[b] + A.scale * (f[b][0] + 2.f * o.x[b] * f[b][1] + o.y[b] * f[b][2]);
    }
}

__global__ void __launch_bounds__(NT) k_ssim_fwd(SsimArgs A) {
    __shared__ float st[2][IH][SW];  // staged x', y'
    __shared__ float sh[5][IH][HW];
    __shared__ double red[NT / 32];
    const PlaneTile P = locate(A, blockIdx.x);
    const float *x = A.x + P.base, *y = A.y + P.base;
    const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5;
    // shift: the tile's first pixel, always inside the image
    const float cx = x[(int64_t)P.y0 * P.W + P.x0], cy = y[(int64_t)P.y0 * P.W + P.x0];
    {
        // every load of the thread is issued before the first shared store
        float vx[SLOADS], vy[SLOADS];
#pragma unroll
        for (int k = 0; k < SLOADS; ++k) {
            const int i = tid + k * NT, r = i / IW, c = i % IW;
            const int gx = P.x0 - R + c, gy = P.y0 - R + r;
            const bool in = i < IH * IW && gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
            const int64_t o = (int64_t)gy * P.W + gx;
            vx[k] = in ? x[o] - cx : 0.f;
            vy[k] = in ? y[o] - cy : 0.f;
        }
#pragma unroll
        for (int k = 0; k < SLOADS; ++k) {
            const int i = tid + k * NT;
            if (i < IH * IW) {
                st[0][i / IW][i % IW] = vx[k];
                st[1][i / IW][i % IW] = vy[k];
            }
        }
    }
    __syncthreads();
    for (int item = tid; item < HITEMS; item += NT) horizontal_fwd(A, st, sh, item);
    __syncthreads();
    ssim_epilogue(A, P, sh, cx, cy, lx, ly, red);
}

__global__ void __launch_bounds__(NT) k_ssim_bwd(SsimArgs A) {
    __shared__ float st[3][IH][SW];
    __shared__ float sh[3][IH][HW];
    const PlaneTile P = locate(A, blockIdx.x);
    const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5;
    const BwdOut out = ssim_bwd_prefetch(A, P, lx, ly);
    {
        float v[3][SLOADS];
#pragma unroll
        for (int k = 0; k < SLOADS; ++k) {
            const int i = tid + k * NT, r = i / IW, c = i % IW;
            const int gx = P.x0 - R + c, gy = P.y0 - R + r;
            const bool in = i < IH * IW && gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
            const int64_t e = P.base + (int64_t)gy * P.W + gx;
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q][k] = in ? A.dmap[q * A.n_elem + e] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < SLOADS; ++k) {
            const int i = tid + k * NT;
            if (i < IH * IW) {
#pragma unroll
                for (int q = 0; q < 3; ++q) st[q][i / IW][i % IW] = v[q][k];
            }
        }
    }
    __syncthreads();
    for (int item = tid; item < HITEMS; item += NT) horizontal<3>(A, st, sh, item);
    __syncthreads();
    ssim_bwd_epilogue(A, P, sh, lx, ly, out);
}


// ---------------------------------------------------------------------------
// TMA staging
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the tile's copies (phase 0) for at most limit_ns.  On time-out it
// sets the flag, waits a tenth of that again so that copies still in flight
// land before the CTA leaves, and returns false.
__device__ __forceinline__ bool tma_wait(uint64_t *bar, uint32_t *flags, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, 0))
        if (global_ns() - t0 > limit_ns) {
            if (threadIdx.x == 0) atomicOr(flags, kFlagTimeout);
            const uint64_t t1 = global_ns();
            while (!mbar_try_wait(bar, 0))
                if (global_ns() - t1 > limit_ns / 10) break;
            return false;
        }
    return true;
}

// Self-test of the bounded wait: a barrier that expects bytes no copy will
// ever deliver (none is issued), so the wait must run out and set the flag.
__global__ void k_wait_selftest(uint32_t *flags, uint64_t limit_ns, int32_t *result) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        mbar_expect_tx(&bar, 16u);
    }
    __syncthreads();
    const bool done = tma_wait(&bar, flags, limit_ns);
    __syncthreads();
    if (threadIdx.x == 0) *result = done ? 0 : 1;
}

__global__ void __launch_bounds__(NT) k_ssim_fwd_tma(SsimArgs A, const __grid_constant__ SsimTma T) {
    __shared__ __align__(128) float tx_[IH][BW];
    __shared__ __align__(128) float ty_[IH][BW];
    __shared__ float sh[5][IH][HW];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double red[NT / 32];
    const PlaneTile P = locate(A, blockIdx.x);
    const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5;
    if (tid == 0) {
        mbar_init(&bar);
        mbar_expect_tx(&bar, 2u * IH * BW * sizeof(float));
        tma_load_3d(&tx_[0][0], &T.x[P.v], P.x0 - R - BOFF, P.y0 - R, P.ch, &bar);
        tma_load_3d(&ty_[0][0], &T.y[P.v], P.x0 - R - BOFF, P.y0 - R, P.ch, &bar);
    }
    __syncthreads();
    if (!tma_wait(&bar, A.flags, A.wait_ns)) return;
    // shift: the tile's first pixel (halo row R, column R)
    const float cx = tx_[R][R + BOFF], cy = ty_[R][R + BOFF];
    for (int item = tid; item < HITEMS; item += NT) {
        const int r = item / (TX / HB), c0 = (item % (TX / HB)) * HB;
        const int gy = P.y0 - R + r;
        const bool row_in = gy >= 0 && gy < P.H;
        float u[HB + 2 * R], w[HB + 2 * R], uu[HB + 2 * R], ww[HB + 2 * R], uw[HB + 2 * R];
#pragma unroll
        for (int j = 0; j < HB + 2 * R; ++j) {
            const int gx = P.x0 - R + c0 + j;
            const bool in = row_in && gx >= 0 && gx < P.W;
            u[j] = in ? tx_[r][c0 + j + BOFF] - cx : 0.f;
            w[j] = in ? ty_[r][c0 + j + BOFF] - cy : 0.f;
            uu[j] = u[j] * u[j];
            ww[j] = w[j] * w[j];
            uw[j] = u[j] * w[j];
        }
#pragma unroll
        for (int o = 0; o < HB; ++o) {
            float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                a = __fmaf_rn(A.g[k], u[o + k], a);
                b = __fmaf_rn(A.g[k], w[o + k], b);
                aa = __fmaf_rn(A.g[k], uu[o + k], aa);
                bb = __fmaf_rn(A.g[k], ww[o + k], bb);
                ab = __fmaf_rn(A.g[k], uw[o + k], ab);
            }
            sh[0][r][c0 + o] = a;
            sh[1][r][c0 + o] = b;
            sh[2][r][c0 + o] = aa;
            sh[3][r][c0 + o] = bb;
            sh[4][r][c0 + o] = ab;
        }
    }
    __syncthreads();
    ssim_epilogue(A, P, sh, cx, cy, lx, ly, red);
}

__global__ void __launch_bounds__(NT) k_ssim_bwd_tma(SsimArgs A, const __grid_constant__ SsimTma T) {
    __shared__ __align__(128) float sd[3][IH][BW];
    __shared__ float sh[3][IH][HW];
    __shared__ __align__(8) uint64_t bar;
    const PlaneTile P = locate(A, blockIdx.x);
    const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5;
    if (tid == 0) {
        mbar_init(&bar);
        mbar_expect_tx(&bar, 3u * IH * BW * sizeof(float));
#pragma unroll
        for (int q = 0; q < 3; ++q) tma_load_4d(&sd[q][0][0], &T.d[P.v], P.x0 - R - BOFF, P.y0 - R, P.ch, q, &bar);
    }
    __syncthreads();
    const BwdOut out = ssim_bwd_prefetch(A, P, lx, ly);
    if (!tma_wait(&bar, A.flags, A.wait_ns)) return;
    for (int item = tid; item < HITEMS; item += NT) {
        const int r = item / (TX / HB), c0 = (item % (TX / HB)) * HB;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float v[HB + 2 * R];
#pragma unroll
            for (int j = 0; j < HB + 2 * R; ++j) v[j] = sd[q][r][c0 + j + BOFF];
#pragma unroll
            for (int o = 0; o < HB; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < K; ++k) acc = __fmaf_rn(A.g[k], v[o + k], acc);
                sh[q][r][c0 + o] = acc;
            }
        }
    }
    __syncthreads();
    ssim_bwd_epilogue(A, P, sh, lx, ly, out);
}

std::once_flag g_encode_once;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode;
}

// The maps of every view, or false if a view or a buffer does not suit TMA.
bool encode_maps(gs_workspace *ws, const float *rgb, const float *target, SsimTma &T) {
    if (ws->n_views > kTmaViews) return false;
    auto enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)rgb | (uintptr_t)target | (uintptr_t)ws->ssim_d) & 15) return false;
    const uint64_t n_elem = 3 * (uint64_t)ws->n_pix;
    for (int v = 0; v < ws->n_views; ++v) {
        const ViewInfo &vi = ws->views_h[v];
        if (vi.W % 4 != 0) return false;
        const uint64_t W = vi.W, H = vi.H, off = 3 * (uint64_t)vi.pix_off;
        const cuuint64_t dim3[3] = {W, H, 3}, str3[2] = {W * 4, W * H * 4};
        const cuuint64_t dim4[4] = {W, H, 3, 3}, str4[3] = {W * 4, W * H * 4, n_elem * 4};
        const cuuint32_t box3[3] = {(cuuint32_t)BW, (cuuint32_t)IH, 1}, box4[4] = {(cuuint32_t)BW, (cuuint32_t)IH, 1, 1};
        const cuuint32_t one[4] = {1, 1, 1, 1};
        CUresult r = enc(&T.x[v], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)(rgb + off), dim3, str3, box3, one,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS)
            r = enc(&T.y[v], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)(target + off), dim3, str3, box3, one,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS)
            r = enc(&T.d[v], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)(ws->ssim_d + off), dim4, str4, box4, one,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
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
    A.flags = &ws->st->flags;
    A.wait_ns = kTmaWaitNs;
    double g[K], sum = 0.0;
    for (int i = 0; i < K; ++i) {
        g[i] = std::exp(-(double)((i - R) * (i - R)) / (2.0 * 1.5 * 1.5));
        sum += g[i];
    }
    A.gsum = 0.f;
    for (int i = 0; i < K; ++i) {
        A.g[i] = (float)(g[i] / sum);
        A.gsum += A.g[i];
    }
    const int grid = (int)ws->n_ssim_tiles;
    if (grid == 0) return GS_OK;
    SsimTma T;
    const bool tma = encode_maps(ws, rgb, target, T);
    StageTimer timer(ws, GS_STAGE_IMAGE_SSIM, s);
    ++ws->kernel_launches;
    if (tma) k_ssim_fwd_tma<<<grid, NT, 0, s>>>(A, T);
    else k_ssim_fwd<<<grid, NT, 0, s>>>(A);
    gs_status r = check_launch("ssim_fwd");
    if (r != GS_OK || !dL_drgb || grad_scale == 0.f) return r;
    ++ws->kernel_launches;
    if (tma) k_ssim_bwd_tma<<<grid, NT, 0, s>>>(A, T);
    else k_ssim_bwd<<<grid, NT, 0, s>>>(A);
    return check_launch("ssim_bwd");
}

}  // namespace gs

extern "C" gs_status gs_selftest_wait_timeout(gs_workspace *ws, int64_t limit_ns, int32_t *result, void *stream) {
    if (!ws || !result || limit_ns <= 0 || limit_ns > 2000000000ll) {
        gs::set_last_error("gs_selftest_wait_timeout: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    ++ws->kernel_launches;
    gs::k_wait_selftest<<<1, 64, 0, (cudaStream_t)stream>>>(&ws->st->flags, (uint64_t)limit_ns, result);
    return gs::check_launch("wait_selftest");
}
