// Tile rasteriser: forward alpha compositing and its adjoint.
//
// One CTA owns one tile at a time and pulls tiles of every view from a global
// work counter, so a single persistent launch covers all cameras of the
// batch, whatever their sizes.  Gaussians of the tile's depth-sorted list are
// staged `batch_depth` at a time in shared memory; each thread walks them for
// its pixels.
//
// Forward (front to back):  alpha = min(alpha_max, o e^{pw}); skip alpha <
// alpha_min; a fragment that would take T below t_min ends the pixel before it
// is blended; C += alpha T c, D += alpha T z, T *= (1 - alpha).  The CTA leaves
// a tile as soon as every pixel has ended.  Per pixel it keeps the list count
// up to the last blended fragment and the final T.
//
// Backward (back to front from that count): alpha is recomputed with the same
// instructions, T is recovered by division, and with h = gC.c + gD z + gA
//   dL/dalpha_j = T_j h_j - (sum_{k>j} w_k h_k) / (1 - alpha_j).
// The 10 image-space gradient components of each Gaussian are summed over the
// thread's pixels and then over the warp with shuffles before one atomic per
// component.
//
// In both passes each thread owns a few vertically adjacent pixels of one
// column (PF forward, PPT backward): the shared memory loads, the loop
// overhead, the column part of the exponent and (backward) the warp
// reduction are paid once per column of pixels.  The backward runs its pixel
// updates without branches: a pixel that a fragment does not reach takes
// alpha = 0, for which each update is exactly the identity.
//
// The VAR variants also render each pixel's depth distribution under the
// weights w: its mean mu = sum w z / W and variance var = sum w (z - mu)^2 / W,
// W = sum w.  They are accumulated front to back by the weighted Welford
// update, in depths relative to the first blended fragment's, c:
//   W += w;  y = z - c;  d = y - m;  m += d w / W;  M2 += w d (y - m),
// so that rounding scales with the spread of the depths, not with the depth
// itself (mu = D / A in float loses ~sqrt(n) ulps of a 5 m depth, which a
// centimetre-scale variance term magnifies).  mu = c + m and var = M2 / W are
// kept per pixel (with 1/W) for the backward, and alpha is written as W
// (1 - T in exact arithmetic).  With sum w (z - mu) = 0 the adjoints are
//   dmu/dw_k = (z_k - mu) / W,                dmu/dz_k = w_k / W,
//   dvar/dw_k = ((z_k - mu)^2 - var) / W,     dvar/dz_k = 2 w_k (z_k - mu) / W,
// so with a = gmu / W and b = gvar / W, h gains a dz + b (dz^2 - var) and
// dL/dz gains w (a + 2 b dz), dz = z - mu.
#include "gs_internal.cuh"

namespace gs {
namespace {

struct RasterArgs {
    const ViewInfo *views;
    int32_t n_views, n_tiles, depth;
    Consts c;
    const float4 *rec;
    const uint32_t *vals;
    const uint2 *ranges;
    const uint32_t *order;  // tiles in work order
    uint32_t *counter;
    uint32_t *last;
    float *tfin;
    // forward outputs
    float *rgb, *depth_out, *alpha_out;
    float *mean_out, *var_out;  // VAR variants: depth mean and variance per pixel
    float4 *vstat;              // VAR variants: (mean, var, 1/W, 0) per pixel, for the backward
    // backward inputs / outputs
    const float *dL_drgb, *dL_ddepth, *dL_dalpha;
    const float *dL_dmean, *dL_dvar;  // VAR variant
    float *g2d;
};

// One CTA works a tile at a time (persistent, tiles taken in the work order);
// a thread holds PF vertically adjacent pixels of one column, which share the
// shared-memory reads and the column part of every fragment's exponent.  A
// pixel stops at the first fragment that would take its transmittance below
// t_min, the thread when all of its pixels have, the CTA when all threads have.
template <int TW, int TH, int PF, bool VAR>
__global__ void __launch_bounds__(TW * TH / PF) k_raster_fwd(RasterArgs A) {
    constexpr int NT = TW * TH / PF;
    static_assert(NT % 32 == 0, "the forward needs whole warps");
    extern __shared__ float4 smem[];
    float4 *sA = smem, *sB = smem + A.depth, *sC = smem + 2 * A.depth;
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    const float amax = A.c.alpha_max, tmin = A.c.t_min, l2amin = A.c.log2_alpha_min;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const uint32_t w = atomicAdd(A.counter, 1u);
            s_tile = w < (uint32_t)A.n_tiles ? (int)A.order[w] : -1;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) break;
        const int v = view_of_tile(A.views, A.n_views, tile);
        const ViewInfo vi = A.views[v];
        const int lt = tile - vi.tile_off;
        const int px = (lt % vi.ntx) * TW + tid % TW;
        const int py0 = (lt / vi.ntx) * TH + (tid / TW) * PF;
        const float pxf = (float)px;
        const uint2 rg = A.ranges[tile];
        float T[PF], Cr[PF], Cg[PF], Cb[PF], D[PF];
        float Wsum[PF], zc[PF], mr[PF], M2[PF];
        uint32_t cnt[PF];
        bool live[PF];
        int nlive = 0;
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            T[i] = 1.f;
            Cr[i] = Cg[i] = Cb[i] = D[i] = 0.f;
            Wsum[i] = zc[i] = mr[i] = M2[i] = 0.f;
            cnt[i] = 0;
            live[i] = px < vi.W && py0 + i < vi.H;
            nlive += live[i];
        }
        for (uint32_t b0 = rg.x; b0 < rg.y; b0 += A.depth) {
            if (__syncthreads_and(nlive == 0)) break;
            const int nb = min((int)(rg.y - b0), A.depth);
            for (int j = tid; j < nb; j += NT) {
                uint32_t pair = A.vals[b0 + j];
                float4 r0 = A.rec[3 * (size_t)pair], r1 = A.rec[3 * (size_t)pair + 1];
                float4 a, bb;
                stage_record(r0, r1, a, bb);
                sA[j] = a;
                sB[j] = bb;
                sC[j] = A.rec[3 * (size_t)pair + 2];
            }
            __syncthreads();
            for (int j = 0; j < nb && nlive > 0; ++j) {
                const float4 a = sA[j], b = sB[j];
                float dxi, u1;
                frag_column(a, b, pxf, dxi, u1);
#pragma unroll
                for (int i = 0; i < PF; ++i) {
                    float t1, t2, dyi;
                    const float e = frag_pixel(a, b, u1, (float)(py0 + i), t1, t2, dyi);
                    if (!live[i] || e < l2amin) continue;
                    const float al = fminf(amax, ex2_approx(e));
                    const float Tn = __fmaf_rn(-T[i], al, T[i]);
                    if (Tn < tmin) {
                        live[i] = false;
                        --nlive;
                        continue;
                    }
                    const float wgt = al * T[i];
                    const float4 c = sC[j];
                    Cr[i] = __fmaf_rn(wgt, c.x, Cr[i]);
                    Cg[i] = __fmaf_rn(wgt, c.y, Cg[i]);
                    Cb[i] = __fmaf_rn(wgt, c.z, Cb[i]);
                    D[i] = __fmaf_rn(wgt, c.w, D[i]);
                    if (VAR) {
                        if (cnt[i] == 0) zc[i] = c.w;
                        Wsum[i] += wgt;
                        const float y = c.w - zc[i];
                        const float d = y - mr[i];
                        mr[i] = __fmaf_rn(d, __fdividef(wgt, Wsum[i]), mr[i]);
                        M2[i] = __fmaf_rn(wgt * d, y - mr[i], M2[i]);
                    }
                    T[i] = Tn;
                    cnt[i] = b0 + j - rg.x + 1;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < PF; ++i) {
            const int py = py0 + i;
            if (px >= vi.W || py >= vi.H) continue;
            const int64_t pl = (int64_t)py * vi.W + px;
            const int64_t pix = vi.pix_off + pl;
            const int64_t hw = (int64_t)vi.W * vi.H;
            float *rgb = A.rgb + 3 * (int64_t)vi.pix_off;
            rgb[pl] = Cr[i];
            rgb[hw + pl] = Cg[i];
            rgb[2 * hw + pl] = Cb[i];
            A.depth_out[pix] = D[i];
            // 1 - T loses the relative precision of a small alpha (T near 1);
            // the variance variant has the direct sum of the weights at hand,
            // which keeps it, as the normalised depth D / alpha needs
            A.alpha_out[pix] = VAR ? Wsum[i] : 1.f - T[i];
            A.last[pix] = cnt[i];
            A.tfin[pix] = T[i];
            if (VAR) {
                const float mean = zc[i] + mr[i];
                const float iw = Wsum[i] > 0.f ? 1.f / Wsum[i] : 0.f;
                const float var = M2[i] * iw;
                A.mean_out[pix] = mean;
                A.var_out[pix] = var;
                A.vstat[pix] = make_float4(mean, var, iw, 0.f);
            }
        }
    }
}

// Sums ten per-lane values over the warp by recursive halving: at each of the
// five butterfly levels a lane keeps half of its remaining components and
// sends the other half to its partner, so 12 shuffles replace 50.  Afterwards
// lane l holds the warp total of component
//   comp(l) = 5*b4 + 3*b3 + 2*b2 + b1      (bK = bit K of l),
// valid when (b3 == 0 and not (b2 and b1)) or (b3 == 1 and b2 == 0); lanes l
// and l^1 hold the same total.  reduce10_component gives comp(l) or -1.
__device__ __forceinline__ float warp_reduce_scatter10(const float v[10], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float a[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float send = b4 ? v[i] : v[i + 5];
        float keep = b4 ? v[i + 5] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float c[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float hiv = i + 3 < 5 ? a[i + 3] : 0.f;
        float send = b3 ? a[i] : hiv;
        float keep = b3 ? hiv : a[i];
        c[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float d[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float hiv = i + 2 < 3 ? c[i + 2] : 0.f;
        float send = b2 ? c[i] : hiv;
        float keep = b2 ? hiv : c[i];
        d[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float send = b1 ? d[0] : d[1];
    float keep = b1 ? d[1] : d[0];
    float e = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    return e + __shfl_xor_sync(0xffffffffu, e, 1);
}

__device__ __forceinline__ int reduce10_component(int lane) {
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
    const bool ok = b3 == 0 ? !(b2 && b1) : b2 == 0;
    return ok ? 5 * b4 + 3 * b3 + 2 * b2 + b1 : -1;
}

// At least 512 resident threads per SM (16 warps, 128 registers a thread):
// with eight pixels a thread, measured best on the 500k orchard (16 one-warp
// blocks: 0.435 ms; 14: 0.441 ms).
template <int TW, int TH, int PPT, bool VAR>
__global__ void __launch_bounds__(TW * TH / PPT, 512 / (TW * TH / PPT)) k_raster_bwd(RasterArgs A) {
    constexpr int NT = TW * TH / PPT;
    static_assert(NT % 32 == 0, "the backward needs whole warps");
    constexpr int NW = (NT + 31) / 32;
    extern __shared__ float4 smem[];
    float4 *sA = smem, *sB = smem + A.depth, *sC = smem + 2 * A.depth;
    float2 *sH = reinterpret_cast<float2 *>(smem + 3 * A.depth);
    uint32_t *sP = reinterpret_cast<uint32_t *>(sH + A.depth);
    __shared__ int s_tile;
    __shared__ uint32_t s_max[NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const float amax = A.c.alpha_max, l2amin = A.c.log2_alpha_min;
    // component this lane adds after the reduction (even lanes only), and the
    // factors c0 + c11 l11 + c22 l22 that turn its raw sum into the gradient
    const int my_comp = (lane & 1) ? -1 : reduce10_component(lane);
    const float sc0 = my_comp == G_QA || my_comp == G_QC ? -0.5f
                      : my_comp == G_QB                  ? -1.f
                      : my_comp == G_U || my_comp == G_V ? 0.f
                                                         : 1.f;
    const float sc11 = my_comp == G_U ? kTwoLn2 : 0.f;
    const float sc22 = my_comp == G_V ? kTwoLn2 : 0.f;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const uint32_t w = atomicAdd(A.counter, 1u);
            s_tile = w < (uint32_t)A.n_tiles ? (int)A.order[w] : -1;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) break;
        const int v = view_of_tile(A.views, A.n_views, tile);
        const ViewInfo vi = A.views[v];
        const int lt = tile - vi.tile_off;
        const int px = (lt % vi.ntx) * TW + tid % TW;
        const int py0 = (lt / vi.ntx) * TH + (tid / TW) * PPT;
        const float pxf = (float)px;
        const uint2 rg = A.ranges[tile];
        const int64_t hw = (int64_t)vi.W * vi.H;
        const float *grgb = A.dL_drgb + 3 * (int64_t)vi.pix_off;
        uint32_t cnt[PPT], mycnt = 0;
        float T[PPT], gR[PPT], gG[PPT], gB[PPT], gD[PPT], gA[PPT], acc[PPT];
        float zmu[PPT], ga[PPT], gb[PPT];
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            const int py = py0 + i;
            cnt[i] = 0;
            T[i] = 1.f;
            gR[i] = gG[i] = gB[i] = gD[i] = gA[i] = acc[i] = 0.f;
            zmu[i] = ga[i] = gb[i] = 0.f;
            if (px < vi.W && py < vi.H) {
                const int64_t pl = (int64_t)py * vi.W + px;
                const int64_t pix = vi.pix_off + pl;
                cnt[i] = A.last[pix];
                T[i] = A.tfin[pix];
                gR[i] = grgb[pl];
                gG[i] = grgb[hw + pl];
                gB[i] = grgb[2 * hw + pl];
                gD[i] = A.dL_ddepth ? A.dL_ddepth[pix] : 0.f;
                gA[i] = A.dL_dalpha ? A.dL_dalpha[pix] : 0.f;
                if (VAR) {
                    const float4 vs = A.vstat[pix];
                    zmu[i] = vs.x;
                    ga[i] = A.dL_dmean ? A.dL_dmean[pix] * vs.z : 0.f;
                    gb[i] = A.dL_dvar ? A.dL_dvar[pix] * vs.z : 0.f;
                    gA[i] = __fmaf_rn(-gb[i], vs.y, gA[i]);  // the -b var part of every h
                }
            }
            mycnt = max(mycnt, cnt[i]);
        }
        uint32_t wmax = mycnt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        if (lane == 0) s_max[wid] = wmax;
        __syncthreads();
        uint32_t maxcnt = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) maxcnt = max(maxcnt, s_max[w]);
        for (int64_t hi = (int64_t)rg.x + maxcnt; hi > (int64_t)rg.x; hi -= A.depth) {
            const int64_t lo = max((int64_t)rg.x, hi - A.depth);
            const int nb = (int)(hi - lo);
            __syncthreads();
            for (int j = tid; j < nb; j += NT) {
                uint32_t pair = A.vals[lo + j];
                float4 r0 = A.rec[3 * (size_t)pair], r1 = A.rec[3 * (size_t)pair + 1];
                float4 a, bb;
                stage_record(r0, r1, a, bb);
                sA[j] = a;
                sB[j] = bb;
                sC[j] = A.rec[3 * (size_t)pair + 2];
                sH[j] = make_float2(r0.z, r0.w);
                sP[j] = pair;
            }
            __syncthreads();
            for (int j = nb - 1; j >= 0; --j) {
                const uint32_t rel = (uint32_t)(lo + j - rg.x);
                if (rel >= wmax) continue;  // no pixel of this warp reached this entry
                const float4 a = sA[j], b = sB[j];
                float dxi, u1;
                frag_column(a, b, pxf, dxi, u1);
                // the forward's alpha decision for each of the thread's pixels:
                // ar = the unclamped alpha of a pixel the fragment reaches, else 0
                float ar[PPT], t1_0 = 0.f, t2_0 = 0.f, dyi_0 = 0.f;
                bool any = false;
#pragma unroll
                for (int i = 0; i < PPT; ++i) {
                    float t1, t2, dyi;
                    const float e = frag_pixel(a, b, u1, (float)(py0 + i), t1, t2, dyi);
                    if (i == 0) {
                        t1_0 = t1;
                        t2_0 = t2;
                        dyi_0 = dyi;
                    }
                    const bool in = rel < cnt[i] && e >= l2amin;
                    ar[i] = in ? ex2_approx(e) : 0.f;
                    any |= in;
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                // Every pixel runs the same instructions: a pixel this fragment
                // does not reach takes alpha = 0, for which each update below is
                // exactly the identity (T * 1, acc + 0 * h, sums + 0).
                const float4 c = sC[j];
                float sR = 0.f, sG = 0.f, sB_ = 0.f, sZ = 0.f;  // sum wgt dL/dc
                // sums of gpw = dL/dpw over the column's pixels i = 0..PPT-1,
                // weighted by 1, i and i^2: the pixel offsets are dx (one per
                // column) and dy_i = dy_0 + i, and t1, t2 are affine in i, so
                // these three give every second-order moment the gradient needs
                float S0 = 0.f, S1 = 0.f, S2 = 0.f;
#pragma unroll
                for (int i = 0; i < PPT; ++i) {
                    const float al = fminf(amax, ar[i]);
                    const float r1m = ar[i] > 0.f ? rcp_approx(1.f - al) : 1.f;
                    T[i] = T[i] * r1m;  // transmittance before this fragment
                    const float wgt = al * T[i];
                    float h = gR[i] * c.x + gG[i] * c.y + gB[i] * c.z + gD[i] * c.w + gA[i];
                    float gz = gD[i];
                    if (VAR) {
                        const float dz = c.w - zmu[i];
                        const float t = __fmaf_rn(gb[i], dz, ga[i]);  // a + b dz
                        h = __fmaf_rn(t, dz, h);
                        gz += __fmaf_rn(gb[i], dz, t);               // a + 2 b dz
                    }
                    const float dLda = T[i] * h - acc[i] * r1m;
                    acc[i] = __fmaf_rn(wgt, h, acc[i]);
                    sR = __fmaf_rn(wgt, gR[i], sR);
                    sG = __fmaf_rn(wgt, gG[i], sG);
                    sB_ = __fmaf_rn(wgt, gB[i], sB_);
                    sZ = __fmaf_rn(wgt, gz, sZ);
                    // gpw with pw = -d^T Q d / 2 (natural log); a clamped alpha
                    // has no gradient through pw
                    const float gpw = ar[i] > 0.f && ar[i] <= amax ? dLda * al : 0.f;
                    S0 += gpw;
                    if (i > 0) {
                        S1 = __fmaf_rn(gpw, (float)i, S1);
                        S2 = __fmaf_rn(gpw, (float)(i * i), S2);
                    }
                }
                // per-lane raw moments; the per-Gaussian factors are applied
                // once after the warp reduction (see below)
                const float2 hh = sH[j];
                const float dx = dxi + hh.x, dy0 = dyi_0 + hh.y;
                const float sy = __fmaf_rn(dy0, S0, S1);  // sum gpw dy
                float g[kGrad];
                g[G_LNO] = S0;
                g[G_U] = __fmaf_rn(t1_0, S0, b.y * S1);  // sum gpw t1, t1_i = t1_0 + l12 i
                g[G_V] = __fmaf_rn(t2_0, S0, b.z * S1);  // sum gpw t2, t2_i = t2_0 + l22 i
                g[G_QA] = dx * dx * S0;                     // sum gpw dx^2
                g[G_QB] = dx * sy;                          // sum gpw dx dy
                g[G_QC] = __fmaf_rn(dy0, sy, __fmaf_rn(dy0, S1, S2));  // sum gpw dy^2
                g[G_R] = sR;
                g[G_G] = sG;
                g[G_B] = sB_;
                g[G_Z] = sZ;
                const float tot = warp_reduce_scatter10(g, lane);
                if (my_comp >= 0) {
                    // dL/dQ = -1/2 sum gpw d d^T; dpw/du = (Q d)_x = l11 t1 / s^2,
                    // dpw/dv = (l12 t1 + l22 t2) / s^2 with 1/s^2 = 2 ln 2: each lane
                    // scales its sum by c0 + c11 l11 + c22 l22 (constants per lane)
                    float *gp = A.g2d + (size_t)sP[j] * kGrad;
                    atomicAdd(gp + my_comp, tot * __fmaf_rn(sc11, b.x, __fmaf_rn(sc22, b.z, sc0)));
                    if (my_comp == G_U) atomicAdd(gp + G_V, kTwoLn2 * b.y * tot);
                }
            }
        }
    }
}

// zero the image-space gradients of the visible pairs
__global__ void k_zero_g2d(const uint32_t *vis_pair, const DevState *st, float *g2d) {
    uint32_t n = st->n_vis;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n * kGrad; i += gridDim.x * blockDim.x)
        g2d[(size_t)vis_pair[i / kGrad] * kGrad + i % kGrad] = 0.f;
}

// Pixels per thread of the backward (the forward uses one, so that a pixel
// leaves the list as soon as it saturates).  More pixels a thread amortise the
// per-fragment warp reduction and the shared-memory reads over more pixels:
// on the 500k orchard with 16x16 tiles, 4 -> 0.467 ms and 8 (one warp a tile)
// -> 0.435 ms.  The VAR variant holds three more values a pixel and keeps 4
// (8 spills).  An 8x8 tile keeps 2 so that its CTA is still a whole warp,
// which the full-mask shuffles and votes require.
template <int TW, int TH, bool VAR>
constexpr int ppt_bwd() { return TW * TH >= 256 ? (VAR ? 4 : 8) : 2; }

size_t fwd_smem(int depth) { return (size_t)depth * 3 * sizeof(float4); }
size_t bwd_smem(int depth) {
    return (size_t)depth * (3 * sizeof(float4) + sizeof(float2) + sizeof(uint32_t));
}

// Pixels per thread of the forward: on the 500k orchard with 16x16 tiles
// 1 -> 0.307 ms, 2 -> 0.268 ms, 4 -> 0.239 ms, 8 -> 0.303 ms; the VAR variant
// (four more values a pixel) 2 -> 0.372 ms, 4 -> 0.400 ms.
template <int TW, int TH, bool VAR>
constexpr int ppt_fwd() { return TW * TH >= 256 && !VAR ? 4 : 2; }

template <int TW, int TH, bool VAR>
cudaError_t configure_variant(gs_workspace *ws, int &grid_f, int &grid_b) {
    constexpr int PPT = ppt_bwd<TW, TH, VAR>(), PF = ppt_fwd<TW, TH, VAR>();
    const int depth = ws->cfg.batch_depth;
    cudaError_t e = cudaFuncSetAttribute(k_raster_fwd<TW, TH, PF, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fwd_smem(256));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_raster_bwd<TW, TH, PPT, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bwd_smem(256));
    int occ_f = 0, occ_b = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, k_raster_fwd<TW, TH, PF, VAR>, TW * TH / PF,
                                                          fwd_smem(depth));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, k_raster_bwd<TW, TH, PPT, VAR>, TW * TH / PPT,
                                                          bwd_smem(depth));
    grid_f = std::max(1, occ_f) * ws->num_sms;
    grid_b = std::max(1, occ_b) * ws->num_sms;
    return e;
}

template <int TW, int TH>
gs_status configure_one(gs_workspace *ws) {
    cudaError_t e = configure_variant<TW, TH, false>(ws, ws->raster_grid_fwd, ws->raster_grid_bwd);
    if (e == cudaSuccess) e = configure_variant<TW, TH, true>(ws, ws->raster_grid_fwd_var, ws->raster_grid_bwd_var);
    if (e != cudaSuccess) {
        set_last_error(std::string("raster_configure: ") + cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

RasterArgs make_args(gs_workspace *ws) {
    RasterArgs A{};
    A.views = ws->views;
    A.n_views = ws->n_views;
    A.n_tiles = (int32_t)ws->n_tiles;
    A.depth = ws->cfg.batch_depth;
    A.c = ws->consts;
    A.rec = ws->rec;
    A.vals = ws->inst_val;
    A.ranges = ws->ranges;
    A.order = ws->tile_order;
    A.last = ws->last;
    A.tfin = ws->tfin;
    return A;
}

template <int TW, int TH>
gs_status run_fwd(gs_workspace *ws, RasterArgs A, cudaStream_t s) {
    StageTimer timer(ws, GS_STAGE_RASTER_FWD, s);
    ++ws->kernel_launches;
    constexpr int PV = ppt_fwd<TW, TH, true>(), P = ppt_fwd<TW, TH, false>();
    if (A.mean_out)
        k_raster_fwd<TW, TH, PV, true><<<ws->raster_grid_fwd_var, TW * TH / PV, fwd_smem(A.depth), s>>>(A);
    else
        k_raster_fwd<TW, TH, P, false><<<ws->raster_grid_fwd, TW * TH / P, fwd_smem(A.depth), s>>>(A);
    return check_launch("raster_fwd");
}
template <int TW, int TH>
gs_status run_bwd(gs_workspace *ws, RasterArgs A, cudaStream_t s) {
    constexpr int PV = ppt_bwd<TW, TH, true>(), P = ppt_bwd<TW, TH, false>();
    StageTimer timer(ws, GS_STAGE_RASTER_BWD, s);
    ++ws->kernel_launches;
    if (A.vstat)
        k_raster_bwd<TW, TH, PV, true><<<ws->raster_grid_bwd_var, TW * TH / PV, bwd_smem(A.depth), s>>>(A);
    else
        k_raster_bwd<TW, TH, P, false><<<ws->raster_grid_bwd, TW * TH / P, bwd_smem(A.depth), s>>>(A);
    return check_launch("raster_bwd");
}

}  // namespace

gs_status raster_configure(gs_workspace *ws) {
    int tw = ws->cfg.tile_w, th = ws->cfg.tile_h;
    if (tw == 8 && th == 8) return configure_one<8, 8>(ws);
    if (tw == 16 && th == 16) return configure_one<16, 16>(ws);
    if (tw == 16 && th == 32) return configure_one<16, 32>(ws);
    if (tw == 32 && th == 16) return configure_one<32, 16>(ws);
    return GS_ERR_INVALID_ARG;
}

gs_status launch_raster_fwd(gs_workspace *ws, float *rgb, float *depth, float *alpha, float *mean,
                            float *var, cudaStream_t s) {
    RasterArgs A = make_args(ws);
    A.counter = &ws->st->fwd_counter;
    A.rgb = rgb;
    A.depth_out = depth;
    A.alpha_out = alpha;
    if (mean) {
        A.mean_out = mean;
        A.var_out = var;
        A.vstat = ws->vstat;
    }
    cudaMemsetAsync(A.counter, 0, sizeof(uint32_t), s);
    int tw = ws->cfg.tile_w, th = ws->cfg.tile_h;
    if (tw == 8 && th == 8) return run_fwd<8, 8>(ws, A, s);
    if (tw == 16 && th == 16) return run_fwd<16, 16>(ws, A, s);
    if (tw == 16 && th == 32) return run_fwd<16, 32>(ws, A, s);
    return run_fwd<32, 16>(ws, A, s);
}

gs_status launch_raster_bwd(gs_workspace *ws, const float *dL_drgb, const float *dL_ddepth,
                            const float *dL_dalpha, bool var, const float *dL_dmean, const float *dL_dvar,
                            cudaStream_t s) {
    RasterArgs A = make_args(ws);
    A.counter = &ws->st->bwd_counter;
    A.dL_drgb = dL_drgb;
    A.dL_ddepth = dL_ddepth;
    A.dL_dalpha = dL_dalpha;
    if (var) {
        A.vstat = ws->vstat;
        A.dL_dmean = dL_dmean;
        A.dL_dvar = dL_dvar;
    }
    A.g2d = ws->g2d;
    {
        StageTimer timer(ws, GS_STAGE_ZERO_GRAD, s);
        ++ws->kernel_launches;
        k_zero_g2d<<<ws->num_sms * 4, 256, 0, s>>>(ws->vis_pair, ws->st, ws->g2d);
    }
    gs_status r = check_launch("zero_g2d");
    if (r != GS_OK) return r;
    cudaMemsetAsync(A.counter, 0, sizeof(uint32_t), s);
    int tw = ws->cfg.tile_w, th = ws->cfg.tile_h;
    if (tw == 8 && th == 8) return run_bwd<8, 8>(ws, A, s);
    if (tw == 16 && th == 16) return run_bwd<16, 16>(ws, A, s);
    if (tw == 16 && th == 32) return run_bwd<16, 32>(ws, A, s);
    return run_bwd<32, 16>(ws, A, s);
}

}  // namespace gs
