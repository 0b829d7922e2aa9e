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
// The VAR variant holds four more values a pixel: at least 640 resident
// threads an SM keeps it at 96 registers without spills (0: no minimum).
template <int TW, int TH, int PF, bool VAR>
__global__ void __launch_bounds__(TW * TH / PF, VAR ? 640 / (TW * TH / PF) : 0) k_raster_fwd(RasterArgs A) {
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
//
// A thread's PPT pixels are worked in Q = PPT/2 packed pairs (pixel p in the
// low half, pixel p + Q in the high half), so that one f32x2 instruction does
// the arithmetic of two pixels.  The alpha decision is taken on
// -e = fma(t1, t1, fma(t2, t2, -log2 o)), which is exactly the negation of
// the forward's e = fma(-t1, t1, fma(-t2, t2, log2 o)) (round to nearest is
// symmetric), so both passes take the same decisions bit for bit.
template <int TW, int TH, int PPT, bool VAR>
__global__ void __launch_bounds__(TW * TH / PPT, 512 / (TW * TH / PPT)) k_raster_bwd(RasterArgs A) {
    constexpr int NT = TW * TH / PPT;
    static_assert(NT % 32 == 0, "the backward needs whole warps");
    static_assert(PPT % 2 == 0, "the backward works pixels in pairs");
    constexpr int NW = (NT + 31) / 32;
    constexpr int Q = PPT / 2;
    extern __shared__ float4 smem[];
    float4 *sA = smem, *sB = smem + A.depth, *sC = smem + 2 * A.depth;
    float2 *sH = reinterpret_cast<float2 *>(smem + 3 * A.depth);
    uint32_t *sP = reinterpret_cast<uint32_t *>(sH + A.depth);
    __shared__ int s_tile;
    __shared__ uint32_t s_max[NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const float amax = A.c.alpha_max, nl2amin = -A.c.log2_alpha_min;
    const f2 ONE = f2_bcast(1.f);
    // component this lane adds after the reduction (even lanes only), and the
    // factors c0 + c11 l11 + c22 l22 that turn its raw sum into the gradient
    // (the colour and depth sums come out negated, see below)
    const int my_comp = (lane & 1) ? -1 : reduce10_component(lane);
    const float sc0 = my_comp == G_QA || my_comp == G_QC ? -0.5f
                      : my_comp == G_QB                  ? -1.f
                      : my_comp == G_U || my_comp == G_V ? 0.f
                      : my_comp == G_LNO                 ? 1.f
                                                         : -1.f;
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
        const f2 PY0 = f2_pack((float)py0, (float)(py0 + Q));
        const uint2 rg = A.ranges[tile];
        const int64_t hw = (int64_t)vi.W * vi.H;
        const float *grgb = A.dL_drgb + 3 * (int64_t)vi.pix_off;
        uint32_t cnt[PPT], mycnt = 0;
        f2 T[Q], gR[Q], gG[Q], gB[Q], gD[Q], gA[Q], nacc[Q];  // nacc = -acc
        f2 zmu[Q], ga[Q], gb[Q];
#pragma unroll
        for (int p = 0; p < Q; ++p) {
            float t_[2], r_[2], g_[2], b_[2], d_[2], a_[2], z_[2], ma_[2], mb_[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = p + h * Q, py = py0 + i;
                cnt[i] = 0;
                t_[h] = 1.f;
                r_[h] = g_[h] = b_[h] = d_[h] = a_[h] = z_[h] = ma_[h] = mb_[h] = 0.f;
                if (px < vi.W && py < vi.H) {
                    const int64_t pl = (int64_t)py * vi.W + px;
                    const int64_t pix = vi.pix_off + pl;
                    cnt[i] = A.last[pix];
                    t_[h] = A.tfin[pix];
                    r_[h] = grgb[pl];
                    g_[h] = grgb[hw + pl];
                    b_[h] = grgb[2 * hw + pl];
                    d_[h] = A.dL_ddepth ? A.dL_ddepth[pix] : 0.f;
                    a_[h] = A.dL_dalpha ? A.dL_dalpha[pix] : 0.f;
                    if (VAR) {
                        const float4 vs = A.vstat[pix];
                        z_[h] = vs.x;
                        ma_[h] = A.dL_dmean ? A.dL_dmean[pix] * vs.z : 0.f;
                        mb_[h] = A.dL_dvar ? A.dL_dvar[pix] * vs.z : 0.f;
                        a_[h] = __fmaf_rn(-mb_[h], vs.y, a_[h]);  // the -b var part of every h
                    }
                }
                mycnt = max(mycnt, cnt[i]);
            }
            T[p] = f2_pack(t_[0], t_[1]);
            gR[p] = f2_pack(r_[0], r_[1]);
            gG[p] = f2_pack(g_[0], g_[1]);
            gB[p] = f2_pack(b_[0], b_[1]);
            gD[p] = f2_pack(d_[0], d_[1]);
            gA[p] = f2_pack(a_[0], a_[1]);
            nacc[p] = f2_bcast(0.f);
            if (VAR) {
                zmu[p] = f2_pack(z_[0], z_[1]);
                ga[p] = f2_pack(ma_[0], ma_[1]);
                gb[p] = f2_pack(mb_[0], mb_[1]);
            }
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
                {
                    const f2 AY = f2_bcast(a.y), L12 = f2_bcast(b.y), L22 = f2_bcast(b.z);
                    const f2 U1 = f2_bcast(u1), K2 = f2_bcast(a.w), NBW = f2_bcast(-b.w);
                    f2 PY = PY0;
#pragma unroll
                    for (int p = 0; p < Q; ++p) {
                        const f2 dy = f2_sub(PY, AY);  // dyi = py - V, exact as in the forward
                        if (p + 1 < Q) PY = f2_add(PY, ONE);
                        const f2 t1 = f2_fma(L12, dy, U1);
                        const f2 t2 = f2_fma(L22, dy, K2);
                        const f2 ne = f2_fma(t1, t1, f2_fma(t2, t2, NBW));  // -e
                        if (p == 0) {
                            t1_0 = f2_lo(t1);
                            t2_0 = f2_lo(t2);
                            dyi_0 = f2_lo(dy);
                        }
                        float n_[2];
                        f2_unpack(ne, n_[0], n_[1]);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int i = p + h * Q;
                            const bool in = rel < cnt[i] && n_[h] <= nl2amin;
                            ar[i] = in ? ex2_approx(-n_[h]) : 0.f;
                            any |= in;
                        }
                    }
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                // Every pixel runs the same instructions: a pixel this fragment
                // does not reach takes alpha = 0, for which each update below is
                // exactly the identity (T * 1, acc + 0 * h, sums + 0; the
                // reciprocal approximation returns 1 for 1 on sm_103, measured).
                // The blended sums are carried negated (nwgt = -wgt), which
                // saves the negations the packed instructions cannot fold.
                const float4 c = sC[j];
                const f2 CX = f2_bcast(c.x), CY = f2_bcast(c.y), CZ = f2_bcast(c.z), CW = f2_bcast(c.w);
                f2 sR, sG, sB_, sZ;  // sums of -wgt dL/dc
                // R_k = sum over pairs p of p^k gpw (k = 0, 1, 2), gpw = dL/dpw
                f2 R0, R1, R2;
#pragma unroll
                for (int p = 0; p < Q; ++p) {
                    const float a0 = ar[p], a1 = ar[p + Q];
                    const f2 nal = f2_pack(fmaxf(-amax, -a0), fmaxf(-amax, -a1));  // -alpha
                    // alpha of an unclamped pixel, else 0: a clamped alpha has no
                    // gradient through pw
                    const f2 ag = f2_pack(a0 <= amax ? a0 : 0.f, a1 <= amax ? a1 : 0.f);
                    float o_[2];
                    f2_unpack(f2_add(ONE, nal), o_[0], o_[1]);
                    const f2 r1m = f2_pack(rcp_approx(o_[0]), rcp_approx(o_[1]));  // 1 / (1 - alpha)
                    T[p] = f2_mul(T[p], r1m);  // transmittance before this fragment
                    const f2 nwgt = f2_mul(nal, T[p]);
                    f2 h = f2_fma(gR[p], CX, f2_fma(gG[p], CY, f2_fma(gB[p], CZ, f2_fma(gD[p], CW, gA[p]))));
                    f2 gz = gD[p];
                    if (VAR) {
                        const f2 dz = f2_sub(CW, zmu[p]);
                        const f2 t = f2_fma(gb[p], dz, ga[p]);  // a + b dz
                        h = f2_fma(t, dz, h);
                        gz = f2_add(gz, f2_fma(gb[p], dz, t));  // a + 2 b dz
                    }
                    // dL/dalpha = T h - acc / (1 - alpha)
                    const f2 dLda = f2_fma(T[p], h, f2_mul(nacc[p], r1m));
                    nacc[p] = f2_fma(nwgt, h, nacc[p]);
                    const f2 gpw = f2_mul(dLda, ag);
                    if (p == 0) {
                        sR = f2_mul(nwgt, gR[p]);
                        sG = f2_mul(nwgt, gG[p]);
                        sB_ = f2_mul(nwgt, gB[p]);
                        sZ = f2_mul(nwgt, gz);
                        R0 = gpw;
                    } else {
                        sR = f2_fma(nwgt, gR[p], sR);
                        sG = f2_fma(nwgt, gG[p], sG);
                        sB_ = f2_fma(nwgt, gB[p], sB_);
                        sZ = f2_fma(nwgt, gz, sZ);
                        R0 = f2_add(R0, gpw);
                    }
                    if (p == 1) {
                        R1 = gpw;
                        R2 = gpw;
                    } else if (p > 1) {
                        R1 = f2_fma(gpw, f2_bcast((float)p), R1);
                        R2 = f2_fma(gpw, f2_bcast((float)(p * p)), R2);
                    }
                }
                if (Q == 1) R1 = R2 = f2_bcast(0.f);
                // S_k = sum over the column's pixels i of i^k gpw: pixel p + Q
                // sits in the high half of pair p
                float r0l, r0h, r1l, r1h, r2l, r2h;
                f2_unpack(R0, r0l, r0h);
                f2_unpack(R1, r1l, r1h);
                f2_unpack(R2, r2l, r2h);
                const float S0 = r0l + r0h;
                const float S1 = __fmaf_rn((float)Q, r0h, r1l + r1h);
                const float S2 = __fmaf_rn((float)(Q * Q), r0h, __fmaf_rn((float)(2 * Q), r1h, r2l + r2h));
                // per-lane raw moments: the pixel offsets are dx (one per column)
                // and dy_i = dy_0 + i, and t1, t2 are affine in i; the
                // per-Gaussian factors are applied once after the warp reduction
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
                g[G_R] = f2_lo(sR) + f2_hi(sR);
                g[G_G] = f2_lo(sG) + f2_hi(sG);
                g[G_B] = f2_lo(sB_) + f2_hi(sB_);
                g[G_Z] = f2_lo(sZ) + f2_hi(sZ);
                const float tot = warp_reduce_scatter10(g, lane);
                if (my_comp >= 0) {
                    // dL/dQ = -1/2 sum gpw d d^T; dpw/du = (Q d)_x = l11 t1 / s^2,
                    // dpw/dv = (l12 t1 + l22 t2) / s^2 with 1/s^2 = 2 ln 2: each lane
                    // scales its sum by c0 + c11 l11 + c22 l22 (constants per lane;
                    // c0 = -1 undoes the negation of the colour and depth sums)
                    float *gp = A.g2d + (size_t)sP[j] * kGrad;
                    atomicAdd(gp + my_comp, tot * __fmaf_rn(sc11, b.x, __fmaf_rn(sc22, b.z, sc0)));
                    if (my_comp == G_U) atomicAdd(gp + G_V, kTwoLn2 * b.y * tot);
                }
            }
        }
    }
}

// zero the image-space gradients of the visible pairs (a backward that does
// not follow its projection directly)
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
// (four more values a pixel, register bound above) 2 -> 0.370 ms, 4 -> 0.352 ms.
template <int TW, int TH, bool VAR>
constexpr int ppt_fwd() { return TW * TH >= 256 ? 4 : 2; }

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
    // the projection clears the rows; a second backward of the same
    // projection clears them itself
    if (!ws->g2d_clear) {
        StageTimer timer(ws, GS_STAGE_ZERO_GRAD, s);
        ++ws->kernel_launches;
        k_zero_g2d<<<ws->num_sms * 4, 256, 0, s>>>(ws->vis_pair, ws->st, ws->g2d);
        gs_status r = check_launch("zero_g2d");
        if (r != GS_OK) return r;
    }
    ws->g2d_clear = false;
    cudaMemsetAsync(A.counter, 0, sizeof(uint32_t), s);
    int tw = ws->cfg.tile_w, th = ws->cfg.tile_h;
    if (tw == 8 && th == 8) return run_bwd<8, 8>(ws, A, s);
    if (tw == 16 && th == 16) return run_bwd<16, 16>(ws, A, s);
    if (tw == 16 && th == 32) return run_bwd<16, 32>(ws, A, s);
    return run_bwd<32, 16>(ws, A, s);
}

}  // namespace gs
