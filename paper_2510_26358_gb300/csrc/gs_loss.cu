// Losses of Sec. III-C.
//
// Depth consistency (Eq. 7): each LiDAR return (u, v, z, view) reads the
// rendered depth at pixel (floor u, floor v).  A return is valid when it lies
// inside the image, z > near_z and the pixel's alpha > 0.  Mode 0 averages
// |D - z|; mode 1 averages KL(N(z, sigma_L^2) || N(D, sigma_U^2)) =
// ln(sigma_U/sigma_L) + (sigma_L^2 + (z - D)^2) / (2 sigma_U^2) - 1/2; both are
// scaled by lambda_L.  The gradient dL/dD = lambda_L/|Omega| dl/dD is added to
// the pixel (atomically: several returns may share a pixel).
//
// Mode 2 takes the renderer's own depth distribution as N(mu_u, sigma_u^2):
// the rendered mean mu_u and sigma_u^2 = max(var, 0) + sigma_U^2 from the
// rendered variance, and
// KL = ln(sigma_u/sigma_L) + (sigma_L^2 + (z - mu_u)^2) / (2 sigma_u^2) - 1/2,
// with gradients to mu_u and var.
//
// Photometric L1 (Eq. 6 with lambda = 0): mean |C - I| over every channel of
// every pixel of every view, gradient sign(C - I)/n.  The full Eq. 6 adds
// lambda (1 - SSIM) (gs_ssim.cu) and scales the L1 gradient by (1 - lambda).
//
// Sums are deterministic: per-block partials in double, then one block adds
// them in block order.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int LT = 256;

__device__ __forceinline__ double block_sum_d(double v, double *sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sm[i];
    return t;
}

// A thread's running sum in float with Kahan's compensation (error about 2
// ulps of the sum whatever the number of terms): the FP64 pipe, a small
// fraction of the FP32 rate on this GPU, is kept for the block and grid sums.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Called by every thread after thread 0 has written the block's partial:
// true in the one block that finishes last (it then sees every partial, and
// puts the counter back to 0 for the next launch when it is done with it).
__device__ __forceinline__ bool last_block(uint32_t *counter) {
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        __threadfence();  // this block's partial before the count
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) __threadfence();  // every other partial before the reads below
    return s_last;
}

struct DepthArgs {
    const ViewInfo *views;
    int32_t n_views, mode;
    float near_z, sigma_L, sigma_U, lambda;
    const float *depth, *alpha, *lidar;
    const float *var;  // mode 2 (`depth` holds the mean)
    int64_t n_pts;
    double *part;  // [2][nb]
    int nb;
    float *loss;
    float *grad;      // dL/dD (mode 2: dL/dmean)
    float *grad_var;  // mode 2: dL/dvar
    DevState *st;
};

// Mode 2 at one pixel: the KL term and its partials w.r.t. (mean, var).
struct VarTerm {
    double kl, dmu, dvar;
};
__device__ __forceinline__ VarTerm var_term(double mu, double var, double z, double sl, double su) {
    VarTerm t;
    const bool clamped = var < 0.0;
    const double v = (clamped ? 0.0 : var) + su * su;
    const double e = mu - z;
    t.kl = 0.5 * log(v) - log(sl) + (sl * sl + e * e) / (2.0 * v) - 0.5;
    const double dmu = e / v;
    const double dv = clamped ? 0.0 : 0.5 / v - (sl * sl + e * e) / (2.0 * v * v);
    t.dmu = dmu;
    t.dvar = dv;
    return t;
}

// Validity of a return: its view exists, it lies inside that image, z > near_z
// and alpha > 0 at pixel (floor u, floor v).  Four returns a thread at a time, i0 + u * stride (u = 0..3): the returns,
// then their pixels' alpha, depth (and variance) gathers, are all in flight
// together; the terms are then taken in the order of the one-at-a-time loop
// (i0, i0 + stride, ...), so the sums are unchanged.
constexpr int kDepthBatch = 4;

struct DepthGather {
    int64_t pix[kDepthBatch];  // -1: not a valid return
    float z[kDepthBatch], dep[kDepthBatch], var[kDepthBatch];
};

__device__ __forceinline__ void gather_returns(const DepthArgs &A, int64_t i0, int64_t stride, DepthGather &G) {
    float4 L[kDepthBatch];
#pragma unroll
    for (int u = 0; u < kDepthBatch; ++u) {
        const int64_t i = i0 + u * stride;
        L[u] = i < A.n_pts ? reinterpret_cast<const float4 *>(A.lidar)[i] : make_float4(0.f, 0.f, 0.f, -1.f);
    }
    float al[kDepthBatch];
#pragma unroll
    for (int u = 0; u < kDepthBatch; ++u) {
        G.pix[u] = -1;
        G.z[u] = L[u].z;
        al[u] = 0.f;
        G.dep[u] = G.var[u] = 0.f;
        const int v = (int)L[u].w;
        if (!(L[u].w >= 0.f) || v >= A.n_views) continue;
        const ViewInfo vi = A.views[v];
        if (!(L[u].x >= 0.f && L[u].x < (float)vi.W && L[u].y >= 0.f && L[u].y < (float)vi.H && L[u].z > A.near_z))
            continue;
        G.pix[u] = vi.pix_off + (int64_t)floorf(L[u].y) * vi.W + (int64_t)floorf(L[u].x);
    }
#pragma unroll
    for (int u = 0; u < kDepthBatch; ++u) {
        if (G.pix[u] < 0) continue;
        al[u] = A.alpha[G.pix[u]];
        G.dep[u] = A.depth[G.pix[u]];
        if (A.mode == 2) G.var[u] = A.var[G.pix[u]];
    }
#pragma unroll
    for (int u = 0; u < kDepthBatch; ++u)
        if (!(al[u] > 0.f)) G.pix[u] = -1;
}

__global__ void __launch_bounds__(LT) k_depth_partial(DepthArgs A) {
    __shared__ double sm[32];
    KahanF sf;
    double s = 0.0;
    uint32_t c = 0;
    const int64_t stride = (int64_t)gridDim.x * LT;
    for (int64_t i0 = (int64_t)blockIdx.x * LT + threadIdx.x; i0 < A.n_pts; i0 += kDepthBatch * stride) {
        DepthGather G;
        gather_returns(A, i0, stride, G);
#pragma unroll
        for (int u = 0; u < kDepthBatch; ++u) {
            if (G.pix[u] < 0) continue;
            const float d = __fsub_rn(G.dep[u], G.z[u]);
            if (A.mode == 0) {
                sf.add(fabsf(d));
            } else if (A.mode == 2) {
                s += var_term(G.dep[u], G.var[u], G.z[u], A.sigma_L, A.sigma_U).kl;
            } else {
                // the KL's point-independent part (its log and constants) is
                // added once per valid point at the end: double logs and
                // divisions per point kept the FP64 pipe busy for tens of
                // microseconds
                sf.add(__fmul_rn(d, d));
            }
            ++c;
        }
    }
    s += sf.value();
    double ts = block_sum_d(s, sm);
    double tc = block_sum_d((double)c, sm);
    if (threadIdx.x == 0) {
        A.part[blockIdx.x] = ts;
        A.part[A.nb + blockIdx.x] = tc;
    }
    if (!last_block(&A.st->done_depth)) return;
    // the last block: grid sums in a fixed order (each thread a fixed strided
    // set, then a fixed tree), the loss and the gradient scale
    s = 0.0;
    double cd = 0.0;
    for (int i = threadIdx.x; i < A.nb; i += LT) {
        s += A.part[i];
        cd += A.part[A.nb + i];
    }
    ts = block_sum_d(s, sm);
    tc = block_sum_d(cd, sm);
    if (threadIdx.x == 0) {
        double scale = tc > 0.0 ? (double)A.lambda / tc : 0.0;
        if (A.mode == 1) {
            // KL(N(z, sL^2) || N(D, sU^2)) = ln(sU / sL) + (sL^2 + (z - D)^2) / (2 sU^2) - 1/2
            const double sl = A.sigma_L, su = A.sigma_U;
            ts = tc * (log(su / sl) + sl * sl / (2.0 * su * su) - 0.5) + ts / (2.0 * su * su);
        }
        *A.loss = (float)(ts * scale);
        A.st->depth_scale = (float)scale;
        A.st->depth_valid = (uint32_t)tc;
        A.st->done_depth = 0u;
    }
}

__global__ void __launch_bounds__(LT) k_depth_grad(DepthArgs A) {
    const float scale = A.st->depth_scale;
    if (scale == 0.f) return;
    const float iv = 1.f / (A.sigma_U * A.sigma_U);
    const int64_t stride = (int64_t)gridDim.x * LT;
    for (int64_t i0 = (int64_t)blockIdx.x * LT + threadIdx.x; i0 < A.n_pts; i0 += kDepthBatch * stride) {
        DepthGather G;
        gather_returns(A, i0, stride, G);
#pragma unroll
        for (int u = 0; u < kDepthBatch; ++u) {
            const int64_t pix = G.pix[u];
            if (pix < 0) continue;
            if (A.mode == 2) {
                const VarTerm t = var_term(G.dep[u], G.var[u], G.z[u], A.sigma_L, A.sigma_U);
                const double k = scale;
                if (A.grad) atomicAdd(A.grad + pix, (float)(k * t.dmu));
                if (A.grad_var) atomicAdd(A.grad_var + pix, (float)(k * t.dvar));
                continue;
            }
            float d = G.dep[u] - G.z[u];
            float g = A.mode == 0 ? (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) : d * iv;
            atomicAdd(A.grad + pix, scale * g);
        }
    }
}

__device__ __forceinline__ float l1_term(float c, float t, float inv, float &g) {
    float d = c - t;
    g += d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
    return fabsf(d);
}

// Target values: float as given, or 8-bit (value / 255, rounded as the
// float division rounds it).  Four at a time: float4 or uchar4.
__device__ __forceinline__ float target_value(float t) { return t; }
__device__ __forceinline__ float target_value(uint8_t t) { return (float)t / 255.f; }
__device__ __forceinline__ float4 target4(const float *t, int64_t i) { return reinterpret_cast<const float4 *>(t)[i]; }
__device__ __forceinline__ float4 target4(const uint8_t *t, int64_t i) {
    const uchar4 b = reinterpret_cast<const uchar4 *>(t)[i];
    return make_float4(target_value(b.x), target_value(b.y), target_value(b.z), target_value(b.w));
}

// Four terms are added in float, each group of four into a thread's
// compensated float sum; the block and grid sums are in double and in a
// fixed order.  A thread works four grid strides at once (more loads in
// flight), in the same order.  With
// `done` set, the last block also writes the mean to *loss (else a separate
// kernel combines the partials).
template <typename TT>
__global__ void __launch_bounds__(LT) k_l1_partial(const float *rgb, const TT *target, int64_t n,
                                                  float *grad, double *part, float inv, uint32_t *done,
                                                  float *loss) {
    constexpr int U = 4;
    __shared__ double sm[32];
    KahanF s;
    const bool vec = ((((uintptr_t)rgb) | ((uintptr_t)grad)) & 15) == 0 &&
                     (((uintptr_t)target) & (4 * sizeof(TT) - 1)) == 0;
    const int64_t n4 = vec ? n / 4 : 0;
    const int64_t stride = (int64_t)gridDim.x * LT;
    for (int64_t i0 = (int64_t)blockIdx.x * LT + threadIdx.x; i0 < n4; i0 += U * stride) {
        float4 c[U], t[U], g[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            c[u] = t[u] = g[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n4) {
                c[u] = reinterpret_cast<const float4 *>(rgb)[i];
                t[u] = target4(target, i);
                if (grad) g[u] = reinterpret_cast<float4 *>(grad)[i];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= n4) break;
            s.add(l1_term(c[u].x, t[u].x, inv, g[u].x) + l1_term(c[u].y, t[u].y, inv, g[u].y) +
                  l1_term(c[u].z, t[u].z, inv, g[u].z) + l1_term(c[u].w, t[u].w, inv, g[u].w));
            if (grad) reinterpret_cast<float4 *>(grad)[i] = g[u];
        }
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * LT + threadIdx.x; i < n; i += stride) {
        float g = grad ? grad[i] : 0.f;
        s.add(l1_term(rgb[i], target_value(target[i]), inv, g));
        if (grad) grad[i] = g;
    }
    double t = block_sum_d(s.value(), sm);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    if (!done || !last_block(done)) return;
    double sd = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += LT) sd += part[i];
    t = block_sum_d(sd, sm);
    if (threadIdx.x == 0) {
        *loss = (float)(t / (double)n);
        *done = 0u;
    }
}

// loss[0] = (1 - lambda) L1 + lambda (1 - SSIM), loss[1] = L1, loss[2] = 1 - SSIM
__global__ void __launch_bounds__(LT) k_image_loss_final(const double *l1part, int nb, const double *spart,
                                                        int64_t ns, int64_t n, float lambda, float *loss) {
    __shared__ double sm[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += LT) a += l1part[i];
    for (int64_t i = threadIdx.x; i < ns; i += LT) b += spart[i];
    const double l1 = block_sum_d(a, sm) / (double)n;
    const double dssim = block_sum_d(b, sm) / (double)n;  // the SSIM partials hold sums of 1 - S
    if (threadIdx.x == 0) {
        loss[0] = (float)((1.0 - (double)lambda) * l1 + (double)lambda * dssim);
        loss[1] = (float)l1;
        loss[2] = (float)dssim;
    }
}

}  // namespace

gs_status launch_depth_loss(gs_workspace *ws, int mode, const float *depth, const float *alpha,
                            const float *var, const float *lidar, int64_t n_pts, float *loss,
                            float *dL_ddepth, float *dL_dvar, cudaStream_t s) {
    DepthArgs A{};
    A.views = ws->views;
    A.n_views = ws->n_views;
    A.mode = mode;
    A.var = var;
    A.grad_var = dL_dvar;
    A.near_z = ws->cfg.near_z;
    A.sigma_L = ws->cfg.sigma_L;
    A.sigma_U = ws->cfg.sigma_U;
    A.lambda = ws->cfg.lambda_L;
    A.depth = depth;
    A.alpha = alpha;
    A.lidar = lidar;
    A.n_pts = n_pts;
    A.part = ws->red_part;
    A.nb = ws->sort_blocks;
    A.loss = loss;
    A.grad = dL_ddepth;
    A.st = ws->st;
    StageTimer timer(ws, GS_STAGE_DEPTH_LOSS, s);
    ++ws->kernel_launches; k_depth_partial<<<A.nb, LT, 0, s>>>(A);
    if ((dL_ddepth || dL_dvar) && n_pts > 0) {
        ++ws->kernel_launches;
        k_depth_grad<<<A.nb, LT, 0, s>>>(A);
    }
    return check_launch("depth_loss");
}

namespace {
template <typename TT>
gs_status image_l1(gs_workspace *ws, const float *rgb, const TT *target, float *loss, float *dL_drgb,
                   cudaStream_t s) {
    int64_t n = 3 * ws->n_pix;
    int nb = ws->sort_blocks;
    StageTimer timer(ws, GS_STAGE_IMAGE_L1, s);
    ++ws->kernel_launches;
    k_l1_partial<TT><<<nb, LT, 0, s>>>(rgb, target, n, dL_drgb, ws->red_part, (float)(1.0 / (double)n),
                                       &ws->st->done_l1, loss);
    return check_launch("image_l1");
}
}  // namespace

gs_status launch_image_l1(gs_workspace *ws, const float *rgb, const float *target, float *loss,
                          float *dL_drgb, cudaStream_t s) {
    return image_l1(ws, rgb, target, loss, dL_drgb, s);
}

gs_status launch_image_l1_u8(gs_workspace *ws, const float *rgb, const uint8_t *target, float *loss,
                             float *dL_drgb, cudaStream_t s) {
    return image_l1(ws, rgb, target, loss, dL_drgb, s);
}

gs_status launch_image_loss(gs_workspace *ws, const float *rgb, const float *target, float lambda, float *loss,
                            float *dL_drgb, cudaStream_t s) {
    const int64_t n = 3 * ws->n_pix;
    const int nb = ws->sort_blocks;
    {
        StageTimer timer(ws, GS_STAGE_IMAGE_L1, s);
        ++ws->kernel_launches;
        k_l1_partial<float><<<nb, LT, 0, s>>>(rgb, target, n, dL_drgb, ws->red_part,
                                       (float)((1.0 - (double)lambda) / (double)n), nullptr, nullptr);
    }
    gs_status r = check_launch("image_loss");
    if (r != GS_OK) return r;
    r = launch_ssim(ws, rgb, target, (float)(-(double)lambda / (double)n), dL_drgb, s);
    if (r != GS_OK) return r;
    ++ws->kernel_launches;
    k_image_loss_final<<<1, LT, 0, s>>>(ws->red_part, nb, ws->ssim_part, ws->n_ssim_tiles, n, lambda, loss);
    return check_launch("image_loss");
}

}  // namespace gs
