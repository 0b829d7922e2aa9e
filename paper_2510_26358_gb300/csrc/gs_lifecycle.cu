// Map lifecycle of the Gaussian map (Sec. III-B, "Gaussian Splats Lifecycle
// Operations") as stream compaction, and the Adam step of its optimiser.
//
// Per splat j (in order), with s = max log-scale and omega the opacity logit,
// every threshold moved to the logit / log domain on the host:
//   prune   omega < logit(tau_opa), s > ln(s_prune_max) or s < ln(s_prune_min)
//   reset   logit(tau_opa) < omega < logit(tau_reset), ln(s_min) < s < ln(s_max):
//           omega = logit(tau_reset)
//   densify g = acc / cnt > gamma_g:  split (s > ln kappa) into two children
//           mu + R(q) diag(exp(ls)) z_k with ls - ln(shrink), or clone
//           (s <= ln clone_scale) into the splat and a copy
// Outputs keep the input order (children / copies in place), so submaps stay
// contiguous.  New splats start with zero optimiser moments.
//
// Three kernels: classify (action and output count per splat, block sums),
// scan (block offsets, total, capacity check, new submap offsets), scatter
// (block-local scan, then the rows; SH rows copied warp-cooperatively so the
// writes coalesce).  A total above the output capacity writes nothing and
// sets the flag gs_lifecycle_status reports.
#include "gs_internal.cuh"
#include "gs_scan.cuh"

#include <cmath>

struct gs_lifecycle {
    int64_t max_in = 0;
    int32_t max_submaps = 0, nblocks_max = 0;
    uint8_t *action = nullptr;      // [max_in] 0 prune, 1 keep, 2 clone, 3 split
    uint32_t *block_sum = nullptr;  // [nblocks]
    uint32_t *block_off = nullptr;  // [nblocks]
    int64_t *state = nullptr;       // [0] outputs needed, [1] capacity flag
    int64_t kernel_launches = 0;
};

namespace gs {
namespace {

constexpr int LT = 256;            // threads per block
constexpr int LCHUNK = 8 * LT;     // splats per block
enum : uint8_t { A_PRUNE = 0, A_KEEP = 1, A_CLONE = 2, A_SPLIT = 3 };
__host__ __device__ constexpr uint32_t out_count(uint8_t a) { return a == A_PRUNE ? 0u : (a == A_KEEP ? 1u : 2u); }

struct Thresholds {
    float opa, smax, smin, grad, split, clone, reset, rmin, rmax, shrink;
    int32_t ops;
};

struct Arrays {
    const float *means, *log_scales, *quats, *omega, *sh;
};
struct OutArrays {
    float *means, *log_scales, *quats, *omega, *sh;
};

__device__ __forceinline__ uint8_t classify(const Thresholds &t, const float *ls, float om, float acc, int32_t cnt,
                                            bool &reset) {
    const float s = fmaxf(fmaxf(ls[0], ls[1]), ls[2]);
    reset = false;
    if ((t.ops & GS_LC_PRUNE) && (om < t.opa || s > t.smax || s < t.smin)) return A_PRUNE;
    reset = (t.ops & GS_LC_RESET) && t.opa < om && om < t.reset && t.rmin < s && s < t.rmax;
    const float g = cnt > 0 ? acc / (float)cnt : 0.f;
    if ((t.ops & GS_LC_DENSIFY) && g > t.grad) {
        if (s > t.split) return A_SPLIT;
        if (s <= t.clone) return A_CLONE;
    }
    return A_KEEP;
}

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *sm) { return gs::block_sum_u32<LT>(v, sm); }
__device__ __forceinline__ uint32_t block_scan_u32(uint32_t v, uint32_t *sm, uint32_t &total) {
    return gs::block_scan_u32<LT>(v, sm, total);
}

__global__ void __launch_bounds__(LT) k_lc_classify(Thresholds t, Arrays in, const float *acc, const int32_t *cnt,
                                                    int64_t n, uint8_t *action, uint32_t *block_sum) {
    __shared__ uint32_t sm[LT / 32];
    const int64_t base = (int64_t)blockIdx.x * LCHUNK;
    uint32_t c = 0;
    for (int i = threadIdx.x; i < LCHUNK; i += LT) {
        const int64_t j = base + i;
        if (j >= n) break;
        bool reset;
        const uint8_t a = classify(t, in.log_scales + 3 * j, in.omega[j], acc ? acc[j] : 0.f, cnt ? cnt[j] : 0, reset);
        action[j] = (uint8_t)(a | (reset ? 0x80 : 0));
        c += out_count(a);
    }
    const uint32_t tot = block_sum_u32(c, sm);
    if (threadIdx.x == 0) block_sum[blockIdx.x] = tot;
}

// One block: exclusive scan of the block sums, the total and the capacity
// check, then the new submap offsets (output position of each submap's first
// splat: the offset of its chunk plus the counts before it in the chunk).
__global__ void __launch_bounds__(LT) k_lc_scan(const uint32_t *block_sum, int nblocks, const uint8_t *action,
                                                int64_t n, const int64_t *offs_in, int n_submaps, int64_t capacity,
                                                uint32_t *block_off, int64_t *offs_out, int64_t *state, int64_t *n_out) {
    __shared__ uint32_t sm[LT / 32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += LT) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nblocks ? block_sum[b] : 0u;
        uint32_t tot;
        const uint32_t ex = block_scan_u32(v, sm, tot);
        if (b < nblocks) block_off[b] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    const int64_t total = carry;
    const bool fits = total <= capacity;
    if (threadIdx.x == 0) {
        state[0] = total;
        state[1] = fits ? 0 : 1;
        if (n_out) *n_out = total;
    }
    if (!fits || !offs_out) return;
    for (int s = 0; s <= n_submaps; ++s) {
        const int64_t j = offs_in[s];
        uint32_t c = 0;
        int64_t pos;
        if (j >= n) {
            pos = total;
        } else {
            const int64_t cb = j / LCHUNK;
            for (int64_t i = cb * LCHUNK + threadIdx.x; i < j; i += LT) c += out_count(action[i] & 0x7f);
            const uint32_t t = block_sum_u32(c, sm);
            pos = (int64_t)block_off[cb] + t;
        }
        if (threadIdx.x == 0) offs_out[s] = pos;
        __syncthreads();
    }
}

__device__ __forceinline__ void quat_rot(const float *q, float R[9]) {
    const float n = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] * n, x = q[1] * n, y = q[2] * n, z = q[3] * n;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

struct ScatterArgs {
    Thresholds t;
    Arrays in, in_m, in_v;
    OutArrays out, out_m, out_v;
    const float *normals;  // [n][2][3]
    const uint8_t *action;
    const uint32_t *block_off;
    const int64_t *state;
    int64_t n;
    int32_t nsh;  // SH floats per splat
    bool moments;
};

// Optimiser moments of one output row (small fields): the source's, or zero
// for a new splat.
__device__ __forceinline__ void copy_moment_row(const Arrays src, const OutArrays dst, int64_t j, int64_t o,
                                                bool fresh) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        dst.means[3 * o + r] = fresh ? 0.f : src.means[3 * j + r];
        dst.log_scales[3 * o + r] = fresh ? 0.f : src.log_scales[3 * j + r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) dst.quats[4 * o + r] = fresh ? 0.f : src.quats[4 * j + r];
    dst.omega[o] = fresh ? 0.f : src.omega[j];
}

// Writes one output row of the small fields (the SH rows are copied apart).
__device__ __forceinline__ void write_row(const ScatterArgs &A, int64_t j, int64_t o, uint8_t a, int k,
                                          bool reset) {
    float mean[3] = {A.in.means[3 * j], A.in.means[3 * j + 1], A.in.means[3 * j + 2]};
    float ls[3] = {A.in.log_scales[3 * j], A.in.log_scales[3 * j + 1], A.in.log_scales[3 * j + 2]};
    const float *q = A.in.quats + 4 * j;
    if (a == A_SPLIT) {
        float R[9];
        quat_rot(q, R);
        const float *z = A.normals + 6 * j + 3 * k;
        const float v0 = expf(ls[0]) * z[0], v1 = expf(ls[1]) * z[1], v2 = expf(ls[2]) * z[2];
#pragma unroll
        for (int r = 0; r < 3; ++r) mean[r] += R[3 * r] * v0 + R[3 * r + 1] * v1 + R[3 * r + 2] * v2;
#pragma unroll
        for (int r = 0; r < 3; ++r) ls[r] -= A.t.shrink;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        A.out.means[3 * o + r] = mean[r];
        A.out.log_scales[3 * o + r] = ls[r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) A.out.quats[4 * o + r] = q[r];
    A.out.omega[o] = reset ? A.t.reset : A.in.omega[j];
    if (A.moments) {
        const bool fresh = a == A_SPLIT || (a == A_CLONE && k == 1);
        copy_moment_row(A.in_m, A.out_m, j, o, fresh);
        copy_moment_row(A.in_v, A.out_v, j, o, fresh);
    }
}

__global__ void __launch_bounds__(LT) k_lc_scatter(ScatterArgs A) {
    __shared__ uint32_t sm[LT / 32];
    __shared__ uint32_t s_carry;
    if (A.state[1]) return;  // over capacity: nothing is written
    const int64_t base = (int64_t)blockIdx.x * LCHUNK;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_carry = A.block_off[blockIdx.x];
    __syncthreads();
    for (int i0 = 0; i0 < LCHUNK; i0 += LT) {
        const int64_t j = base + i0 + threadIdx.x;
        const uint8_t code = j < A.n ? A.action[j] : (uint8_t)A_PRUNE;
        const uint8_t a = code & 0x7f;
        const bool reset = code & 0x80;
        const uint32_t c = out_count(a);
        uint32_t tot;
        const uint32_t ex = block_scan_u32(c, sm, tot);
        const int64_t o = (int64_t)s_carry + ex;
        for (uint32_t k = 0; k < c; ++k) write_row(A, j, o + k, a, (int)k, reset);
        // SH rows: each warp copies the rows of its 32 splats, lanes along the row
        for (int src = 0; src < 32; ++src) {
            const uint32_t cs = __shfl_sync(0xffffffffu, c, src);
            if (cs == 0) continue;
            const int64_t js = __shfl_sync(0xffffffffu, j, src);
            const int64_t os = __shfl_sync(0xffffffffu, o, src);
            const uint8_t as = (uint8_t)__shfl_sync(0xffffffffu, (uint32_t)a, src);
            for (uint32_t k = 0; k < cs; ++k) {
                const bool fresh = as == A_SPLIT || (as == A_CLONE && k == 1);
                for (int e = lane; e < A.nsh; e += 32) {
                    A.out.sh[(os + k) * A.nsh + e] = A.in.sh[js * A.nsh + e];
                    if (A.moments) {
                        A.out_m.sh[(os + k) * A.nsh + e] = fresh ? 0.f : A.in_m.sh[js * A.nsh + e];
                        A.out_v.sh[(os + k) * A.nsh + e] = fresh ? 0.f : A.in_v.sh[js * A.nsh + e];
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
        if (base + i0 + LT >= A.n) break;
    }
}

// Adam over the five parameter arrays.  Each block takes a chunk of
// kAdamChunk elements of one array (blocks are assigned to arrays in
// proportion to their lengths, so the long SH array gets most of them);
// float4 accesses where the chunk is 16-byte aligned.  With a = lr / bc1 and
// r = 1 / sqrt(bc2): p -= a m / (sqrt(v) r + eps), the formula of R22.
constexpr int kAdamChunk = 4 * 4 * LT;  // 4 float4 per thread
struct AdamSeg {
    float *p, *m, *v;
    const float *g;
    int64_t n;
    float a;       // lr / (1 - beta1^step)
    int32_t b0;    // first block of this array
};
struct AdamArgs {
    AdamSeg seg[5];
    float b1, b2, eps, r;  // r = 1 / sqrt(1 - beta2^step)
};

__device__ __forceinline__ void adam_one(float &p, float &m, float &v, float g, float a, const AdamArgs &A) {
    m = __fmaf_rn(A.b1, m - g, g);           // b1 m + (1 - b1) g
    v = __fmaf_rn(A.b2, v - g * g, g * g);   // b2 v + (1 - b2) g^2
    p -= a * m / __fmaf_rn(sqrtf(v), A.r, A.eps);
}

__global__ void __launch_bounds__(LT) k_adam(AdamArgs A) {
    const int b = blockIdx.x;
    const int s = (b >= A.seg[1].b0) + (b >= A.seg[2].b0) + (b >= A.seg[3].b0) + (b >= A.seg[4].b0);
    AdamSeg S;
    switch (s) {
        case 0: S = A.seg[0]; break;
        case 1: S = A.seg[1]; break;
        case 2: S = A.seg[2]; break;
        case 3: S = A.seg[3]; break;
        default: S = A.seg[4]; break;
    }
    const int64_t lo = (int64_t)(b - S.b0) * kAdamChunk;
    const int64_t hi = min(S.n, lo + (int64_t)kAdamChunk);
    const bool vec = ((((uintptr_t)S.p) | ((uintptr_t)S.m) | ((uintptr_t)S.v) | ((uintptr_t)S.g)) & 15) == 0 &&
                     hi - lo == kAdamChunk;
    if (vec) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = lo + 4 * ((int64_t)k * LT + threadIdx.x);
            float4 p = *reinterpret_cast<float4 *>(S.p + i), m = *reinterpret_cast<float4 *>(S.m + i);
            float4 v = *reinterpret_cast<float4 *>(S.v + i);
            const float4 g = *reinterpret_cast<const float4 *>(S.g + i);
            adam_one(p.x, m.x, v.x, g.x, S.a, A);
            adam_one(p.y, m.y, v.y, g.y, S.a, A);
            adam_one(p.z, m.z, v.z, g.z, S.a, A);
            adam_one(p.w, m.w, v.w, g.w, S.a, A);
            *reinterpret_cast<float4 *>(S.p + i) = p;
            *reinterpret_cast<float4 *>(S.m + i) = m;
            *reinterpret_cast<float4 *>(S.v + i) = v;
        }
    } else {
        for (int64_t i = lo + threadIdx.x; i < hi; i += LT) {
            float p = S.p[i], m = S.m[i], v = S.v[i];
            adam_one(p, m, v, S.g[i], S.a, A);
            S.p[i] = p;
            S.m[i] = m;
            S.v[i] = v;
        }
    }
}

// Zeroing of up to kZeroMax device buffers in one launch: blocks are given to
// the buffers in proportion to their sizes, 16 bytes per store where aligned.
constexpr int kZeroMax = 16;
constexpr int kZeroChunk = 16 * 4 * LT;  // bytes per block
struct ZeroArgs {
    unsigned char *p[kZeroMax];
    int64_t bytes[kZeroMax];
    int32_t b0[kZeroMax + 1];  // first block of each buffer
    int32_t n;
};

__global__ void __launch_bounds__(LT) k_zero(ZeroArgs A) {
    const int b = blockIdx.x;
    int s = 0;
#pragma unroll 1
    while (s + 1 < A.n && b >= A.b0[s + 1]) ++s;
    unsigned char *p = A.p[s];
    const int64_t lo = (int64_t)(b - A.b0[s]) * kZeroChunk;
    const int64_t hi = min(A.bytes[s], lo + (int64_t)kZeroChunk);
    if ((((uintptr_t)p) & 15) == 0) {
        const int64_t v_lo = (lo + 15) / 16, v_hi = hi / 16;
        for (int64_t i = v_lo + threadIdx.x; i < v_hi; i += LT)
            reinterpret_cast<float4 *>(p)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t i = lo + threadIdx.x; i < min(hi, v_lo * 16); i += LT) p[i] = 0;
        for (int64_t i = max(lo, v_hi * 16) + threadIdx.x; i < hi; i += LT) p[i] = 0;
    } else {
        for (int64_t i = lo + threadIdx.x; i < hi; i += LT) p[i] = 0;
    }
}

Thresholds thresholds(const gs_lifecycle_params &p) {
    auto logit = [](double t) { return (float)std::log(t / (1.0 - t)); };
    Thresholds t{};
    t.opa = logit(p.prune_opacity);
    t.smax = (float)std::log((double)p.prune_scale_max);
    t.smin = (float)std::log((double)p.prune_scale_min);
    t.grad = p.densify_grad;
    t.split = (float)std::log((double)p.split_scale);
    t.clone = (float)std::log((double)p.clone_scale);
    t.reset = logit(p.reset_opacity);
    t.rmin = (float)std::log((double)p.reset_scale_min);
    t.rmax = (float)std::log((double)p.reset_scale_max);
    t.shrink = (float)std::log((double)p.split_shrink);
    t.ops = p.ops;
    return t;
}

bool all_set(const gs_param_arrays *a) {
    return a && a->means && a->log_scales && a->quats && a->opacity_logits && a->sh;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_lifecycle_create(int64_t max_in, int32_t max_submaps, gs_lifecycle **out) {
    if (!out || max_in < 0 || max_in > 0x3FFFFFFFll || max_submaps < 1 || max_submaps > GS_MAX_SUBMAPS) {
        set_last_error("gs_lifecycle_create: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    gs_lifecycle *lc = new gs_lifecycle();
    lc->max_in = max_in;
    lc->max_submaps = max_submaps;
    lc->nblocks_max = (int32_t)std::max<int64_t>(1, (max_in + LCHUNK - 1) / LCHUNK);
    cudaError_t e = cudaMalloc(&lc->action, std::max<int64_t>(1, max_in));
    if (e == cudaSuccess) e = cudaMalloc(&lc->block_sum, sizeof(uint32_t) * lc->nblocks_max);
    if (e == cudaSuccess) e = cudaMalloc(&lc->block_off, sizeof(uint32_t) * lc->nblocks_max);
    if (e == cudaSuccess) e = cudaMalloc(&lc->state, sizeof(int64_t) * 2);
    if (e == cudaSuccess) e = cudaMemset(lc->state, 0, sizeof(int64_t) * 2);
    if (e != cudaSuccess) {
        set_last_error(std::string("gs_lifecycle_create: ") + cudaGetErrorString(e));
        gs_lifecycle_destroy(lc);
        return GS_ERR_CUDA;
    }
    *out = lc;
    return GS_OK;
}

void gs_lifecycle_destroy(gs_lifecycle *lc) {
    if (!lc) return;
    cudaFree(lc->action);
    cudaFree(lc->block_sum);
    cudaFree(lc->block_off);
    cudaFree(lc->state);
    delete lc;
}

gs_status gs_lifecycle_run(gs_lifecycle *lc, const gs_lifecycle_params *p, int32_t sh_degree, int64_t n_in,
                           int32_t n_submaps, const int64_t *submap_offsets_in, const gs_param_arrays *in,
                           const gs_param_arrays *in_m, const gs_param_arrays *in_v, const float *densify_acc,
                           const int32_t *densify_cnt, const float *split_normals, const gs_param_arrays *out,
                           const gs_param_arrays *out_m, const gs_param_arrays *out_v, int64_t out_capacity,
                           int64_t *submap_offsets_out, int64_t *n_out, void *stream) {
    if (!lc || !p || !in || !out || !submap_offsets_in) {
        set_last_error("gs_lifecycle_run: NULL argument");
        return GS_ERR_INVALID_ARG;
    }
    if (n_in < 0 || n_in > lc->max_in || n_submaps < 1 || n_submaps > lc->max_submaps || sh_degree < 0 ||
        sh_degree > 3 || out_capacity < 0 || out_capacity > 0x7FFFFFFFll) {
        set_last_error("gs_lifecycle_run: size out of range");
        return GS_ERR_INVALID_ARG;
    }
    const bool moments = in_m || in_v || out_m || out_v;
    if ((n_in > 0 && !all_set(in)) || (out_capacity > 0 && !all_set(out)) ||
        (moments && !(all_set(in_m) && all_set(in_v) && all_set(out_m) && all_set(out_v)))) {
        set_last_error("gs_lifecycle_run: a parameter array is NULL");
        return GS_ERR_INVALID_ARG;
    }
    if ((p->ops & GS_LC_DENSIFY) && (!densify_acc || !densify_cnt || !split_normals)) {
        set_last_error("gs_lifecycle_run: densification needs the statistic and the split normals");
        return GS_ERR_INVALID_ARG;
    }
    if ((p->ops & ~(GS_LC_PRUNE | GS_LC_DENSIFY | GS_LC_RESET)) || !(p->prune_opacity > 0.f && p->prune_opacity < 1.f) ||
        !(p->reset_opacity > 0.f && p->reset_opacity < 1.f) || !(p->prune_scale_max > 0.f) ||
        !(p->prune_scale_min > 0.f) || !(p->split_scale > 0.f) || !(p->clone_scale > 0.f) ||
        !(p->split_shrink > 0.f) || !(p->reset_scale_min > 0.f) || !(p->reset_scale_max > 0.f)) {
        set_last_error("gs_lifecycle_run: bad parameters");
        return GS_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Thresholds t = thresholds(*p);
    const int nblocks = (int)std::max<int64_t>(1, (n_in + LCHUNK - 1) / LCHUNK);
    auto arr = [](const gs_param_arrays *a) {
        return a ? Arrays{a->means, a->log_scales, a->quats, a->opacity_logits, a->sh} : Arrays{};
    };
    auto oarr = [](const gs_param_arrays *a) {
        return a ? OutArrays{a->means, a->log_scales, a->quats, a->opacity_logits, a->sh} : OutArrays{};
    };
    if (n_in > 0) {
        ++lc->kernel_launches;
        k_lc_classify<<<nblocks, LT, 0, s>>>(t, arr(in), densify_acc, densify_cnt, n_in, lc->action, lc->block_sum);
    } else {
        cudaMemsetAsync(lc->block_sum, 0, sizeof(uint32_t), s);
    }
    ++lc->kernel_launches;
    k_lc_scan<<<1, LT, 0, s>>>(lc->block_sum, n_in > 0 ? nblocks : 0, lc->action, n_in, submap_offsets_in, n_submaps,
                               out_capacity, lc->block_off, submap_offsets_out, lc->state, n_out);
    gs_status r = check_launch("lifecycle");
    if (r != GS_OK || n_in == 0) return r;
    ScatterArgs A{};
    A.t = t;
    A.in = arr(in);
    A.in_m = arr(in_m);
    A.in_v = arr(in_v);
    A.out = oarr(out);
    A.out_m = oarr(out_m);
    A.out_v = oarr(out_v);
    A.normals = split_normals;
    A.action = lc->action;
    A.block_off = lc->block_off;
    A.state = lc->state;
    A.n = n_in;
    A.nsh = 3 * (sh_degree + 1) * (sh_degree + 1);
    A.moments = moments;
    ++lc->kernel_launches;
    k_lc_scatter<<<nblocks, LT, 0, s>>>(A);
    return check_launch("lifecycle_scatter");
}

gs_status gs_lifecycle_status(gs_lifecycle *lc, void *stream, int64_t *n_needed) {
    if (!lc) {
        set_last_error("gs_lifecycle_status: NULL argument");
        return GS_ERR_INVALID_ARG;
    }
    int64_t h[2] = {0, 0};
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(h, lc->state, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_last_error(std::string("gs_lifecycle_status: ") + cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    if (n_needed) *n_needed = h[0];
    return h[1] ? GS_ERR_CAPACITY : GS_OK;
}

gs_status gs_zero_buffers(void *const *ptrs, const int64_t *bytes, int32_t count, void *stream) {
    if (count < 0 || count > kZeroMax || (count > 0 && (!ptrs || !bytes))) {
        set_last_error("gs_zero_buffers: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    ZeroArgs A{};
    int64_t blocks = 0;
    for (int i = 0; i < count; ++i) {
        if (bytes[i] < 0 || (bytes[i] > 0 && !ptrs[i])) {
            set_last_error("gs_zero_buffers: bad buffer");
            return GS_ERR_INVALID_ARG;
        }
        if (bytes[i] == 0) continue;
        A.p[A.n] = static_cast<unsigned char *>(ptrs[i]);
        A.bytes[A.n] = bytes[i];
        A.b0[A.n] = (int32_t)blocks;
        blocks += (bytes[i] + kZeroChunk - 1) / kZeroChunk;
        ++A.n;
    }
    if (A.n == 0) return GS_OK;
    if (blocks > 0x7FFFFFFF) {
        set_last_error("gs_zero_buffers: too large");
        return GS_ERR_INVALID_ARG;
    }
    A.b0[A.n] = (int32_t)blocks;
    k_zero<<<(unsigned)blocks, LT, 0, (cudaStream_t)stream>>>(A);
    return check_launch("zero_buffers");
}

gs_status gs_adam_step(const gs_param_arrays *param, const gs_param_arrays *grad, const gs_param_arrays *m,
                       const gs_param_arrays *v, int64_t n, int32_t sh_degree, const gs_adam_params *p,
                       void *stream) {
    if (!p || n < 0 || sh_degree < 0 || sh_degree > 3 || p->step < 1 || !(p->beta1 >= 0.f && p->beta1 < 1.f) ||
        !(p->beta2 >= 0.f && p->beta2 < 1.f) || !(p->eps >= 0.f)) {
        set_last_error("gs_adam_step: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    if (n == 0) return GS_OK;
    if (!all_set(param) || !all_set(grad) || !all_set(m) || !all_set(v)) {
        set_last_error("gs_adam_step: a parameter array is NULL");
        return GS_ERR_INVALID_ARG;
    }
    AdamArgs A{};
    const int64_t len[5] = {3 * n, 3 * n, 4 * n, n, 3 * n * (sh_degree + 1) * (sh_degree + 1)};
    float *ps[5] = {param->means, param->log_scales, param->quats, param->opacity_logits, param->sh};
    const float *gs_[5] = {grad->means, grad->log_scales, grad->quats, grad->opacity_logits, grad->sh};
    float *ms[5] = {m->means, m->log_scales, m->quats, m->opacity_logits, m->sh};
    float *vs[5] = {v->means, v->log_scales, v->quats, v->opacity_logits, v->sh};
    const double bc1 = 1.0 - std::pow((double)p->beta1, (double)p->step);
    const double bc2 = 1.0 - std::pow((double)p->beta2, (double)p->step);
    int64_t blocks = 0;
    for (int s = 0; s < 5; ++s) {
        A.seg[s] = AdamSeg{ps[s], ms[s], vs[s], gs_[s], len[s], (float)((double)p->lr[s] / bc1), (int32_t)blocks};
        blocks += (len[s] + kAdamChunk - 1) / kAdamChunk;
    }
    if (blocks > 0x7FFFFFFF) {
        set_last_error("gs_adam_step: too many parameters");
        return GS_ERR_INVALID_ARG;
    }
    A.b1 = p->beta1;
    A.b2 = p->beta2;
    A.eps = p->eps;
    A.r = (float)(1.0 / std::sqrt(bc2));
    k_adam<<<(unsigned)blocks, LT, 0, (cudaStream_t)stream>>>(A);
    return check_launch("adam");
}

}  // extern "C"
