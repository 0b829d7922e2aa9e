// Voxel-hash insertion of fused points (Sec. III-B, Eq. 5) and the LRU active
// set of the incremental map ("Memory Management").
//
// Keys: k = floor(x/v) P1 + floor(y/v) P2 + floor(z/v) P3 in unsigned 64-bit
// arithmetic (wrap-around), P = Teschner et al.'s primes, x/v divided in
// float32 (IEEE) before the floor.  The all-ones key is folded onto its
// predecessor so that it can mark empty hash slots.
//
// Insertion of a batch of points at frame f uses one open-addressing table
// over the batch's point keys (capacity a power of two >= 2 points, linear
// probing; each slot keeps the smallest point index that carries its key):
//   1. every point inserts its key (atomicCAS) and records its slot;
//   2. every device splat probes its key: found -> last_used = f and the
//      voxel is marked known; every host-resident key likewise -> reload flag;
//   3. the points that are the first of an unknown voxel create new splats,
//      compacted in point order (deterministic): mean = the point, isotropic
//      log-scale ln(s_init), identity rotation, opacity o_init, SH DC =
//      (rgb - 1/2) / Y00, higher coefficients 0.
// LRU selection: with n > tau splats, the (n - tau) smallest (last_used,
// index) pairs are flagged, by an exact radix select of the last_used value
// (four 8-bit passes) and an ordered count of the ties.
// Partition: a stable split of the splat rows by a flag array into a kept and
// a moved set; either side may live in host-mapped memory (offload, reload).
#include "gs_internal.cuh"
#include "gs_scan.cuh"

#include <cmath>

namespace {
constexpr unsigned long long kEmpty = ~0ull;
}

struct gs_voxel {
    int64_t max_points = 0, max_items = 0;
    uint64_t cap = 0;
    int cap_bits = 0;
    unsigned long long *tkey = nullptr;  // [cap]
    int32_t *tmin = nullptr;             // [cap]
    int32_t *tknown = nullptr;           // [cap]
    uint32_t *pslot = nullptr;           // [max_points]
    uint32_t *block_sum = nullptr, *block_off = nullptr;  // [nblocks]
    uint32_t *hist = nullptr;            // [256]
    uint32_t *sel = nullptr;             // [4] prefix, mask, remaining rank
    int64_t *state = nullptr;            // [0] new splats needed, [1] capacity flag, [2] kept, [3] moved
    int64_t kernel_launches = 0;
};

namespace gs {
namespace {

constexpr int VT = 256;
constexpr int VCHUNK = 8 * VT;
constexpr unsigned long long kP1 = 73856093ull, kP2 = 19349663ull, kP3 = 83492791ull;
constexpr float kY00 = 0.28209479177387814f;

__device__ __forceinline__ unsigned long long voxel_key(float x, float y, float z, float v) {
    const long long cx = (long long)floorf(__fdiv_rn(x, v));
    const long long cy = (long long)floorf(__fdiv_rn(y, v));
    const long long cz = (long long)floorf(__fdiv_rn(z, v));
    const unsigned long long k = (unsigned long long)cx * kP1 + (unsigned long long)cy * kP2 +
                                 (unsigned long long)cz * kP3;
    return k == kEmpty ? kEmpty - 1 : k;
}

__device__ __forceinline__ uint32_t slot_of(unsigned long long k, int bits) {
    return (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

__global__ void __launch_bounds__(VT) k_voxel_keys(const float *xyz, int64_t n, int32_t stride, float v,
                                                   unsigned long long *keys) {
    for (int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT) {
        const float *p = xyz + i * stride;
        keys[i] = voxel_key(p[0], p[1], p[2], v);
    }
}

__global__ void __launch_bounds__(VT) k_table_insert(const float *pts, int64_t n, float v, unsigned long long *tkey,
                                                     int32_t *tmin, uint32_t *pslot, int bits) {
    const uint32_t mask = (1u << bits) - 1u;
    for (int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT) {
        const float *p = pts + 6 * i;
        const unsigned long long k = voxel_key(p[0], p[1], p[2], v);
        uint32_t s = slot_of(k, bits);
        // at most n distinct keys in a table of >= 2n slots: a free or
        // matching slot exists, so the probe ends within (mask + 1) steps
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long cur = atomicCAS(tkey + s, kEmpty, k);
            if (cur == kEmpty || cur == k) {
                atomicMin(tmin + s, (int32_t)i);
                pslot[i] = s;
                break;
            }
            s = (s + 1u) & mask;
        }
    }
}

// Probes keys[j] in the table: found -> out[j] = value (or leaves it when
// `only_found`), and marks the voxel known; not found -> out[j] = miss.
__global__ void __launch_bounds__(VT) k_table_probe(const unsigned long long *keys, int64_t n,
                                                    const unsigned long long *tkey, int32_t *tknown, int bits,
                                                    int32_t *out, int32_t value, bool only_found, int32_t miss) {
    const uint32_t mask = (1u << bits) - 1u;
    for (int64_t j = (int64_t)blockIdx.x * VT + threadIdx.x; j < n; j += (int64_t)gridDim.x * VT) {
        unsigned long long k = keys[j];
        if (k == kEmpty) k = kEmpty - 1;
        uint32_t s = slot_of(k, bits);
        bool found = false;
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long cur = tkey[s];
            if (cur == kEmpty) break;
            if (cur == k) {
                found = true;
                tknown[s] = 1;
                break;
            }
            s = (s + 1u) & mask;
        }
        if (found) out[j] = value;
        else if (!only_found) out[j] = miss;
    }
}

__device__ __forceinline__ uint32_t is_creator(int64_t i, int64_t n, const uint32_t *pslot, const int32_t *tmin,
                                               const int32_t *tknown) {
    if (i >= n) return 0u;
    const uint32_t s = pslot[i];
    return (tknown[s] == 0 && tmin[s] == (int32_t)i) ? 1u : 0u;
}

__global__ void __launch_bounds__(VT) k_creator_count(int64_t n, const uint32_t *pslot, const int32_t *tmin,
                                                      const int32_t *tknown, uint32_t *block_sum) {
    __shared__ uint32_t sm[VT / 32];
    const int64_t base = (int64_t)blockIdx.x * VCHUNK;
    uint32_t c = 0;
    for (int i = threadIdx.x; i < VCHUNK; i += VT) c += is_creator(base + i, n, pslot, tmin, tknown);
    const uint32_t t = block_sum_u32<VT>(c, sm);
    if (threadIdx.x == 0) block_sum[blockIdx.x] = t;
}

// One block: exclusive scan of the block sums; total -> state[0] (and *total_out),
// total > capacity -> state[1].
__global__ void __launch_bounds__(VT) k_scan_blocks(const uint32_t *block_sum, int nblocks, uint32_t *block_off,
                                                    int64_t capacity, int64_t *state, int64_t *total_out) {
    __shared__ uint32_t sm[VT / 32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += VT) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nblocks ? block_sum[b] : 0u;
        uint32_t tot;
        const uint32_t ex = block_scan_u32<VT>(v, sm, tot);
        if (b < nblocks) block_off[b] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        state[0] = carry;
        state[1] = (int64_t)carry > capacity ? 1 : 0;
        if (total_out) *total_out = carry;
    }
}

struct EmitArgs {
    const float *pts;
    int64_t n;
    float v, log_s, omega;
    const uint32_t *pslot;
    const int32_t *tmin, *tknown;
    const uint32_t *block_off;
    const int64_t *state;
    float *means, *log_scales, *quats, *opacity, *sh;
    unsigned long long *keys;
    int32_t nsh;
};

__global__ void __launch_bounds__(VT) k_creator_emit(EmitArgs A) {
    __shared__ uint32_t sm[VT / 32];
    __shared__ uint32_t carry;
    if (A.state[1]) return;
    const int64_t base = (int64_t)blockIdx.x * VCHUNK;
    if (threadIdx.x == 0) carry = A.block_off[blockIdx.x];
    __syncthreads();
    for (int i0 = 0; i0 < VCHUNK; i0 += VT) {
        const int64_t i = base + i0 + threadIdx.x;
        const uint32_t c = is_creator(i, A.n, A.pslot, A.tmin, A.tknown);
        uint32_t tot;
        const uint32_t ex = block_scan_u32<VT>(c, sm, tot);
        if (c) {
            const int64_t o = (int64_t)carry + ex;
            const float *p = A.pts + 6 * i;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                A.means[3 * o + r] = p[r];
                A.log_scales[3 * o + r] = A.log_s;
            }
            A.quats[4 * o] = 1.f;
            A.quats[4 * o + 1] = A.quats[4 * o + 2] = A.quats[4 * o + 3] = 0.f;
            A.opacity[o] = A.omega;
            float *sh = A.sh + o * A.nsh;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) sh[ch] = (p[3 + ch] - 0.5f) / kY00;
            for (int e = 3; e < A.nsh; ++e) sh[e] = 0.f;
            A.keys[o] = voxel_key(p[0], p[1], p[2], A.v);
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
        if (base + i0 + VT >= A.n) break;
    }
}

// ---------------------------------------------------------------------------
// LRU selection
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t lru_bits(int32_t v) { return (uint32_t)v ^ 0x80000000u; }

__global__ void __launch_bounds__(VT) k_sel_hist(const int32_t *lu, int64_t n, const uint32_t *sel, int shift,
                                                 uint32_t *hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t prefix = sel[0], mask = sel[1];
    for (int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT) {
        const uint32_t u = lru_bits(lu[i]);
        if ((u & mask) == prefix) atomicAdd(h + ((u >> shift) & 255u), 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(hist + threadIdx.x, h[threadIdx.x]);
}

// one block of 256: the digit where the remaining rank falls
__global__ void __launch_bounds__(256) k_sel_pick(uint32_t *hist, uint32_t *sel, int shift) {
    __shared__ uint32_t sm[8];
    const uint32_t c = hist[threadIdx.x];
    uint32_t tot;
    const uint32_t before = block_scan_u32<256>(c, sm, tot);
    const uint32_t r = sel[2];
    __syncthreads();
    if (before < r && before + c >= r) {
        sel[0] |= threadIdx.x << shift;
        sel[1] |= 255u << shift;
        sel[2] = r - before;
    }
    hist[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(VT) k_sel_eqcount(const int32_t *lu, int64_t n, const uint32_t *sel,
                                                    uint32_t *block_sum) {
    __shared__ uint32_t sm[VT / 32];
    const int64_t base = (int64_t)blockIdx.x * VCHUNK;
    const uint32_t f = sel[0];
    uint32_t c = 0;
    for (int i = threadIdx.x; i < VCHUNK; i += VT) {
        const int64_t j = base + i;
        if (j < n && lru_bits(lu[j]) == f) ++c;
    }
    const uint32_t t = block_sum_u32<VT>(c, sm);
    if (threadIdx.x == 0) block_sum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(VT) k_sel_mark(const int32_t *lu, int64_t n, const uint32_t *sel,
                                                 const uint32_t *block_off, int32_t *flags) {
    __shared__ uint32_t sm[VT / 32];
    __shared__ uint32_t carry;
    const int64_t base = (int64_t)blockIdx.x * VCHUNK;
    const uint32_t f = sel[0], r = sel[2];
    if (threadIdx.x == 0) carry = block_off[blockIdx.x];
    __syncthreads();
    for (int i0 = 0; i0 < VCHUNK; i0 += VT) {
        const int64_t j = base + i0 + threadIdx.x;
        const uint32_t u = j < n ? lru_bits(lu[j]) : 0xFFFFFFFFu;
        const uint32_t eq = (j < n && u == f) ? 1u : 0u;
        uint32_t tot;
        const uint32_t ex = block_scan_u32<VT>(eq, sm, tot);
        if (j < n) flags[j] = (u < f || (eq && carry + ex < r)) ? 1 : 0;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
        if (base + i0 + VT >= n) break;
    }
}

__global__ void k_sel_init(uint32_t *sel, uint32_t m) {
    sel[0] = 0u;
    sel[1] = 0u;
    sel[2] = m;
    sel[3] = 0u;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---------------------------------------------------------------------------
// stable partition
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(VT) k_flag_count(const int32_t *flags, int64_t n, uint32_t *block_sum) {
    __shared__ uint32_t sm[VT / 32];
    const int64_t base = (int64_t)blockIdx.x * VCHUNK;
    uint32_t c = 0;
    for (int i = threadIdx.x; i < VCHUNK; i += VT) {
        const int64_t j = base + i;
        if (j < n && flags[j]) ++c;
    }
    const uint32_t t = block_sum_u32<VT>(c, sm);
    if (threadIdx.x == 0) block_sum[blockIdx.x] = t;
}

struct PartArgs {
    const int32_t *flags;
    int64_t n;
    const uint32_t *block_off;
    const float *in[5];
    float *kept[5], *moved[5];
    const unsigned long long *in_keys;
    unsigned long long *kept_keys, *moved_keys;
    const int32_t *in_lu;
    int32_t *kept_lu, *moved_lu;
    int32_t nsh;
};

__device__ __forceinline__ void copy_small(const PartArgs &A, int64_t j, int64_t o, bool mv) {
    float *const *dst = mv ? A.moved : A.kept;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        dst[0][3 * o + r] = A.in[0][3 * j + r];
        dst[1][3 * o + r] = A.in[1][3 * j + r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) dst[2][4 * o + r] = A.in[2][4 * j + r];
    dst[3][o] = A.in[3][j];
    if (A.in_keys) (mv ? A.moved_keys : A.kept_keys)[o] = A.in_keys[j];
    if (A.in_lu) (mv ? A.moved_lu : A.kept_lu)[o] = A.in_lu[j];
}

__global__ void __launch_bounds__(VT) k_partition(PartArgs A) {
    __shared__ uint32_t sm[VT / 32];
    __shared__ uint32_t carry;
    const int64_t base = (int64_t)blockIdx.x * VCHUNK;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) carry = A.block_off[blockIdx.x];
    __syncthreads();
    for (int i0 = 0; i0 < VCHUNK; i0 += VT) {
        const int64_t j = base + i0 + threadIdx.x;
        const bool valid = j < A.n;
        const uint32_t f = valid && A.flags[j] ? 1u : 0u;
        uint32_t tot;
        const uint32_t ex = block_scan_u32<VT>(f, sm, tot);
        const int64_t moved_before = (int64_t)carry + ex;
        const int64_t o = f ? moved_before : j - moved_before;
        if (valid) copy_small(A, j, o, f);
        // SH rows: each warp copies the rows of its 32 splats, lanes along the row
        for (int src = 0; src < 32; ++src) {
            const bool vs = __shfl_sync(0xffffffffu, valid, src);
            if (!vs) continue;
            const int64_t js = __shfl_sync(0xffffffffu, j, src);
            const int64_t os = __shfl_sync(0xffffffffu, o, src);
            const bool fs = __shfl_sync(0xffffffffu, f, src);
            float *dst = fs ? A.moved[4] : A.kept[4];
            for (int e = lane; e < A.nsh; e += 32) dst[os * A.nsh + e] = A.in[4][js * A.nsh + e];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
        if (base + i0 + VT >= A.n) break;
    }
}

__global__ void k_partition_counts(const int64_t *state, int64_t n, int64_t *out) {
    out[0] = n - state[0];
    out[1] = state[0];
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + VT - 1) / VT, 152 * 16)); }
int nblocks_for(int64_t n) { return (int)std::max<int64_t>(1, (n + VCHUNK - 1) / VCHUNK); }

bool params_set(const gs_param_arrays *a) {
    return a && a->means && a->log_scales && a->quats && a->opacity_logits && a->sh;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_voxel_keys(const float *xyz, int64_t n, int32_t stride, float voxel, uint64_t *keys, void *stream) {
    if (n < 0 || stride < 3 || !(voxel > 0.f) || (n > 0 && (!xyz || !keys))) {
        set_last_error("gs_voxel_keys: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    if (n == 0) return GS_OK;
    k_voxel_keys<<<grid_for(n), VT, 0, (cudaStream_t)stream>>>(xyz, n, stride, voxel,
                                                                 reinterpret_cast<unsigned long long *>(keys));
    return check_launch("voxel_keys");
}

gs_status gs_voxel_create(int64_t max_points, int64_t max_items, gs_voxel **out) {
    if (!out || max_points < 0 || max_items < 0 || max_points > (1ll << 29) || max_items > (1ll << 30)) {
        set_last_error("gs_voxel_create: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    gs_voxel *vx = new gs_voxel();
    vx->max_points = max_points;
    vx->max_items = max_items;
    vx->cap_bits = 4;
    while ((1ll << vx->cap_bits) < 2 * std::max<int64_t>(1, max_points)) ++vx->cap_bits;
    vx->cap = 1ull << vx->cap_bits;
    const int nb = nblocks_for(std::max(max_points, max_items));
    cudaError_t e = cudaMalloc(&vx->tkey, sizeof(unsigned long long) * vx->cap);
    if (e == cudaSuccess) e = cudaMalloc(&vx->tmin, sizeof(int32_t) * vx->cap);
    if (e == cudaSuccess) e = cudaMalloc(&vx->tknown, sizeof(int32_t) * vx->cap);
    if (e == cudaSuccess) e = cudaMalloc(&vx->pslot, sizeof(uint32_t) * std::max<int64_t>(1, max_points));
    if (e == cudaSuccess) e = cudaMalloc(&vx->block_sum, sizeof(uint32_t) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&vx->block_off, sizeof(uint32_t) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&vx->hist, sizeof(uint32_t) * 256);
    if (e == cudaSuccess) e = cudaMalloc(&vx->sel, sizeof(uint32_t) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&vx->state, sizeof(int64_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(vx->state, 0, sizeof(int64_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(vx->hist, 0, sizeof(uint32_t) * 256);
    if (e != cudaSuccess) {
        set_last_error(std::string("gs_voxel_create: ") + cudaGetErrorString(e));
        gs_voxel_destroy(vx);
        return GS_ERR_CUDA;
    }
    *out = vx;
    return GS_OK;
}

void gs_voxel_destroy(gs_voxel *vx) {
    if (!vx) return;
    void *ptrs[] = {vx->tkey, vx->tmin, vx->tknown, vx->pslot, vx->block_sum, vx->block_off, vx->hist, vx->sel,
                    vx->state};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete vx;
}

gs_status gs_voxel_insert(gs_voxel *vx, const gs_insert_params *p, const float *points, int64_t n_points,
                          const uint64_t *splat_keys, int32_t *last_used, int64_t n_splats, const uint64_t *host_keys,
                          int32_t *reload, int64_t n_host, int32_t sh_degree, const gs_param_arrays *new_splats,
                          uint64_t *new_keys, int64_t new_capacity, int64_t *n_new, void *stream) {
    if (!vx || !p || n_points < 0 || n_points > vx->max_points || n_splats < 0 || n_host < 0 || sh_degree < 0 ||
        sh_degree > 3 || new_capacity < 0 || new_capacity > 0x7FFFFFFFll || !(p->voxel > 0.f) ||
        !(p->s_init > 0.f) || !(p->o_init > 0.f && p->o_init < 1.f)) {
        set_last_error("gs_voxel_insert: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    if ((n_points > 0 && !points) || (n_splats > 0 && (!splat_keys || !last_used)) ||
        (n_host > 0 && (!host_keys || !reload)) || (new_capacity > 0 && (!params_set(new_splats) || !new_keys))) {
        set_last_error("gs_voxel_insert: NULL array");
        return GS_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned long long *sk = reinterpret_cast<const unsigned long long *>(splat_keys);
    const unsigned long long *hk = reinterpret_cast<const unsigned long long *>(host_keys);
    cudaMemsetAsync(vx->tkey, 0xFF, sizeof(unsigned long long) * vx->cap, s);
    cudaMemsetAsync(vx->tmin, 0x7F, sizeof(int32_t) * vx->cap, s);
    cudaMemsetAsync(vx->tknown, 0, sizeof(int32_t) * vx->cap, s);
    if (n_points > 0) {
        ++vx->kernel_launches;
        k_table_insert<<<grid_for(n_points), VT, 0, s>>>(points, n_points, p->voxel, vx->tkey, vx->tmin, vx->pslot,
                                                         vx->cap_bits);
    }
    if (n_splats > 0) {
        ++vx->kernel_launches;
        k_table_probe<<<grid_for(n_splats), VT, 0, s>>>(sk, n_splats, vx->tkey, vx->tknown, vx->cap_bits, last_used,
                                                        p->frame, true, 0);
    }
    if (n_host > 0) {
        ++vx->kernel_launches;
        k_table_probe<<<grid_for(n_host), VT, 0, s>>>(hk, n_host, vx->tkey, vx->tknown, vx->cap_bits, reload, 1, false,
                                                      0);
    }
    const int nb = nblocks_for(n_points);
    if (n_points > 0) {
        ++vx->kernel_launches;
        k_creator_count<<<nb, VT, 0, s>>>(n_points, vx->pslot, vx->tmin, vx->tknown, vx->block_sum);
    } else {
        cudaMemsetAsync(vx->block_sum, 0, sizeof(uint32_t), s);
    }
    ++vx->kernel_launches;
    k_scan_blocks<<<1, VT, 0, s>>>(vx->block_sum, n_points > 0 ? nb : 0, vx->block_off, new_capacity, vx->state,
                                   n_new);
    gs_status r = check_launch("voxel_insert");
    if (r != GS_OK || n_points == 0) return r;
    EmitArgs A{};
    A.pts = points;
    A.n = n_points;
    A.v = p->voxel;
    A.log_s = (float)std::log((double)p->s_init);
    A.omega = (float)std::log((double)p->o_init / (1.0 - (double)p->o_init));
    A.pslot = vx->pslot;
    A.tmin = vx->tmin;
    A.tknown = vx->tknown;
    A.block_off = vx->block_off;
    A.state = vx->state;
    if (new_capacity > 0) {
        A.means = new_splats->means;
        A.log_scales = new_splats->log_scales;
        A.quats = new_splats->quats;
        A.opacity = new_splats->opacity_logits;
        A.sh = new_splats->sh;
        A.keys = reinterpret_cast<unsigned long long *>(new_keys);
    }
    A.nsh = 3 * (sh_degree + 1) * (sh_degree + 1);
    if (new_capacity > 0) {
        ++vx->kernel_launches;
        k_creator_emit<<<nb, VT, 0, s>>>(A);
    }
    return check_launch("voxel_emit");
}

gs_status gs_voxel_status(gs_voxel *vx, void *stream, int64_t *n_new) {
    if (!vx) {
        set_last_error("gs_voxel_status: NULL argument");
        return GS_ERR_INVALID_ARG;
    }
    int64_t h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(h, vx->state, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_last_error(std::string("gs_voxel_status: ") + cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    if (n_new) *n_new = h[0];
    return h[1] ? GS_ERR_CAPACITY : GS_OK;
}

gs_status gs_active_select(gs_voxel *vx, const int32_t *last_used, int64_t n, int64_t tau, int32_t *flags,
                           void *stream) {
    if (!vx || n < 0 || n > vx->max_items || tau < 0 || (n > 0 && (!last_used || !flags))) {
        set_last_error("gs_active_select: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    if (n == 0) return GS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = n - tau;
    if (m <= 0 || m >= n) {
        ++vx->kernel_launches;
        k_fill_i32<<<grid_for(n), VT, 0, s>>>(flags, n, m <= 0 ? 0 : 1);
        return check_launch("active_select");
    }
    ++vx->kernel_launches;
    k_sel_init<<<1, 1, 0, s>>>(vx->sel, (uint32_t)m);
    for (int shift = 24; shift >= 0; shift -= 8) {
        vx->kernel_launches += 2;
        k_sel_hist<<<grid_for(n), VT, 0, s>>>(last_used, n, vx->sel, shift, vx->hist);
        k_sel_pick<<<1, 256, 0, s>>>(vx->hist, vx->sel, shift);
    }
    const int nb = nblocks_for(n);
    vx->kernel_launches += 3;
    k_sel_eqcount<<<nb, VT, 0, s>>>(last_used, n, vx->sel, vx->block_sum);
    k_scan_blocks<<<1, VT, 0, s>>>(vx->block_sum, nb, vx->block_off, INT64_MAX, vx->state + 2, nullptr);
    k_sel_mark<<<nb, VT, 0, s>>>(last_used, n, vx->sel, vx->block_off, flags);
    return check_launch("active_select");
}

gs_status gs_partition(gs_voxel *vx, const int32_t *flags, int64_t n, int32_t sh_degree, const gs_param_arrays *in,
                       const uint64_t *in_keys, const int32_t *in_last_used, const gs_param_arrays *kept,
                       uint64_t *kept_keys, int32_t *kept_last_used, const gs_param_arrays *moved, uint64_t *moved_keys,
                       int32_t *moved_last_used, int64_t *counts, void *stream) {
    if (!vx || n < 0 || n > vx->max_items || sh_degree < 0 || sh_degree > 3 ||
        (n > 0 && (!flags || !params_set(in) || !params_set(kept) || !params_set(moved))) ||
        (in_keys && (!kept_keys || !moved_keys)) || (in_last_used && (!kept_last_used || !moved_last_used))) {
        set_last_error("gs_partition: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = nblocks_for(n);
    if (n > 0) {
        ++vx->kernel_launches;
        k_flag_count<<<nb, VT, 0, s>>>(flags, n, vx->block_sum);
    } else {
        cudaMemsetAsync(vx->block_sum, 0, sizeof(uint32_t), s);
    }
    vx->kernel_launches += 1;
    k_scan_blocks<<<1, VT, 0, s>>>(vx->block_sum, n > 0 ? nb : 0, vx->block_off, INT64_MAX, vx->state + 2, nullptr);
    if (counts) {
        ++vx->kernel_launches;
        k_partition_counts<<<1, 1, 0, s>>>(vx->state + 2, n, counts);
    }
    if (n == 0) return check_launch("partition");
    PartArgs A{};
    A.flags = flags;
    A.n = n;
    A.block_off = vx->block_off;
    const float *ins[5] = {in->means, in->log_scales, in->quats, in->opacity_logits, in->sh};
    float *ks[5] = {kept->means, kept->log_scales, kept->quats, kept->opacity_logits, kept->sh};
    float *ms[5] = {moved->means, moved->log_scales, moved->quats, moved->opacity_logits, moved->sh};
    for (int i = 0; i < 5; ++i) {
        A.in[i] = ins[i];
        A.kept[i] = ks[i];
        A.moved[i] = ms[i];
    }
    A.in_keys = reinterpret_cast<const unsigned long long *>(in_keys);
    A.kept_keys = reinterpret_cast<unsigned long long *>(kept_keys);
    A.moved_keys = reinterpret_cast<unsigned long long *>(moved_keys);
    A.in_lu = in_last_used;
    A.kept_lu = kept_last_used;
    A.moved_lu = moved_last_used;
    A.nsh = 3 * (sh_degree + 1) * (sh_degree + 1);
    ++vx->kernel_launches;
    k_partition<<<nb, VT, 0, s>>>(A);
    return check_launch("partition");
}

}  // extern "C"
