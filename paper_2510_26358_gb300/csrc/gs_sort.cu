// Binning: one instance per (visible pair, covered tile), ordered by the
// 64-bit key (global tile << 32 | float bits of depth), ties by pair order.
// A pair's rectangle tiles are all emitted; those its alpha >= alpha_min
// ellipse misses carry the invalid tile id (see the emission below).
//
// Instead of radix-sorting 64-bit keys over every instance, the visible pairs
// are first sorted by their 32-bit depth key (N_vis elements), the instances
// are then emitted in that order, and a stable sort by tile id alone (the
// bits of the value n_tiles, so that the invalid id sorts after every real
// one) finishes the job.  Stability makes the result identical to the stable
// 64-bit sort: within a tile the instances stay in (depth, pair) order.
// Per-tile ranges come from key changes.
//
// Every count lives on the device (capacity overflow sets a flag), so the
// sequence needs no host round trip and can be captured in a CUDA graph.  All
// kernels run a fixed grid of `sort_blocks` blocks, each owning a contiguous
// chunk of ceil(n / blocks) rounded to a whole tile.
//
// The radix sort is a reduce-then-scan LSD sort with 8-bit digits:
//   hist     per-block digit counts -> table[digit][block]
//   scan     exclusive scan of the table (digit-major) -> global offsets
//   scatter  per block, tile by tile in order: stable in-tile ranks from warp
//            match masks and per-warp digit counts, a local reorder in shared
//            memory, then coalesced runs written at the global offsets.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int T = kSortThreads;
constexpr int W = T / 32;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// block-wide exclusive scan of one value per thread (blockDim == T); returns
// the exclusive prefix and writes the block total to *total
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *sm, uint32_t *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < W ? sm[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < W) sm[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t base = w > 0 ? sm[w - 1] : 0u;
    *total = sm[W - 1];
    __syncthreads();
    return base + x - v;
}

// ---------------------------------------------------------------------------
// visible-pair compaction
// ---------------------------------------------------------------------------

// Both compaction kernels split the pairs into the same per-block chunks,
// whole multiples of kCompactStep keys (8 a thread, read as two 16-byte
// loads), so that the compaction takes few block-wide scans.
constexpr int kCompactStep = 8 * T;

__global__ void __launch_bounds__(T) k_count_visible(const uint32_t *pkey, uint32_t n, uint32_t *part,
                                                    int nb) {
    __shared__ uint32_t sm[32];
    uint32_t lo, hi;
    chunk_range(n, blockIdx.x, nb, kCompactStep, lo, hi);
    uint32_t c = 0;
    for (uint32_t i = lo + threadIdx.x; i < hi; i += T) c += pkey[i] != kInvalidKey;
    uint32_t tot;
    block_exclusive_scan(c, sm, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// exclusive scan of part[0..nb) in place by one block; the total goes to *total
// and, when cap > 0, is checked against the capacity
__global__ void k_scan_parts(uint32_t *part, int nb, uint32_t *total, DevState *st, uint64_t cap,
                             int mode) {
    __shared__ uint32_t sm[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += T) {
        int i = base + threadIdx.x;
        uint32_t v = i < nb ? part[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(v, sm, &tot);
        if (i < nb) part[i] = (uint32_t)(carry + ex);
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        unsigned long long t = carry;
        if (mode == 0) {
            *total = (uint32_t)t;
        } else {
            st->n_inst_needed = t;
            // every binning starts the flags afresh: capacity for this one,
            // no device-wait time-out yet
            if (t > cap) {
                st->flags = kFlagCapacity;
                st->n_inst = 0;
            } else {
                st->flags = 0u;
                st->n_inst = (uint32_t)t;
            }
        }
    }
}

__global__ void __launch_bounds__(T) k_compact_visible(const uint32_t *pkey, uint32_t n, const uint32_t *part,
                                                      int nb, uint32_t *vis_key, uint32_t *vis_pair) {
    __shared__ uint32_t sm[32];
    uint32_t lo, hi;
    chunk_range(n, blockIdx.x, nb, kCompactStep, lo, hi);
    uint32_t base = part[blockIdx.x];
    // this thread's 8 consecutive keys of a step, in pair order; the next
    // step's keys are loaded before this step's block-wide scan
    auto load8 = [&](uint32_t t0, uint32_t k[8]) {
        const uint32_t i0 = t0 + 8 * threadIdx.x;
        if (i0 + 8 <= hi) {
            const uint4 a = reinterpret_cast<const uint4 *>(pkey + i0)[0];
            const uint4 b = reinterpret_cast<const uint4 *>(pkey + i0)[1];
            k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w;
            k[4] = b.x; k[5] = b.y; k[6] = b.z; k[7] = b.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) k[j] = i0 + j < hi ? pkey[i0 + j] : kInvalidKey;
        }
    };
    uint32_t kn[8];
    if (lo < hi) load8(lo, kn);
    for (uint32_t t0 = lo; t0 < hi; t0 += kCompactStep) {
        const uint32_t i0 = t0 + 8 * threadIdx.x;
        uint32_t k[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) k[j] = kn[j];
        if (t0 + kCompactStep < hi) load8(t0 + kCompactStep, kn);
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) c += k[j] != kInvalidKey;
        uint32_t tot;
        uint32_t o = base + block_exclusive_scan(c, sm, &tot);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (k[j] != kInvalidKey) {
                vis_key[o] = k[j];
                vis_pair[o] = i0 + j;
                ++o;
            }
        base += tot;
    }
}

// ---------------------------------------------------------------------------
// radix sort passes (count n read from the device)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(T) k_radix_hist(const uint32_t *keys, const uint32_t *n_ptr, int shift,
                                                 uint32_t *hist, int nb, int tile) {
    __shared__ uint32_t h[W][256];
    for (int i = threadIdx.x; i < W * 256; i += T) (&h[0][0])[i] = 0;
    __syncthreads();
    uint32_t lo, hi;
    chunk_range(*n_ptr, blockIdx.x, nb, tile, lo, hi);
    int w = threadIdx.x >> 5;
    for (uint32_t i = lo + threadIdx.x; i < hi; i += T) atomicAdd(&h[w][(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) s += h[j][threadIdx.x];
    hist[threadIdx.x * nb + blockIdx.x] = s;
}

// Exclusive scan of each digit's row of the [256][nb] table: block d turns
// row d into offsets relative to the digit's first slot and writes the row
// total to dtot[d].  The digit bases (prefix of dtot) are added by the
// scatter kernel.  nb <= 4 * T.
__global__ void __launch_bounds__(T) k_radix_scan(uint32_t *hist, int nb, uint32_t *dtot) {
    __shared__ uint32_t sm[32];
    uint32_t *row = hist + (size_t)blockIdx.x * nb;
    const int t = threadIdx.x;
    uint32_t v[4];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int i = 4 * t + k;
        v[k] = i < nb ? row[i] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, sm, &tot);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int i = 4 * t + k;
        if (i < nb) row[i] = run;
        run += v[k];
    }
    if (t == 0) dtot[blockIdx.x] = tot;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Tiles of 1024 keys and more are copied into shared memory asynchronously,
// one tile ahead (tile k lands in buffer k & 1 while tile k - 1 is worked;
// the buffer then holds tile k's reordered run): 0.452 -> 0.433 ms for the
// two passes over 25.1M instances, 0.165 -> 0.154 ms for the depth sort's
// 1024-key tiles over 3.08M pairs.  512-key tiles load into registers (the
// copy ahead measured 0.175 -> 0.179 ms there).
template <int R>
constexpr bool kScatterAhead = R >= 4;

template <int R>
struct ScatterSmem {
    uint32_t key[kScatterAhead<R> ? 2 : 1][T * R];
    uint32_t val[kScatterAhead<R> ? 2 : 1][T * R];
    uint32_t wcnt[W][256];  // per-warp digit counts, then per-warp digit offsets
    uint32_t base[256], tcnt[256], tstart[256];
    uint32_t scan[32];
};

// One block tile = T*R keys, split into W contiguous warp sub-tiles of 32*R
// keys.  Each warp ranks its own sub-tile round by round (the mask of the
// lanes holding the same digit, built from one ballot per digit bit, which
// measured faster than __match_any_sync: 0.473 -> 0.452 ms for the two passes
// over 25.1M instances; it gives the rank among equal digits of the round,
// per-warp counters carry it across rounds, no block barrier); one
// block-wide pass then turns the per-warp counts into offsets, the keys are
// reordered by digit in shared memory and written out in coalesced runs at
// the global offsets.  Stable: sub-tiles, rounds and lanes follow the input
// order.
template <int R>
__global__ void __launch_bounds__(T) k_radix_scatter(const uint32_t *kin, const uint32_t *vin,
                                                    uint32_t *kout, uint32_t *vout,
                                                    const uint32_t *n_ptr, int shift,
                                                    const uint32_t *hist, const uint32_t *dtot, int nb) {
    constexpr int TILE = T * R;
    constexpr int WT = 32 * R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<R> &S = *reinterpret_cast<ScatterSmem<R> *>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t lo, hi;
    chunk_range(*n_ptr, blockIdx.x, nb, TILE, lo, hi);
    if (lo >= hi) return;
    {
        uint32_t tot;
        uint32_t digit_base = block_exclusive_scan(dtot[t], S.scan, &tot);
        S.base[t] = digit_base + hist[t * nb + blockIdx.x];
    }
    const uint32_t lt = lanemask_lt();
    // asynchronous copy of the tile at t1 into buffer bi in sixteen-byte
    // pieces of keys and of values (consecutive threads, consecutive pieces),
    // the tail's short piece zero-filled (only its in-range bytes are read)
    auto fetch = [&](uint32_t t1, int bi) {
        const uint32_t tn1 = min((uint32_t)TILE, hi - t1);
#pragma unroll
        for (int q = 0; q < (TILE / 4 + T - 1) / T; ++q) {
            if (q * T + t >= TILE / 4) break;
            const uint32_t e = 4 * (q * T + t);  // first key of the piece
            const uint32_t nbytes = e < tn1 ? 4u * min(4u, tn1 - e) : 0u;
            const uint32_t src = t1 + (e < tn1 ? e : 0u);
            cp_async16(&S.key[bi][e], kin + src, nbytes);
            cp_async16(&S.val[bi][e], vin + src, nbytes);
        }
        cp_async_commit();
    };
    constexpr bool AHEAD = kScatterAhead<R>;
    if constexpr (AHEAD) fetch(lo, 0);
    int bi = 0;
    for (uint32_t t0 = lo; t0 < hi; t0 += TILE, bi = AHEAD ? bi ^ 1 : 0) {
        const uint32_t tn = min((uint32_t)TILE, hi - t0);
        if constexpr (AHEAD) {
            if (t0 + TILE < hi) {
                fetch(t0 + TILE, bi ^ 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
        }
#pragma unroll
        for (int j = 0; j < W; ++j) S.wcnt[j][t] = 0;
        __syncthreads();
        uint32_t key[R], val[R], rank[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t i = w * WT + r * 32 + lane;
            key[r] = i >= tn ? 0u : AHEAD ? S.key[bi][i] : kin[t0 + i];
            val[r] = i >= tn ? 0u : AHEAD ? S.val[bi][i] : vin[t0 + i];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const bool valid = (uint32_t)(w * WT + r * 32 + lane) < tn;
            const uint32_t d = (key[r] >> shift) & 255u;
            uint32_t m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint32_t bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                m &= ((d >> b) & 1u) ? bb : ~bb;
            }
            const uint32_t below = m & lt;
            const uint32_t before = valid ? S.wcnt[w][d] : 0u;
            rank[r] = before + __popc(below);
            __syncwarp();
            if (valid && below == 0) S.wcnt[w][d] = before + __popc(m);
            __syncwarp();
        }
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint32_t c = S.wcnt[j][t];
            S.wcnt[j][t] = run;
            run += c;
        }
        S.tcnt[t] = run;
        uint32_t tot;
        S.tstart[t] = block_exclusive_scan(run, S.scan, &tot);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((uint32_t)(w * WT + r * 32 + lane) < tn) {
                const uint32_t d = (key[r] >> shift) & 255u;
                const uint32_t lp = S.tstart[d] + S.wcnt[w][d] + rank[r];
                S.key[bi][lp] = key[r];
                S.val[bi][lp] = val[r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t j = t + r * T;
            if (j < tn) {
                const uint32_t k = S.key[bi][j];
                const uint32_t d = (k >> shift) & 255u;
                const uint32_t o = S.base[d] + (j - S.tstart[d]);
                kout[o] = k;
                vout[o] = S.val[bi][j];
            }
        }
        __syncthreads();
        S.base[t] += S.tcnt[t];
    }
}

// ---------------------------------------------------------------------------
// instance emission and ranges
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t rect_tiles(short4 r) {
    int nx = (int)r.z - (int)r.x + 1, ny = (int)r.w - (int)r.y + 1;
    return (nx > 0 && ny > 0) ? (uint32_t)(nx * ny) : 0u;
}

// Both kernels below split the sorted visible pairs into the same per-block
// chunks of whole kOffsetStep steps: a thread takes four consecutive pairs a
// step (four independent rectangle gathers in flight; one block-wide scan per
// step of the offsets), on the compaction's wide grid.
constexpr int kOffsetStep = 4 * T;

// instance count of every sorted visible pair (into ioff) and of every block's chunk
__global__ void __launch_bounds__(T) k_count_instances(const uint32_t *vis_pair, const short4 *rect,
                                                      const DevState *st, uint32_t *ioff, uint32_t *part,
                                                      int nb) {
    __shared__ uint32_t sm[32];
    uint32_t n = st->n_vis;
    uint32_t lo, hi;
    chunk_range(n, blockIdx.x, nb, kOffsetStep, lo, hi);
    uint32_t c = 0;
    for (uint32_t i0 = lo + 4 * threadIdx.x; i0 < hi; i0 += kOffsetStep) {
        uint32_t pr[4];
        short4 rc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) pr[u] = i0 + u < hi ? vis_pair[i0 + u] : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) rc[u] = i0 + u < hi ? rect[pr[u]] : make_short4(1, 1, 0, 0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i0 + u >= hi) break;
            const uint32_t k = rect_tiles(rc[u]);
            ioff[i0 + u] = k;
            c += k;
        }
    }
    uint32_t tot;
    block_exclusive_scan(c, sm, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// ioff[i] <- first output slot of sorted pair i (exclusive scan of the counts);
// win_pair[w] <- the pair that owns slot w * kEmitWindow (every slot belongs to
// exactly one pair, so each window start is written once)
__global__ void __launch_bounds__(T) k_instance_offsets(const DevState *st, const uint32_t *part, int nb,
                                                       uint32_t *ioff, uint32_t *win_pair, uint32_t n_win) {
    __shared__ uint32_t sm[32];
    // over capacity the offsets are not used (emission writes nothing) and
    // would index past the window table
    if (st->flags & kFlagCapacity) return;
    uint32_t n = st->n_vis;
    uint32_t lo, hi;
    chunk_range(n, blockIdx.x, nb, kOffsetStep, lo, hi);
    uint32_t base = part[blockIdx.x];
    for (uint32_t t0 = lo; t0 < hi; t0 += kOffsetStep) {
        const uint32_t i0 = t0 + 4 * threadIdx.x;
        uint32_t c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = i0 + u < hi ? ioff[i0 + u] : 0u;
        uint32_t tot;
        uint32_t start = base + block_exclusive_scan(c[0] + c[1] + c[2] + c[3], sm, &tot);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t i = i0 + u;
            if (i >= hi) break;
            ioff[i] = start;
            for (uint32_t w = (start + kEmitWindow - 1) / kEmitWindow;
                 c[u] > 0 && w < n_win && w * (uint64_t)kEmitWindow < (uint64_t)start + c[u]; ++w)
                win_pair[w] = i;
            start += c[u];
        }
        base += tot;
    }
}

// Instances of the depth-sorted visible pairs, in that order, each pair's
// tiles row-major.  The work is split by output slot, not by pair (pairs in
// depth order have very uneven rectangles): a block takes a window of
// kEmitWindow consecutive slots, takes the pairs that cover it from the
// window-start table (the pairs owning its first slot and the next window's),
// stages them in shared memory, and every thread writes one instance per
// step, reading its pair from the window's slot-owner table.
//
// A rectangle tile that the Gaussian's padded alpha >= alpha_min ellipse
// misses (about a fifth of them on wide scenes: the corners of the rectangles
// of large or tilted ellipses) is written with tile id kInvalidKey.  The tile
// sort puts these after every real tile (the sort covers whole bytes above
// the highest tile id), the ranges skip them, and the rasterisers never walk
// them.

// Does the tile whose pixels span [X0, X1] x [Y0, Y1] hold an instance of the
// pair with record r0 = (U, V, hx, hy), r1 = (l11, l12, l22, log2 o)?  The
// rasterisers keep a fragment where log2 o - |t|^2 >= log2 alpha_min, with
// t = L d, L = [[l11, l12], [0, l22]] and d = (px - U + hx, py - V + hy) the
// offset of pixel (px, py)'s centre from the mean.  The tile is kept iff the
// minimum of |L d|^2 over the box of its pixel centres, grown by ext_abs_pad,
// is within (log2 o - log2 alpha_min) (1 + ext_rel_pad)^2: the same padding as
// the rectangle's extents, which dwarfs the rounding of this test and of the
// rasterisers' own evaluation, so a dropped tile has no fragment to keep.  The
// minimum of the convex quadratic is 0 when the box holds the mean, else it
// lies on an edge, at the edge's stationary point clamped to the edge.
// The pair's own factors of the test: the stationary slopes on an edge
// dx = const (sy = dy/dx) and dy = const (sx = dx/dy), and the padded
// threshold.  (Staging them per pair in the window, with the record load that
// needs, measured slower than recomputing them per instance: the load lands
// on the staging's critical path.)
__device__ __forceinline__ float4 reach_terms(const float4 r1, const Consts &k) {
    const float l11 = r1.x, l12 = r1.y, l22 = r1.z;
    const float pad = 1.f + k.ext_rel_pad;
    // (the slopes by the fast division, within 2 ulps: the quadratic is
    // stationary there, so a slope off by e moves the edge minimum by O(e^2);
    // orchard4m emission 0.239 -> 0.228 ms)
    return make_float4(__fdividef(-l11 * l12, l12 * l12 + l22 * l22), __fdividef(-l12, l11),
                       (r1.w - k.log2_alpha_min) * pad * pad, 0.f);
}

__device__ __forceinline__ bool tile_reached(const float4 r0, const float4 r1, const float4 q, int X0, int X1,
                                             int Y0, int Y1, const Consts &k) {
    const float ax = __fadd_rn((float)X0 - r0.x, r0.z) - k.ext_abs_pad;
    const float bx = __fadd_rn((float)X1 - r0.x, r0.z) + k.ext_abs_pad;
    const float ay = __fadd_rn((float)Y0 - r0.y, r0.w) - k.ext_abs_pad;
    const float by = __fadd_rn((float)Y1 - r0.y, r0.w) + k.ext_abs_pad;
    if (ax <= 0.f && bx >= 0.f && ay <= 0.f && by >= 0.f) return true;
    const float l11 = r1.x, l12 = r1.y, l22 = r1.z;
    const float sy = q.x, sx = q.y;
    float m = INFINITY;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float cx = e ? bx : ax;
        const float dy = fminf(fmaxf(sy * cx, ay), by);
        const float t1 = l11 * cx + l12 * dy, t2 = l22 * dy;
        m = fminf(m, t1 * t1 + t2 * t2);
        const float cy = e ? by : ay;
        const float dx = fminf(fmaxf(sx * cy, ax), bx);
        const float u1 = l11 * dx + l12 * cy, u2 = l22 * cy;
        m = fminf(m, u1 * u1 + u2 * u2);
    }
    return m <= q.z;
}

// Blocks of the emission an SM keeps resident: a window's staging is a short
// chain of dependent loads (slot owners, pair ids, rectangles) that every
// thread of the block waits for, so several blocks per SM hide it.
constexpr int kEmitBlocksPerSM = 6;
constexpr int kEmitPerThread = kEmitWindow / T;
static_assert(kEmitWindow == T * kEmitPerThread, "a window is a whole number of slots a thread");

// Per window, staged once per covering pair: its first slot, pair id,
// rectangle origin, width, 1 / width (for the row of a slot) and view.  The
// owner of every slot of the window comes from one block-wide max-scan of the
// pairs' start marks (pair j >= 1 starts inside the window, pair 0 owns its
// first slot; every visible pair has at least one tile), so a slot finds its
// pair with one shared-memory read instead of a binary search over the
// staged pairs: 0.323 -> 0.270 ms for 25.1M instances of 3.08M pairs.
__global__ void __launch_bounds__(T, kEmitBlocksPerSM) k_emit_instances(
    const uint32_t *vis_pair, const short4 *rect, const float4 *rec, const ViewInfo *views, int n_views,
    const Consts k, const DevState *st, const uint32_t *ioff, const uint32_t *win_pair, uint32_t *inst_tile,
    uint32_t *inst_val) {
    __shared__ uint32_t s_off[kEmitWindow];
    __shared__ uint32_t s_pair[kEmitWindow];
    __shared__ short4 s_rect[kEmitWindow];    // (x0, y0, width, view)
    __shared__ float s_rw[kEmitWindow];       // 1 / width
    __shared__ uint16_t s_own[kEmitWindow];   // owner (staged pair) of each slot of the window
    __shared__ int4 s_view[GS_MAX_VIEWS];     // (tile_off, ntx, W, H)
    __shared__ int32_t s_poff[GS_MAX_VIEWS];  // first pair of each view
    __shared__ uint32_t s_range[2];
    __shared__ uint32_t s_wmax[T / 32];
    if (st->flags & kFlagCapacity) return;
    const uint32_t n = st->n_vis, total = st->n_inst;
    const uint32_t windows = (total + kEmitWindow - 1) / kEmitWindow;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int v = t; v < n_views; v += T) {
        s_view[v] = make_int4(views[v].tile_off, views[v].ntx, views[v].W, views[v].H);
        s_poff[v] = views[v].pair_off;
    }
    for (uint32_t wdw = blockIdx.x; wdw < windows; wdw += gridDim.x) {
        const uint32_t o0 = wdw * kEmitWindow;
        const uint32_t o1 = min(o0 + kEmitWindow, total);
        if (t == 0) s_range[0] = win_pair[wdw];
        if (t == 1) {
            // the pair owning slot o1 - 1: the last pair if this is the last
            // window, else the owner of the next window's first slot, or the
            // pair before it when that one starts exactly at o1
            uint32_t p1 = n - 1;
            if (wdw + 1 < windows) {
                p1 = win_pair[wdw + 1];
                if (ioff[p1] == o1) --p1;
            }
            s_range[1] = p1;
        }
#pragma unroll
        for (int i = 0; i < kEmitPerThread; ++i) s_own[t * kEmitPerThread + i] = 0;
        __syncthreads();
        const uint32_t s0 = s_range[0], np = s_range[1] - s0 + 1;  // np <= window: every pair has >= 1 slot
        for (uint32_t j = t; j < np; j += T) {
            const uint32_t pair = vis_pair[s0 + j];
            int lo_v = 0, hi_v = n_views - 1;
            while (lo_v < hi_v) {
                int mid = (lo_v + hi_v + 1) >> 1;
                if ((uint32_t)s_poff[mid] <= pair) lo_v = mid; else hi_v = mid - 1;
            }
            const uint32_t off = ioff[s0 + j];
            const short4 r = rect[pair];
            const int wdt = (int)r.z - (int)r.x + 1;
            s_off[j] = off;
            s_pair[j] = pair;
            s_rect[j] = make_short4(r.x, r.y, (short)wdt, (short)lo_v);
            s_rw[j] = 1.f / (float)wdt;
            if (j > 0) s_own[off - o0] = (uint16_t)j;
        }
        __syncthreads();
        // inclusive max-scan of the marks: thread t owns slots [4t, 4t + 4)
        {
            uint32_t v[kEmitPerThread], run = 0;
#pragma unroll
            for (int i = 0; i < kEmitPerThread; ++i) {
                run = max(run, (uint32_t)s_own[t * kEmitPerThread + i]);
                v[i] = run;
            }
            uint32_t x = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x = max(x, y);
            }
            if (lane == 31) s_wmax[wid] = x;
            uint32_t before = __shfl_up_sync(0xffffffffu, x, 1);
            if (lane == 0) before = 0;
            __syncthreads();
            for (int w = 0; w < wid; ++w) before = max(before, s_wmax[w]);
#pragma unroll
            for (int i = 0; i < kEmitPerThread; ++i) s_own[t * kEmitPerThread + i] = (uint16_t)max(before, v[i]);
        }
        __syncthreads();
        for (uint32_t o = o0 + t; o < o1; o += T) {
            const uint32_t a = s_own[o - o0];
            const short4 r = s_rect[a];
            const float rw = s_rw[a];
            const int4 vw = s_view[r.w];
            const uint32_t pair = s_pair[a];
            const int wdt = r.z;
            const int local = (int)(o - s_off[a]);
            // row = local / wdt from the staged reciprocal, corrected to the
            // exact quotient (the estimate is within one of it)
            int row = (int)((float)local * rw);
            if (row * wdt > local) --row;
            else if ((row + 1) * wdt <= local) ++row;
            const int ty = r.y + row, tx = r.x + (local - row * wdt);
            const int X0 = tx * k.tile_w, Y0 = ty * k.tile_h;
            const float4 r1 = __ldg(rec + 3 * (size_t)pair + 1);
            const bool keep = tile_reached(__ldg(rec + 3 * (size_t)pair), r1, reach_terms(r1, k), X0,
                                           min(X0 + k.tile_w, vw.z) - 1, Y0, min(Y0 + k.tile_h, vw.w) - 1, k);
            inst_tile[o] = keep ? (uint32_t)(vw.x + ty * vw.y + tx) : kInvalidKey;
            inst_val[o] = pair;
        }
        __syncthreads();
    }
}

// [start, end) of every tile's run in the sorted instances; the dropped
// rectangle tiles (kInvalidKey, sorted last) belong to no tile
// (a thread takes four consecutive ids with one 16-byte load, plus the ids
// on either side)
__global__ void k_ranges(const uint32_t *tile, const DevState *st, uint32_t n_tiles, uint2 *ranges,
                         uint32_t *order_tot) {
    if (blockIdx.x == 0 && threadIdx.x < kOrderBuckets) order_tot[threadIdx.x] = 0u;  // for the work order
    const uint32_t n = st->n_inst;
    const uint32_t n4 = (n + 3) / 4;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4 * q;
        uint32_t t[6];
        t[0] = i0 > 0 ? tile[i0 - 1] : kInvalidKey;
        if (i0 + 4 <= n) {
            const uint4 v = reinterpret_cast<const uint4 *>(tile)[q];
            t[1] = v.x; t[2] = v.y; t[3] = v.z; t[4] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) t[1 + j] = i0 + j < n ? tile[i0 + j] : kInvalidKey;
        }
        t[5] = i0 + 4 < n ? tile[i0 + 4] : kInvalidKey;
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            const uint32_t i = i0 + j - 1;
            if (i >= n || t[j] >= n_tiles) continue;
            if (t[j - 1] != t[j]) ranges[t[j]].x = i;
            if (t[j + 1] != t[j]) ranges[t[j]].y = i + 1;
        }
    }
}

// Raster work order: tiles by decreasing list length, so that the longest
// lists start first and the persistent rasterisers finish together.  A
// counting sort into kOrderBuckets length buckets; the order inside a bucket
// is whatever the atomics give (tiles are independent, so it does not change
// any result).
__device__ __forceinline__ uint32_t order_bucket(uint2 r) {
    const uint32_t len = r.y - r.x;
    return kOrderBuckets - 1 - min((uint32_t)(kOrderBuckets - 1), len >> kOrderShift);
}

// Two kernels over kOrderBlocks blocks (one block over every tile took 47 us
// on 54k tiles, its shared-memory atomics on 64 counters serialised):
// k_order_count adds each block's bucket counts to the bucket totals, the
// atomic's old value giving the block its base inside each bucket;
// k_order_place takes the totals' prefix and puts each tile at its bucket's
// start + its block's base + its rank in the block.  The totals are cleared by
// k_ranges (block 0), which runs before.

__global__ void __launch_bounds__(256) k_order_count(const uint2 *ranges, int n_tiles, uint32_t *tot,
                                                    uint32_t *bbase) {
    __shared__ uint32_t cnt[kOrderBuckets];
    const int t = threadIdx.x;
    if (t < kOrderBuckets) cnt[t] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + t; i < n_tiles; i += gridDim.x * blockDim.x)
        atomicAdd(&cnt[order_bucket(ranges[i])], 1u);
    __syncthreads();
    if (t < kOrderBuckets) bbase[blockIdx.x * kOrderBuckets + t] = cnt[t] ? atomicAdd(&tot[t], cnt[t]) : 0u;
}

__global__ void __launch_bounds__(256) k_order_place(const uint2 *ranges, int n_tiles, const uint32_t *tot,
                                                    const uint32_t *bbase, uint32_t *order) {
    static_assert(kOrderBuckets == 64, "the prefix below takes two counts a lane of one warp");
    __shared__ uint32_t cur[kOrderBuckets];
    const int t = threadIdx.x;
    if (t < 32) {  // exclusive prefix of the 64 bucket totals by one warp, plus this block's bases
        const uint32_t a = tot[t], b = tot[t + 32];
        uint32_t x = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (t >= o) x += y;
        }
        const uint32_t tot_a = __shfl_sync(0xffffffffu, x, 31);
        uint32_t z = b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (t >= o) z += y;
        }
        cur[t] = x - a + bbase[blockIdx.x * kOrderBuckets + t];
        cur[t + 32] = tot_a + z - b + bbase[blockIdx.x * kOrderBuckets + t + 32];
    }
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + t; i < n_tiles; i += gridDim.x * blockDim.x)
        order[atomicAdd(&cur[order_bucket(ranges[i])], 1u)] = (uint32_t)i;
}

// One stable pass over bits [shift, shift+8) by nb blocks; swaps in/out.
// R = 8 rounds (2048-key tiles) on twice the blocks for the instance sort
// (64 registers: one full wave of four blocks per SM; measured 0.0725 ->
// 0.068 ms against R = 16 on one block per two SMs' worth), R = 2 or 4 for
// the smaller sort of the visible pairs (see its launch).
template <int R>
gs_status radix_pass(gs_workspace *ws, uint32_t *&k, uint32_t *&v, uint32_t *&k2, uint32_t *&v2,
                     const uint32_t *n_ptr, int shift, int nb, cudaStream_t s) {
    // the digit table has a column per block, and the scan takes at most 4 T
    if (nb < 1 || nb > ws->hist_cols || nb > 4 * T) {
        set_last_error("radix_pass: " + std::to_string(nb) + " blocks exceed the digit table (" +
                       std::to_string(ws->hist_cols) + " columns)");
        return GS_ERR_INVALID_ARG;
    }
    ++ws->kernel_launches; k_radix_hist<<<nb, T, 0, s>>>(k, n_ptr, shift, ws->hist, nb, T * R);
    ++ws->kernel_launches; k_radix_scan<<<256, T, 0, s>>>(ws->hist, nb, ws->digit_tot);
    ++ws->kernel_launches;
    k_radix_scatter<R><<<nb, T, sizeof(ScatterSmem<R>), s>>>(k, v, k2, v2, n_ptr, shift, ws->hist,
                                                             ws->digit_tot, nb);
    std::swap(k, k2);
    std::swap(v, v2);
    return check_launch("radix_pass");
}

}  // namespace

gs_status sort_configure() {
    cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(ScatterSmem<8>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_radix_scatter<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(ScatterSmem<2>));

    if (e != cudaSuccess) {
        set_last_error(std::string("sort_configure: ") + cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

gs_status launch_bin_sort(gs_workspace *ws, cudaStream_t s) {
    int nb = ws->sort_blocks;
    uint32_t n_pairs = (uint32_t)ws->n_pairs;
    DevState *st = ws->st;
    cudaMemsetAsync(&st->n_vis, 0, sizeof(uint32_t) * 2 + sizeof(unsigned long long) + sizeof(uint32_t), s);
    // 1. compaction of visible pairs (more blocks than the other stages: each
    //    block's chunk is a chain of block-wide scans)
    gs_status r;
    const int nw = ws->wide_blocks;
    {
    StageTimer timer(ws, GS_STAGE_COMPACT, s);
    ++ws->kernel_launches; k_count_visible<<<nw, T, 0, s>>>(ws->pkey, n_pairs, ws->part, nw);
    ++ws->kernel_launches; k_scan_parts<<<1, T, 0, s>>>(ws->part, nw, &st->n_vis, st, 0, 0);
    ++ws->kernel_launches; k_compact_visible<<<nw, T, 0, s>>>(ws->pkey, n_pairs, ws->part, nw, ws->vis_key, ws->vis_pair);
    r = check_launch("compact");
    if (r != GS_OK) return r;
    }
    // 2. stable sort of the visible pairs by depth key (32 bits)
    uint32_t *k = ws->vis_key, *v = ws->vis_pair, *k2 = ws->vis_key_alt, *v2 = ws->vis_pair_alt;
    {
    StageTimer timer(ws, GS_STAGE_DEPTH_SORT, s);
    // (blocks grow with the pairs: a tenth of them or so are visible; more
    // blocks than keys to fill them only lengthen the digit-table scans)
    const int nd = (int)std::min<int64_t>(nw, std::max<int64_t>(nb, ws->n_pairs / 16384));
    // four keys a thread once the blocks hold several tiles each (orchard4m,
    // 3.08 M visible of 24 M pairs: 0.175 -> 0.164 ms), two below (orchard500k,
    // 148k of 1.5 M: 0.063 ms against 0.065 with four)
    const bool wide = ws->n_pairs >= (int64_t)8 << 20;
    for (int sh = 0; sh < 32; sh += 8)
        if ((r = wide ? radix_pass<4>(ws, k, v, k2, v2, &st->n_vis, sh, nd, s)
                      : radix_pass<2>(ws, k, v, k2, v2, &st->n_vis, sh, nd, s)) != GS_OK)
            return r;
    }
    // after 4 passes the sorted data are back in vis_key / vis_pair
    // 3. instance offsets, capacity check, emission in depth order
    // emit into whichever buffer makes the last tile pass end in inst_tile/inst_val
    int passes = (ws->tile_bits + 7) / 8;
    uint32_t *tk = (passes & 1) ? ws->inst_tile_alt : ws->inst_tile;
    uint32_t *tv = (passes & 1) ? ws->inst_val_alt : ws->inst_val;
    uint32_t *tk2 = (passes & 1) ? ws->inst_tile : ws->inst_tile_alt;
    uint32_t *tv2 = (passes & 1) ? ws->inst_val : ws->inst_val_alt;
    {
    StageTimer timer(ws, GS_STAGE_EMIT, s);
    ++ws->kernel_launches; k_count_instances<<<nw, T, 0, s>>>(v, ws->rect, st, ws->ioff, ws->part, nw);
    ++ws->kernel_launches; k_scan_parts<<<1, T, 0, s>>>(ws->part, nw, nullptr, st, (uint64_t)ws->inst_cap, 1);
    ++ws->kernel_launches; k_instance_offsets<<<nw, T, 0, s>>>(st, ws->part, nw, ws->ioff, ws->win_pair,
                                                                  (uint32_t)(ws->inst_cap / kEmitWindow + 2));
    ++ws->kernel_launches;
    k_emit_instances<<<kEmitBlocksPerSM * ws->num_sms, T, 0, s>>>(v, ws->rect, ws->rec, ws->views, ws->n_views,
                                                                    ws->consts, st, ws->ioff, ws->win_pair, tk, tv);
    if ((r = check_launch("emit")) != GS_OK) return r;
    }
    // 4. stable sort of the instances by tile id
    {
    StageTimer timer(ws, GS_STAGE_TILE_SORT, s);
    for (int p = 0; p < passes; ++p)
        if ((r = radix_pass<8>(ws, tk, tv, tk2, tv2, &st->n_inst, 8 * p, std::min(4 * T, 2 * nb), s)) != GS_OK) return r;
    }
    // 5. ranges
    StageTimer timer(ws, GS_STAGE_RANGES, s);
    cudaMemsetAsync(ws->ranges, 0, sizeof(uint2) * ws->n_tiles, s);
    ++ws->kernel_launches;
    // (eight blocks an SM, every thread resident: 0.054 -> 0.044 ms with the
    // work order on orchard4m's 25.1 M instances, against four)
    k_ranges<<<ws->num_sms * 8, 256, 0, s>>>(ws->inst_tile, st, (uint32_t)ws->n_tiles, ws->ranges, ws->order_tot);
    // 6. raster work order
    ++ws->kernel_launches;
    k_order_count<<<kOrderBlocks, 256, 0, s>>>(ws->ranges, (int)ws->n_tiles, ws->order_tot, ws->order_base);
    ++ws->kernel_launches;
    k_order_place<<<kOrderBlocks, 256, 0, s>>>(ws->ranges, (int)ws->n_tiles, ws->order_tot, ws->order_base,
                                               ws->tile_order);
    return check_launch("ranges");
}

}  // namespace gs
