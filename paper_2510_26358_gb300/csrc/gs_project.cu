// Per-camera EWA projection of the shared Gaussian set and its adjoint.
//
// Forward (Sec. III-B, Eqs. 3-4): for every (view, Gaussian) pair of the same
// submap, Sigma = R S S^T R^T, p = W mu + t, Sigma' = J W Sigma W^T J^T +
// dilation*I, the scaled Cholesky factor of Sigma'^-1, opacity, the extent of
// the alpha >= alpha_min ellipse and its tile rectangle, and the SH colour.
// One thread per Gaussian loops over the cameras of its submap, so the 3-D
// covariance and the parameter loads are shared by all views.
//
// Precision: the view-space depth key is the double-precision dot product
// ((R0 mu0 + R1 mu1) + R2 mu2) + t (exact products of float inputs), rounded to
// float, so keys are reproducible bit for bit; it is read off the float-float
// depth wherever that determines it (all but about one pair in 2^14).  The pixel
// mean is formed in float-float arithmetic (error-free products and sums,
// about 48 bits) and kept as an integer pixel plus a small float offset, so
// that per-fragment offsets are exact integers plus that offset.  Only the
// depth key uses double: GB300's FP64 rate is a small fraction of its FP32
// rate, and the visible pairs are a sparse subset of every warp.
// The image covariance is built from the rows of J W R S, its determinant
// through the Lagrange identity (a sum of squares) with the minors taken by
// the Binet-Cauchy identity from the camera and the Gaussian's axes, so no
// step cancels, not even for a long thin Gaussian.
//
// Backward (chain rule through the same steps), over chunks of one submap:
// each block first packs the chunk's Gaussians that some view sees (most are
// outside every frustum), then
//   k_sh_bwd       three lanes (one per colour channel) per Gaussian: SH
//                  coefficient gradients, written once per Gaussian, and the
//                  colour's gradient w.r.t. the view direction per pair;
//   k_project_bwd  one lane per Gaussian walks its views and accumulates the
//                  geometric gradients in registers, written once; the pose
//                  twist of each view is reduced over the block and summed
//                  per view by k_pose_reduce in a fixed order.
// The forward stores a clamped colour channel as -0, so the backward reads
// the clamp decision from the record instead of recomputing the colour.
#include "gs_internal.cuh"

namespace gs {
namespace {

// real orthonormal SH, no Condon-Shortley phase, ordered by l then m = -l..l
constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.48860251190291992f;
constexpr float kC2a = 1.09254843059207907f;
constexpr float kC2b = 0.31539156525252001f;
constexpr float kC2c = 0.54627421529603954f;
constexpr float kC3a = 0.59004358992664352f;
constexpr float kC3b = 2.89061144264055405f;
constexpr float kC3c = 0.45704579946446572f;
constexpr float kC3d = 0.37317633259011540f;
constexpr float kC3e = 1.44530572132027729f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    Y[0] = kC0;
    if (DEG >= 1) {
        Y[1] = kC1 * y;
        Y[2] = kC1 * z;
        Y[3] = kC1 * x;
    }
    if (DEG >= 2) {
        Y[4] = kC2a * x * y;
        Y[5] = kC2a * y * z;
        Y[6] = kC2b * (2.f * z * z - x * x - y * y);
        Y[7] = kC2a * x * z;
        Y[8] = kC2c * (x * x - y * y);
    }
    if (DEG >= 3) {
        Y[9] = kC3a * y * (3.f * x * x - y * y);
        Y[10] = kC3b * x * y * z;
        Y[11] = kC3c * y * (4.f * z * z - x * x - y * y);
        Y[12] = kC3d * z * (2.f * z * z - 3.f * x * x - 3.f * y * y);
        Y[13] = kC3c * x * (4.f * z * z - x * x - y * y);
        Y[14] = kC3e * z * (x * x - y * y);
        Y[15] = kC3a * x * (x * x - 3.f * y * y);
    }
}

// d Y_k / d(x, y, z)
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float dY[16][3]) {
#pragma unroll
    for (int k = 0; k < 16; ++k) dY[k][0] = dY[k][1] = dY[k][2] = 0.f;
    if (DEG >= 1) {
        dY[1][1] = kC1;
        dY[2][2] = kC1;
        dY[3][0] = kC1;
    }
    if (DEG >= 2) {
        dY[4][0] = kC2a * y; dY[4][1] = kC2a * x;
        dY[5][1] = kC2a * z; dY[5][2] = kC2a * y;
        dY[6][0] = -2.f * kC2b * x; dY[6][1] = -2.f * kC2b * y; dY[6][2] = 4.f * kC2b * z;
        dY[7][0] = kC2a * z; dY[7][2] = kC2a * x;
        dY[8][0] = 2.f * kC2c * x; dY[8][1] = -2.f * kC2c * y;
    }
    if (DEG >= 3) {
        dY[9][0] = kC3a * 6.f * x * y; dY[9][1] = kC3a * 3.f * (x * x - y * y);
        dY[10][0] = kC3b * y * z; dY[10][1] = kC3b * x * z; dY[10][2] = kC3b * x * y;
        dY[11][0] = -2.f * kC3c * x * y;
        dY[11][1] = kC3c * (4.f * z * z - x * x - 3.f * y * y);
        dY[11][2] = 8.f * kC3c * y * z;
        dY[12][0] = -6.f * kC3d * x * z; dY[12][1] = -6.f * kC3d * y * z;
        dY[12][2] = kC3d * (6.f * z * z - 3.f * x * x - 3.f * y * y);
        dY[13][0] = kC3c * (4.f * z * z - 3.f * x * x - y * y);
        dY[13][1] = -2.f * kC3c * x * y;
        dY[13][2] = 8.f * kC3c * x * z;
        dY[14][0] = 2.f * kC3e * x * z; dY[14][1] = -2.f * kC3e * y * z;
        dY[14][2] = kC3e * (x * x - y * y);
        dY[15][0] = 3.f * kC3a * (x * x - y * y); dY[15][1] = -6.f * kC3a * x * y;
    }
}

struct Cam {
    float fx, fy, cx, cy;
    float T[12];
};

__device__ __forceinline__ Cam load_cam(const gs_camera *cams, int v) {
    Cam c;
    const gs_camera *cp = cams + v;
    c.fx = __ldg(&cp->fx);
    c.fy = __ldg(&cp->fy);
    c.cx = __ldg(&cp->cx);
    c.cy = __ldg(&cp->cy);
#pragma unroll
    for (int i = 0; i < 12; ++i) c.T[i] = __ldg(&cp->T_cw[i]);
    return c;
}

// p = W mu + t in double with the fixed summation order
__device__ __forceinline__ double view_coord(const float *Ti, float m0, float m1, float m2) {
    double s = __fma_rn((double)Ti[1], (double)m1, (double)Ti[0] * (double)m0);
    s = __fma_rn((double)Ti[2], (double)m2, s);
    return s + (double)Ti[3];
}

// float-float arithmetic: (hi, lo) with |lo| <= ulp(hi) / 2.  The rounded
// operations are explicit so that no multiply-add contraction changes them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float2 renorm(float s, float e) {
    const float hi = __fadd_rn(s, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

// W_i . mu + t_i: exact products (fma residuals), compensated sums
__device__ __forceinline__ float2 view_coord_ff(const float *Ti, float m0, float m1, float m2) {
    const float p0 = __fmul_rn(Ti[0], m0), p1 = __fmul_rn(Ti[1], m1), p2 = __fmul_rn(Ti[2], m2);
    float err = __fadd_rn(__fadd_rn(__fmaf_rn(Ti[0], m0, -p0), __fmaf_rn(Ti[1], m1, -p1)),
                          __fmaf_rn(Ti[2], m2, -p2));
    float s, t;
    two_sum(p0, p1, s, t);
    err = __fadd_rn(err, t);
    two_sum(s, p2, s, t);
    err = __fadd_rn(err, t);
    two_sum(s, Ti[3], s, t);
    err = __fadd_rn(err, t);
    return renorm(s, err);
}

// f x / z + c for float-float x, z
__device__ __forceinline__ float2 ff_pinhole(float f, float2 x, float2 z, float c) {
    const float q0 = __fdiv_rn(x.x, z.x);
    // remainder x - q0 z: the hi part exactly (fma), plus the small terms
    const float r = __fadd_rn(__fmaf_rn(-q0, z.x, x.x), __fmaf_rn(-q0, z.y, x.y));
    const float q1 = __fdiv_rn(r, z.x);
    const float a = __fmul_rn(f, q0);
    const float ea = __fmaf_rn(f, q0, -a);
    float s, es;
    two_sum(a, c, s, es);
    return renorm(s, __fadd_rn(__fadd_rn(ea, es), __fmul_rn(f, q1)));
}

// The depth key z32 = float(D) and the near-plane decision D > near, where D
// is the double sum ((W0 mu0 + W1 mu1) + W2 mu2) + t (products of floats are
// exact in double, so D is within 3 ulps (2^-53) of the terms' magnitudes
// `mag` of the exact sum), taken from the float-float z = hi + lo of the same
// sum (within ~40 x 2^-48 mag of it) wherever that decides them: hi is
// float(D) when z lies farther than 2^-38 mag inside hi's rounding interval,
// and D > near when z - near exceeds 2^-38 mag in either direction.  Only
// the rare pair closer than that to a rounding boundary or to the near plane
// (about one in 2^14) computes D itself, so the FP64 pipe (a small fraction
// of the FP32 rate, and paid by the whole warp for any lane) stays idle.
// Returns the decision; z32 receives the key when it is visible.
__device__ __forceinline__ bool depth_key(const float *Tz, const float mu[3], float2 z, float near, float &z32) {
    const float mag = fabsf(Tz[0] * mu[0]) + fabsf(Tz[1] * mu[1]) + fabsf(Tz[2] * mu[2]) + fabsf(Tz[3]);
    const float margin = mag * 0x1p-38f;
    const float d = __fadd_rn(__fsub_rn(z.x, near), z.y);
    if (z.x > 0.f && fabsf(d) > margin) {
        const float up = __int_as_float(__float_as_int(z.x) + 1), dn = __int_as_float(__float_as_int(z.x) - 1);
        const float half = 0.5f * (z.y >= 0.f ? up - z.x : z.x - dn);
        if (fabsf(z.y) < half - margin) {
            z32 = z.x;
            return d > 0.f;
        }
    }
    const double D = view_coord(Tz, mu[0], mu[1], mu[2]);
    z32 = __double2float_rn(D);
    return D > (double)near;
}

// floor / ceil of hi + lo (|lo| <= ulp(hi) / 2, |hi| < 2^23): a non-integer
// hi keeps its floor / ceil; an integer hi moves by one if lo points away
__device__ __forceinline__ float floor_ff(float2 v) {
    const float f = floorf(v.x);
    return (f == v.x && v.y < 0.f) ? f - 1.f : f;
}
__device__ __forceinline__ float ceil_ff(float2 v) {
    const float c = ceilf(v.x);
    return (c == v.x && v.y > 0.f) ? c + 1.f : c;
}

// v - d for float-float v and a float d
__device__ __forceinline__ float2 ff_sub(float2 v, float d) {
    float s, e;
    two_sum(v.x, -d, s, e);
    return renorm(s, __fadd_rn(e, v.y));
}

__device__ __forceinline__ int submap_of(const SubmapInfo *subs, int n_submaps, int64_t g) {
    int lo = 0, hi = n_submaps - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (subs[mid].g0 <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// quaternion (w,x,y,z) -> rotation of the normalised quaternion; returns |q|
__device__ __forceinline__ float quat_rot(const float q[4], float qh[4], float R[9]) {
    float n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    float qn = sqrtf(n2);
    float inv = qn > 0.f ? 1.f / qn : 0.f;
    float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    qh[0] = w; qh[1] = x; qh[2] = y; qh[3] = z;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
    return qn;
}

// The rotation of q correctly rounded to float, R = M(q) / |q|^2 with the
// quadratic entries of M formed in double (products of floats are exact in
// double).  Used for strongly anisotropic Gaussians: a long axis s_L rounded
// by an ulp leans by ~1e-7 rad, which its projection onto a thin image
// direction turns into an error of the thin variance relative to itself of
// ~1e-7 s_L / s_thin (1e-5 for a 180:1 needle); correct rounding keeps each
// entry's error at half an ulp.  Not inlined: its double-precision code in the
// body of the projection kernels, even untaken, slowed them by a sixth.
__device__ __noinline__ void quat_rot_rn(const float q[4], float R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double ww = w * w, xx = x * x, yy = y * y, zz = z * z;
    const double inv = 1.0 / ((ww + xx) + (yy + zz));
    const double i2 = 2.0 * inv;
    R[0] = (float)(((ww + xx) - (yy + zz)) * inv);
    R[1] = (float)((x * y - w * z) * i2);
    R[2] = (float)((x * z + w * y) * i2);
    R[3] = (float)((x * y + w * z) * i2);
    R[4] = (float)(((ww + yy) - (xx + zz)) * inv);
    R[5] = (float)((y * z - w * x) * i2);
    R[6] = (float)((x * z - w * y) * i2);
    R[7] = (float)((y * z + w * x) * i2);
    R[8] = (float)(((ww + zz) - (xx + yy)) * inv);
}

// Axis-scale ratio above which the rotation is formed by quat_rot_rn: a float
// rotation leaves the thin variance ~6e-8 x the ratio off, 1.9e-6 at 32:1 (the
// bar is 1e-5), and the double path costs a warp its FP64 instructions
// whenever one lane takes it (a threshold of 8:1 sent most warps of the
// orchard's trunks and canopies there: projection 0.54 -> 0.77 ms at 4M).
constexpr float kAnisoLogRatio = 3.4657359f;  // ln 32

struct ProjArgs {
    const float *means, *log_scales, *quats, *opac, *sh;
    int64_t n;
    const gs_camera *cams;
    const ViewInfo *views;
    const SubmapInfo *subs;
    const int32_t *sub_views;
    int32_t n_submaps, maxv;
    Consts c;
    float4 *rec;
    uint32_t *pkey;
    short4 *rect;
    float *g2d_zero;  // forward: the image-space gradient rows of the visible pairs, cleared here
    // backward
    const float *g2d;
    float *gm, *gls, *gq, *gom, *gsh, *pose_part, *dens_acc;
    float4 *gdir;     // [pairs] dL/d(view direction) of the colour (x, y, z, unused)
    int32_t *dens_cnt;
    int32_t overwrite;  // gradients written (=) instead of accumulated, zeros for unseen Gaussians
    int32_t sh_vec;     // the SH array starts on a 16-byte boundary
    int32_t gsh_vec;    // the SH gradient array starts on a 16-byte boundary
};

// Projection of one pair in float after the exact depth: Jacobian, image
// covariance rows T2 = J W R S, and the derived quantities.
struct PairGeom {
    float pxf, pyf, pzf;          // view-space mean (rounded)
    float J00, J02, J11, J12;     // projection Jacobian
    bool clx, cly;                // tangent clamped
    float txc, tyc;               // clamped tangent times z
    float WM[9];                  // W R S
    float r0[3], r1[3];           // rows of J W R S
    float a, b, c, det;           // Sigma' and its determinant
    float cx, cy, cz;             // r0 x r1 (its 2x2 minors)
};

__device__ __forceinline__ void pair_geom(const Cam &cam, int W, int H, const Consts &k, float px, float py,
                                          float pz, const float R[9], const float S[3], PairGeom &G) {
    G.pxf = px;
    G.pyf = py;
    G.pzf = pz;
    float limx = k.jac_clamp * fmaxf(cam.cx, (float)W - cam.cx) / cam.fx;
    float limy = k.jac_clamp * fmaxf(cam.cy, (float)H - cam.cy) / cam.fy;
    float xr = G.pxf / G.pzf, yr = G.pyf / G.pzf;
    G.clx = xr < -limx || xr > limx;
    G.cly = yr < -limy || yr > limy;
    G.txc = fminf(fmaxf(xr, -limx), limx) * G.pzf;
    G.tyc = fminf(fmaxf(yr, -limy), limy) * G.pzf;
    float iz = 1.f / G.pzf;
    float iz2 = iz * iz;
    G.J00 = cam.fx * iz;
    G.J02 = -cam.fx * G.txc * iz2;
    G.J11 = cam.fy * iz;
    G.J12 = -cam.fy * G.tyc * iz2;
    const float *T = cam.T;
    // U = W R: the Gaussian's unit axes in camera coordinates (columns); W R S = U S
    float U[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            U[3 * i + j] = T[4 * i + 0] * R[j] + T[4 * i + 1] * R[3 + j] + T[4 * i + 2] * R[6 + j];
            G.WM[3 * i + j] = U[3 * i + j] * S[j];
        }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        G.r0[j] = G.J00 * G.WM[j] + G.J02 * G.WM[6 + j];
        G.r1[j] = G.J11 * G.WM[3 + j] + G.J12 * G.WM[6 + j];
    }
    float n0 = G.r0[0] * G.r0[0] + G.r0[1] * G.r0[1] + G.r0[2] * G.r0[2];
    float n1 = G.r1[0] * G.r1[0] + G.r1[1] * G.r1[1] + G.r1[2] * G.r1[2];
    G.b = G.r0[0] * G.r1[0] + G.r0[1] * G.r1[1] + G.r0[2] * G.r1[2];
    G.a = n0 + k.dilation;
    G.c = n1 + k.dilation;
    // r0 x r1, whose components are the 2x2 minors of T2 = J U S: by the
    // Binet-Cauchy identity the minor of columns (k, l) is
    //   s_k s_l (j0 x j1) . (u_k x u_l) = s_k s_l (j0 x j1) . u_m
    // for (k, l, m) cyclic (the columns u of a rotation: u_k x u_l = u_m), with
    // j0 = (J00, 0, J02), j1 = (0, J11, J12) the rows of J.  Taken from the
    // entries of r0 and r1 instead, a minor of a long thin Gaussian is a
    // difference of products of its long axis's large terms: their rounding
    // (about an ulp of s_long^2) swamps the true value s_long s_thin.
    const float nx = -G.J02 * G.J11, ny = -G.J00 * G.J12, nz = G.J00 * G.J11;
    G.cx = S[1] * S[2] * (nx * U[0] + ny * U[3] + nz * U[6]);
    G.cy = S[2] * S[0] * (nx * U[1] + ny * U[4] + nz * U[7]);
    G.cz = S[0] * S[1] * (nx * U[2] + ny * U[5] + nz * U[8]);
    G.det = (G.cx * G.cx + G.cy * G.cy + G.cz * G.cz) + k.dilation * (n0 + n1) + k.dilation * k.dilation;
}

template <int DEG>
__device__ __forceinline__ void load_sh(const float *sh, int64_t g, float C[16][3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float *p = sh + g * (3 * K);
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) C[k][ch] = __ldg(p + 3 * k + ch);
}

// unit viewing direction mu - C, C = -R^T t the camera centre
__device__ __forceinline__ void view_dir(const Cam &cam, const float mu[3], float w[3], float &wn) {
    const float *T = cam.T;
    float C0 = -(T[0] * T[3] + T[4] * T[7] + T[8] * T[11]);
    float C1 = -(T[1] * T[3] + T[5] * T[7] + T[9] * T[11]);
    float C2 = -(T[2] * T[3] + T[6] * T[7] + T[10] * T[11]);
    w[0] = mu[0] - C0;
    w[1] = mu[1] - C1;
    w[2] = mu[2] - C2;
    wn = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
}

template <int DEG>
__global__ void __launch_bounds__(kProjThreads) k_project_fwd(ProjArgs A) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= A.n) return;
    const Consts &k = A.c;
    int s = submap_of(A.subs, A.n_submaps, g);
    const SubmapInfo sub = A.subs[s];

    float mu[3] = {__ldg(A.means + 3 * g), __ldg(A.means + 3 * g + 1), __ldg(A.means + 3 * g + 2)};
    float ls[3] = {__ldg(A.log_scales + 3 * g), __ldg(A.log_scales + 3 * g + 1),
                   __ldg(A.log_scales + 3 * g + 2)};
    float q[4] = {__ldg(A.quats + 4 * g), __ldg(A.quats + 4 * g + 1), __ldg(A.quats + 4 * g + 2),
                  __ldg(A.quats + 4 * g + 3)};
    float om = __ldg(A.opac + g);
    float qh[4], R[9];
    float qn = quat_rot(q, qh, R);
    float S[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
    if (fmaxf(ls[0], fmaxf(ls[1], ls[2])) - fminf(ls[0], fminf(ls[1], ls[2])) > kAnisoLogRatio && qn > 0.f)
        quat_rot_rn(q, R);
    // ln o = -ln(1 + e^-omega); support threshold E = 2 ln(o / alpha_min)
    // largest axis scale, for the conservative frustum test below
    const float smax = fmaxf(S[0], fmaxf(S[1], S[2]));
    float lno = -log1pf(expf(-om));
    float log2o = lno * kLog2e;
    float E = 2.f * (lno - k.ln_alpha_min);
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float *shg = A.sh + g * (3 * K);
    const float mabs = fabsf(mu[0]) + fabsf(mu[1]) + fabsf(mu[2]);

    for (int kv = 0; kv < sub.nviews; ++kv) {
        int v = A.sub_views[s * A.maxv + kv];
        const ViewInfo vi = A.views[v];
        int64_t pair = (int64_t)vi.pair_off + (g - vi.g0);
        Cam cam = load_cam(A.cams, v);
        // float estimate of the view point: pairs clearly behind the near plane
        // or clearly outside the image skip the float-float mean and the exact
        // depth key (measured: projection 0.543 -> 0.491 ms on orchard4m)
        const float x_est = __fmaf_rn(cam.T[2], mu[2], __fmaf_rn(cam.T[1], mu[1], __fmaf_rn(cam.T[0], mu[0], cam.T[3])));
        const float y_est = __fmaf_rn(cam.T[6], mu[2], __fmaf_rn(cam.T[5], mu[1], __fmaf_rn(cam.T[4], mu[0], cam.T[7])));
        const float z_est = __fmaf_rn(cam.T[10], mu[2], __fmaf_rn(cam.T[9], mu[1], __fmaf_rn(cam.T[8], mu[0], cam.T[11])));
        const float tabs = fabsf(cam.T[3]) + fabsf(cam.T[7]) + fabsf(cam.T[11]);
        bool vis = qn > 0.f && E > 0.f && z_est > k.near_z - 1e-5f * (mabs + tabs + 1.f);
        if (vis) {
            // The rows of W R S have norm <= smax, so Sigma'_xx <= (|J00| + |J02|)^2 smax^2 + dil:
            // a pair whose mean lies farther outside the image than that bound on the
            // support's half-extent (plus margins for these float estimates) has no pixel.
            // Each estimate is within 4 ulps of (mabs + |t|) of the exact coordinate.
            const float iz = 1.f / z_est;
            const float limx = k.jac_clamp * fmaxf(cam.cx, (float)vi.W - cam.cx) / cam.fx;
            const float limy = k.jac_clamp * fmaxf(cam.cy, (float)vi.H - cam.cy) / cam.fy;
            const float tx = fminf(fmaxf(x_est * iz, -limx), limx), ty = fminf(fmaxf(y_est * iz, -limy), limy);
            const float jx = cam.fx * iz * (1.f + fabsf(tx)), jy = cam.fy * iz * (1.f + fabsf(ty));
            const float bx = sqrtf(E * (jx * jx * smax * smax + k.dilation)) * 1.01f * (1.f + k.ext_rel_pad) +
                             k.ext_abs_pad + 1.f;
            const float by = sqrtf(E * (jy * jy * smax * smax + k.dilation)) * 1.01f * (1.f + k.ext_rel_pad) +
                             k.ext_abs_pad + 1.f;
            const float uf = cam.fx * x_est * iz + cam.cx, vf = cam.fy * y_est * iz + cam.cy;
            const float est = 1e-6f * (mabs + tabs) * iz * (1.f + fabsf(x_est * iz) + fabsf(y_est * iz));
            const float mu_ = 1e-4f * (fabsf(uf) + fabsf(vf));
            const float mx = mu_ + cam.fx * est, my = mu_ + cam.fy * est;
            if (uf < 0.5f - bx - mx || uf > (float)vi.W - 0.5f + bx + mx ||
                vf < 0.5f - by - my || vf > (float)vi.H - 0.5f + by + my)
                vis = false;
        }
        float z32 = 0.f;
        float2 pxx = make_float2(0.f, 0.f), pyy = pxx, pzz = pxx;
        if (vis) {
            pzz = view_coord_ff(cam.T + 8, mu[0], mu[1], mu[2]);
            vis = depth_key(cam.T + 8, mu, pzz, k.near_z, z32);  // the exact depth key (R10)
        }
        if (vis) {
            pxx = view_coord_ff(cam.T, mu[0], mu[1], mu[2]);
            pyy = view_coord_ff(cam.T + 4, mu[0], mu[1], mu[2]);
        }
        PairGeom G;
        float4 r0 = make_float4(0, 0, 0, 0), r1 = r0, r2 = r0;
        short4 rc = make_short4(1, 1, 0, 0);
        if (vis) {
            pair_geom(cam, vi.W, vi.H, k, pxx.x, pyy.x, pzz.x, R, S, G);
            vis = G.det > 0.f;
        }
        if (vis) {
            // pixel mean (float-float), split into integer pixel + offset
            const float2 u = ff_pinhole(cam.fx, pxx, pzz, cam.cx);
            const float2 vv = ff_pinhole(cam.fy, pyy, pzz, cam.cy);
            const float Uf = floor_ff(u), Vf = floor_ff(vv);
            float hx = __fsub_rn(0.5f, __fadd_rn(__fsub_rn(u.x, Uf), u.y));
            float hy = __fsub_rn(0.5f, __fadd_rn(__fsub_rn(vv.x, Vf), vv.y));
            // padded axis-aligned extent of {d : d^T Sigma'^-1 d <= E}
            float ex = sqrtf(E * G.a) * (1.f + k.ext_rel_pad) + k.ext_abs_pad;
            float ey = sqrtf(E * G.c) * (1.f + k.ext_rel_pad) + k.ext_abs_pad;
            float xlo = ceil_ff(ff_sub(u, ex + 0.5f)), xhi = floor_ff(ff_sub(u, 0.5f - ex));
            float ylo = ceil_ff(ff_sub(vv, ey + 0.5f)), yhi = floor_ff(ff_sub(vv, 0.5f - ey));
            xlo = fmaxf(xlo, 0.f);
            ylo = fmaxf(ylo, 0.f);
            xhi = fminf(xhi, (float)(vi.W - 1));
            yhi = fminf(yhi, (float)(vi.H - 1));
            vis = xlo <= xhi && ylo <= yhi;
            if (vis) {
                rc = make_short4((short)((int)xlo / k.tile_w), (short)((int)ylo / k.tile_h),
                                 (short)((int)xhi / k.tile_w), (short)((int)yhi / k.tile_h));
                // Cholesky factor L (upper) of Sigma'^-1 = L^T L, scaled by kCholScale
                float l22 = kCholScale / sqrtf(G.c);
                float l11 = kCholScale * sqrtf(G.c / G.det);
                float l12 = -kCholScale * G.b / sqrtf(G.c * G.det);
                // colour seen from the camera centre
                float w[3], wn;
                view_dir(cam, mu, w, wn);
                float iw = 1.f / wn;
                float Y[16];
                sh_basis<DEG>(w[0] * iw, w[1] * iw, w[2] * iw, Y);
                float rgb[3];
                float acc[3] = {0.5f, 0.5f, 0.5f};
                if constexpr ((3 * K) % 4 == 0) {
                    // the row in 16-byte pieces when it starts on a 16-byte
                    // boundary: a warp's load then touches its 32 rows with a
                    // quarter of the instructions (orchard4m projection
                    // 0.486 -> 0.323 ms); coefficients in the same order
                    if (A.sh_vec) {
#pragma unroll
                        for (int q = 0; q < 3 * K / 4; ++q) {
                            const float4 c4 = __ldg(reinterpret_cast<const float4 *>(shg) + q);
                            const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int e = 4 * q + i, kk = e / 3, ch = e % 3;
                                acc[ch] = __fmaf_rn(cv[i], Y[kk], acc[ch]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < K; ++kk)
#pragma unroll
                            for (int ch = 0; ch < 3; ++ch)
                                acc[ch] = __fmaf_rn(__ldg(shg + 3 * kk + ch), Y[kk], acc[ch]);
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < K; ++kk)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) acc[ch] = __fmaf_rn(__ldg(shg + 3 * kk + ch), Y[kk], acc[ch]);
                }
                // a clamped channel is stored as -0: it renders as 0, and its
                // sign bit hands the clamp decision to the backward
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) rgb[ch] = acc[ch] < 0.f ? -0.f : acc[ch];
                r0 = make_float4(Uf, Vf, hx, hy);
                r1 = make_float4(l11, l12, l22, log2o);
                r2 = make_float4(rgb[0], rgb[1], rgb[2], z32);
            }
        }
        if (vis) {
            A.rec[3 * pair + 0] = r0;
            A.rec[3 * pair + 1] = r1;
            A.rec[3 * pair + 2] = r2;
            // the backward's atomics add into these rows: cleared next to the
            // record (neighbouring threads, neighbouring rows) instead of by a
            // gather over the sorted visible pairs later
            float2 *row = reinterpret_cast<float2 *>(A.g2d_zero + pair * kGrad);
#pragma unroll
            for (int i = 0; i < kGrad / 2; ++i) row[i] = make_float2(0.f, 0.f);
            // (read only for visible pairs, like the record: an invisible
            // pair's rectangle is not written)
            A.rect[pair] = rc;
        }
        A.pkey[pair] = vis ? __float_as_uint(r2.w) : kInvalidKey;
    }
}

// submap of projection-backward block b (blocks never straddle a submap)
__device__ __forceinline__ int submap_of_block(const ProjArgs &A, int b) {
    int lo = 0, hi = A.n_submaps - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (A.subs[mid].block0 <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The Gaussians of chunk c0 of submap s that at least one of the submap's
// views sees, in index order: s_item gets the chunk index, s_mask the views.
// Most Gaussians lie outside every frustum; packing the visible ones keeps
// the lanes of the backward busy.  All visibility loads are issued before
// the one barrier; positions come from per-warp ballots.  Returns the count
// (the same in every thread); the whole block must call it.  s_cnt holds
// kProjBwdChunk / 32 counters.
template <class Unseen>
__device__ int chunk_visible(const ProjArgs &A, int s, const SubmapInfo &sub, int64_t c0, int *s_item,
                             unsigned long long *s_mask, uint32_t *s_cnt, Unseen unseen) {
    constexpr int F = kProjBwdChunk / kProjBwdThreads, NW = kProjBwdThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long m[F];
#pragma unroll
    for (int f = 0; f < F; ++f) m[f] = 0ull;
    for (int kv = 0; kv < sub.nviews; ++kv) {
        const ViewInfo &vi = A.views[A.sub_views[s * A.maxv + kv]];
        const uint32_t *pk = A.pkey + (int64_t)vi.pair_off + (sub.g0 + c0 - vi.g0);
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const int loc = f * kProjBwdThreads + threadIdx.x;
            if (c0 + loc < sub.ng && pk[loc] != kInvalidKey) m[f] |= 1ull << kv;
        }
    }
    // the chunk's Gaussians that no view sees (in overwrite mode their
    // gradient rows are written here, as zeros)
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const int loc = f * kProjBwdThreads + threadIdx.x;
        if (c0 + loc < sub.ng && m[f] == 0ull) unseen(sub.g0 + c0 + loc);
    }
    uint32_t bal[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
        bal[f] = __ballot_sync(0xffffffffu, m[f] != 0ull);
        if (lane == 0) s_cnt[f * NW + wid] = __popc(bal[f]);
    }
    __syncthreads();
    // exclusive prefix in (f, warp) order, which is chunk index order
    uint32_t run = 0, base[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
        for (int w = 0; w < NW; ++w) {
            if (w == wid) base[f] = run;
            run += s_cnt[f * NW + w];
        }
    }
    const uint32_t below = (1u << lane) - 1u;
#pragma unroll
    for (int f = 0; f < F; ++f)
        if (m[f]) {
            const uint32_t pos = base[f] + __popc(bal[f] & below);
            s_item[pos] = f * kProjBwdThreads + threadIdx.x;
            s_mask[pos] = m[f];
        }
    __syncthreads();
    return (int)run;
}

// Adjoint of the SH colour, c_ch = max(0, 1/2 + sum_k sh_(k, ch) Y_k(d)) with
// d the unit direction from the camera centre to the mean: dL/dsh_(k, ch) =
// gc_ch Y_k and dL/dd = sum_(k, ch) gc_ch sh_(k, ch) grad Y_k, where gc is the
// pixel-space colour gradient of the pair, zero on a clamped channel.  Three
// lanes (one per channel) work one visible Gaussian: they read its SH row
// together (consecutive floats), keep their channel's coefficients and
// gradient sums in registers across the Gaussian's views, and write the row
// once; dL/dd of each pair goes to gdir for the geometric adjoint.
template <int DEG>
__global__ void __launch_bounds__(kProjBwdThreads) k_sh_bwd(ProjArgs A) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int NWARP = kProjBwdThreads / 32, GPW = 10;  // ten groups of three lanes a warp
    __shared__ int s_item[kProjBwdChunk];
    __shared__ unsigned long long s_mask[kProjBwdChunk];
    __shared__ uint32_t s_scan[kProjBwdChunk / 32];
    __shared__ uint8_t s_unseen[kProjBwdChunk];
    constexpr int R4 = (3 * K) % 4 == 0 ? 3 * K / 4 : 1;
    // the warp's ten gradient rows staged for 16-byte stores (orchard4m
    // adjoints 0.529 -> 0.518 ms); a row stride of R4 + 1 pieces keeps the
    // groups' lanes on different banks
    constexpr int SR = 4 * (R4 + 1);
    __shared__ __align__(16) float s_out[kProjBwdThreads / 32][GPW * SR];
    const bool vec = (3 * K) % 4 == 0 && A.gsh_vec;
    const int b = blockIdx.x, s = submap_of_block(A, b);
    const SubmapInfo sub = A.subs[s];
    const int64_t c0 = (int64_t)(b - sub.block0) * kProjBwdChunk;
    for (int i = threadIdx.x; i < kProjBwdChunk; i += kProjBwdThreads) s_unseen[i] = 0;
    __syncthreads();
    const int n_items = chunk_visible(A, s, sub, c0, s_item, s_mask, s_scan, [&](int64_t gu) {
        if (!A.overwrite) return;
        if (vec) {
            s_unseen[gu - sub.g0 - c0] = 1;  // cleared by the whole block below
            return;
        }
        float *row = A.gsh + gu * (3 * K);
#pragma unroll
        for (int i = 0; i < 3 * K; ++i) row[i] = 0.f;
    });
    // the unseen rows, consecutive threads on consecutive 16-byte pieces (a
    // thread writing a whole row of its own Gaussian spread each store over 32
    // rows: orchard4m SH and geometric adjoints 0.586 -> 0.529 ms)
    if (vec && A.overwrite) {
        const int nloc = (int)min((int64_t)kProjBwdChunk, sub.ng - c0);
        float4 *rows = reinterpret_cast<float4 *>(A.gsh + (sub.g0 + c0) * (3 * K));
        for (int i = threadIdx.x; i < nloc * R4; i += kProjBwdThreads)
            if (s_unseen[i / R4]) rows[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int grp = lane / 3, ch = lane - 3 * grp, lead = 3 * grp;  // lanes 30, 31 idle
    for (int base = wid * GPW; base < n_items; base += NWARP * GPW) {
        const int it = base + grp;
        const bool live = grp < GPW && it < n_items;
        unsigned long long mask = live ? s_mask[it] : 0ull;
        const int64_t g = sub.g0 + c0 + (live ? s_item[it] : 0);
        float mu[3] = {0.f, 0.f, 0.f}, shc[K], gacc[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            shc[kk] = live ? __ldg(A.sh + g * (3 * K) + 3 * kk + ch) : 0.f;
            gacc[kk] = 0.f;
        }
        if (live) {
            mu[0] = __ldg(A.means + 3 * g);
            mu[1] = __ldg(A.means + 3 * g + 1);
            mu[2] = __ldg(A.means + 3 * g + 2);
        }
        for (;;) {
            const bool act = mask != 0ull;
            if (!__any_sync(0xffffffffu, act)) break;
            float gd[3] = {0.f, 0.f, 0.f};
            int64_t pair = 0;
            if (act) {
                const int kv = __ffsll((long long)mask) - 1;
                mask &= mask - 1ull;
                const int v = A.sub_views[s * A.maxv + kv];
                const ViewInfo vi = A.views[v];
                pair = (int64_t)vi.pair_off + (g - vi.g0);
                // the forward marked a clamped channel by the sign of its colour
                // (both loads issued before the camera's arithmetic)
                const float cf = reinterpret_cast<const float *>(A.rec + 3 * pair + 2)[ch];
                const float graw = A.g2d[pair * kGrad + G_R + ch];
                const Cam cam = load_cam(A.cams, v);
                float w[3], wn;
                view_dir(cam, mu, w, wn);
                const float iw = 1.f / wn;
                const float d[3] = {w[0] * iw, w[1] * iw, w[2] * iw};
                const float gc = signbit(cf) ? 0.f : graw;
                float Y[16], dY[16][3];
                sh_basis<DEG>(d[0], d[1], d[2], Y);
                sh_basis_grad<DEG>(d[0], d[1], d[2], dY);
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    gacc[kk] = __fmaf_rn(gc, Y[kk], gacc[kk]);
                    const float t = gc * shc[kk];
                    gd[0] = __fmaf_rn(t, dY[kk][0], gd[0]);
                    gd[1] = __fmaf_rn(t, dY[kk][1], gd[1]);
                    gd[2] = __fmaf_rn(t, dY[kk][2], gd[2]);
                }
            }
            // sum over the three channels of the group, in channel order
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float a1 = __shfl_sync(0xffffffffu, gd[i], min(lead + 1, 31));
                const float a2 = __shfl_sync(0xffffffffu, gd[i], min(lead + 2, 31));
                gd[i] = (gd[i] + a1) + a2;
            }
            if (act && ch == 0) A.gdir[pair] = make_float4(gd[0], gd[1], gd[2], 0.f);
        }
        if (vec && A.overwrite) {
            float *so = s_out[wid];
            if (live) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) so[grp * SR + 3 * kk + ch] = gacc[kk];
            }
            __syncwarp();
            for (int i = lane; i < GPW * R4; i += 32) {
                const int r = i / R4, q = i - r * R4;
                if (base + r < n_items) {
                    const int64_t gr = sub.g0 + c0 + s_item[base + r];
                    reinterpret_cast<float4 *>(A.gsh + gr * (3 * K))[q] =
                        reinterpret_cast<const float4 *>(so + r * SR)[q];
                }
            }
            __syncwarp();
        } else if (live) {
            float *gsh = A.gsh + g * (3 * K) + ch;
            if (A.overwrite) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) gsh[3 * kk] = gacc[kk];
            } else {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) gsh[3 * kk] += gacc[kk];
            }
        }
    }
}

// Five blocks an SM (96 registers, a few spilled outside the view loop):
// orchard4m 0.657 -> 0.635 ms for the two adjoint kernels, against four
// blocks at 116 registers; six (80 registers) spill inside the loop.
template <int DEG>
__global__ void __launch_bounds__(kProjBwdThreads, 5) k_project_bwd(ProjArgs A) {
    constexpr int NWARP = kProjBwdThreads / 32;
    extern __shared__ float red[];  // [views of the submap][warps][6] pose twist sums
    __shared__ int s_item[kProjBwdChunk];                  // chunk index of a visible Gaussian
    __shared__ unsigned long long s_mask[kProjBwdChunk];  // the views that see it
    __shared__ uint32_t s_scan[kProjBwdChunk / 32];
    const Consts &k = A.c;
    // blocks are laid out per submap, kProjBwdChunk Gaussians each
    const int b = blockIdx.x, s = submap_of_block(A, b);
    const SubmapInfo sub = A.subs[s];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t c0 = (int64_t)(b - sub.block0) * kProjBwdChunk;
    for (int i = tid; i < sub.nviews * NWARP * 6; i += kProjBwdThreads) red[i] = 0.f;

    // 1. the chunk's Gaussians that some view sees (in overwrite mode the
    //    others' rows get zeros)
    const int n_items = chunk_visible(A, s, sub, c0, s_item, s_mask, s_scan, [&](int64_t gu) {
        if (!A.overwrite) return;
#pragma unroll
        for (int i = 0; i < 3; ++i) A.gm[3 * gu + i] = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) A.gls[3 * gu + i] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) A.gq[4 * gu + i] = 0.f;
        A.gom[gu] = 0.f;
        if (A.dens_acc) A.dens_acc[gu] = 0.f;
        if (A.dens_cnt) A.dens_cnt[gu] = 0;
    });

    // 2. each warp takes 32 of them at a time; a lane walks the views of its
    //    Gaussian in order and is the only writer of its gradients
    for (int base = wid * 32; base < n_items; base += kProjBwdThreads) {
        const int it = base + lane;
        const bool live = it < n_items;
        unsigned long long mask = live ? s_mask[it] : 0ull;
        const int64_t g = sub.g0 + c0 + (live ? s_item[it] : 0);
        float mu[3] = {0, 0, 0}, ls[3] = {0, 0, 0}, q[4] = {1, 0, 0, 0}, om = 0.f;
        if (live) {
            mu[0] = __ldg(A.means + 3 * g); mu[1] = __ldg(A.means + 3 * g + 1); mu[2] = __ldg(A.means + 3 * g + 2);
            ls[0] = __ldg(A.log_scales + 3 * g); ls[1] = __ldg(A.log_scales + 3 * g + 1);
            ls[2] = __ldg(A.log_scales + 3 * g + 2);
            q[0] = __ldg(A.quats + 4 * g); q[1] = __ldg(A.quats + 4 * g + 1);
            q[2] = __ldg(A.quats + 4 * g + 2); q[3] = __ldg(A.quats + 4 * g + 3);
            om = __ldg(A.opac + g);
        }
        float qh[4], R[9];
        float qn = quat_rot(q, qh, R);
        float S[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
        if (fmaxf(ls[0], fmaxf(ls[1], ls[2])) - fminf(ls[0], fminf(ls[1], ls[2])) > kAnisoLogRatio && qn > 0.f)
            quat_rot_rn(q, R);  // the forward's rotation
        float o = 1.f / (1.f + expf(-om));

        float gmu[3] = {0, 0, 0}, gM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gom = 0.f;
        float gls[3] = {0, 0, 0};
        float dacc = 0.f;
        int dcnt = 0;
        for (;;) {
            const bool act = mask != 0ull;
            if (!__any_sync(0xffffffffu, act)) break;
            const int kv = act ? __ffsll((long long)mask) - 1 : -1;
            if (act) mask &= mask - 1ull;
            float gpose[6] = {0, 0, 0, 0, 0, 0};
            if (act) {
                int v = A.sub_views[s * A.maxv + kv];
                const ViewInfo vi = A.views[v];
                int64_t pair = (int64_t)vi.pair_off + (g - vi.g0);
                    const float *gg = A.g2d + pair * kGrad;
                    float gu = gg[G_U], gv = gg[G_V], gqa = gg[G_QA], gqb = gg[G_QB], gqc = gg[G_QC];
                    float glno = gg[G_LNO], gz = gg[G_Z];
                    // view-direction gradient of the colour, from the SH adjoint
                    // (loaded with the image-space row, before the pair's geometry)
                    const float4 gd4 = A.gdir[pair];
                    Cam cam = load_cam(A.cams, v);
                    PairGeom G;
                    pair_geom(cam, vi.W, vi.H, k, view_coord_ff(cam.T, mu[0], mu[1], mu[2]).x,
                              view_coord_ff(cam.T + 4, mu[0], mu[1], mu[2]).x, view_coord_ff(cam.T + 8, mu[0], mu[1], mu[2]).x,
                              R, S, G);
                    const float p[3] = {G.pxf, G.pyf, G.pzf};
                    const float *T = cam.T;
                    float gp[3] = {0.f, 0.f, gz};
                    // pixel mean
                    float iz = 1.f / p[2], iz2 = iz * iz;
                    gp[0] += gu * cam.fx * iz;
                    gp[1] += gv * cam.fy * iz;
                    gp[2] -= (gu * cam.fx * p[0] + gv * cam.fy * p[1]) * iz2;
                    // colour
                    float w[3], wn;
                    view_dir(cam, mu, w, wn);
                    float iw = 1.f / wn;
                    float d[3] = {w[0] * iw, w[1] * iw, w[2] * iw};
                    const float gdir[3] = {gd4.x, gd4.y, gd4.z};
                    float dd = d[0] * gdir[0] + d[1] * gdir[1] + d[2] * gdir[2];
                    float gw[3] = {(gdir[0] - d[0] * dd) * iw, (gdir[1] - d[1] * dd) * iw, (gdir[2] - d[2] * dd) * iw};
                    // Sigma' = T2 T2^T + dil I with T2 = J W M, rows r0, r1 and columns
                    // v_k (the image-space axes), Q = Sigma'^-1, G = [[gqa, gqb/2],
                    // [gqb/2, gqc]]: dL/dSigma' = -Q G Q, so column k of dL/dT2 is
                    // 2 dL/dSigma' v_k = -2 Q G Y_k with Y_k = Q v_k, and
                    // dL/dls_k = v_k . (column k) = -2 Y_k^T G Y_k (M = R diag(S)
                    // scales column k).  Q is applied through the adjugate
                    // adj(Sigma') = sum_m w_m w_m^T + dil I, w_m = (r1_m, -r0_m): in
                    // Y_k det = sum_{m != k} w_m (w_m . v_k) + dil v_k axis k's own term
                    // vanishes identically, and w_m . v_k are the minors of r0 x r1.
                    // The entries of -Q G Q would cancel for a long thin Gaussian (Q's
                    // small eigenvalue, along its long axis, is a difference of large
                    // entries).
                    const float idet = 1.f / G.det;
                    const float hb = 0.5f * gqb;
                    float gr0[3], gr1[3];
                    {
                        const float cr[3][3] = {{0.f, G.cz, -G.cy}, {-G.cz, 0.f, G.cx}, {G.cy, -G.cx, 0.f}};
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) {
                            float y0 = k.dilation * G.r0[kk], y1 = k.dilation * G.r1[kk];
#pragma unroll
                            for (int m = 0; m < 3; ++m) {
                                if (m == kk) continue;
                                // w_m . v_k = r1_m r0_k - r0_m r1_k = cr[kk][m]
                                y0 += G.r1[m] * cr[kk][m];
                                y1 -= G.r0[m] * cr[kk][m];
                            }
                            y0 *= idet;
                            y1 *= idet;
                            const float z0 = gqa * y0 + hb * y1, z1 = hb * y0 + gqc * y1;  // G Y_k
                            gls[kk] -= 2.f * (z0 * y0 + z1 * y1);
                            // Q z = (sum_m w_m (w_m . z) + dil z) / det
                            float q0 = k.dilation * z0, q1 = k.dilation * z1;
#pragma unroll
                            for (int m = 0; m < 3; ++m) {
                                const float wz = G.r1[m] * z0 - G.r0[m] * z1;
                                q0 += G.r1[m] * wz;
                                q1 -= G.r0[m] * wz;
                            }
                            gr0[kk] = -2.f * q0 * idet;
                            gr1[kk] = -2.f * q1 * idet;
                        }
                    }
                    // T2 = J WM: rows r0 = J00 WM0 + J02 WM2, r1 = J11 WM1 + J12 WM2
                    float gJ00 = gr0[0] * G.WM[0] + gr0[1] * G.WM[1] + gr0[2] * G.WM[2];
                    float gJ02 = gr0[0] * G.WM[6] + gr0[1] * G.WM[7] + gr0[2] * G.WM[8];
                    float gJ11 = gr1[0] * G.WM[3] + gr1[1] * G.WM[4] + gr1[2] * G.WM[5];
                    float gJ12 = gr1[0] * G.WM[6] + gr1[1] * G.WM[7] + gr1[2] * G.WM[8];
                    float gWM[9];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        gWM[j] = G.J00 * gr0[j];
                        gWM[3 + j] = G.J11 * gr1[j];
                        gWM[6 + j] = G.J02 * gr0[j] + G.J12 * gr1[j];
                    }
                    // J as a function of p (clamped tangent: J02 = -fx c / z)
                    gp[2] += -(gJ00 * cam.fx + gJ11 * cam.fy) * iz2;
                    if (!G.clx) {
                        gp[0] += -gJ02 * cam.fx * iz2;
                        gp[2] += 2.f * gJ02 * cam.fx * p[0] * iz2 * iz;
                    } else {
                        gp[2] += gJ02 * cam.fx * (G.txc * iz) * iz2;
                    }
                    if (!G.cly) {
                        gp[1] += -gJ12 * cam.fy * iz2;
                        gp[2] += 2.f * gJ12 * cam.fy * p[1] * iz2 * iz;
                    } else {
                        gp[2] += gJ12 * cam.fy * (G.tyc * iz) * iz2;
                    }
                    // WM = Rb M: dL/dM += Rb^T gWM ; pose rotation: Rb -> (I + [phi]x) Rb
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            gM[3 * i + j] += T[i] * gWM[j] + T[4 + i] * gWM[3 + j] + T[8 + i] * gWM[6 + j];
                    // dL/dphi from WM: delta WM = [phi]x WM -> dL/dphi = sum_j WM_j x gWM_j (columns)
                    float A_[9];  // A = gWM WM^T
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            A_[3 * i + j] = gWM[3 * i] * G.WM[3 * j] + gWM[3 * i + 1] * G.WM[3 * j + 1] +
                                            gWM[3 * i + 2] * G.WM[3 * j + 2];
                    // tr(A^T [phi]x WM...) : dL = sum_ij gWM_ij ([phi]x WM)_ij = tr(gWM^T [phi]x WM)
                    //   = tr([phi]x WM gWM^T) = tr([phi]x A^T); axial part
                    gpose[3] += A_[7] - A_[5];
                    gpose[4] += A_[2] - A_[6];
                    gpose[5] += A_[3] - A_[1];
                    // mean and pose translation: p = Rb mu + t
                    gmu[0] += T[0] * gp[0] + T[4] * gp[1] + T[8] * gp[2] + gw[0];
                    gmu[1] += T[1] * gp[0] + T[5] * gp[1] + T[9] * gp[2] + gw[1];
                    gmu[2] += T[2] * gp[0] + T[6] * gp[1] + T[10] * gp[2] + gw[2];
                    float gwc[3] = {T[0] * gw[0] + T[1] * gw[1] + T[2] * gw[2],
                                    T[4] * gw[0] + T[5] * gw[1] + T[6] * gw[2],
                                    T[8] * gw[0] + T[9] * gw[1] + T[10] * gw[2]};
                    gpose[0] += gp[0] + gwc[0];
                    gpose[1] += gp[1] + gwc[1];
                    gpose[2] += gp[2] + gwc[2];
                    gpose[3] += p[1] * gp[2] - p[2] * gp[1];
                    gpose[4] += p[2] * gp[0] - p[0] * gp[2];
                    gpose[5] += p[0] * gp[1] - p[1] * gp[0];
                    // opacity: d ln o / d omega = 1 - o
                    gom += glno * (1.f - o);
                    dacc += sqrtf(gu * gu + gv * gv);
                    dcnt += 1;
            }
            // pose twist: one warp sum per view that some lane worked in this
            // step, added to the warp's slot of that view (fixed order)
            unsigned pend = __ballot_sync(0xffffffffu, act);
            while (pend) {
                const int kv0 = __shfl_sync(0xffffffffu, kv, __ffs(pend) - 1);
                const bool mine = kv == kv0;
                pend &= ~__ballot_sync(0xffffffffu, mine);
                float t[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    t[i] = mine ? gpose[i] : 0.f;
#pragma unroll
                    for (int o2 = 16; o2 > 0; o2 >>= 1) t[i] += __shfl_xor_sync(0xffffffffu, t[i], o2);
                }
                if (lane == 0)
#pragma unroll
                    for (int i = 0; i < 6; ++i) red[(kv0 * NWARP + wid) * 6 + i] += t[i];
            }
        }
        if (live) {
            // M = R diag(S): dL/dR_ik = gM_ik S_k (dL/dls_k was summed per view above)
            float gR[9];
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                gR[kk] = gM[kk] * S[kk];
                gR[3 + kk] = gM[3 + kk] * S[kk];
                gR[6 + kk] = gM[6 + kk] * S[kk];
            }
            // rotation of the normalised quaternion, then the normalisation
            float w = qh[0], x = qh[1], y = qh[2], z = qh[3];
            float gw_ = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
            float gx_ = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] +
                               w * gR[7] - 2.f * x * gR[8]);
            float gy_ = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] +
                               z * gR[7] - 2.f * y * gR[8]);
            float gz_ = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] +
                               y * gR[5] + x * gR[6] + y * gR[7]);
            float dq = w * gw_ + x * gx_ + y * gy_ + z * gz_;
            float iq = qn > 0.f ? 1.f / qn : 0.f;
            float gq[4] = {(gw_ - w * dq) * iq, (gx_ - x * dq) * iq, (gy_ - y * dq) * iq, (gz_ - z * dq) * iq};

#pragma unroll
            for (int i = 0; i < 3; ++i) A.gm[3 * g + i] = (A.overwrite ? 0.f : A.gm[3 * g + i]) + gmu[i];
#pragma unroll
            for (int i = 0; i < 3; ++i) A.gls[3 * g + i] = (A.overwrite ? 0.f : A.gls[3 * g + i]) + gls[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) A.gq[4 * g + i] = (A.overwrite ? 0.f : A.gq[4 * g + i]) + gq[i];
            A.gom[g] = (A.overwrite ? 0.f : A.gom[g]) + gom;
            if (A.dens_acc) A.dens_acc[g] = (A.overwrite ? 0.f : A.dens_acc[g]) + dacc;
            if (A.dens_cnt) A.dens_cnt[g] = (A.overwrite ? 0 : A.dens_cnt[g]) + dcnt;
        }
    }
    __syncthreads();
    for (int idx = tid; idx < sub.nviews * 6; idx += kProjBwdThreads) {
        int kv = idx / 6, i = idx % 6;
        float t = 0.f;
        for (int w = 0; w < NWARP; ++w) t += red[(kv * NWARP + w) * 6 + i];
        A.pose_part[((int64_t)b * A.maxv + kv) * 6 + i] = t;
    }
}

// pose[v][i] += sum over the blocks of v's submap of the partials of v's slot;
// one block per (view, component), fixed summation order
__global__ void __launch_bounds__(256) k_pose_reduce(const float *pose_part, const ViewInfo *views,
                                                    const SubmapInfo *subs, int maxv, float *pose, int overwrite) {
    __shared__ double sm[8];
    const int v = blockIdx.x / 6, i = blockIdx.x % 6;
    const ViewInfo vi = views[v];
    const SubmapInfo sub = subs[vi.submap];
    double acc = 0.0;
    for (int b = sub.block0 + threadIdx.x; b < sub.block0 + sub.nblocks; b += 256)
        acc += (double)pose_part[((int64_t)b * maxv + vi.k_in_submap) * 6 + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w];
        pose[6 * v + i] = (overwrite ? 0.f : pose[6 * v + i]) + (float)t;
    }
}

ProjArgs make_args(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams) {
    ProjArgs A{};
    A.means = g->means;
    A.log_scales = g->log_scales;
    A.quats = g->quats;
    A.opac = g->opacity_logits;
    A.sh = g->sh;
    A.n = g->n;
    A.cams = cams;
    A.views = ws->views;
    A.subs = ws->subs;
    A.sub_views = ws->sub_views;
    A.n_submaps = ws->n_submaps;
    A.maxv = ws->max_views_per_submap;
    A.c = ws->consts;
    A.rec = ws->rec;
    A.pkey = ws->pkey;
    A.rect = ws->rect;
    A.g2d = ws->g2d;
    A.sh_vec = (((uintptr_t)g->sh) & 15) == 0;
    return A;
}

}  // namespace

gs_status launch_project_fwd(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams,
                             cudaStream_t s) {
    ProjArgs A = make_args(ws, g, cams);
    A.g2d_zero = ws->g2d;
    ws->g2d_clear = true;  // (set before the early return: no pair, nothing to clear)
    if (ws->n == 0) return GS_OK;
    StageTimer timer(ws, GS_STAGE_PROJECT, s);
    int grid = (int)((ws->n + kProjThreads - 1) / kProjThreads);
    switch (ws->sh_degree) {
        case 0: ++ws->kernel_launches; k_project_fwd<0><<<grid, kProjThreads, 0, s>>>(A); break;
        case 1: ++ws->kernel_launches; k_project_fwd<1><<<grid, kProjThreads, 0, s>>>(A); break;
        case 2: ++ws->kernel_launches; k_project_fwd<2><<<grid, kProjThreads, 0, s>>>(A); break;
        default: ++ws->kernel_launches; k_project_fwd<3><<<grid, kProjThreads, 0, s>>>(A); break;
    }
    return check_launch("project_fwd");
}

gs_status launch_project_bwd(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams,
                             const gs_grads *out, cudaStream_t s) {
    ProjArgs A = make_args(ws, g, cams);
    A.gm = out->means;
    A.gls = out->log_scales;
    A.gq = out->quats;
    A.gom = out->opacity_logits;
    A.gsh = out->sh;
    A.pose_part = ws->pose_part;
    A.dens_acc = out->densify_acc;
    A.dens_cnt = out->densify_cnt;
    A.gdir = ws->gdir;
    A.overwrite = out->overwrite;
    A.gsh_vec = (((uintptr_t)out->sh) & 15) == 0;
    StageTimer timer(ws, GS_STAGE_PROJECT_BWD, s);
    if (ws->proj_blocks > 0) {
        size_t smem = sizeof(float) * ws->max_views_per_submap * (kProjBwdThreads / 32) * 6;
        switch (ws->sh_degree) {
            case 0: ++ws->kernel_launches; k_sh_bwd<0><<<ws->proj_blocks, kProjBwdThreads, 0, s>>>(A); break;
            case 1: ++ws->kernel_launches; k_sh_bwd<1><<<ws->proj_blocks, kProjBwdThreads, 0, s>>>(A); break;
            case 2: ++ws->kernel_launches; k_sh_bwd<2><<<ws->proj_blocks, kProjBwdThreads, 0, s>>>(A); break;
            default: ++ws->kernel_launches; k_sh_bwd<3><<<ws->proj_blocks, kProjBwdThreads, 0, s>>>(A); break;
        }
        switch (ws->sh_degree) {
            case 0: ++ws->kernel_launches; k_project_bwd<0><<<ws->proj_blocks, kProjBwdThreads, smem, s>>>(A); break;
            case 1: ++ws->kernel_launches; k_project_bwd<1><<<ws->proj_blocks, kProjBwdThreads, smem, s>>>(A); break;
            case 2: ++ws->kernel_launches; k_project_bwd<2><<<ws->proj_blocks, kProjBwdThreads, smem, s>>>(A); break;
            default: ++ws->kernel_launches; k_project_bwd<3><<<ws->proj_blocks, kProjBwdThreads, smem, s>>>(A); break;
        }
        gs_status st = check_launch("project_bwd");
        if (st != GS_OK) return st;
    }
    if (out->pose) {
        ++ws->kernel_launches;
        k_pose_reduce<<<6 * ws->n_views, 256, 0, s>>>(ws->pose_part, ws->views, ws->subs,
                                                      ws->max_views_per_submap, out->pose, out->overwrite);
        return check_launch("pose_reduce");
    }
    return GS_OK;
}

}  // namespace gs
