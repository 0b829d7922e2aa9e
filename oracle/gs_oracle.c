/*
 * FP64 CPU oracle for multi-view differentiable Gaussian splatting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  The product path (the CUDA
 * library under paper_2510_26358_gb300/csrc) never calls it, and the two share
 * no code, header, table or constant generator.
 *
 * Everything is computed in double precision, one pixel and one Gaussian at a
 * time, in the order the method defines it, with no blocking or fusion.
 * Paper: AgriGS-SLAM, Sec. III-B (multi-view 3DGS, Eqs. 2-4) and Sec. III-C
 * (losses, Eqs. 6-8).  The paper defers the rasteriser itself to standard
 * 3D Gaussian Splatting; the constants it leaves open are taken as
 *   dilation 0.3 px, alpha = min(0.99, o*exp(-d^T Sigma'^-1 d / 2)),
 *   skip alpha < 1/255, stop before blending when T would drop below 1e-4,
 * and the readings below.
 *
 * Readings (where the paper is silent):
 *   R1  quaternion order (w,x,y,z), normalised before use; |q| = 0 culls.
 *   R2  cameras use OpenCV axes; W_b is the world->camera [R|t].
 *   R3  near plane: a pair is visible only if view-space z > near_z.
 *   R4  Jacobian of the pinhole with the tangent x/z clamped to
 *       +-jac_clamp*max(cx, W-cx)/fx (same for y); derivative taken of the
 *       clamped function as written.
 *   R5  pixel (i,j) is sampled at its centre (i+0.5, j+0.5).
 *   R6  support: a Gaussian contributes to a pixel iff alpha >= alpha_min there;
 *       its tile rectangle covers the pixel centres inside the padded
 *       axis-aligned extent of the ellipse {d : d^T Q d <= 2 ln(o/alpha_min)}.
 *       Images therefore do not depend on the tile size.
 *   R6b a tile of that rectangle holds an instance iff the box of its pixel
 *       centres (clipped to the image), grown by ext_abs_pad on every side,
 *       meets the padded ellipse {d : d^T Q d <= E (1 + ext_rel_pad)^2},
 *       E = 2 ln(o/alpha_min): the rectangle's corner tiles that the ellipse
 *       misses hold no pixel the Gaussian reaches and get no instance.  Only
 *       the instance lists change: every pixel with alpha >= alpha_min lies
 *       in a kept tile, so images do not depend on this reading.
 *   R7  colour: real orthonormal SH basis without Condon-Shortley phase,
 *       ordered by l then m=-l..l, evaluated at the unit direction from the
 *       camera centre to the mean; rgb = max(0.5 + sum_k c_k Y_k, 0).
 *   R8  opacity o = sigmoid(omega).
 *   R9  compositing order: ascending (fp32-rounded view depth, Gaussian index);
 *       depth output is the alpha-weighted view-space z, not normalised.
 *   R10 depth is exact: p = R mu + t summed as ((R0 mu0 + R1 mu1) + R2 mu2) + t
 *       in double (products of float inputs are exact), then z32 = (float)p_z.
 *   R11 pose tangent: left perturbation T_cw <- exp(xi^) T_cw, xi = (rho, phi).
 *   R12 depth loss (Eq. 7): nearest pixel of each LiDAR return; fixed sigma_u;
 *       points are valid if inside the image, z_L > near_z and alpha > 0.
 *   R13 image loss (Eq. 6 with lambda = 0): mean |C - I| over all channels,
 *       pixels and views.
 *   R14 densification statistic: per view where the pair is visible,
 *       acc += ||(dL/du, dL/dv)|| in pixels and cnt += 1.
 *   R17 SSIM term of Eq. (6): per channel of every view, the structural
 *       similarity of Wang et al. (2004) with an 11x11 Gaussian window of
 *       sigma 1.5 (weights normalised to sum 1), zero padding outside the
 *       image ('same' output size), C1 = 0.01^2, C2 = 0.03^2 (unit dynamic
 *       range), averaged over all channels, pixels and views.
 *   R16 rendered depth distribution (for Eq. 7 with a predicted sigma_u):
 *       the weights w_k = alpha_k T_k of a pixel's blended fragments, of total
 *       W = sum w (= A), spread over their depths z_k: mean mu_u = D/W and
 *       variance var = sum w (z - mu_u)^2 / W (both 0 where nothing blends);
 *       sigma_u^2 = max(var, 0) + sigma_U^2 (sigma_U is the floor).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* interface types                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t width, height, submap, pad_;
    double fx, fy, cx, cy;
    double T[12]; /* row-major [R | t], world -> camera */
} oc_camera;

typedef struct {
    int32_t tile_w, tile_h;
    double near_z, dilation, alpha_min, alpha_max, t_min, jac_clamp;
    double ext_rel_pad, ext_abs_pad; /* padding of the extent used for tile rectangles */
    double rect_eps_abs, rect_eps_rel; /* width of the ambiguity band for rect decisions */
    double tile_eps_rel, tile_eps_cond; /* relative band of the R6b tile decisions: rel + cond *
                                         * (a c + b^2) / det of Sigma' (the rounding of the
                                         * inverse grows with its condition) */
} oc_config;

/* columns of a projected record (one row of OC_NCOL doubles per pair) */
enum {
    C_VIS = 0, C_TX0, C_TY0, C_TX1, C_TY1, /* tile rectangle, inclusive */
    C_U, C_V, C_Z, C_Z32,                 /* pixel mean, view depth, depth as float */
    C_SA, C_SB, C_SC,                     /* Sigma' (2x2, with dilation) */
    C_QA, C_QB, C_QC,                     /* Q = Sigma'^-1 */
    C_OPA, C_E, C_EX, C_EY,               /* opacity, support threshold, padded extents */
    C_R, C_G, C_B,                        /* colour */
    C_CLR, C_CLG, C_CLB,                  /* 1 where the colour is clamped at 0 */
    C_RGB_MARGIN,                         /* min |0.5 + sum c Y| over channels */
    C_RECT_AMBIG,                         /* 1 if a rect or tile decision lies inside the eps band */
    C_GAUSS, C_VIEW,                      /* Gaussian index, view index */
    C_NTILE,                              /* tiles of the rectangle that hold an instance (R6b) */
    OC_NCOL
};

/* columns of the per-pair image-space gradient */
enum { G_U = 0, G_V, G_QA, G_QB, G_QC, G_LNO, G_R, G_G, G_B, G_Z, OC_NGRAD };

/* layout check for the Python wrapper: OC_NCOL*100 + OC_NGRAD */
int64_t oracle_layout(void) { return (int64_t)OC_NCOL * 100 + OC_NGRAD; }

/* Host threads of the per-pair and per-pixel loops (OpenMP when compiled with
 * it).  Each pair and each pixel is computed alone, exactly as with one
 * thread; only the order in which the backward adds contributions of
 * different pixels into one pair's gradient (and of different pairs into a
 * view's pose gradient) depends on the threads, so results with more than
 * one thread can differ from the one-thread results by rounding.  Default 1. */
static int oc_threads = 1;
void oracle_set_threads(int n) { oc_threads = n > 0 ? n : 1; }
int oracle_get_threads(void) { return oc_threads; }

/* a += v, atomic when several threads may add to the same location */
static void acc_add(double *a, double v) {
#ifdef _OPENMP
#pragma omp atomic
#endif
    *a += v;
}

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void mat3_transpose(const double A[9], double B[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[3 * j + i] = A[3 * i + j];
}

/* rotation of a unit quaternion (w,x,y,z) */
static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR/dq_k for the same formula, k = w,x,y,z (q need not be unit here) */
static void quat_to_rot_jac(const double q[4], double dR[4][9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], Dw, sizeof Dw);
    memcpy(dR[1], Dx, sizeof Dx);
    memcpy(dR[2], Dy, sizeof Dy);
    memcpy(dR[3], Dz, sizeof Dz);
}

/* real orthonormal SH basis (R7) and its gradient w.r.t. the direction */
static void sh_basis(int deg, const double d[3], double Y[16], double dY[16][3]) {
    const double PI = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    double c0 = 0.5 * sqrt(1.0 / PI);
    double c1 = sqrt(3.0 / (4.0 * PI));
    double c2a = 0.5 * sqrt(15.0 / PI), c2b = 0.25 * sqrt(5.0 / PI), c2c = 0.25 * sqrt(15.0 / PI);
    double c3a = 0.25 * sqrt(35.0 / (2.0 * PI)), c3b = 0.5 * sqrt(105.0 / PI);
    double c3c = 0.25 * sqrt(21.0 / (2.0 * PI)), c3d = 0.25 * sqrt(7.0 / PI);
    double c3e = 0.25 * sqrt(105.0 / PI);
    memset(dY, 0, sizeof(double) * 16 * 3);
    Y[0] = c0;
    if (deg < 1) return;
    Y[1] = c1 * y; dY[1][1] = c1;
    Y[2] = c1 * z; dY[2][2] = c1;
    Y[3] = c1 * x; dY[3][0] = c1;
    if (deg < 2) return;
    Y[4] = c2a * x * y;               dY[4][0] = c2a * y; dY[4][1] = c2a * x;
    Y[5] = c2a * y * z;               dY[5][1] = c2a * z; dY[5][2] = c2a * y;
    Y[6] = c2b * (2 * z * z - x * x - y * y);
    dY[6][0] = -2 * c2b * x; dY[6][1] = -2 * c2b * y; dY[6][2] = 4 * c2b * z;
    Y[7] = c2a * x * z;               dY[7][0] = c2a * z; dY[7][2] = c2a * x;
    Y[8] = c2c * (x * x - y * y);     dY[8][0] = 2 * c2c * x; dY[8][1] = -2 * c2c * y;
    if (deg < 3) return;
    Y[9] = c3a * y * (3 * x * x - y * y);
    dY[9][0] = c3a * 6 * x * y; dY[9][1] = c3a * (3 * x * x - 3 * y * y);
    Y[10] = c3b * x * y * z;
    dY[10][0] = c3b * y * z; dY[10][1] = c3b * x * z; dY[10][2] = c3b * x * y;
    Y[11] = c3c * y * (4 * z * z - x * x - y * y);
    dY[11][0] = c3c * (-2 * x * y); dY[11][1] = c3c * (4 * z * z - x * x - 3 * y * y);
    dY[11][2] = c3c * 8 * y * z;
    Y[12] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
    dY[12][0] = c3d * (-6 * x * z); dY[12][1] = c3d * (-6 * y * z);
    dY[12][2] = c3d * (6 * z * z - 3 * x * x - 3 * y * y);
    Y[13] = c3c * x * (4 * z * z - x * x - y * y);
    dY[13][0] = c3c * (4 * z * z - 3 * x * x - y * y); dY[13][1] = c3c * (-2 * x * y);
    dY[13][2] = c3c * 8 * x * z;
    Y[14] = c3e * z * (x * x - y * y);
    dY[14][0] = c3e * 2 * x * z; dY[14][1] = -c3e * 2 * y * z; dY[14][2] = c3e * (x * x - y * y);
    Y[15] = c3a * x * (x * x - 3 * y * y);
    dY[15][0] = c3a * (3 * x * x - 3 * y * y); dY[15][1] = c3a * (-6 * x * y);
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* ------------------------------------------------------------------------ */
/* view layout                                                              */
/* ------------------------------------------------------------------------ */

/* Pairs are laid out view-major: view v owns pairs [pair_off[v], pair_off[v] +
 * N_s) for its submap s, in Gaussian order.  Tiles of view v are numbered
 * tile_off[v] + ty*ntx + tx; pixels pix_off[v] + y*W + x. */
typedef struct {
    int64_t pair_off, tile_off, pix_off;
    int64_t g0, ng;
    int32_t ntx, nty;
} oc_view;

static void make_views(int n_views, const oc_camera *cams, const int64_t *sub_off,
                       const oc_config *cfg, oc_view *V) {
    int64_t po = 0, to = 0, xo = 0;
    for (int v = 0; v < n_views; ++v) {
        int s = cams[v].submap;
        V[v].g0 = sub_off[s];
        V[v].ng = sub_off[s + 1] - sub_off[s];
        V[v].pair_off = po;
        V[v].tile_off = to;
        V[v].pix_off = xo;
        V[v].ntx = (cams[v].width + cfg->tile_w - 1) / cfg->tile_w;
        V[v].nty = (cams[v].height + cfg->tile_h - 1) / cfg->tile_h;
        po += V[v].ng;
        to += (int64_t)V[v].ntx * V[v].nty;
        xo += (int64_t)cams[v].width * cams[v].height;
    }
}

int64_t oracle_count_pairs(int n_views, const oc_camera *cams, const int64_t *sub_off) {
    int64_t p = 0;
    for (int v = 0; v < n_views; ++v) p += sub_off[cams[v].submap + 1] - sub_off[cams[v].submap];
    return p;
}

int64_t oracle_count_tiles(int n_views, const oc_camera *cams, const oc_config *cfg) {
    int64_t t = 0;
    for (int v = 0; v < n_views; ++v)
        t += (int64_t)((cams[v].width + cfg->tile_w - 1) / cfg->tile_w) *
             ((cams[v].height + cfg->tile_h - 1) / cfg->tile_h);
    return t;
}

/* ------------------------------------------------------------------------ */
/* 3-D covariance, Eq. (3)                                                   */
/* ------------------------------------------------------------------------ */

/* Sigma = R S S^T R^T with S = diag(exp(log_scale)), R from the normalised
 * quaternion.  Output: full 3x3 row-major. Returns 0 if |q| = 0. */
int oracle_cov3d(const double *quat, const double *log_scale, double *Sigma) {
    double qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    if (!(qn > 0.0)) return 0;
    double qh[4] = {quat[0] / qn, quat[1] / qn, quat[2] / qn, quat[3] / qn};
    double R[9];
    quat_to_rot(qh, R);
    double S2[3] = {exp(2 * log_scale[0]), exp(2 * log_scale[1]), exp(2 * log_scale[2])};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += R[3 * i + k] * S2[k] * R[3 * j + k];
            Sigma[3 * i + j] = s;
        }
    return 1;
}

void oracle_sh_basis(int deg, const double *dir, double *Y) {
    double dY[16][3];
    double Yl[16] = {0};
    sh_basis(deg, dir, Yl, dY);
    int K = (deg + 1) * (deg + 1);
    for (int k = 0; k < K; ++k) Y[k] = Yl[k];
}

/* ------------------------------------------------------------------------ */
/* projection, Eqs. (2)-(4)                                                  */
/* ------------------------------------------------------------------------ */

/* tile index of the first covered pixel for a lower extent argument a:
 * first pixel = ceil(a) clipped to >= 0 */
static int64_t lo_tile(double a, int tw) {
    double p = ceil(a);
    if (p < 0) p = 0;
    return (int64_t)p / tw;
}
static int64_t hi_tile(double a, int W, int tw) {
    double p = floor(a);
    if (p > W - 1) p = W - 1;
    return (int64_t)p / tw;
}

/* R6b: minimum of d^T Q d over the box [x0, x1] x [y0, y1] of offsets d from
 * the mean.  Q is positive definite, so the minimum is 0 when the box holds
 * the mean and otherwise lies on one of the four edges, where q is a convex
 * parabola along the edge minimised at its stationary point clamped to the
 * edge. */
static double box_min_quad(double qa, double qb, double qc, double x0, double x1, double y0, double y1) {
    if (x0 <= 0.0 && 0.0 <= x1 && y0 <= 0.0 && 0.0 <= y1) return 0.0;
    double best = INFINITY;
    double xs[2] = {x0, x1}, ys[2] = {y0, y1};
    for (int i = 0; i < 2; ++i) {
        double x = xs[i], y = dmin(dmax(-qb * x / qc, y0), y1); /* edge dx = x */
        best = dmin(best, qa * x * x + 2.0 * qb * x * y + qc * y * y);
        y = ys[i];
        x = dmin(dmax(-qb * y / qa, x0), x1); /* edge dy = y */
        best = dmin(best, qa * x * x + 2.0 * qb * x * y + qc * y * y);
    }
    return best;
}

/* R6b: minimum of d^T Q d over the pixel centres of tile (tx, ty), clipped
 * to the image, with the box grown by `grow` pixels on every side */
static double tile_min_q(const double *r, int64_t tx, int64_t ty, const oc_camera *cam,
                         const oc_config *cfg, double grow) {
    int64_t X0 = tx * cfg->tile_w, Y0 = ty * cfg->tile_h;
    int64_t X1 = (X0 + cfg->tile_w < cam->width ? X0 + cfg->tile_w : cam->width) - 1;
    int64_t Y1 = (Y0 + cfg->tile_h < cam->height ? Y0 + cfg->tile_h : cam->height) - 1;
    return box_min_quad(r[C_QA], r[C_QB], r[C_QC], (double)X0 + 0.5 - r[C_U] - grow,
                        (double)X1 + 0.5 - r[C_U] + grow, (double)Y0 + 0.5 - r[C_V] - grow,
                        (double)Y1 + 0.5 - r[C_V] + grow);
}

static double tile_threshold(const double *r, const oc_config *cfg) {
    return r[C_E] * (1.0 + cfg->ext_rel_pad) * (1.0 + cfg->ext_rel_pad);
}

static int tile_kept(const double *r, int64_t tx, int64_t ty, const oc_camera *cam, const oc_config *cfg) {
    return tile_min_q(r, tx, ty, cam, cfg, cfg->ext_abs_pad) <= tile_threshold(r, cfg);
}

static void project_pair(const double *mu, const double *ls, const double *q, double omega,
                         const double *sh, int sh_degree, const oc_camera *cam,
                         const oc_config *cfg, double *rec) {
    memset(rec, 0, sizeof(double) * OC_NCOL);
    const double *T = cam->T;
    /* R10: view-space point, fixed summation order */
    double p[3];
    for (int i = 0; i < 3; ++i)
        p[i] = ((T[4 * i + 0] * mu[0] + T[4 * i + 1] * mu[1]) + T[4 * i + 2] * mu[2]) + T[4 * i + 3];
    rec[C_Z] = p[2];
    rec[C_Z32] = (double)(float)p[2];
    if (!(p[2] > cfg->near_z)) return; /* R3 */
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(qn > 0.0)) return; /* R1 */

    /* Eq. (3): Sigma = R S S^T R^T */
    double Sigma[9];
    oracle_cov3d(q, ls, Sigma);
    /* W Sigma W^T with W the rotation of the world->camera transform */
    double Rb[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double RbT[9], tmp[9], Sc[9];
    mat3_transpose(Rb, RbT);
    mat3_mul(Rb, Sigma, tmp);
    mat3_mul(tmp, RbT, Sc);
    /* R4: Jacobian of the pinhole with clamped tangents */
    double W = cam->width, H = cam->height;
    double limx = cfg->jac_clamp * dmax(cam->cx, W - cam->cx) / cam->fx;
    double limy = cfg->jac_clamp * dmax(cam->cy, H - cam->cy) / cam->fy;
    double tx = dmin(dmax(p[0] / p[2], -limx), limx) * p[2];
    double ty = dmin(dmax(p[1] / p[2], -limy), limy) * p[2];
    double J[6] = {cam->fx / p[2], 0.0, -cam->fx * tx / (p[2] * p[2]),
                   0.0, cam->fy / p[2], -cam->fy * ty / (p[2] * p[2])};
    /* Eq. (4): Sigma' = J W Sigma W^T J^T, top-left 2x2, plus dilation */
    double S2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) s += J[3 * i + k] * Sc[3 * k + l] * J[3 * j + l];
            S2[2 * i + j] = s;
        }
    double a = S2[0] + cfg->dilation, b = S2[1], c = S2[3] + cfg->dilation;
    double det = a * c - b * b;
    rec[C_SA] = a; rec[C_SB] = b; rec[C_SC] = c;
    if (!(det > 0.0)) return;
    rec[C_QA] = c / det; rec[C_QB] = -b / det; rec[C_QC] = a / det;
    /* R5: pixel-space mean */
    double u = cam->fx * p[0] / p[2] + cam->cx;
    double v = cam->fy * p[1] / p[2] + cam->cy;
    rec[C_U] = u; rec[C_V] = v;
    /* R8 */
    double o = 1.0 / (1.0 + exp(-omega));
    rec[C_OPA] = o;
    /* R6: support threshold and padded axis-aligned extent */
    double E = 2.0 * log(o / cfg->alpha_min);
    rec[C_E] = E;
    if (!(E > 0.0)) return;
    double ex = sqrt(E * a) * (1.0 + cfg->ext_rel_pad) + cfg->ext_abs_pad;
    double ey = sqrt(E * c) * (1.0 + cfg->ext_rel_pad) + cfg->ext_abs_pad;
    rec[C_EX] = ex; rec[C_EY] = ey;
    double xa = u - ex - 0.5, xb = u + ex - 0.5, ya = v - ey - 0.5, yb = v + ey - 0.5;
    int tw = cfg->tile_w, th = cfg->tile_h;
    int vis = ceil(xa) <= floor(xb) && ceil(xa) <= W - 1 && floor(xb) >= 0 &&
              ceil(ya) <= floor(yb) && ceil(ya) <= H - 1 && floor(yb) >= 0;
    /* ambiguity band: does a small perturbation of the arguments change a
     * tile index or the visibility decision? */
    {
        double epsx = cfg->rect_eps_abs + cfg->rect_eps_rel * ex;
        double epsy = cfg->rect_eps_abs + cfg->rect_eps_rel * ey;
        int amb = 0;
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            double dxa = xa + sgn * epsx, dxb = xb - sgn * epsx;
            double dya = ya + sgn * epsy, dyb = yb - sgn * epsy;
            int vis2 = ceil(dxa) <= floor(dxb) && ceil(dxa) <= W - 1 && floor(dxb) >= 0 &&
                       ceil(dya) <= floor(dyb) && ceil(dya) <= H - 1 && floor(dyb) >= 0;
            if (vis2 != vis) amb = 1;
            if (vis && vis2) {
                if (lo_tile(dxa, tw) != lo_tile(xa, tw) || hi_tile(dxb, cam->width, tw) != hi_tile(xb, cam->width, tw) ||
                    lo_tile(dya, th) != lo_tile(ya, th) || hi_tile(dyb, cam->height, th) != hi_tile(yb, cam->height, th))
                    amb = 1;
            }
        }
        rec[C_RECT_AMBIG] = amb;
    }
    if (!vis) return;
    rec[C_TX0] = (double)lo_tile(xa, tw);
    rec[C_TX1] = (double)hi_tile(xb, cam->width, tw);
    rec[C_TY0] = (double)lo_tile(ya, th);
    rec[C_TY1] = (double)hi_tile(yb, cam->height, th);
    rec[C_VIS] = 1.0;
    /* R6b: kept tiles, and whether a small perturbation of a tile's box (the
     * pixel band of the rectangle decisions) or of the threshold (relative
     * band eta) changes a decision */
    {
        double thr = tile_threshold(rec, cfg);
        double eps = cfg->rect_eps_abs + cfg->rect_eps_rel * (dmax(ex, ey) + dmax(tw, th));
        double eta = cfg->tile_eps_rel + cfg->tile_eps_cond * (a * c + b * b) / det;
        int64_t kept = 0;
        for (int64_t ty = (int64_t)rec[C_TY0]; ty <= (int64_t)rec[C_TY1]; ++ty)
            for (int64_t tx = (int64_t)rec[C_TX0]; tx <= (int64_t)rec[C_TX1]; ++tx) {
                kept += tile_kept(rec, tx, ty, cam, cfg);
                int hi = tile_min_q(rec, tx, ty, cam, cfg, cfg->ext_abs_pad + eps) <= thr * (1.0 + eta);
                int lo = tile_min_q(rec, tx, ty, cam, cfg, cfg->ext_abs_pad - eps) <= thr * (1.0 - eta);
                if (hi != lo) rec[C_RECT_AMBIG] = 1.0;
            }
        rec[C_NTILE] = (double)kept;
    }
    /* R7: view-dependent colour from the camera centre C = -R^T t */
    double Cb[3];
    for (int i = 0; i < 3; ++i) Cb[i] = -(RbT[3 * i + 0] * T[3] + RbT[3 * i + 1] * T[7] + RbT[3 * i + 2] * T[11]);
    double w[3] = {mu[0] - Cb[0], mu[1] - Cb[1], mu[2] - Cb[2]};
    double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double dir[3] = {w[0] / wn, w[1] / wn, w[2] / wn};
    double Y[16], dY[16][3];
    sh_basis(sh_degree, dir, Y, dY);
    int K = (sh_degree + 1) * (sh_degree + 1);
    double margin = 1e300;
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.5;
        for (int k = 0; k < K; ++k) s += sh[3 * k + ch] * Y[k];
        rec[C_R + ch] = s < 0 ? 0.0 : s;
        rec[C_CLR + ch] = s < 0 ? 1.0 : 0.0;
        margin = dmin(margin, fabs(s));
    }
    rec[C_RGB_MARGIN] = margin;
}

/* Project every (view, Gaussian) pair.  Inputs are the float parameters
 * widened to double.  rec: [n_pairs][OC_NCOL]. */
int oracle_project(int64_t n, const double *means, const double *log_scales, const double *quats,
                   const double *opacity_logits, const double *sh, int sh_degree,
                   int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                   const oc_config *cfg, double *rec) {
    (void)n;
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    int K = (sh_degree + 1) * (sh_degree + 1);
    for (int v = 0; v < n_views; ++v) {
#pragma omp parallel for schedule(dynamic, 1024) num_threads(oc_threads)
        for (int64_t k = 0; k < V[v].ng; ++k) {
            int64_t g = V[v].g0 + k;
            double *r = rec + (V[v].pair_off + k) * OC_NCOL;
            project_pair(means + 3 * g, log_scales + 3 * g, quats + 4 * g, opacity_logits[g],
                         sh + (int64_t)3 * K * g, sh_degree, &cams[v], cfg, r);
            r[C_GAUSS] = (double)g;
            r[C_VIEW] = (double)v;
        }
    }
    free(V);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* binning: 64-bit (tile | depth) keys, stable sort, per-tile ranges         */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; int64_t seq; int64_t pair; } oc_inst;

static int inst_cmp(const void *pa, const void *pb) {
    const oc_inst *a = (const oc_inst *)pa, *b = (const oc_inst *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->seq > b->seq) - (a->seq < b->seq); /* stable: emission order */
}

static uint32_t float_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* Count instances: sum over visible pairs of their kept tiles (R6b). */
int64_t oracle_count_instances(int64_t n_pairs, const double *rec) {
    int64_t total = 0;
    for (int64_t p = 0; p < n_pairs; ++p) {
        const double *r = rec + p * OC_NCOL;
        if (r[C_VIS] == 0.0) continue;
        total += (int64_t)r[C_NTILE];
    }
    return total;
}

/* Stable sort of the emitted instances I[0..m) by key, then the keys, the
 * pair of each instance and ranges[2t], ranges[2t+1] = [first, end) of every
 * tile t (0,0 when empty). */
static void sort_and_range(oc_inst *I, int64_t m, int64_t n_tiles, uint64_t *keys_out, int64_t *vals_out,
                           int64_t *ranges) {
    qsort(I, (size_t)m, sizeof(oc_inst), inst_cmp);
    for (int64_t t = 0; t < 2 * n_tiles; ++t) ranges[t] = 0;
    for (int64_t i = 0; i < m; ++i) {
        keys_out[i] = I[i].key;
        vals_out[i] = I[i].pair;
        int64_t t = (int64_t)(I[i].key >> 32);
        if (i == 0 || (I[i - 1].key >> 32) != (uint64_t)t) ranges[2 * t] = i;
        if (i == m - 1 || (I[i + 1].key >> 32) != (uint64_t)t) ranges[2 * t + 1] = i + 1;
    }
}

/* Emit one key per (visible pair, kept tile of its rectangle, R6b) in pair
 * order with the tiles of a rectangle row-major, key = (global tile << 32) |
 * bits(z32); stable sort by key; ranges[2t], ranges[2t+1] = [first, end) of
 * tile t (0,0 when empty). */
int oracle_bin(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
               const oc_config *cfg, const double *rec, uint64_t *keys_out, int64_t *vals_out,
               int64_t *ranges) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    int64_t n_pairs = oracle_count_pairs(n_views, cams, submap_offsets);
    int64_t n_tiles = oracle_count_tiles(n_views, cams, cfg);
    int64_t n_inst = oracle_count_instances(n_pairs, rec);
    oc_inst *I = (oc_inst *)malloc(sizeof(oc_inst) * (n_inst > 0 ? n_inst : 1));
    int64_t m = 0;
    for (int v = 0; v < n_views; ++v)
        for (int64_t k = 0; k < V[v].ng; ++k) {
            int64_t p = V[v].pair_off + k;
            const double *r = rec + p * OC_NCOL;
            if (r[C_VIS] == 0.0) continue;
            uint32_t zb = float_bits((float)r[C_Z32]);
            for (int64_t ty = (int64_t)r[C_TY0]; ty <= (int64_t)r[C_TY1]; ++ty)
                for (int64_t tx = (int64_t)r[C_TX0]; tx <= (int64_t)r[C_TX1]; ++tx) {
                    if (!tile_kept(r, tx, ty, &cams[v], cfg)) continue;
                    uint64_t tile = (uint64_t)(V[v].tile_off + ty * V[v].ntx + tx);
                    I[m].key = (tile << 32) | zb;
                    I[m].seq = m;
                    I[m].pair = p;
                    ++m;
                }
        }
    sort_and_range(I, m, n_tiles, keys_out, vals_out, ranges);
    free(I);
    free(V);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* stage-isolated binning: R6b and the sort from given float32 records      */
/* ------------------------------------------------------------------------ */

/* The binning stage alone, on the projection outputs of the float32 path:
 * per pair the record (U, V, hx, hy | l11, l12, l22, log2 o | r, g, b, z) of
 * 12 floats, the tile rectangle (tx0, ty0, tx1, ty1) as int16 and the depth
 * key (float bits of z, 0xFFFFFFFF for a pair that is not visible).  The pixel
 * mean is u = U + 1/2 - hx, v = V + 1/2 - hy, so that the offset of pixel
 * centre (X + 1/2, Y + 1/2) from it is (X - U + hx, Y - V + hy); L is the
 * upper Cholesky factor [[l11, l12], [0, l22]] of Q log2(e)/2, so that
 * log2 alpha = log2 o - |L d|^2 before the clamp.  R6b keeps a rectangle tile
 * iff min over the box of its pixel-centre offsets (clipped to the image,
 * grown by ext_abs_pad) of |L d|^2 <= (log2 o - log2 alpha_min)(1 +
 * ext_rel_pad)^2.  Here that minimum and that threshold are taken exactly (in
 * double, from the float inputs; products of two floats are exact in double). */

static int rec32_visible(const int16_t *rect, uint32_t pkey) {
    return pkey != 0xFFFFFFFFu && rect[2] >= rect[0] && rect[3] >= rect[1];
}

/* Number of rectangle tiles of the visible pairs (the decisions to take). */
int64_t oracle_rect_tiles32(int64_t n_pairs, const int16_t *rect, const uint32_t *pkey) {
    int64_t total = 0;
    for (int64_t p = 0; p < n_pairs; ++p)
        if (rec32_visible(rect + 4 * p, pkey[p]))
            total += (int64_t)(rect[4 * p + 2] - rect[4 * p] + 1) * (rect[4 * p + 3] - rect[4 * p + 1] + 1);
    return total;
}

/* R6b decision of every rectangle tile of every visible pair, in emission
 * order (pairs in order, each rectangle row-major): dec = 1 keep, 0 drop.
 * margin[i] = (threshold - minimum) / scale, where scale bounds the size of
 * the terms a float32 evaluation of the same test rounds: the threshold's
 * factors and the largest |L d|^2 over the box corners.  A float32 evaluation
 * can take the other decision only where |margin| is a few float ulps. */
int oracle_tile_decisions32(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                            const oc_config *cfg, int64_t n_pairs, const float *rec32, const int16_t *rect,
                            const uint32_t *pkey, int8_t *dec, double *margin) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    double l2amin = log2(cfg->alpha_min);
    double pad = 1.0 + cfg->ext_rel_pad;
    int64_t m = 0;
    for (int v = 0; v < n_views; ++v)
        for (int64_t k = 0; k < V[v].ng; ++k) {
            int64_t p = V[v].pair_off + k;
            if (p >= n_pairs) break;
            const int16_t *rc = rect + 4 * p;
            if (!rec32_visible(rc, pkey[p])) continue;
            const float *r = rec32 + 12 * p;
            double U = r[0], Vv = r[1], hx = r[2], hy = r[3];
            double l11 = r[4], l12 = r[5], l22 = r[6], log2o = r[7];
            /* |L d|^2 = qa dx^2 + 2 qb dx dy + qc dy^2 */
            double qa = l11 * l11, qb = l11 * l12, qc = l12 * l12 + l22 * l22;
            double thr = (log2o - l2amin) * pad * pad;
            for (int64_t ty = rc[1]; ty <= rc[3]; ++ty)
                for (int64_t tx = rc[0]; tx <= rc[2]; ++tx) {
                    int64_t X0 = tx * cfg->tile_w, Y0 = ty * cfg->tile_h;
                    int64_t X1 = (X0 + cfg->tile_w < cams[v].width ? X0 + cfg->tile_w : cams[v].width) - 1;
                    int64_t Y1 = (Y0 + cfg->tile_h < cams[v].height ? Y0 + cfg->tile_h : cams[v].height) - 1;
                    double ax = ((double)X0 - U + hx) - cfg->ext_abs_pad;
                    double bx = ((double)X1 - U + hx) + cfg->ext_abs_pad;
                    double ay = ((double)Y0 - Vv + hy) - cfg->ext_abs_pad;
                    double by = ((double)Y1 - Vv + hy) + cfg->ext_abs_pad;
                    double mq = box_min_quad(qa, qb, qc, ax, bx, ay, by);
                    double big = 0.0;
                    for (int c = 0; c < 4; ++c) {
                        double x = (c & 1) ? bx : ax, y = (c & 2) ? by : ay;
                        double t1 = fabs(l11 * x) + fabs(l12 * y), t2 = fabs(l22 * y);
                        big = dmax(big, t1 * t1 + t2 * t2);
                    }
                    double scale = big + (fabs(log2o) + fabs(l2amin)) * pad * pad;
                    dec[m] = mq <= thr;
                    margin[m] = (thr - mq) / scale;
                    ++m;
                }
        }
    free(V);
    return 0;
}

/* Instances, keys and ranges from the float32 path's projection outputs and
 * one decision per rectangle tile (emission order, as oracle_tile_decisions32
 * writes them): key = (global tile << 32) | pkey, stable sort by key,
 * per-tile [first, end).  Returns the number of instances. */
int64_t oracle_bin_decided(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                           const oc_config *cfg, int64_t n_pairs, const int16_t *rect, const uint32_t *pkey,
                           const int8_t *dec, uint64_t *keys_out, int64_t *vals_out, int64_t *ranges) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    int64_t n_tiles = oracle_count_tiles(n_views, cams, cfg);
    int64_t n_dec = oracle_rect_tiles32(n_pairs, rect, pkey);
    oc_inst *I = (oc_inst *)malloc(sizeof(oc_inst) * (n_dec > 0 ? n_dec : 1));
    int64_t m = 0, d = 0;
    for (int v = 0; v < n_views; ++v)
        for (int64_t k = 0; k < V[v].ng; ++k) {
            int64_t p = V[v].pair_off + k;
            if (p >= n_pairs) break;
            const int16_t *rc = rect + 4 * p;
            if (!rec32_visible(rc, pkey[p])) continue;
            for (int64_t ty = rc[1]; ty <= rc[3]; ++ty)
                for (int64_t tx = rc[0]; tx <= rc[2]; ++tx) {
                    if (dec[d++]) {
                        uint64_t tile = (uint64_t)(V[v].tile_off + ty * V[v].ntx + tx);
                        I[m].key = (tile << 32) | pkey[p];
                        I[m].seq = m;
                        I[m].pair = p;
                        ++m;
                    }
                }
        }
    sort_and_range(I, m, n_tiles, keys_out, vals_out, ranges);
    free(I);
    free(V);
    return m;
}

/* ------------------------------------------------------------------------ */
/* forward compositing                                                      */
/* ------------------------------------------------------------------------ */

/* alpha of pair record r at pixel centre (px, py); *raw gets o*exp(pw) */
static double frag_alpha(const double *r, double px, double py, const oc_config *cfg, double *raw) {
    double dx = px - r[C_U], dy = py - r[C_V];
    double pw = -0.5 * (r[C_QA] * dx * dx + 2.0 * r[C_QB] * dx * dy + r[C_QC] * dy * dy);
    double al = r[C_OPA] * exp(pw);
    *raw = al;
    return dmin(cfg->alpha_max, al);
}

typedef struct {
    double C[3], D, T, mean, var;
    int64_t last;    /* list position of the last blended fragment, -1 if none */
    int64_t n_blend; /* number of blended fragments */
    double margin;   /* min log-distance of a discrete decision to its threshold */
    double clamp_margin;
    uint64_t sig;    /* order-sensitive signature of the blended set */
} oc_pix;

/* Composite the candidate pairs cand[0..n) (already in compositing order) at
 * pixel centre (px, py).  pos[i] is the list position reported as `last`. */
static void composite(const double *rec, const int64_t *cand, const int64_t *pos, int64_t n,
                      double px, double py, const oc_config *cfg, oc_pix *out) {
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0, margin = 1e300, cm = 1e300;
    double *wz = (double *)malloc(sizeof(double) * 2 * (n > 0 ? n : 1)); /* blended (w, z) */
    int64_t last = -1, nb = 0;
    uint64_t sig = 1469598103934665603ull;
    double lmin = log(cfg->alpha_min), ltmin = log(cfg->t_min), lmax = log(cfg->alpha_max);
    for (int64_t i = 0; i < n; ++i) {
        const double *r = rec + cand[i] * OC_NCOL;
        double raw, al = frag_alpha(r, px, py, cfg, &raw);
        if (raw > 0) {
            margin = dmin(margin, fabs(log(raw) - lmin));
            cm = dmin(cm, fabs(log(raw) - lmax));
        }
        if (al < cfg->alpha_min) continue;
        double Tn = T * (1.0 - al);
        margin = dmin(margin, fabs(log(Tn) - ltmin));
        if (Tn < cfg->t_min) break; /* stop before blending this fragment */
        double w = al * T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += w * r[C_R + ch];
        D += w * r[C_Z];
        wz[2 * nb] = w;
        wz[2 * nb + 1] = r[C_Z];
        T = Tn;
        last = pos[i];
        ++nb;
        sig = (sig ^ (uint64_t)cand[i]) * 1099511628211ull;
    }
    /* R16: mean and variance of the blended depths, by definition */
    double W = 0.0, M2 = 0.0;
    for (int64_t k = 0; k < nb; ++k) W += wz[2 * k];
    double mu = nb > 0 ? D / W : 0.0;
    for (int64_t k = 0; k < nb; ++k) M2 += wz[2 * k] * (wz[2 * k + 1] - mu) * (wz[2 * k + 1] - mu);
    free(wz);
    memcpy(out->C, C, sizeof C);
    out->D = D; out->T = T; out->mean = mu; out->var = nb > 0 ? M2 / W : 0.0;
    out->last = last; out->n_blend = nb;
    out->margin = margin; out->clamp_margin = cm; out->sig = sig;
}

static void write_pix(const oc_pix *o, int64_t pix, int64_t W, int64_t H, int64_t pix_off,
                      double *rgb, double *depth, double *alpha, double *Tfin, int64_t *last,
                      int64_t *nblend, double *margin, uint64_t *sig) {
    int64_t local = pix - pix_off;
    for (int ch = 0; ch < 3; ++ch) rgb[3 * pix_off + ch * W * H + local] = o->C[ch];
    depth[pix] = o->D;
    alpha[pix] = 1.0 - o->T;
    if (Tfin) Tfin[pix] = o->T;
    if (last) last[pix] = o->last;
    if (nblend) nblend[pix] = o->n_blend;
    if (margin) margin[pix] = o->margin;
    if (sig) sig[pix] = o->sig;
}

/* Tiled forward: every pixel walks the sorted list of its tile.
 * rgb is planar per view: view v occupies [3*pix_off, 3*pix_off + 3*W*H).
 * last holds the list position of the last blended fragment (-1 if none). */
int oracle_render_fwd(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                      const oc_config *cfg, const double *rec, const int64_t *vals,
                      const int64_t *ranges, double *rgb, double *depth, double *alpha,
                      double *Tfin, int64_t *last, int64_t *nblend, double *margin, uint64_t *sig) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    for (int v = 0; v < n_views; ++v) {
        int64_t W = cams[v].width, H = cams[v].height;
#pragma omp parallel for schedule(dynamic, 1) num_threads(oc_threads)
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                int64_t t = V[v].tile_off + (y / cfg->tile_h) * V[v].ntx + x / cfg->tile_w;
                int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
                int64_t n = e - s;
                int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
                for (int64_t i = 0; i < n; ++i) pos[i] = s + i;
                oc_pix o;
                composite(rec, vals + s, pos, n, x + 0.5, y + 0.5, cfg, &o);
                free(pos);
                write_pix(&o, V[v].pix_off + y * W + x, W, H, V[v].pix_off, rgb, depth, alpha,
                          Tfin, last, nblend, margin, sig);
            }
    }
    free(V);
    return 0;
}

/* Mean and variance of the blended depths per pixel (R16). */
int oracle_render_depth_dist(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                             const oc_config *cfg, const double *rec, const int64_t *vals,
                             const int64_t *ranges, double *mean, double *var) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    for (int v = 0; v < n_views; ++v) {
        int64_t W = cams[v].width, H = cams[v].height;
#pragma omp parallel for schedule(dynamic, 1) num_threads(oc_threads)
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                int64_t t = V[v].tile_off + (y / cfg->tile_h) * V[v].ntx + x / cfg->tile_w;
                int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
                int64_t n = e - s;
                int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
                for (int64_t i = 0; i < n; ++i) pos[i] = s + i;
                oc_pix o;
                composite(rec, vals + s, pos, n, x + 0.5, y + 0.5, cfg, &o);
                free(pos);
                mean[V[v].pix_off + y * W + x] = o.mean;
                var[V[v].pix_off + y * W + x] = o.var;
            }
    }
    free(V);
    return 0;
}

/* Tiled forward for a list of pixels only (global pixel indices), for
 * sampled checks of full-size images; outputs are per listed pixel:
 * rgb [n_sel][3], depth, alpha, T, last, margin. */
int oracle_render_fwd_pixels(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                             const oc_config *cfg, const double *rec, const int64_t *vals,
                             const int64_t *ranges, int64_t n_sel, const int64_t *pix,
                             double *rgb, double *depth, double *alpha, double *Tfin,
                             int64_t *last, double *margin) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
#pragma omp parallel for schedule(dynamic, 64) num_threads(oc_threads)
    for (int64_t k = 0; k < n_sel; ++k) {
        int v = 0;
        while (v + 1 < n_views && V[v + 1].pix_off <= pix[k]) ++v;
        int64_t W = cams[v].width;
        int64_t local = pix[k] - V[v].pix_off;
        int64_t y = local / W, x = local % W;
        int64_t t = V[v].tile_off + (y / cfg->tile_h) * V[v].ntx + x / cfg->tile_w;
        int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
        int64_t n = e - s;
        int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) pos[i] = s + i;
        oc_pix o;
        composite(rec, vals + s, pos, n, x + 0.5, y + 0.5, cfg, &o);
        free(pos);
        for (int ch = 0; ch < 3; ++ch) rgb[3 * k + ch] = o.C[ch];
        depth[k] = o.D;
        alpha[k] = 1.0 - o.T;
        Tfin[k] = o.T;
        last[k] = o.last;
        margin[k] = o.margin;
    }
    free(V);
    return 0;
}

/* Brute-force forward without tiles: every pixel composites all visible pairs
 * of its view in ascending (z32, Gaussian index) order; membership is decided
 * by alpha alone.  `last` here is the index into that per-view order. */
typedef struct { double z32; int64_t g; int64_t pair; } oc_zs;
static int zs_cmp(const void *pa, const void *pb) {
    const oc_zs *a = (const oc_zs *)pa, *b = (const oc_zs *)pb;
    if (a->z32 != b->z32) return a->z32 < b->z32 ? -1 : 1;
    return (a->g > b->g) - (a->g < b->g);
}

int oracle_render_brute(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                        const oc_config *cfg, const double *rec, double *rgb, double *depth,
                        double *alpha, double *Tfin, int64_t *nblend, uint64_t *sig) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    for (int v = 0; v < n_views; ++v) {
        int64_t W = cams[v].width, H = cams[v].height;
        oc_zs *Z = (oc_zs *)malloc(sizeof(oc_zs) * (V[v].ng > 0 ? V[v].ng : 1));
        int64_t n = 0;
        for (int64_t k = 0; k < V[v].ng; ++k) {
            int64_t p = V[v].pair_off + k;
            const double *r = rec + p * OC_NCOL;
            /* every projected pair in front of the camera is a candidate; the
             * rectangle is not consulted */
            if (!(r[C_Z] > cfg->near_z) || !(r[C_E] > 0.0) || r[C_QA] == 0.0) continue;
            Z[n].z32 = r[C_Z32]; Z[n].g = (int64_t)r[C_GAUSS]; Z[n].pair = p; ++n;
        }
        qsort(Z, (size_t)n, sizeof(oc_zs), zs_cmp);
        int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
        int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) { cand[i] = Z[i].pair; pos[i] = i; }
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                oc_pix o;
                composite(rec, cand, pos, n, x + 0.5, y + 0.5, cfg, &o);
                write_pix(&o, V[v].pix_off + y * W + x, W, H, V[v].pix_off, rgb, depth, alpha,
                          Tfin, NULL, nblend, NULL, sig);
            }
        free(cand); free(pos); free(Z);
    }
    free(V);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* losses, Eqs. (6)-(7)                                                      */
/* ------------------------------------------------------------------------ */

/* R13: L = mean |C - I| over n values; dL/dC = sign(C - I)/n (sign(0) = 0). */
double oracle_image_l1(int64_t n, const double *C, const double *I, double *grad) {
    double s = 0;
    for (int64_t i = 0; i < n; ++i) {
        double d = C[i] - I[i];
        s += fabs(d);
        if (grad) grad[i] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)n;
    }
    return n > 0 ? s / (double)n : 0.0;
}

/* R17: the normalised 11-tap Gaussian window, sigma 1.5 */
#define OC_SSIM_R 5
static void ssim_window(double g[2 * OC_SSIM_R + 1]) {
    double s = 0.0;
    for (int i = -OC_SSIM_R; i <= OC_SSIM_R; ++i) {
        g[i + OC_SSIM_R] = exp(-(double)(i * i) / (2.0 * 1.5 * 1.5));
        s += g[i + OC_SSIM_R];
    }
    for (int i = 0; i < 2 * OC_SSIM_R + 1; ++i) g[i] /= s;
}

/* Mean SSIM (R17) of planar images rgb against target, views laid out as in
 * the renderer's outputs.  grad (nullable) receives d(mean SSIM)/d rgb.
 * Each pixel q takes window sums of x, y, x^2, y^2, xy over its 11x11
 * neighbourhood (zero outside the image):
 *   mu_x, mu_y, s_xx = E[x^2] - mu_x^2, s_yy, s_xy = E[xy] - mu_x mu_y,
 *   S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)).
 * Adjoint: S depends on x only through m1 = E[x], m2 = E[x^2] and m12 = E[xy];
 * with A = 2 mu_x mu_y + C1, B = 2 s_xy + C2, Cc = mu_x^2 + mu_y^2 + C1,
 * D = s_xx + s_yy + C2:
 *   dS/dmu_x (s fixed) = (B/D) (2 mu_y Cc - 2 mu_x A) / Cc^2,
 *   dS/ds_xx = -A B / (Cc D^2),   dS/ds_xy = 2 A / (Cc D),
 *   dS/dm1 = dS/dmu_x - 2 mu_x dS/ds_xx - mu_y dS/ds_xy,
 *   dS/dm2 = dS/ds_xx,  dS/dm12 = dS/ds_xy,
 * and x_p enters m1, m2, m12 of every q whose window holds p with weight
 * g(p - q): d/dx_p = g (dS/dm1 + 2 x_p dS/dm2 + y_p dS/dm12). */
double oracle_ssim(int n_views, const oc_camera *cams, const double *rgb, const double *target,
                   double *grad) {
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double g[2 * OC_SSIM_R + 1];
    ssim_window(g);
    int64_t n_all = 0;
    for (int v = 0; v < n_views; ++v) n_all += 3 * (int64_t)cams[v].width * cams[v].height;
    if (grad)
        for (int64_t i = 0; i < n_all; ++i) grad[i] = 0.0;
    double total = 0.0;
    int64_t off = 0;
    for (int v = 0; v < n_views; ++v) {
        const int W = cams[v].width, H = cams[v].height;
        for (int ch = 0; ch < 3; ++ch, off += (int64_t)W * H) {
            const double *x = rgb + off, *y = target + off;
            for (int qy = 0; qy < H; ++qy)
                for (int qx = 0; qx < W; ++qx) {
                    double mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
                    for (int j = -OC_SSIM_R; j <= OC_SSIM_R; ++j)
                        for (int i = -OC_SSIM_R; i <= OC_SSIM_R; ++i) {
                            int px = qx + i, py = qy + j;
                            if (px < 0 || px >= W || py < 0 || py >= H) continue;
                            double w = g[i + OC_SSIM_R] * g[j + OC_SSIM_R];
                            double a = x[(int64_t)py * W + px], b = y[(int64_t)py * W + px];
                            mx += w * a; my += w * b;
                            exx += w * a * a; eyy += w * b * b; exy += w * a * b;
                        }
                    double sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
                    double A = 2.0 * mx * my + C1, B = 2.0 * sxy + C2;
                    double Cc = mx * mx + my * my + C1, D = sxx + syy + C2;
                    total += A * B / (Cc * D);
                    if (!grad) continue;
                    double dmu = (B / D) * (2.0 * my * Cc - 2.0 * mx * A) / (Cc * Cc);
                    double dsxx = -A * B / (Cc * D * D);
                    double dsxy = 2.0 * A / (Cc * D);
                    double d1 = dmu - 2.0 * mx * dsxx - my * dsxy, d2 = dsxx, d12 = dsxy;
                    for (int j = -OC_SSIM_R; j <= OC_SSIM_R; ++j)
                        for (int i = -OC_SSIM_R; i <= OC_SSIM_R; ++i) {
                            int px = qx + i, py = qy + j;
                            if (px < 0 || px >= W || py < 0 || py >= H) continue;
                            double w = g[i + OC_SSIM_R] * g[j + OC_SSIM_R];
                            int64_t p = (int64_t)py * W + px;
                            grad[off + p] += w * (d1 + 2.0 * x[p] * d2 + y[p] * d12);
                        }
                }
        }
    }
    if (n_all == 0) return 0.0;
    if (grad)
        for (int64_t i = 0; i < n_all; ++i) grad[i] /= (double)n_all;
    return total / (double)n_all;
}

/* KL(N(m1, s1^2) || N(m2, s2^2)) */
double oracle_kl_normal(double m1, double s1, double m2, double s2) {
    return log(s2 / s1) + (s1 * s1 + (m1 - m2) * (m1 - m2)) / (2.0 * s2 * s2) - 0.5;
}

/* R12 / Eq. (7).  lidar rows (u, v, z, view).  mode 0: mean |D - z|;
 * mode 1: mean KL(N(z, sigma_L^2) || N(D, sigma_U^2)); scaled by lambda.
 * grad (nullable) receives dL/dD per pixel (accumulated over points). */
double oracle_depth_loss(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                         const oc_config *cfg, const double *depth, const double *alpha,
                         int64_t n_pts, const double *lidar, int mode, double sigma_L,
                         double sigma_U, double lambda, double *grad, int64_t *n_valid) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    double s = 0;
    int64_t nv = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t i = 0; i < n_pts; ++i) {
            const double *L = lidar + 4 * i;
            int v = (int)L[3];
            if (v < 0 || v >= n_views) continue;
            double W = cams[v].width, H = cams[v].height;
            if (!(L[0] >= 0 && L[0] < W && L[1] >= 0 && L[1] < H && L[2] > cfg->near_z)) continue;
            int64_t pix = V[v].pix_off + (int64_t)floor(L[1]) * cams[v].width + (int64_t)floor(L[0]);
            if (!(alpha[pix] > 0)) continue;
            double Dh = depth[pix], z = L[2];
            if (pass == 0) {
                ++nv;
                s += mode == 0 ? fabs(Dh - z) : oracle_kl_normal(z, sigma_L, Dh, sigma_U);
            } else if (grad) {
                double g = mode == 0 ? (Dh > z ? 1.0 : (Dh < z ? -1.0 : 0.0))
                                     : (Dh - z) / (sigma_U * sigma_U);
                grad[pix] += lambda * g / (double)nv;
            }
        }
        if (nv == 0) break;
    }
    free(V);
    if (n_valid) *n_valid = nv;
    return nv > 0 ? lambda * s / (double)nv : 0.0;
}

/* Eq. (7) with the renderer's predicted distribution (R16):
 * sigma_u^2 = max(var, 0) + sigma_U^2; mean over valid points (R12) of
 * KL(N(z, sigma_L^2) || N(mean, sigma_u^2)) times lambda.  Gradients (each
 * accumulated per pixel, nullable) w.r.t. mean and var. */
double oracle_depth_loss_var(int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                             const oc_config *cfg, const double *alpha, const double *mean,
                             const double *var_in, int64_t n_pts, const double *lidar, double sigma_L,
                             double sigma_U, double lambda, double *gmean, double *gvar,
                             int64_t *n_valid) {
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    double s = 0;
    int64_t nv = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t i = 0; i < n_pts; ++i) {
            const double *L = lidar + 4 * i;
            int v = (int)L[3];
            if (v < 0 || v >= n_views) continue;
            double W = cams[v].width, H = cams[v].height;
            if (!(L[0] >= 0 && L[0] < W && L[1] >= 0 && L[1] < H && L[2] > cfg->near_z)) continue;
            int64_t pix = V[v].pix_off + (int64_t)floor(L[1]) * cams[v].width + (int64_t)floor(L[0]);
            double A = alpha[pix];
            if (!(A > 0)) continue;
            double z = L[2];
            double mu = mean[pix];
            double var = var_in[pix];
            int clamped = var < 0;
            double su2 = (clamped ? 0.0 : var) + sigma_U * sigma_U;
            double e = mu - z;
            if (pass == 0) {
                ++nv;
                s += 0.5 * log(su2) - log(sigma_L) + (sigma_L * sigma_L + e * e) / (2.0 * su2) - 0.5;
            } else {
                double k = lambda / (double)nv;
                double dmu = e / su2;                                                  /* dKL/dmu */
                double dv = clamped ? 0.0 : 0.5 / su2 - (sigma_L * sigma_L + e * e) / (2.0 * su2 * su2);
                if (gmean) gmean[pix] += k * dmu;
                if (gvar) gvar[pix] += k * dv;
            }
        }
        if (nv == 0) break;
    }
    free(V);
    if (n_valid) *n_valid = nv;
    return nv > 0 ? lambda * s / (double)nv : 0.0;
}

/* ------------------------------------------------------------------------ */
/* backward                                                                 */
/* ------------------------------------------------------------------------ */

/* Raster adjoint for one pixel: replay the forward to list the blended
 * fragments with their alpha and transmittance, then apply
 *   dL/dc_j = w_j gC, dL/dz_j = w_j gD,
 *   dL/dalpha_j = T_j h_j - (sum_{k>j} w_k h_k) / (1 - alpha_j),
 * with w_k = alpha_k T_k and h_k = gC.c_k + gD z_k + gA (A = sum_k w_k). */
static void pixel_adjoint(const double *rec, const int64_t *cand, int64_t n, double px, double py,
                          const oc_config *cfg, const double gC[3], double gD, double gA,
                          double gmean, double gvar, double *g2d) {
    int64_t *bl = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    double *al = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *raw = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *Tb = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    int64_t m = 0;
    double T = 1.0;
    for (int64_t i = 0; i < n; ++i) {
        const double *r = rec + cand[i] * OC_NCOL;
        double rw, a = frag_alpha(r, px, py, cfg, &rw);
        if (a < cfg->alpha_min) continue;
        double Tn = T * (1.0 - a);
        if (Tn < cfg->t_min) break;
        bl[m] = cand[i]; al[m] = a; raw[m] = rw; Tb[m] = T; ++m;
        T = Tn;
    }
    /* R16: mu = sum w z / W, W = sum w, var = M2 / W, M2 = sum w (z - mu)^2.
     * dmu/dw_k = (z_k - mu)/W, dmu/dz_k = w_k/W; with R = sum w (z - mu),
     *   dM2/dw_k = (z_k - mu)^2 - 2 R dmu/dw_k,  dM2/dz_k = 2 w_k (z_k - mu) - 2 R dmu/dz_k,
     *   dvar/dw_k = dM2/dw_k / W - M2/W^2,       dvar/dz_k = dM2/dz_k / W. */
    double W = 0.0, Dz = 0.0, R = 0.0, M2 = 0.0;
    for (int64_t j = 0; j < m; ++j) {
        W += al[j] * Tb[j];
        Dz += al[j] * Tb[j] * rec[bl[j] * OC_NCOL + C_Z];
    }
    double mu = m > 0 ? Dz / W : 0.0;
    for (int64_t j = 0; j < m; ++j) {
        double e = rec[bl[j] * OC_NCOL + C_Z] - mu;
        R += al[j] * Tb[j] * e;
        M2 += al[j] * Tb[j] * e * e;
    }
    double suffix = 0.0;
    for (int64_t j = m - 1; j >= 0; --j) {
        const double *r = rec + bl[j] * OC_NCOL;
        double *g = g2d + bl[j] * OC_NGRAD;
        double w = al[j] * Tb[j];
        double dz = r[C_Z] - mu;
        double dmu_dw = dz / W, dmu_dz = w / W;
        double dvar_dw = (dz * dz - 2.0 * R * dmu_dw) / W - M2 / (W * W);
        double dvar_dz = (2.0 * w * dz - 2.0 * R * dmu_dz) / W;
        /* h = dL/dw_j through C, D, A = sum w, mu and var */
        double h = gC[0] * r[C_R] + gC[1] * r[C_G] + gC[2] * r[C_B] + gD * r[C_Z] + gA +
                   gmean * dmu_dw + gvar * dvar_dw;
        double dal = Tb[j] * h - suffix / (1.0 - al[j]);
        suffix += w * h;
        acc_add(&g[G_R], w * gC[0]); acc_add(&g[G_G], w * gC[1]); acc_add(&g[G_B], w * gC[2]);
        acc_add(&g[G_Z], w * gD + gmean * dmu_dz + gvar * dvar_dz);
        if (raw[j] > cfg->alpha_max) continue; /* clamped: no dependence on o, pw */
        /* alpha = o exp(pw): dalpha/dln(o) = alpha, dalpha/dpw = alpha */
        double gpw = dal * al[j];
        acc_add(&g[G_LNO], gpw);
        double dx = px - r[C_U], dy = py - r[C_V];
        /* pw = -1/2 (qa dx^2 + 2 qb dx dy + qc dy^2), d = pixel - mean */
        acc_add(&g[G_QA], -0.5 * gpw * dx * dx);
        acc_add(&g[G_QB], -gpw * dx * dy);
        acc_add(&g[G_QC], -0.5 * gpw * dy * dy);
        acc_add(&g[G_U], gpw * (r[C_QA] * dx + r[C_QB] * dy));
        acc_add(&g[G_V], gpw * (r[C_QB] * dx + r[C_QC] * dy));
    }
    free(bl); free(al); free(raw); free(Tb);
}

/* Projection adjoint for one visible pair: from the image-space gradient g to
 * the Gaussian parameters (accumulated) and the pose twist of the view. */
static void project_adjoint(const double *mu, const double *ls, const double *q, double omega,
                            const double *sh, int sh_degree, const oc_camera *cam,
                            const oc_config *cfg, const double *rec, const double *g,
                            double *g_mu, double *g_ls, double *g_q, double *g_om, double *g_sh,
                            double *g_pose) {
    (void)omega; /* the opacity enters through rec[C_OPA] */
    const double *T = cam->T;
    double p[3];
    for (int i = 0; i < 3; ++i)
        p[i] = ((T[4 * i + 0] * mu[0] + T[4 * i + 1] * mu[1]) + T[4 * i + 2] * mu[2]) + T[4 * i + 3];
    double Rb[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double RbT[9];
    mat3_transpose(Rb, RbT);
    double fx = cam->fx, fy = cam->fy;
    double gp[3] = {0, 0, 0};   /* dL/dp, p the view-space mean */
    double gw[3] = {0, 0, 0};   /* dL/dw, w = mu - C the SH viewing vector */

    /* colour: rgb_c = max(0.5 + sum_k sh_kc Y_k(dir), 0), dir = w/|w| */
    double Cb[3];
    for (int i = 0; i < 3; ++i) Cb[i] = -(RbT[3 * i + 0] * T[3] + RbT[3 * i + 1] * T[7] + RbT[3 * i + 2] * T[11]);
    double w[3] = {mu[0] - Cb[0], mu[1] - Cb[1], mu[2] - Cb[2]};
    double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double dir[3] = {w[0] / wn, w[1] / wn, w[2] / wn};
    double Y[16], dY[16][3];
    sh_basis(sh_degree, dir, Y, dY);
    int K = (sh_degree + 1) * (sh_degree + 1);
    double gdir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
        if (rec[C_CLR + ch] != 0.0) continue;
        double gc = g[G_R + ch];
        for (int k = 0; k < K; ++k) {
            g_sh[3 * k + ch] += gc * Y[k];
            for (int i = 0; i < 3; ++i) gdir[i] += gc * sh[3 * k + ch] * dY[k][i];
        }
    }
    /* dir = w/|w|: dL/dw = (I - dir dir^T) gdir / |w| */
    double dd = dir[0] * gdir[0] + dir[1] * gdir[1] + dir[2] * gdir[2];
    for (int i = 0; i < 3; ++i) gw[i] = (gdir[i] - dir[i] * dd) / wn;

    /* depth output: z = p_z */
    gp[2] += g[G_Z];
    /* pixel mean: u = fx p_x/p_z + cx, v = fy p_y/p_z + cy */
    gp[0] += g[G_U] * fx / p[2];
    gp[1] += g[G_V] * fy / p[2];
    gp[2] += -(g[G_U] * fx * p[0] + g[G_V] * fy * p[1]) / (p[2] * p[2]);

    /* conic Q = Sigma'^-1: with G the symmetric matrix of dL/dQ (off-diagonal
     * halved, since qb appears twice), dL/dSigma' = -Q G Q */
    double Q[4] = {rec[C_QA], rec[C_QB], rec[C_QB], rec[C_QC]};
    double G[4] = {g[G_QA], 0.5 * g[G_QB], 0.5 * g[G_QB], g[G_QC]};
    double QG[4], M[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) QG[2 * i + j] = Q[2 * i] * G[j] + Q[2 * i + 1] * G[2 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) M[2 * i + j] = -(QG[2 * i] * Q[j] + QG[2 * i + 1] * Q[2 + j]);
    /* M is dL/dSigma' as a symmetric matrix (full-matrix convention) */

    /* Sigma' = J Sc J^T + dil I with Sc = Rb Sigma Rb^T */
    double Sigma[9], tmp[9], Sc[9];
    oracle_cov3d(q, ls, Sigma);
    mat3_mul(Rb, Sigma, tmp);
    mat3_mul(tmp, RbT, Sc);
    double W = cam->width, H = cam->height;
    double limx = cfg->jac_clamp * dmax(cam->cx, W - cam->cx) / fx;
    double limy = cfg->jac_clamp * dmax(cam->cy, H - cam->cy) / fy;
    double xr = p[0] / p[2], yr = p[1] / p[2];
    int clx = xr < -limx || xr > limx, cly = yr < -limy || yr > limy;
    double tx = dmin(dmax(xr, -limx), limx) * p[2];
    double ty = dmin(dmax(yr, -limy), limy) * p[2];
    double J[6] = {fx / p[2], 0.0, -fx * tx / (p[2] * p[2]),
                   0.0, fy / p[2], -fy * ty / (p[2] * p[2])};
    /* dL/dSc = J^T M J ; dL/dJ = 2 M J Sc */
    double gSc[9];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double s = 0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) s += J[3 * i + k] * M[2 * i + j] * J[3 * j + l];
            gSc[3 * k + l] = s;
        }
    double gJ[6];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            double s = 0;
            for (int j = 0; j < 2; ++j)
                for (int l = 0; l < 3; ++l) s += M[2 * i + j] * J[3 * j + l] * Sc[3 * l + k];
            gJ[3 * i + k] = 2.0 * s;
        }
    /* J entries as functions of p (clamped tangent: tx = c*p_z, J02 = -fx c/p_z) */
    double z2 = p[2] * p[2], z3 = z2 * p[2];
    gp[2] += gJ[0] * (-fx / z2) + gJ[4] * (-fy / z2);
    if (!clx) {
        gp[0] += gJ[2] * (-fx / z2);
        gp[2] += gJ[2] * (2.0 * fx * p[0] / z3);
    } else {
        double cx_ = tx / p[2];
        gp[2] += gJ[2] * (fx * cx_ / z2);
    }
    if (!cly) {
        gp[1] += gJ[5] * (-fy / z2);
        gp[2] += gJ[5] * (2.0 * fy * p[1] / z3);
    } else {
        double cy_ = ty / p[2];
        gp[2] += gJ[5] * (fy * cy_ / z2);
    }

    /* Sc = Rb Sigma Rb^T: dL/dSigma = Rb^T gSc Rb */
    double gSig[9], t2[9];
    mat3_mul(RbT, gSc, t2);
    mat3_mul(t2, Rb, gSig);
    /* Sigma = R diag(S^2) R^T = M3 M3^T with M3 = R diag(S): dL/dM3 = (G + G^T) M3 */
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qh[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
    double R[9];
    quat_to_rot(qh, R);
    double S[3] = {exp(ls[0]), exp(ls[1]), exp(ls[2])};
    double gM3[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double s = 0;
            for (int j = 0; j < 3; ++j) s += (gSig[3 * i + j] + gSig[3 * j + i]) * R[3 * j + k] * S[k];
            gM3[3 * i + k] = s;
        }
    /* M3_ik = R_ik S_k with S_k = exp(ls_k): dL/dls_k = sum_i gM3_ik R_ik S_k */
    double gR[9];
    for (int k = 0; k < 3; ++k) {
        double s = 0;
        for (int i = 0; i < 3; ++i) {
            s += gM3[3 * i + k] * R[3 * i + k];
            gR[3 * i + k] = gM3[3 * i + k] * S[k];
        }
        g_ls[k] += s * S[k];
    }
    /* R from the normalised quaternion, then the normalisation */
    double dR[4][9];
    quat_to_rot_jac(qh, dR);
    double gqh[4];
    for (int a = 0; a < 4; ++a) {
        double s = 0;
        for (int e = 0; e < 9; ++e) s += gR[e] * dR[a][e];
        gqh[a] = s;
    }
    double dq = qh[0] * gqh[0] + qh[1] * gqh[1] + qh[2] * gqh[2] + qh[3] * gqh[3];
    for (int a = 0; a < 4; ++a) g_q[a] += (gqh[a] - qh[a] * dq) / qn;

    /* opacity: ln o = -ln(1 + e^-omega), d ln o / d omega = 1 - o */
    *g_om += g[G_LNO] * (1.0 - rec[C_OPA]);

    /* mean: p = Rb mu + t and w = mu - C */
    for (int i = 0; i < 3; ++i)
        g_mu[i] += RbT[3 * i + 0] * gp[0] + RbT[3 * i + 1] * gp[1] + RbT[3 * i + 2] * gp[2] + gw[i];

    /* pose, left perturbation (R11): p -> p + rho + phi x p, Rb -> (I + [phi]x) Rb,
     * w -> w + Rb^T rho.  dL/drho = gp + Rb gw; dL/dphi = p x gp + cov term. */
    double gw_c[3];
    for (int i = 0; i < 3; ++i) gw_c[i] = Rb[3 * i + 0] * gw[0] + Rb[3 * i + 1] * gw[1] + Rb[3 * i + 2] * gw[2];
    g_pose[0] += gp[0] + gw_c[0];
    g_pose[1] += gp[1] + gw_c[1];
    g_pose[2] += gp[2] + gw_c[2];
    g_pose[3] += p[1] * gp[2] - p[2] * gp[1];
    g_pose[4] += p[2] * gp[0] - p[0] * gp[2];
    g_pose[5] += p[0] * gp[1] - p[1] * gp[0];
    /* Sc -> Sc + [phi]x Sc - Sc [phi]x: dL/dphi = 2 * axial(A - A^T)/..., A = Sc gSc */
    double A[9];
    mat3_mul(Sc, gSc, A);
    g_pose[3] += 2.0 * (A[5] - A[7]);
    g_pose[4] += 2.0 * (A[6] - A[2]);
    g_pose[5] += 2.0 * (A[1] - A[3]);
}

/* Full backward: raster adjoint for every pixel (using the oracle's own sorted
 * lists), then the projection adjoint of every visible pair.
 * dC: planar like rgb; dD, dA per pixel (dA nullable).
 * Outputs (accumulated, caller zeroes): g2d [n_pairs][OC_NGRAD], parameter
 * gradients, pose [n_views][6], densify acc/cnt [n]. */
int oracle_render_bwd(int64_t n, const double *means, const double *log_scales, const double *quats,
                      const double *opacity_logits, const double *sh, int sh_degree,
                      int n_views, const oc_camera *cams, const int64_t *submap_offsets,
                      const oc_config *cfg, const double *rec, const int64_t *vals,
                      const int64_t *ranges, const double *dC, const double *dD, const double *dA,
                      const double *dmean, const double *dvar, double *g2d, double *g_means, double *g_ls, double *g_quats, double *g_om,
                      double *g_sh, double *g_pose, double *dens_acc, double *dens_cnt) {
    (void)n;
    oc_view *V = (oc_view *)malloc(sizeof(oc_view) * (n_views > 0 ? n_views : 1));
    make_views(n_views, cams, submap_offsets, cfg, V);
    for (int v = 0; v < n_views; ++v) {
        int64_t W = cams[v].width, H = cams[v].height;
#pragma omp parallel for schedule(dynamic, 1) num_threads(oc_threads)
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                int64_t pix = V[v].pix_off + y * W + x, local = y * W + x;
                double gC[3];
                for (int ch = 0; ch < 3; ++ch) gC[ch] = dC[3 * V[v].pix_off + ch * W * H + local];
                double gD = dD ? dD[pix] : 0.0, gA = dA ? dA[pix] : 0.0;
                double gmu = dmean ? dmean[pix] : 0.0, gv = dvar ? dvar[pix] : 0.0;
                if (gC[0] == 0 && gC[1] == 0 && gC[2] == 0 && gD == 0 && gA == 0 && gmu == 0 && gv == 0)
                    continue;
                int64_t t = V[v].tile_off + (y / cfg->tile_h) * V[v].ntx + x / cfg->tile_w;
                int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
                pixel_adjoint(rec, vals + s, e - s, x + 0.5, y + 0.5, cfg, gC, gD, gA, gmu, gv, g2d);
            }
    }
    int K = (sh_degree + 1) * (sh_degree + 1);
    /* a Gaussian appears once per view, so the pairs of one view update
     * disjoint parameter rows; each thread sums its pairs' pose terms apart */
    for (int v = 0; v < n_views; ++v) {
#pragma omp parallel num_threads(oc_threads)
        {
            double pose_t[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 1024)
            for (int64_t k = 0; k < V[v].ng; ++k) {
                int64_t p = V[v].pair_off + k, g = V[v].g0 + k;
                const double *r = rec + p * OC_NCOL;
                if (r[C_VIS] == 0.0) continue;
                const double *gg = g2d + p * OC_NGRAD;
                project_adjoint(means + 3 * g, log_scales + 3 * g, quats + 4 * g, opacity_logits[g],
                                sh + (int64_t)3 * K * g, sh_degree, &cams[v], cfg, r, gg,
                                g_means + 3 * g, g_ls + 3 * g, g_quats + 4 * g, g_om + g,
                                g_sh + (int64_t)3 * K * g, pose_t);
                /* R14: image-space gradient magnitude at the projected centre, pixels */
                if (dens_acc) dens_acc[g] += sqrt(gg[G_U] * gg[G_U] + gg[G_V] * gg[G_V]);
                if (dens_cnt) dens_cnt[g] += 1.0;
            }
            for (int i = 0; i < 6; ++i) acc_add(&g_pose[6 * v + i], pose_t[i]);
        }
    }
    free(V);
    return 0;
}
