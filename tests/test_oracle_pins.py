"""Pins for the FP64 oracle against facts that do not come from the oracle itself.

Each test ties one part of the oracle to a closed form, an invariant, an
independent library routine or brute force, so that a dropped term, a wrong
sign, a transposed operand or a wrong index in the oracle fails at least one:

  covariance (Eq. 3)        eigen-structure; scipy's quaternion rotation
  projection (Eq. 4)        isotropic on-axis closed form; pinhole; J by FD
  colour                    SH orthonormality by quadrature; DC reproduces rgb
  compositing               single-Gaussian closed form; stacked-alpha closed
                            form with the stop rule; sum of weights = alpha
  binning                   keys rebuilt with numpy's stable sort, each tile's
                            test redone as a bounded least-squares problem
                            (scipy's BVLS); every pixel with alpha >= alpha_min
                            in a kept tile (brute force); brute-force renderer
                            (no tiles) equal bitwise for 3 tile sizes
  backward                  central differences of every parameter type and
                            every pose twist; translation identity
  losses (Eqs. 6-7)         KL by numerical integration; FD of both losses
  SSIM (Eq. 6)              scipy's separable Gaussian filters; constant-image
                            closed form; SSIM(x, x) = 1 with zero gradient;
                            central differences; Eq. 6 composition
  rendered depth mean/var   two-fragment closed form; zero variance for equal
                            depths; Popoviciu bound; invariance to a common
                            depth shift; KL with the rendered variance by
                            quadrature, reduced to the fixed-sigma mode, and
                            FD through the whole render
"""
import copy
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2510_26358_gb300 import scenes as S

scipy = pytest.importorskip("scipy")
from scipy.spatial.transform import Rotation  # noqa: E402
from scipy.optimize import lsq_linear  # noqa: E402


CFG = O.Config()


def _cam(W=64, H=48, f=60.0, T=None, cx=None, cy=None):
    T = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) if T is None else T
    return S.Camera(W, H, f, f, W / 2 if cx is None else cx, H / 2 if cy is None else cy, T, 0)


def _params(means, log_scales, quats, omega, sh, deg=0):
    n = len(means)
    return O.Params(np.asarray(means, np.float64).reshape(n, 3),
                    np.asarray(log_scales, np.float64).reshape(n, 3),
                    np.asarray(quats, np.float64).reshape(n, 4),
                    np.asarray(omega, np.float64).reshape(n),
                    np.asarray(sh, np.float64).reshape(n, (deg + 1) ** 2, 3), deg,
                    np.array([0, n], np.int64))


# ---------------------------------------------------------------------------
# covariance, Eq. (3)
# ---------------------------------------------------------------------------

def test_cov3d_eigenvalues_and_rotation():
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.normal(size=4) * rng.uniform(0.1, 5.0)   # not unit on purpose
        s = rng.normal(-2, 1, 3)
        Sig = O.cov3d(q, s)
        assert np.allclose(Sig, Sig.T, atol=1e-15)
        ev = np.sort(np.linalg.eigvalsh(Sig))
        assert np.allclose(ev, np.sort(np.exp(2 * s)), rtol=1e-10, atol=1e-15)
        # scipy's rotation of the same quaternion (scipy order is x,y,z,w)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        assert np.allclose(Sig, R @ np.diag(np.exp(2 * s)) @ R.T, rtol=1e-10, atol=1e-14)


def test_cov3d_zero_quaternion_is_rejected():
    # a zero quaternion culls the pair (reading R1)
    cam = _cam()
    P = _params([[0, 0, 3]], [[-2, -2, -2]], [[0, 0, 0, 0]], [2.0], [[0, 0, 0]])
    rec = O.project(P, [cam], CFG)
    assert rec[0, O.C_VIS] == 0


# ---------------------------------------------------------------------------
# projection, Eq. (4)
# ---------------------------------------------------------------------------

def test_isotropic_on_axis_image_covariance():
    f, z, s = 60.0, 3.0, math.log(0.05)
    cam = _cam(f=f)
    P = _params([[0, 0, z]], [[s, s, s]], [[0.3, -0.2, 0.5, 0.7]], [1.0], [[0, 0, 0]])
    r = O.project(P, [cam], CFG)[0]
    var = (f * 0.05 / z) ** 2 + float(np.float32(0.3))
    assert r[O.C_SA] == pytest.approx(var, rel=1e-12)
    assert r[O.C_SC] == pytest.approx(var, rel=1e-12)
    assert abs(r[O.C_SB]) < 1e-15
    assert r[O.C_U] == pytest.approx(32.0, abs=1e-12) and r[O.C_V] == pytest.approx(24.0, abs=1e-12)
    assert r[O.C_QA] == pytest.approx(1 / var, rel=1e-12)
    assert r[O.C_Z] == z and r[O.C_Z32] == z


def test_pinhole_mean_and_pose():
    # a rotated, translated camera: the mean lands where the pinhole model says
    R = Rotation.from_euler("xyz", [0.1, -0.2, 0.3]).as_matrix()
    t = np.array([0.2, -0.1, 0.5])
    cam = S.Camera(80, 60, 70.0, 65.0, 41.0, 29.0, np.concatenate([R, t[:, None]], 1), 0)
    mu = np.array([0.3, 0.2, 2.5])
    P = _params([mu], [[-3, -3, -3]], [[1, 0, 0, 0]], [1.0], [[0, 0, 0]])
    r = O.project(P, [cam], CFG)[0]
    pc = R @ mu + t
    assert r[O.C_U] == pytest.approx(70.0 * pc[0] / pc[2] + 41.0, rel=1e-13)
    assert r[O.C_V] == pytest.approx(65.0 * pc[1] / pc[2] + 29.0, rel=1e-13)
    assert r[O.C_Z] == pytest.approx(pc[2], rel=1e-15)


def test_image_covariance_is_linearised_pinhole():
    # Sigma' - dil*I = J (R Sigma R^T) J^T with J the derivative of the pinhole
    # map, here taken by central differences of (fx x/z + cx, fy y/z + cy)
    rng = np.random.default_rng(5)
    R = Rotation.from_euler("xyz", [0.05, 0.1, -0.3]).as_matrix()
    t = np.array([0.1, 0.0, 0.2])
    cam = S.Camera(100, 80, 90.0, 85.0, 50.0, 40.0, np.concatenate([R, t[:, None]], 1), 0)
    for _ in range(10):
        mu = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(1.5, 4)])
        q = rng.normal(size=4)
        s = rng.normal(-2.5, 0.5, 3)
        P = _params([mu], [s], [q], [1.0], [[0, 0, 0]])
        r = O.project(P, [cam], CFG)[0]
        pc = R @ mu + t

        def pin(p):
            return np.array([90.0 * p[0] / p[2] + 50.0, 85.0 * p[1] / p[2] + 40.0])
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-6
            J[:, k] = (pin(pc + e) - pin(pc - e)) / 2e-6
        Sc = R @ O.cov3d(q, s) @ R.T
        S2 = J @ Sc @ J.T
        dil = float(np.float32(0.3))
        assert np.allclose([r[O.C_SA] - dil, r[O.C_SB], r[O.C_SC] - dil],
                           [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-7, atol=1e-9)


def test_near_plane_culls():
    cam = _cam()
    P = _params([[0, 0, 0.19], [0, 0, 0.21]], [[-3] * 3] * 2, [[1, 0, 0, 0]] * 2, [2.0, 2.0],
                [[0, 0, 0]] * 2)
    rec = O.project(P, [cam], CFG)
    assert rec[0, O.C_VIS] == 0 and rec[1, O.C_VIS] == 1


# ---------------------------------------------------------------------------
# colour
# ---------------------------------------------------------------------------

def test_sh_basis_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for the degree <= 6
    # products of degree-3 harmonics
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phis = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            d = np.array([st * math.cos(ph), st * math.sin(ph), ct])
            Y = O.sh_basis(3, d)
            G += w * (2 * np.pi / nphi) * np.outer(Y, Y)
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_sh_degree0_reproduces_rgb():
    cam = _cam()
    rgb = np.array([0.1, 0.6, 0.95])
    sh0 = (rgb - 0.5) * 2 * math.sqrt(math.pi)
    P = _params([[0.1, 0.05, 2.0]], [[-3] * 3], [[1, 0, 0, 0]], [2.0], [sh0])
    r = O.project(P, [cam], CFG)[0]
    assert np.allclose(r[[O.C_R, O.C_G, O.C_B]], rgb, atol=1e-14)


# ---------------------------------------------------------------------------
# compositing
# ---------------------------------------------------------------------------

def test_single_isotropic_gaussian_closed_form():
    W, H, f, z, sc = 40, 32, 50.0, 2.0, 0.04
    cam = _cam(W, H, f)
    omega, rgb = 1.3, np.array([0.2, 0.7, 0.4])
    sh0 = (rgb - 0.5) * 2 * math.sqrt(math.pi)
    P = _params([[0, 0, z]], [[math.log(sc)] * 3], [[1, 0, 0, 0]], [omega], [sh0])
    rec, keys, vals, ranges, out = O.forward(P, [cam], CFG)
    o = 1 / (1 + math.exp(-omega))
    var = (f * sc / z) ** 2 + float(np.float32(0.3))
    amin, amax = float(np.float32(1 / 255)), float(np.float32(0.99))
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
    raw = o * np.exp(-0.5 * d2 / var)
    al = np.where(raw >= amin, np.minimum(amax, raw), 0.0).ravel()
    assert np.allclose(out["alpha"], al, atol=1e-14)
    assert np.allclose(out["depth"], al * z, atol=1e-13)
    for c in range(3):
        assert np.allclose(out["rgb"][c * W * H:(c + 1) * W * H], al * rgb[c], atol=1e-14)
    assert (out["alpha"] > 0).sum() > 20


def test_stacked_alphas_and_stop_rule():
    # k identical opaque discs at increasing depth: T after j blends = (1-a)^j;
    # the fragment that would take T below t_min is not blended
    cam = _cam(16, 16, 20.0)
    a = 0.95
    omega = math.log(a / (1 - a))
    n = 6
    P = _params([[0, 0, 1.0 + 0.1 * i] for i in range(n)], [[math.log(0.5)] * 3] * n,
                [[1, 0, 0, 0]] * n, [omega] * n, [[1.0, 1.0, 1.0]] * n)
    rec, keys, vals, ranges, out = O.forward(P, [cam], CFG)
    pix = 8 * 16 + 8
    # near the centre alpha ~ a; T: 0.05, 2.5e-3, 1.25e-4, then 6.25e-6 < 1e-4 stops
    assert out["nblend"][pix] == 3
    T = out["T"][pix]
    assert 1e-4 <= T < 2e-4
    assert out["alpha"][pix] == pytest.approx(1 - T, rel=0, abs=1e-15)


def test_weights_sum_to_alpha():
    # with every colour equal to 1, each channel equals the accumulated alpha
    sc = S.random_box_scene(300, 48, 40, 45.0, seed=2)
    sh = np.zeros_like(sc.sh)
    sh[:, 0, :] = 0.5 * 2 * math.sqrt(math.pi)
    P = O.Params(sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sh, 0, sc.submap_offsets)
    cams = O.as_float32_cameras(sc.cameras)
    rec, keys, vals, ranges, out = O.forward(P, cams, CFG)
    npx = 48 * 40
    for c in range(3):
        assert np.allclose(out["rgb"][c * npx:(c + 1) * npx], out["alpha"], atol=1e-13)
    assert np.all(out["T"] >= float(np.float32(1e-4)))
    assert np.allclose(out["alpha"], 1 - out["T"], atol=0)
    # the alpha-weighted depth lies between the nearest and farthest blended depth
    zs = rec[rec[:, O.C_VIS] > 0, O.C_Z]
    m = out["alpha"] > 0
    dn = out["depth"][m] / out["alpha"][m]
    assert dn.min() >= zs.min() - 1e-12 and dn.max() <= zs.max() + 1e-12


# ---------------------------------------------------------------------------
# binning and tiling
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("tile,scene", [((8, 8), "box"), ((16, 16), "box"), ((16, 32), "box"),
                                        ((8, 8), "needles")])
def test_tiled_equals_brute_force(tile, scene):
    cfg = O.Config(tile_w=tile[0], tile_h=tile[1])
    if scene == "box":
        sc = S.random_box_scene(500, 72, 56, 60.0, seed=11, sh_degree=3)
    else:  # most rectangle tiles dropped by the tile-exact rule
        sc = S.needle_scene(400, 72, 56, 60.0, seed=12)
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    rec, keys, vals, ranges, out = O.forward(P, cams, cfg)
    br = O.render_brute(P, cams, cfg, rec)
    for k in ("rgb", "depth", "alpha", "T", "nblend", "sig"):
        assert np.array_equal(out[k], br[k]), k
    assert out["nblend"].max() >= 3


@pytest.mark.parametrize("scene", ["submaps", "needles"])
def test_keys_rebuilt_with_numpy_stable_sort(scene):
    cfg = O.Config(tile_w=8, tile_h=8)
    if scene == "submaps":
        sc = S.uneven_submaps(3, 200, 800, seed=4, scale=1.0, resolutions=((48, 40), (64, 32)))
    else:  # long thin ellipses: most rectangle tiles dropped, badly conditioned covariances
        sc = S.needle_scene(600, 96, 72, 90.0, seed=7)
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    rec = O.project(P, cams, cfg)
    keys, vals, ranges = O.bin(P, cams, cfg, rec)
    cc = cfg.c()
    rho, kappa = cc.ext_rel_pad, cc.ext_abs_pad
    # independent rebuild: per view, per visible pair, per tile of its
    # rectangle; the tile is kept iff min ||L d||^2 over the tile's grown box
    # of pixel-centre offsets d (Q = L^T L) is within the padded threshold,
    # solved as bounded linear least squares; then argsort
    ek, ev = [], []
    toff, poff = 0, 0
    n_rect = n_reach = 0
    for v, c in enumerate(cams):
        ntx, nty = -(-c.width // 8), -(-c.height // 8)
        ng = int(sc.submap_offsets[c.submap + 1] - sc.submap_offsets[c.submap])
        for k in range(ng):
            r = rec[poff + k]
            if r[O.C_VIS] == 0:
                continue
            Q = np.array([[r[O.C_QA], r[O.C_QB]], [r[O.C_QB], r[O.C_QC]]])
            L = np.linalg.cholesky(Q).T
            thr = r[O.C_E] * (1 + rho) ** 2
            zb = np.array([r[O.C_Z32]], np.float32).view(np.uint32)[0]
            for ty in range(int(r[O.C_TY0]), int(r[O.C_TY1]) + 1):
                for tx in range(int(r[O.C_TX0]), int(r[O.C_TX1]) + 1):
                    n_rect += 1
                    px = np.arange(tx * 8, min(tx * 8 + 8, c.width)) + 0.5 - r[O.C_U]
                    py = np.arange(ty * 8, min(ty * 8 + 8, c.height)) + 0.5 - r[O.C_V]
                    lo, hi = [px[0] - kappa, py[0] - kappa], [px[-1] + kappa, py[-1] + kappa]
                    qmin = 2 * lsq_linear(L, np.zeros(2), bounds=(lo, hi), method="bvls").cost
                    assert abs(qmin - thr) > 1e-9 * thr  # no decision this close in the fixture
                    # brute force: a pixel where the Gaussian reaches alpha_min lies in a kept tile
                    dx, dy = np.meshgrid(px, py)
                    reach = (Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy <= r[O.C_E]).any()
                    assert qmin <= thr or not reach
                    if qmin <= thr:
                        n_reach += reach
                        ek.append((np.uint64(toff + ty * ntx + tx) << np.uint64(32)) | np.uint64(zb))
                        ev.append(poff + k)
        toff += ntx * nty
        poff += ng
    ek, ev = np.array(ek, np.uint64), np.array(ev, np.int64)
    # convexity: in every rectangle row a pair's kept tiles are those whose
    # grown box overlaps the one x-interval of the ellipse within the row's
    # strip, so they form a single run
    toffs = np.cumsum([0] + [-(-c.width // 8) * -(-c.height // 8) for c in cams])
    ntxs = [-(-c.width // 8) for c in cams]
    tiles_o = (keys >> np.uint64(32)).astype(np.int64)
    for pair in np.unique(vals):
        t = tiles_o[vals == pair]
        v = int(np.searchsorted(toffs, t[0], side="right") - 1)
        tx, ty = (t - toffs[v]) % ntxs[v], (t - toffs[v]) // ntxs[v]
        for row in np.unique(ty):
            xs = np.sort(tx[ty == row])
            assert np.array_equal(xs, np.arange(xs[0], xs[-1] + 1))
    # the fixture exercises both outcomes: corner tiles dropped, most kept ones reached
    assert n_rect - len(ek) >= 50 and n_reach > 0.8 * len(ek), (n_rect, len(ek), n_reach)
    order = np.argsort(ek, kind="stable")
    assert np.array_equal(keys, ek[order]) and np.array_equal(vals, ev[order])
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    for t in range(ranges.shape[0]):
        idx = np.nonzero(tiles == t)[0]
        if len(idx):
            assert ranges[t, 0] == idx[0] and ranges[t, 1] == idx[-1] + 1
        else:
            assert ranges[t, 0] == ranges[t, 1] == 0
    # views only see the Gaussians of their own submap
    g = rec[:, O.C_GAUSS].astype(int)
    vw = rec[:, O.C_VIEW].astype(int)
    for v, c in enumerate(cams):
        gs = g[vw == v]
        assert gs.min() >= sc.submap_offsets[c.submap] and gs.max() < sc.submap_offsets[c.submap + 1]


def _float32_records(rec):
    """Projection outputs in the float32 path's layout, made from the FP64
    oracle's records: (U, V, hx, hy | l11, l12, l22, log2 o | r, g, b, z) with
    U = floor(u), hx = U + 1/2 - u, L the upper Cholesky factor of
    Q log2(e)/2; the tile rectangles; depth keys (0xFFFFFFFF: not visible)."""
    n = rec.shape[0]
    out = np.zeros((n, 12), np.float32)
    rect = np.zeros((n, 4), np.int16)
    pkey = np.full(n, 0xFFFFFFFF, np.uint32)
    s2 = math.log2(math.e) / 2
    for i, r in enumerate(rec):
        if r[O.C_VIS] == 0:
            continue
        U, V = math.floor(r[O.C_U]), math.floor(r[O.C_V])
        l11 = math.sqrt(r[O.C_QA] * s2)
        l12 = r[O.C_QB] * s2 / l11
        l22 = math.sqrt(r[O.C_QC] * s2 - l12 * l12)
        out[i] = (U, V, U + 0.5 - r[O.C_U], V + 0.5 - r[O.C_V], l11, l12, l22, math.log2(r[O.C_OPA]),
                  r[O.C_R], r[O.C_G], r[O.C_B], r[O.C_Z32])
        rect[i] = (r[O.C_TX0], r[O.C_TY0], r[O.C_TX1], r[O.C_TY1])
        pkey[i] = np.float32(r[O.C_Z32]).view(np.uint32)
    return out, rect, pkey


@pytest.mark.parametrize("scene", ["submaps", "needles"])
def test_stage_isolated_binning_rebuilt(scene):
    """The binning stage on float32 projection outputs: every rectangle
    tile's R6b decision redone as bounded least squares on the float inputs
    (the box of pixel-centre offsets X - U + hx, grown by ext_abs_pad, and L
    as given), keys rebuilt with numpy's stable sort, ranges from the sorted
    tile ids; and on records made from the FP64 projection the decisions
    agree with the end-to-end binning wherever neither is near its threshold."""
    cfg = O.Config(tile_w=8, tile_h=8)
    if scene == "submaps":
        sc = S.uneven_submaps(3, 200, 800, seed=4, scale=1.0, resolutions=((48, 40), (64, 32)))
    else:
        sc = S.needle_scene(600, 96, 72, 90.0, seed=7)
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    rec = O.project(P, cams, cfg)
    rec32, rect, pkey = _float32_records(rec)
    dec, margin = O.tile_decisions32(P, cams, cfg, rec32, rect, pkey)
    cc = cfg.c()
    rho, kappa, l2amin = cc.ext_rel_pad, cc.ext_abs_pad, math.log2(cc.alpha_min)
    ek, ev, exp_dec = [], [], []
    toff, poff = 0, 0
    for v, c in enumerate(cams):
        ntx, nty = -(-c.width // 8), -(-c.height // 8)
        ng = int(sc.submap_offsets[c.submap + 1] - sc.submap_offsets[c.submap])
        for k in range(ng):
            p = poff + k
            if pkey[p] == 0xFFFFFFFF:
                continue
            r = rec32[p].astype(np.float64)
            L = np.array([[r[4], r[5]], [0.0, r[6]]])
            thr = (r[7] - l2amin) * (1 + rho) ** 2
            for ty in range(int(rect[p, 1]), int(rect[p, 3]) + 1):
                for tx in range(int(rect[p, 0]), int(rect[p, 2]) + 1):
                    X1, Y1 = min(tx * 8 + 8, c.width) - 1, min(ty * 8 + 8, c.height) - 1
                    lo = [tx * 8 - r[0] + r[2] - kappa, ty * 8 - r[1] + r[3] - kappa]
                    hi = [X1 - r[0] + r[2] + kappa, Y1 - r[1] + r[3] + kappa]
                    qmin = 2 * lsq_linear(L, np.zeros(2), bounds=(lo, hi), method="bvls").cost
                    assert abs(qmin - thr) > 1e-9 * (abs(thr) + 1)  # no decision this close in the fixture
                    keep = qmin <= thr
                    exp_dec.append(keep)
                    if keep:
                        ek.append((np.uint64(toff + ty * ntx + tx) << np.uint64(32)) | np.uint64(pkey[p]))
                        ev.append(p)
        toff += ntx * nty
        poff += ng
    exp_dec = np.array(exp_dec, bool)
    assert np.array_equal(dec.astype(bool), exp_dec)
    assert np.all(np.sign(margin[margin != 0]) == np.where(exp_dec, 1, -1)[margin != 0])
    assert (~exp_dec).sum() >= 50 and exp_dec.sum() >= 50
    keys, vals, ranges = O.bin_decided(P, cams, cfg, rect, pkey, dec)
    ek, ev = np.array(ek, np.uint64), np.array(ev, np.int64)
    order = np.argsort(ek, kind="stable")
    assert np.array_equal(keys, ek[order]) and np.array_equal(vals, ev[order])
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    T = ranges.shape[0]
    first = np.searchsorted(tiles, np.arange(T), side="left")
    last = np.searchsorted(tiles, np.arange(T), side="right")
    empty = first == last
    assert np.array_equal(ranges[~empty, 0], first[~empty]) and np.array_equal(ranges[~empty, 1], last[~empty])
    assert np.all(ranges[empty] == 0)
    # against the end-to-end binning (FP64 projection): the same instances
    # except where the end-to-end band marks the pair
    k0, v0, _ = O.bin(P, cams, cfg, rec)
    amb = np.nonzero(rec[:, O.C_RECT_AMBIG] > 0)[0]
    a = ~np.isin(vals, amb)
    b = ~np.isin(v0, amb)
    assert np.array_equal(keys[a], k0[b]) and np.array_equal(vals[a], v0[b])


# ---------------------------------------------------------------------------
# backward: central differences and the translation identity
# ---------------------------------------------------------------------------

def _se3_left(T, xi):
    rho, phi = xi[:3], xi[3:]
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        R, V = np.eye(3) + K, np.eye(3) + 0.5 * K
    else:
        R = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * K + (th - math.sin(th)) / th ** 3 * K @ K
    return np.concatenate([R @ T[:, :3], (R @ T[:, 3] + V @ rho)[:, None]], 1)


def _fd_case(scene, cams, n_samples, seed, h=1e-7):
    P = O.Params.from_scene(scene)
    rng = np.random.default_rng(seed)
    npx = sum(c.width * c.height for c in cams)
    wC, wD, wA = rng.normal(size=3 * npx), 0.1 * rng.normal(size=npx), rng.normal(size=npx)
    rec = O.project(P, cams, CFG)
    vis = np.unique(rec[rec[:, O.C_VIS] > 0, O.C_GAUSS].astype(int))
    pix_view = np.concatenate([np.full(c.width * c.height, v) for v, c in enumerate(cams)])
    rgb_pix = np.concatenate([np.tile(np.arange(c.width * c.height) + sum(d.width * d.height for d in cams[:v]), 3)
                              for v, c in enumerate(cams)])
    del pix_view

    def run(Pp, cc):
        return O.forward(Pp, cc, CFG)[4]

    def masked(flip):
        keep = ~flip
        return wC * keep[rgb_pix], wD * keep, wA * keep

    def check(Pp, Pm, cp, cm, pick):
        op, om = run(Pp, cp), run(Pm, cm)
        flip = op["sig"] != om["sig"]
        mC, mD, mA = masked(flip)
        fd = (mC @ (op["rgb"] - om["rgb"]) + mD @ (op["depth"] - om["depth"]) +
              mA @ (op["alpha"] - om["alpha"])) / (2 * h)
        r0, k0, v0, rg0, o0 = O.forward(P, cams, CFG)
        g = O.render_bwd(P, cams, CFG, r0, v0, rg0, mC, mD, mA)
        return fd, pick(g), int(flip.sum())

    results = []
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        for _ in range(n_samples):
            gi = int(rng.choice(vis))
            A = getattr(P, name)
            idx = (gi,) + tuple(int(rng.integers(0, s)) for s in A.shape[1:])
            Pp, Pm = P.copy(), P.copy()
            getattr(Pp, name)[idx] += h
            getattr(Pm, name)[idx] -= h
            fd, an, nf = check(Pp, Pm, cams, cams, lambda g: g[name][idx])
            results.append((name, fd, an, nf))
    for v in range(len(cams)):
        for k in range(6):
            xi = np.zeros(6); xi[k] = h
            cp, cm = copy.deepcopy(cams), copy.deepcopy(cams)
            cp[v].T_cw = _se3_left(cams[v].T_cw, xi)
            cm[v].T_cw = _se3_left(cams[v].T_cw, -xi)
            fd, an, nf = check(P, P, cp, cm, lambda g: g["pose"][v, k])
            results.append((f"pose{v}.{k}", fd, an, nf))
    return results


def _assert_fd(results, rtol=1e-5):
    scale = {}
    for name, fd, an, _ in results:
        key = name.split(".")[0].rstrip("0123456789") if name.startswith("pose") else name
        scale[key] = max(scale.get(key, 0.0), abs(an))
    for name, fd, an, nf in results:
        key = name.split(".")[0].rstrip("0123456789") if name.startswith("pose") else name
        # relative to the gradient and, for near-zero entries, to the tensor's scale
        tol = rtol * max(abs(an), 1e-3 * scale[key]) + 1e-9
        assert abs(fd - an) <= tol, (name, fd, an, nf)


def test_fd_box_scene_sh3():
    sc = S.random_box_scene(250, 48, 40, 45.0, seed=7, sh_degree=3)
    cams = O.as_float32_cameras(sc.cameras)
    _assert_fd(_fd_case(sc, cams, 4, seed=1))


def test_fd_orchard_crop_posed_rig():
    # the pose-gradient workload at toy size: orchard rows, a perturbed 4-camera
    # rig, every camera cropped to a 64x48 window around its principal point
    sc = S.orchard_scene(6_000, 3, 4, 1440, 1080, rear=True, pose_noise=True,
                         lidar_per_view=0, seed=3)
    cams = [c.crop(int(c.cx) - 32, int(c.cy) - 24, 64, 48) for c in sc.cameras]
    cams = O.as_float32_cameras(cams)
    res = _fd_case(sc, cams, 3, seed=2)
    _assert_fd(res)
    assert sum(1 for r in res if r[0].startswith("pose")) == 24


def test_fd_pose_rig_config_step():
    """Central differences with the pose-refinement workload's own step
    h = 1e-4, on that workload: the 1M-Gaussian orchard and its four
    perturbed 1440x1080 cameras, each cropped to a 64x48 window; the
    Gaussians are restricted to those visible in a crop (the others have no
    instance in any crop's tiles and so no effect on the images).  All 24
    pose twists, and 13 entries of each parameter type among the Gaussians
    that blend somewhere (most visible ones sit behind saturated pixels and
    have no gradient).  A rotation of 1e-4 moves the image by ~0.13 px, so
    the plain differences carry an O(h^2) truncation of ~1e-2 of the
    gradient; Richardson's extrapolation (4 D(h/2) - D(h)) / 3 removes it,
    and that must agree with the analytic gradient to 1e-4.  Pixels whose
    blended set changes in any of the four evaluations are masked on both
    sides."""
    from tests.rig_crop import pose_rig_crop, visible_subset
    sc = pose_rig_crop()
    cams = O.as_float32_cameras(sc.cameras)
    prev = O.set_threads(os.cpu_count() or 1)
    try:
        rec = O.project(O.Params.from_scene(sc), cams, CFG)
        sub = visible_subset(sc, np.unique(rec[rec[:, O.C_VIS] > 0, O.C_GAUSS].astype(np.int64)))
        P = O.Params.from_scene(sub)
        npx = sub.n_pix
        rng = np.random.default_rng(5)
        wC, wD, wA = rng.normal(size=3 * npx), 0.1 * rng.normal(size=npx), rng.normal(size=npx)
        rgb_pix = np.concatenate([np.tile(np.arange(c.width * c.height) + sum(d.width * d.height for d in cams[:v]), 3)
                                  for v, c in enumerate(cams)])
        r0, k0, v0, rg0, o0 = O.forward(P, cams, CFG)
        g_all = O.render_bwd(P, cams, CFG, r0, v0, rg0, wC, wD, wA)
        blending = np.nonzero(np.abs(g_all["opacity_logits"]) > 1e-8 * np.abs(g_all["opacity_logits"]).max())[0]
        assert len(blending) >= 200

        def loss(o, keep):
            return (wC * keep[rgb_pix]) @ o["rgb"] + (wD * keep) @ o["depth"] + (wA * keep) @ o["alpha"]

        def richardson(move):
            """move(s) -> (Params, cameras) displaced by s along the direction."""
            h = 1e-4
            outs = {s: O.forward(*move(s), CFG)[4] for s in (h, -h, h / 2, -h / 2)}
            keep = np.logical_and.reduce([o["sig"] == o0["sig"] for o in outs.values()])
            d1 = (loss(outs[h], keep) - loss(outs[-h], keep)) / (2 * h)
            d2 = (loss(outs[h / 2], keep) - loss(outs[-h / 2], keep)) / h
            return d1, (4 * d2 - d1) / 3, keep

        results = []
        for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            for _ in range(13):
                gi = int(rng.choice(blending))
                A = getattr(P, name)
                idx = (gi,) + tuple(int(rng.integers(0, n)) for n in A.shape[1:])

                def move(s, name=name, idx=idx):
                    Pm = P.copy()
                    getattr(Pm, name)[idx] += s
                    return Pm, cams
                d1, dr, keep = richardson(move)
                an = O.render_bwd(P, cams, CFG, r0, v0, rg0, wC * keep[rgb_pix], wD * keep, wA * keep)[name][idx]
                results.append((name, dr, an, int((~keep).sum())))
        raw = []
        for v in range(len(cams)):
            for k in range(6):
                def move(s, v=v, k=k):
                    cm = copy.deepcopy(cams)
                    xi = np.zeros(6)
                    xi[k] = s
                    cm[v].T_cw = _se3_left(cams[v].T_cw, xi)
                    return P, cm
                d1, dr, keep = richardson(move)
                an = O.render_bwd(P, cams, CFG, r0, v0, rg0, wC * keep[rgb_pix], wD * keep, wA * keep)["pose"][v, k]
                results.append((f"pose{v}.{k}", dr, an, int((~keep).sum())))
                raw.append(abs(d1 - an) / max(abs(an), 1e-12))
    finally:
        O.set_threads(prev)
    assert sum(1 for r in results if r[0].startswith("pose")) == 24
    zero = [r for r in results if r[2] == 0]
    print("entries with a zero gradient (clamped colour channels):", [(r[0], r[1]) for r in zero])
    assert len(zero) <= 8 and all(r[0] == "sh" and r[1] == 0 for r in zero)
    _assert_fd(results, rtol=1e-4)
    print(f"plain central differences at h = 1e-4: pose error up to {max(raw):.1e} of the gradient")


def test_translation_identity():
    # shifting every mean by delta equals moving the camera by -delta:
    # dL/drho = R_b sum_g dL/dmu_g for a single view
    sc = S.random_box_scene(300, 48, 40, 45.0, seed=9, sh_degree=3)
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    R = np.array([[0.96, -0.2, 0.19], [0.21, 0.98, -0.03], [-0.18, 0.07, 0.98]])
    u, _, vt = np.linalg.svd(R)
    cams[0].T_cw = np.concatenate([u @ vt, np.array([[0.1], [-0.05], [0.3]])], 1)
    rng = np.random.default_rng(0)
    npx = 48 * 40
    rec, keys, vals, ranges, out = O.forward(P, cams, CFG)
    g = O.render_bwd(P, cams, CFG, rec, vals, ranges, rng.normal(size=3 * npx),
                     rng.normal(size=npx), rng.normal(size=npx))
    lhs = cams[0].T_cw[:, :3] @ g["means"].sum(0)
    assert np.allclose(g["pose"][0, :3], lhs, rtol=1e-10, atol=1e-10)
    assert np.abs(g["pose"][0, 3:]).max() > 0


# ---------------------------------------------------------------------------
# image-space gradients and the densification statistic (Sec. III-B: the
# image-space gradient magnitude at the projected splat centre)
# ---------------------------------------------------------------------------

# record column perturbed for each component of the per-pair image-space
# gradient (the opacity enters through ln o)
_G2D_COLS = {O.G_U: O.C_U, O.G_V: O.C_V, O.G_QA: O.C_QA, O.G_QB: O.C_QB, O.G_QC: O.C_QC, O.G_LNO: O.C_OPA,
             O.G_R: O.C_R, O.G_G: O.C_G, O.G_B: O.C_B, O.G_Z: O.C_Z}


def test_image_space_gradients_and_densify_statistic_fd():
    """Each of the ten image-space gradient components of a pair (mean u, v;
    conic qa, qb, qc; ln o; colour; depth) against central differences of
    the loss with that record entry moved and the tile lists kept; then the
    densification statistic against the same differences: for every
    Gaussian, the sum over the views where it is visible of the Euclidean
    norm of (dL/du, dL/dv) in pixels, and the number of those views."""
    sc = S.random_box_scene(300, 56, 44, 50.0, seed=21, sh_degree=1)
    rng = np.random.default_rng(21)
    cam0 = sc.cameras[0]
    cams = O.as_float32_cameras([cam0, S.perturb_pose(cam0, rng, sigma_t=0.1, sigma_deg=3.0)])
    P = O.Params.from_scene(sc)
    rec, keys, vals, ranges, out = O.forward(P, cams, CFG)
    npx = sum(c.width * c.height for c in cams)
    wC, wD, wA = rng.normal(size=3 * npx), 0.1 * rng.normal(size=npx), rng.normal(size=npx)
    rgb_pix = np.concatenate([np.tile(np.arange(c.width * c.height) + sum(d.width * d.height for d in cams[:v]), 3)
                              for v, c in enumerate(cams)])
    vis = np.nonzero(rec[:, O.C_VIS] > 0)[0]
    gauss = rec[:, O.C_GAUSS].astype(int)
    shared = [g for g in np.unique(gauss[vis]) if (gauss[vis] == g).sum() == 2]
    assert len(shared) >= 20

    def loss_with(rec_p, mask):
        o = O.render_fwd(P, cams, CFG, rec_p, vals, ranges)
        return (wC * mask[rgb_pix]) @ o["rgb"] + (wD * mask) @ o["depth"] + (wA * mask) @ o["alpha"], o["sig"]

    def fd(p, col, h):
        rp, rm = rec.copy(), rec.copy()
        if col == O.C_OPA:        # d/d ln o
            rp[p, col] *= math.exp(h)
            rm[p, col] *= math.exp(-h)
        else:
            rp[p, col] += h
            rm[p, col] -= h
        ones = np.ones(npx, bool)
        _, sp = loss_with(rp, ones)
        _, sm = loss_with(rm, ones)
        keep = sp == sm           # pixels whose blended set does not change
        lp, _ = loss_with(rp, keep)
        lm, _ = loss_with(rm, keep)
        return (lp - lm) / (2 * h), keep

    h = 1e-6
    picked = list(rng.choice(vis, 12, replace=False))
    for g in shared[:10]:
        picked += list(np.nonzero((gauss == g) & (rec[:, O.C_VIS] > 0))[0])
    fd_uv, clean = {}, {}
    for p in picked:
        comps = {}
        masks = []
        for k, col in _G2D_COLS.items():
            comps[k], keep = fd(p, col, h)
            masks.append(keep)
        keep = np.logical_and.reduce(masks)
        go = O.render_bwd(P, cams, CFG, rec, vals, ranges, wC * keep[rgb_pix], wD * keep, wA * keep)
        g2d = go["g2d"][p]
        scale = max(abs(g2d).max(), 1e-12)
        for k in _G2D_COLS:
            assert abs(comps[k] - g2d[k]) <= 1e-6 * scale + 1e-9, (p, k, comps[k], g2d[k])
        fd_uv[p] = (comps[O.G_U], comps[O.G_V])
        clean[p] = bool(keep.all())    # no pixel's blended set changed under the moves
    # the statistic of the Gaussians seen by both views whose moves flip no pixel
    go = O.render_bwd(P, cams, CFG, rec, vals, ranges, wC, wD, wA)
    n_ok = 0
    for g in shared[:10]:
        pairs = np.nonzero((gauss == g) & (rec[:, O.C_VIS] > 0))[0]
        if not all(clean[p] for p in pairs):
            continue
        ref = sum(math.hypot(*fd_uv[p]) for p in pairs)
        assert abs(go["dens_acc"][g] - ref) <= 1e-6 * ref, (g, go["dens_acc"][g], ref)
        assert go["dens_cnt"][g] == len(pairs) == 2
        n_ok += 1
    assert n_ok >= 3


def test_densify_statistic_closed_form():
    """One isotropic Gaussian seen twice (two identical views) under the loss
    L = sum over pixel centres of w * A, with w a smooth bump (3 px wide,
    polynomial-tilted) that vanishes long before the alpha >= alpha_min edge
    of the Gaussian's support.  Since alpha depends on (pixel - mean),
    dL/du = -sum w d(alpha)/dx = sum alpha dw/dx, because the lattice sum of
    the derivative of the smooth, rapidly decaying w alpha is 0 (to ~1e-12
    for these widths); likewise dL/dv = sum alpha dw/dy.  The statistic is
    then the sum over the two views of the Euclidean norm of (dL/du, dL/dv)
    in pixels (not squared, not normalised), the count is 2, and a third
    camera that looks away adds nothing."""
    W, H, f, z = 96, 96, 80.0, 4.0
    s_world = 6.0 * z / f                         # 6 px image standard deviation before the dilation
    o = 0.9
    mu = np.array([[0.25 * z / f, -0.5 * z / f, z]])
    P = _params(mu, np.log([s_world] * 3), [1, 0, 0, 0], math.log(o / (1 - o)), np.zeros(3))
    T_away = np.concatenate([np.diag([-1.0, 1.0, -1.0]), np.zeros((3, 1))], 1)
    cams = O.as_float32_cameras([_cam(W, H, f), _cam(W, H, f), _cam(W, H, f, T=T_away)])
    rec, keys, vals, ranges, out = O.forward(P, cams, CFG)
    npx = W * H
    # pinhole mean of the Gaussian, the bump 1.3 px right of and 0.7 px above it
    u = f * mu[0, 0] / z + W / 2
    v = f * mu[0, 1] / z + H / 2
    u0, v0, b = u + 1.3, v - 0.7, 3.0
    X, Y = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    ex, ey = (X - u0) / b, (Y - v0) / b
    bump = np.exp(-0.5 * (ex * ex + ey * ey))
    poly = 1.0 + 0.5 * ex + 0.3 * ey
    w = (bump * poly).ravel()
    dw_dx = (bump * (0.5 / b - ex / b * poly)).ravel()
    dw_dy = (bump * (0.3 / b - ey / b * poly)).ravel()
    A = out["alpha"][:npx]
    exp_u, exp_v = A @ dw_dx, A @ dw_dy
    g = O.render_bwd(P, cams, CFG, rec, vals, ranges, np.zeros(9 * npx), np.zeros(3 * npx),
                     np.concatenate([w, w, np.zeros(npx)]))
    scale = math.hypot(exp_u, exp_v)
    assert abs(exp_u) > 0.05 and abs(exp_v) > 0.05
    for p in (0, 1):
        assert abs(g["g2d"][p, O.G_U] - exp_u) <= 1e-8 * scale, (g["g2d"][p, O.G_U], exp_u)
        assert abs(g["g2d"][p, O.G_V] - exp_v) <= 1e-8 * scale, (g["g2d"][p, O.G_V], exp_v)
    assert rec[2, O.C_VIS] == 0
    assert g["dens_cnt"][0] == 2
    assert abs(g["dens_acc"][0] - 2 * scale) <= 1e-8 * scale


# ---------------------------------------------------------------------------
# losses, Eqs. (6)-(7)
# ---------------------------------------------------------------------------

def test_kl_closed_form_by_integration():
    from scipy.integrate import quad
    for (m1, s1, m2, s2) in [(3.0, 0.05, 3.1, 0.05), (2.0, 0.1, 1.7, 0.3), (5.0, 0.5, 5.0, 0.2)]:
        p = lambda x: math.exp(-0.5 * ((x - m1) / s1) ** 2) / (s1 * math.sqrt(2 * math.pi))
        q = lambda x: math.exp(-0.5 * ((x - m2) / s2) ** 2) / (s2 * math.sqrt(2 * math.pi))
        val, _ = quad(lambda x: p(x) * (math.log(p(x)) - math.log(q(x))) if p(x) > 0 else 0.0,
                      m1 - 12 * s1, m1 + 12 * s1, limit=200, epsabs=1e-13, epsrel=1e-12)
        assert O.kl_normal(m1, s1, m2, s2) == pytest.approx(val, rel=1e-8, abs=1e-10)


@pytest.mark.parametrize("mode", [0, 1])
def test_depth_loss_gradient_and_validity(mode):
    rng = np.random.default_rng(1)
    cams = [_cam(20, 16, 20.0), _cam(12, 10, 15.0)]
    P = O.Params(np.zeros((1, 3)), np.zeros((1, 3)), np.ones((1, 4)), np.zeros(1),
                 np.zeros((1, 1, 3)), 0, np.array([0, 1]))
    npx = 20 * 16 + 12 * 10
    depth = rng.uniform(1, 5, npx)
    alpha = rng.uniform(0, 1, npx)
    alpha[rng.random(npx) < 0.2] = 0.0
    lid = np.stack([rng.uniform(-2, 22, 300), rng.uniform(-2, 18, 300), rng.uniform(0.1, 6, 300),
                    rng.integers(0, 2, 300)], 1)
    loss, grad, nv = O.depth_loss(P, cams, CFG, depth, alpha, lid, mode=mode, sigma_L=0.05,
                                  sigma_U=0.08, lam=0.7)
    # count of valid points by the stated rule
    cnt = 0
    for u, v, z, vw in lid:
        c = cams[int(vw)]
        if 0 <= u < c.width and 0 <= v < c.height and z > 0.2:
            off = 0 if vw == 0 else 320
            if alpha[off + int(v) * c.width + int(u)] > 0:
                cnt += 1
    assert nv == cnt and nv > 50
    h = 1e-6
    for pix in rng.choice(np.nonzero(grad)[0], 10, replace=False):
        dp, dm = depth.copy(), depth.copy()
        dp[pix] += h
        dm[pix] -= h
        fd = (O.depth_loss(P, cams, CFG, dp, alpha, lid, mode, 0.05, 0.08, 0.7)[0] -
              O.depth_loss(P, cams, CFG, dm, alpha, lid, mode, 0.05, 0.08, 0.7)[0]) / (2 * h)
        assert fd == pytest.approx(grad[pix], rel=1e-6, abs=1e-9)


def test_image_l1_gradient():
    rng = np.random.default_rng(2)
    C, I = rng.random(50), rng.random(50)
    loss, g = O.image_l1(C, I)
    assert loss == pytest.approx(np.abs(C - I).sum() / 50)
    h = 1e-7
    for i in range(0, 50, 7):
        Cp, Cm = C.copy(), C.copy()
        Cp[i] += h
        Cm[i] -= h
        assert (O.image_l1(Cp, I)[0] - O.image_l1(Cm, I)[0]) / (2 * h) == pytest.approx(g[i], rel=1e-6)


# ---------------------------------------------------------------------------
# rendered depth distribution: Eq. (7) with a predicted variance
# ---------------------------------------------------------------------------

def _dist(P, cams, cfg=CFG):
    rec, keys, vals, ranges, out = O.forward(P, cams, cfg)
    mean, var = O.render_depth_dist(P, cams, cfg, rec, vals, ranges)
    return rec, vals, ranges, out, mean, var


def test_two_fragment_variance_closed_form():
    # two discs at z1 < z2 with weights w1, w2: mean (w1 z1 + w2 z2) / A and
    # variance w1 w2 (z2 - z1)^2 / A^2
    cam = _cam(16, 16, 20.0)
    a1, a2, z1, z2 = 0.6, 0.8, 1.3, 1.75
    P = _params([[0, 0, z1], [0, 0, z2]], [[math.log(0.5)] * 3] * 2, [[1, 0, 0, 0]] * 2,
                [math.log(a1 / (1 - a1)), math.log(a2 / (1 - a2))], [[1.0, 1.0, 1.0]] * 2)
    rec, vals, ranges, out, mean, var = _dist(P, [cam])
    pix = 8 * 16 + 8
    A, D = out["alpha"][pix], out["depth"][pix]
    # the two weights from alpha and depth: D = w1 z1 + w2 z2, A = w1 + w2
    w2 = (D - z1 * A) / (z2 - z1)
    w1 = A - w2
    assert w1 > 0.5 and w2 > 0.2
    # w1 is the disc's own alpha at the pixel centre; w2 = alpha_2 (1 - w1)
    assert w1 == pytest.approx(a1 * math.exp(-0.5 * 0.5 / ((20 * 0.5 / z1) ** 2 + 0.3)), rel=1e-6)
    assert mean[pix] == pytest.approx((w1 * z1 + w2 * z2) / A, rel=1e-13)
    assert var[pix] == pytest.approx(w1 * w2 * (z2 - z1) ** 2 / A ** 2, rel=1e-12)


def test_equal_depth_fragments_have_zero_variance():
    cam = _cam(16, 16, 20.0)
    n = 4
    P = _params([[0.01 * i, -0.01 * i, 1.5] for i in range(n)], [[math.log(0.3)] * 3] * n,
                [[1, 0, 0, 0]] * n, [0.5] * n, [[1.0, 1.0, 1.0]] * n)
    rec, vals, ranges, out, mean, var = _dist(P, [cam])
    assert (out["nblend"] >= 3).any()
    assert np.abs(var).max() < 1e-28
    m = out["alpha"] > 0
    assert np.allclose(mean[m], 1.5, rtol=0, atol=1e-14) and np.all(mean[~m] == 0)


def test_rendered_variance_bounds():
    # 0 <= variance <= (z_max - z_min)^2 / 4 (Popoviciu); the mean lies in the
    # blended depth range
    sc = S.random_box_scene(400, 48, 40, 45.0, seed=5)
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    rec, vals, ranges, out, mean, var = _dist(P, cams)
    zs = rec[rec[:, O.C_VIS] > 0, O.C_Z]
    m = out["alpha"] > 0
    assert var[m].min() >= 0.0
    assert var[m].max() <= (zs.max() - zs.min()) ** 2 / 4 + 1e-12
    assert mean[m].min() >= zs.min() - 1e-12 and mean[m].max() <= zs.max() + 1e-12
    assert np.allclose(mean[m], out["depth"][m] / out["alpha"][m], rtol=1e-12)
    assert (var[m] > 1e-4).sum() > 100


def test_variance_is_shift_free():
    # moving every Gaussian and the camera by the same offset along the view
    # axis moves the depths, not their spread: var is unchanged, the mean
    # moves by the offset
    sc = S.random_box_scene(300, 48, 40, 45.0, seed=6)
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    rec, vals, ranges, out, mean, var = _dist(P, cams)
    P2 = P.copy()
    P2.means[:, 2] += 3.0
    cams2 = copy.deepcopy(cams)
    cams2[0].T_cw = cams[0].T_cw.copy()
    cams2[0].T_cw[2, 3] -= 3.0
    rec2, vals2, ranges2, out2, mean2, var2 = _dist(P2, cams2)
    assert np.array_equal(out["nblend"], out2["nblend"])
    assert np.allclose(var2, var, rtol=1e-9, atol=1e-12)
    assert np.allclose(mean2, mean, rtol=1e-12, atol=1e-12)


def _var_loss_inputs(rng, n_pts=300):
    # per-pixel (alpha, mean, variance) and LiDAR returns whose depth lies
    # within a few decimetres of the rendered mean where they land
    cams = [_cam(20, 16, 20.0), _cam(12, 10, 15.0)]
    P = O.Params(np.zeros((1, 3)), np.zeros((1, 3)), np.ones((1, 4)), np.zeros(1),
                 np.zeros((1, 1, 3)), 0, np.array([0, 1]))
    npx = 20 * 16 + 12 * 10
    alpha = rng.uniform(0.05, 1, npx)
    alpha[rng.random(npx) < 0.2] = 0.0
    mean = np.where(alpha > 0, rng.uniform(1, 5, npx), 0.0)
    var = np.where(alpha > 0, rng.uniform(0.0, 0.2, npx) ** 2, 0.0)
    vw = rng.integers(0, 2, n_pts)
    u, v = rng.uniform(-2, 22, n_pts), rng.uniform(-2, 18, n_pts)
    z = rng.uniform(0.1, 6, n_pts)
    for i in range(n_pts):
        cm = cams[vw[i]]
        if 0 <= u[i] < cm.width and 0 <= v[i] < cm.height:
            pix = (0 if vw[i] == 0 else 320) + int(v[i]) * cm.width + int(u[i])
            z[i] = mean[pix] + rng.normal(0, 0.2)
    lid = np.stack([u, v, z, vw], 1)
    return P, cams, alpha, mean, var, lid


def test_variance_kl_reduces_to_fixed_sigma():
    # zero rendered variance: sigma_u = sigma_U, so the loss is the fixed-sigma
    # KL mode evaluated on the mean depth
    rng = np.random.default_rng(4)
    P, cams, alpha, mean, var, lid = _var_loss_inputs(rng)
    lv = O.depth_loss_var(P, cams, CFG, alpha, mean, np.zeros_like(var), lid, 0.05, 0.08, 0.7)
    lk, gk, nk = O.depth_loss(P, cams, CFG, mean, alpha, lid, 1, 0.05, 0.08, 0.7)
    assert lv[0] == pytest.approx(lk, rel=1e-13) and lv[3] == nk
    assert np.allclose(lv[1], gk, rtol=1e-12, atol=1e-15)


def test_variance_kl_matches_integration():
    # one point: the loss is KL(N(z, sL^2) || N(mu, var + sU^2)) by quadrature
    from scipy.integrate import quad
    cams = [_cam(4, 4, 5.0)]
    P = O.Params(np.zeros((1, 3)), np.zeros((1, 3)), np.ones((1, 4)), np.zeros(1),
                 np.zeros((1, 1, 3)), 0, np.array([0, 1]))
    A, mu, sd, z = 0.7, 3.2, 0.11, 3.3
    sL, sU = float(np.float32(0.05)), float(np.float32(0.04))
    alpha, mean, var = np.zeros(16), np.zeros(16), np.zeros(16)
    alpha[5], mean[5], var[5] = A, mu, sd ** 2
    lid = np.array([[1.5, 1.5, z, 0]])
    loss = O.depth_loss_var(P, cams, CFG, alpha, mean, var, lid, sL, sU, 1.0)[0]
    s2 = math.sqrt(sd ** 2 + sU ** 2)
    p = lambda x: math.exp(-0.5 * ((x - z) / sL) ** 2) / (sL * math.sqrt(2 * math.pi))
    lq = lambda x: -0.5 * ((x - mu) / s2) ** 2 - math.log(s2 * math.sqrt(2 * math.pi))
    val, _ = quad(lambda x: p(x) * (math.log(p(x)) - lq(x)) if p(x) > 0 else 0.0,
                  z - 12 * sL, z + 12 * sL, limit=200, epsabs=1e-13, epsrel=1e-12)
    assert loss == pytest.approx(val, rel=1e-8)


def test_variance_kl_gradient_fd():
    rng = np.random.default_rng(6)
    P, cams, alpha, mean, var, lid = _var_loss_inputs(rng)
    args = (0.05, 0.08, 0.7)
    loss, gm, gv, nv = O.depth_loss_var(P, cams, CFG, alpha, mean, var, lid, *args)
    assert nv > 50
    h = 1e-7
    ins = [mean, var]
    for k, g in enumerate((gm, gv)):
        for pix in rng.choice(np.nonzero(g)[0], 8, replace=False):
            xp = [x.copy() for x in ins]
            xm = [x.copy() for x in ins]
            xp[k][pix] += h
            xm[k][pix] -= h
            fd = (O.depth_loss_var(P, cams, CFG, alpha, *xp, lid, *args)[0] -
                  O.depth_loss_var(P, cams, CFG, alpha, *xm, lid, *args)[0]) / (2 * h)
            assert fd == pytest.approx(g[pix], rel=1e-5, abs=1e-8), (k, pix)


def test_variance_kl_chain_fd():
    # loss(render(params)) with the rendered mean and variance: the adjoint
    # against central differences of every parameter type and every pose twist
    sc = S.random_box_scene(250, 48, 40, 45.0, seed=12, sh_degree=1)
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    rng = np.random.default_rng(8)
    rec, vals, ranges, out, mean, var = _dist(P, cams)
    hit = np.nonzero(out["alpha"] > 0.2)[0]
    pix = rng.choice(hit, 200, replace=False)
    lid = np.stack([pix % 48 + 0.5, pix // 48 + 0.5, mean[pix] + rng.normal(0, 0.1, len(pix)),
                    np.zeros(len(pix))], 1)
    args = (0.05, 0.03, 1.0)

    def loss_of(Pp, cc):
        r, k, v, rg, o = O.forward(Pp, cc, CFG)
        a, b = O.render_depth_dist(Pp, cc, CFG, r, v, rg)
        return O.depth_loss_var(Pp, cc, CFG, o["alpha"], a, b, lid, *args)[0], o

    L0, gm, gv, nv = O.depth_loss_var(P, cams, CFG, out["alpha"], mean, var, lid, *args)
    assert nv == len(pix)
    z = np.zeros(3 * 48 * 40)
    g = O.render_bwd(P, cams, CFG, rec, vals, ranges, z, np.zeros(48 * 40), None, gm, gv)
    h = 1e-7
    checked = 0
    vis = np.unique(rec[rec[:, O.C_VIS] > 0, O.C_GAUSS].astype(int))
    for name in ("means", "log_scales", "quats", "opacity_logits"):
        for _ in range(4):
            gi = int(rng.choice(vis))
            Arr = getattr(P, name)
            idx = (gi,) + tuple(int(rng.integers(0, s)) for s in Arr.shape[1:])
            Pp, Pm = P.copy(), P.copy()
            getattr(Pp, name)[idx] += h
            getattr(Pm, name)[idx] -= h
            (lp, op), (lm, om) = loss_of(Pp, cams), loss_of(Pm, cams)
            if np.any(op["sig"] != om["sig"]):
                continue  # a support or stop decision flipped inside the step
            fd = (lp - lm) / (2 * h)
            assert fd == pytest.approx(g[name][idx], rel=1e-5, abs=1e-7), (name, idx)
            checked += 1
    for k in range(6):
        xi = np.zeros(6); xi[k] = h
        cp, cm = copy.deepcopy(cams), copy.deepcopy(cams)
        cp[0].T_cw = _se3_left(cams[0].T_cw, xi)
        cm[0].T_cw = _se3_left(cams[0].T_cw, -xi)
        (lp, op), (lm, om) = loss_of(P, cp), loss_of(P, cm)
        if np.any(op["sig"] != om["sig"]):
            continue
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g["pose"][0, k], rel=1e-5, abs=1e-7), ("pose", k)
        checked += 1
    assert checked >= 15
    assert np.abs(g["means"]).max() > 0


# ---------------------------------------------------------------------------
# SSIM term of Eq. (6)
# ---------------------------------------------------------------------------

def _ssim_by_scipy(x, y):
    """SSIM map per Wang et al. with scipy's separable Gaussian filter: sigma
    1.5 truncated at radius 5, zero padding (an implementation independent of
    the oracle's direct window sums)."""
    from scipy.ndimage import gaussian_filter
    f = lambda a: gaussian_filter(a, sigma=1.5, truncate=5.0 / 1.5, mode="constant", cval=0.0)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    mx, my = f(x), f(y)
    sxx, syy, sxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    return (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def _planes(rng, cams, smooth=False):
    out = []
    for c in cams:
        a = rng.random((3, c.height, c.width))
        if smooth:
            from scipy.ndimage import gaussian_filter
            a = np.stack([gaussian_filter(p, 2.0) for p in a])
        out.append(a.ravel())
    return np.concatenate(out)


def test_ssim_matches_scipy_filters():
    rng = np.random.default_rng(21)
    cams = [_cam(37, 23), _cam(16, 40)]
    x = _planes(rng, cams)
    y = np.clip(x + 0.2 * rng.normal(size=x.size), 0, 1)
    val, _ = O.ssim(cams, x, y, grad=False)
    maps, off = [], 0
    for c in cams:
        for ch in range(3):
            n = c.width * c.height
            maps.append(_ssim_by_scipy(x[off:off + n].reshape(c.height, c.width),
                                       y[off:off + n].reshape(c.height, c.width)).ravel())
            off += n
    ref = np.concatenate(maps).mean()
    assert val == pytest.approx(ref, rel=1e-12, abs=1e-14)
    assert 0.2 < val < 0.95


def test_ssim_constant_images_closed_form():
    # away from the border the windows see constants a, b: sigma terms vanish
    # and SSIM = (2ab + C1) / (a^2 + b^2 + C1) (the border windows are cut by
    # the zero padding, so compare a 5-pixel-wide interior through the map)
    cams = [_cam(25, 21)]
    a, b = 0.7, 0.4
    C1 = 0.01 ** 2
    x = np.full(3 * 25 * 21, a)
    y = np.full(3 * 25 * 21, b)
    val, g = O.ssim(cams, x, y)
    m = _ssim_by_scipy(np.full((21, 25), a), np.full((21, 25), b))
    assert m[5:-5, 5:-5] == pytest.approx((2 * a * b + C1) / (a * a + b * b + C1), rel=1e-12)
    assert val == pytest.approx(m.mean(), rel=1e-12)


def test_ssim_identity_is_maximum():
    rng = np.random.default_rng(22)
    cams = [_cam(30, 20)]
    x = _planes(rng, cams)
    val, g = O.ssim(cams, x, x)
    assert val == pytest.approx(1.0, abs=1e-14)
    assert np.abs(g).max() < 1e-14


@pytest.mark.parametrize("smooth", [False, True])
def test_ssim_gradient_fd(smooth):
    rng = np.random.default_rng(23 + smooth)
    cams = [_cam(19, 14), _cam(12, 17)]
    x = _planes(rng, cams, smooth)
    y = _planes(rng, cams, smooth)
    val, g = O.ssim(cams, x, y)
    h = 1e-6
    for i in rng.choice(x.size, 25, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (O.ssim(cams, xp, y, grad=False)[0] - O.ssim(cams, xm, y, grad=False)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-6, abs=2e-10), i  # FD rounding ~1e-16 / h
    # Eq. (6) composes the two terms
    lam = 0.2
    L, gL = O.image_loss(cams, x, y, lam)
    assert L == pytest.approx((1 - lam) * np.abs(x - y).mean() + lam * (1 - val), rel=1e-14)
