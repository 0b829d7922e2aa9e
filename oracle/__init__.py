"""Python access to the FP64 CPU oracle (``gs_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports
it.  Every function widens its float32 inputs to float64 and returns float64
results computed one pixel / one Gaussian at a time (see the C file's header
for the readings of the paper it implements).

Parity status per function (see the pins in ``tests/test_oracle_pins.py``):
  project      pinned: closed forms (covariance eigen-structure, isotropic
               on-axis image covariance, pinhole), SH orthonormality, FD of J
  bin          pinned: brute-force renderer equality, independent key rebuild
               with every tile decision redone by bounded least squares, every
               reached pixel in a kept tile (brute force)
  tile_decisions32 / bin_decided (the binning stage alone, from float32
               projection outputs): pinned by the same key rebuild with the
               decisions redone by bounded least squares on the float inputs
  render_fwd   pinned: single-Gaussian closed form, T invariants, brute force
  render_bwd   pinned: central finite differences, translation identity
  depth_loss   pinned: KL closed form vs numerical integration, FD
  image_l1     pinned: FD
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

NCOL = 30
(C_VIS, C_TX0, C_TY0, C_TX1, C_TY1, C_U, C_V, C_Z, C_Z32, C_SA, C_SB, C_SC, C_QA, C_QB, C_QC,
 C_OPA, C_E, C_EX, C_EY, C_R, C_G, C_B, C_CLR, C_CLG, C_CLB, C_RGB_MARGIN, C_RECT_AMBIG,
 C_GAUSS, C_VIEW, C_NTILE) = range(30)
NGRAD = 10
G_U, G_V, G_QA, G_QB, G_QC, G_LNO, G_R, G_G, G_B, G_Z = range(10)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("submap", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("T", ctypes.c_double * 12)]


class _Config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("near_z", ctypes.c_double), ("dilation", ctypes.c_double),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("t_min", ctypes.c_double), ("jac_clamp", ctypes.c_double),
                ("ext_rel_pad", ctypes.c_double), ("ext_abs_pad", ctypes.c_double),
                ("rect_eps_abs", ctypes.c_double), ("rect_eps_rel", ctypes.c_double),
                ("tile_eps_rel", ctypes.c_double), ("tile_eps_cond", ctypes.c_double)]


@dataclass
class Config:
    tile_w: int = 16
    tile_h: int = 16
    near_z: float = 0.2
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    jac_clamp: float = 1.3
    ext_rel_pad: float = 1e-3
    ext_abs_pad: float = 1e-2
    rect_eps_abs: float = 1e-4
    rect_eps_rel: float = 1e-5
    tile_eps_rel: float = 1e-3
    tile_eps_cond: float = 2.0 ** -20

    def c(self) -> _Config:
        # the float32 values the GPU path uses, widened exactly
        f = lambda x: float(np.float32(x))
        return _Config(self.tile_w, self.tile_h, f(self.near_z), f(self.dilation), f(self.alpha_min),
                       f(self.alpha_max), f(self.t_min), f(self.jac_clamp), f(self.ext_rel_pad),
                       f(self.ext_abs_pad), self.rect_eps_abs, self.rect_eps_rel, self.tile_eps_rel,
                       self.tile_eps_cond)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, d = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        _lib.oracle_project.argtypes = [i64, P, P, P, P, P, i32, i32, P, P, P, P]
        _lib.oracle_bin.argtypes = [i32, P, P, P, P, P, P, P]
        _lib.oracle_count_pairs.argtypes = [i32, P, P]
        _lib.oracle_count_pairs.restype = i64
        _lib.oracle_count_tiles.argtypes = [i32, P, P]
        _lib.oracle_count_tiles.restype = i64
        _lib.oracle_count_instances.argtypes = [i64, P]
        _lib.oracle_count_instances.restype = i64
        _lib.oracle_render_fwd.argtypes = [i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        _lib.oracle_render_brute.argtypes = [i32, P, P, P, P, P, P, P, P, P, P]
        _lib.oracle_render_fwd_pixels.argtypes = [i32, P, P, P, P, P, P, i64, P, P, P, P, P, P, P]
        _lib.oracle_render_bwd.argtypes = [i64, P, P, P, P, P, i32, i32, P, P, P, P, P, P, P, P, P,
                                           P, P, P, P, P, P, P, P, P, P, P]
        _lib.oracle_render_depth_dist.argtypes = [i32, P, P, P, P, P, P, P, P]
        _lib.oracle_depth_loss_var.argtypes = [i32, P, P, P, P, P, P, i64, P, d, d, d, P, P, P]
        _lib.oracle_depth_loss_var.restype = d
        _lib.oracle_image_l1.argtypes = [i64, P, P, P]
        _lib.oracle_image_l1.restype = d
        _lib.oracle_ssim.argtypes = [i32, P, P, P, P]
        _lib.oracle_ssim.restype = d
        _lib.oracle_kl_normal.argtypes = [d, d, d, d]
        _lib.oracle_kl_normal.restype = d
        _lib.oracle_depth_loss.argtypes = [i32, P, P, P, P, P, i64, P, i32, d, d, d, P, P]
        _lib.oracle_depth_loss.restype = d
        _lib.oracle_cov3d.argtypes = [P, P, P]
        _lib.oracle_cov3d.restype = i32
        _lib.oracle_sh_basis.argtypes = [i32, P, P]
        _lib.oracle_layout.restype = i64
        _lib.oracle_rect_tiles32.argtypes = [i64, P, P]
        _lib.oracle_rect_tiles32.restype = i64
        _lib.oracle_tile_decisions32.argtypes = [i32, P, P, P, i64, P, P, P, P, P]
        _lib.oracle_bin_decided.argtypes = [i32, P, P, P, i64, P, P, P, P, P, P]
        _lib.oracle_bin_decided.restype = i64
        _lib.oracle_set_threads.argtypes = [i32]
        _lib.oracle_get_threads.restype = i32
        assert _lib.oracle_layout() == NCOL * 100 + NGRAD, "oracle column layout mismatch"
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the oracle's per-pair and per-pixel loops (default 1,
    which reproduces results bit for bit; more threads change only the order
    of the backward's additions).  Returns the previous value."""
    prev = int(lib().oracle_get_threads())
    lib().oracle_set_threads(int(n))
    return prev


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def cameras(cams) -> ctypes.Array:
    """ctypes array of oracle cameras from scene Camera objects (float64 copies
    of the float32 values the GPU path receives, unless ``exact`` floats are
    already given)."""
    arr = (_Camera * max(1, len(cams)))()
    for i, c in enumerate(cams):
        T = np.asarray(c.T_cw, np.float64).reshape(12)
        arr[i].width, arr[i].height, arr[i].submap = int(c.width), int(c.height), int(c.submap)
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        for k in range(12):
            arr[i].T[k] = float(T[k])
    return arr


def as_float32_cameras(cams):
    """Copies of the cameras whose numbers are rounded to float32, so that the
    oracle sees exactly what the CUDA path sees."""
    import copy
    out = []
    for c in cams:
        c2 = copy.copy(c)
        c2.fx, c2.fy, c2.cx, c2.cy = (float(np.float32(x)) for x in (c.fx, c.fy, c.cx, c.cy))
        c2.T_cw = np.asarray(c.T_cw, np.float32).astype(np.float64)
        out.append(c2)
    return out


class Params:
    """Gaussian parameters as float64 arrays (widened from the float32 inputs)."""

    def __init__(self, means, log_scales, quats, opacity_logits, sh, sh_degree, submap_offsets):
        self.means = _d(means)
        self.log_scales = _d(log_scales)
        self.quats = _d(quats)
        self.opacity_logits = _d(opacity_logits)
        self.sh = _d(sh)
        self.sh_degree = int(sh_degree)
        self.submap_offsets = np.ascontiguousarray(np.asarray(submap_offsets, np.int64))

    @classmethod
    def from_scene(cls, s):
        return cls(s.means, s.log_scales, s.quats, s.opacity_logits, s.sh, s.sh_degree, s.submap_offsets)

    @property
    def n(self):
        return self.means.shape[0]

    def copy(self):
        return Params(self.means.copy(), self.log_scales.copy(), self.quats.copy(),
                      self.opacity_logits.copy(), self.sh.copy(), self.sh_degree,
                      self.submap_offsets.copy())


def n_pairs(cams, offsets) -> int:
    ca = cameras(cams)
    return int(lib().oracle_count_pairs(len(cams), ca, _p(np.asarray(offsets, np.int64))))


def n_tiles(cams, cfg: Config) -> int:
    cc = cfg.c()
    return int(lib().oracle_count_tiles(len(cams), cameras(cams), ctypes.byref(cc)))


def project(P: Params, cams, cfg: Config) -> np.ndarray:
    ca, cc = cameras(cams), cfg.c()
    n_p = n_pairs(cams, P.submap_offsets)
    rec = np.zeros((max(n_p, 1), NCOL), np.float64)
    lib().oracle_project(P.n, _p(P.means), _p(P.log_scales), _p(P.quats), _p(P.opacity_logits),
                         _p(P.sh), P.sh_degree, len(cams), ca, _p(P.submap_offsets),
                         ctypes.byref(cc), _p(rec))
    return rec[:n_p]


def bin(P: Params, cams, cfg: Config, rec: np.ndarray):
    """Returns (keys uint64 [I], vals int64 [I], ranges int64 [T,2])."""
    ca, cc = cameras(cams), cfg.c()
    rec = np.ascontiguousarray(rec)
    n_inst = int(lib().oracle_count_instances(rec.shape[0], _p(rec)))
    keys = np.zeros(max(n_inst, 1), np.uint64)
    vals = np.zeros(max(n_inst, 1), np.int64)
    T = n_tiles(cams, cfg)
    ranges = np.zeros((max(T, 1), 2), np.int64)
    lib().oracle_bin(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc), _p(rec), _p(keys),
                     _p(vals), _p(ranges))
    return keys[:n_inst], vals[:n_inst], ranges[:T]


def tile_decisions32(P: Params, cams, cfg: Config, rec32, rect, pkey):
    """The binning stage alone, from the float32 path's projection outputs
    (records [n_pairs][12] f32, rectangles [n_pairs][4] i16, depth keys
    [n_pairs] u32): R6b's decision for every rectangle tile of every visible
    pair, taken exactly from those float inputs, in emission order.  Returns
    (keep int8 [D], margin float64 [D]): |margin| of a few float ulps marks a
    decision a float32 evaluation may take the other way."""
    ca, cc = cameras(cams), cfg.c()
    rec32 = np.ascontiguousarray(rec32, np.float32).reshape(-1, 12)
    rect = np.ascontiguousarray(rect, np.int16).reshape(-1, 4)
    pkey = np.ascontiguousarray(pkey, np.uint32)
    n_p = rec32.shape[0]
    D = int(lib().oracle_rect_tiles32(n_p, _p(rect), _p(pkey)))
    dec = np.zeros(max(D, 1), np.int8)
    margin = np.zeros(max(D, 1))
    lib().oracle_tile_decisions32(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc), n_p, _p(rec32),
                                  _p(rect), _p(pkey), _p(dec), _p(margin))
    return dec[:D], margin[:D]


def bin_decided(P: Params, cams, cfg: Config, rect, pkey, dec):
    """Keys (uint64), pair of each instance (int64) and per-tile ranges [T, 2]
    of the stable key sort, from the float32 path's rectangles and depth keys
    and one keep decision per rectangle tile (emission order)."""
    ca, cc = cameras(cams), cfg.c()
    rect = np.ascontiguousarray(rect, np.int16).reshape(-1, 4)
    pkey = np.ascontiguousarray(pkey, np.uint32)
    dec = np.ascontiguousarray(dec, np.int8)
    n_keep = int(np.count_nonzero(dec))
    keys = np.zeros(max(n_keep, 1), np.uint64)
    vals = np.zeros(max(n_keep, 1), np.int64)
    T = n_tiles(cams, cfg)
    ranges = np.zeros((max(T, 1), 2), np.int64)
    m = lib().oracle_bin_decided(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc), rect.shape[0], _p(rect),
                                 _p(pkey), _p(dec), _p(keys), _p(vals), _p(ranges))
    assert m == n_keep
    return keys[:m], vals[:m], ranges[:T]


def _npix(cams):
    return int(sum(c.width * c.height for c in cams))


def render_fwd(P: Params, cams, cfg: Config, rec, vals, ranges) -> dict:
    ca, cc = cameras(cams), cfg.c()
    npx = _npix(cams)
    out = dict(rgb=np.zeros(3 * npx), depth=np.zeros(npx), alpha=np.zeros(npx), T=np.zeros(npx),
               last=np.zeros(npx, np.int64), nblend=np.zeros(npx, np.int64),
               margin=np.zeros(npx), sig=np.zeros(npx, np.uint64))
    vals = np.ascontiguousarray(vals, np.int64)
    ranges = np.ascontiguousarray(ranges, np.int64)
    lib().oracle_render_fwd(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc), _p(rec),
                            _p(vals), _p(ranges), _p(out["rgb"]), _p(out["depth"]),
                            _p(out["alpha"]), _p(out["T"]), _p(out["last"]), _p(out["nblend"]),
                            _p(out["margin"]), _p(out["sig"]))
    return out


def render_fwd_pixels(P: Params, cams, cfg: Config, rec, vals, ranges, pix) -> dict:
    """Tiled forward of the listed global pixel indices only."""
    ca, cc = cameras(cams), cfg.c()
    pix = np.ascontiguousarray(pix, np.int64)
    n = pix.size
    out = dict(rgb=np.zeros((max(n, 1), 3)), depth=np.zeros(max(n, 1)), alpha=np.zeros(max(n, 1)),
               T=np.zeros(max(n, 1)), last=np.zeros(max(n, 1), np.int64), margin=np.zeros(max(n, 1)))
    lib().oracle_render_fwd_pixels(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc),
                                   _p(np.ascontiguousarray(rec)), _p(np.ascontiguousarray(vals, np.int64)),
                                   _p(np.ascontiguousarray(ranges, np.int64)), n, _p(pix), _p(out["rgb"]),
                                   _p(out["depth"]), _p(out["alpha"]), _p(out["T"]), _p(out["last"]),
                                   _p(out["margin"]))
    return {k: v[:n] for k, v in out.items()}


def render_brute(P: Params, cams, cfg: Config, rec) -> dict:
    ca, cc = cameras(cams), cfg.c()
    npx = _npix(cams)
    out = dict(rgb=np.zeros(3 * npx), depth=np.zeros(npx), alpha=np.zeros(npx), T=np.zeros(npx),
               nblend=np.zeros(npx, np.int64), sig=np.zeros(npx, np.uint64))
    lib().oracle_render_brute(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc), _p(rec),
                              _p(out["rgb"]), _p(out["depth"]), _p(out["alpha"]), _p(out["T"]),
                              _p(out["nblend"]), _p(out["sig"]))
    return out


def render_depth_dist(P: Params, cams, cfg: Config, rec, vals, ranges):
    """(mean, var) per pixel: weighted mean and variance of the blended depths
    under the weights w = alpha T (reading R16 of the C file)."""
    ca, cc = cameras(cams), cfg.c()
    mean, var = np.zeros(_npix(cams)), np.zeros(_npix(cams))
    lib().oracle_render_depth_dist(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc),
                                   _p(np.ascontiguousarray(rec)), _p(np.ascontiguousarray(vals, np.int64)),
                                   _p(np.ascontiguousarray(ranges, np.int64)), _p(mean), _p(var))
    return mean, var


def depth_loss_var(P: Params, cams, cfg: Config, alpha, mean, var, lidar, sigma_L=0.05, sigma_U=0.05, lam=1.0):
    """Eq. (7) with the rendered depth distribution. Returns (loss, g_mean, g_var, n_valid)."""
    ca, cc = cameras(cams), cfg.c()
    alpha, mean, var = _d(alpha), _d(mean), _d(var)
    lid = _d(lidar).reshape(-1, 4)
    g = [np.zeros_like(mean) for _ in range(2)]
    nv = ctypes.c_int64(0)
    loss = lib().oracle_depth_loss_var(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc), _p(alpha),
                                       _p(mean), _p(var), lid.shape[0], _p(lid),
                                       float(np.float32(sigma_L)), float(np.float32(sigma_U)),
                                       float(np.float32(lam)), *(_p(x) for x in g), ctypes.byref(nv))
    return (loss, *g, int(nv.value))


def render_bwd(P: Params, cams, cfg: Config, rec, vals, ranges, dC, dD, dA=None, dmean=None, dvar=None) -> dict:
    ca, cc = cameras(cams), cfg.c()
    K = (P.sh_degree + 1) ** 2
    n_p = rec.shape[0]
    g = dict(g2d=np.zeros((max(n_p, 1), NGRAD)), means=np.zeros((P.n, 3)),
             log_scales=np.zeros((P.n, 3)), quats=np.zeros((P.n, 4)),
             opacity_logits=np.zeros(P.n), sh=np.zeros((P.n, K, 3)),
             pose=np.zeros((len(cams), 6)), dens_acc=np.zeros(P.n), dens_cnt=np.zeros(P.n))
    dC, dD = _d(dC), _d(dD)
    opt = [(_d(x) if x is not None else None) for x in (dA, dmean, dvar)]
    dAp, dmp, dvp = (_p(x) if x is not None else None for x in opt)
    lib().oracle_render_bwd(P.n, _p(P.means), _p(P.log_scales), _p(P.quats),
                            _p(P.opacity_logits), _p(P.sh), P.sh_degree, len(cams), ca,
                            _p(P.submap_offsets), ctypes.byref(cc), _p(np.ascontiguousarray(rec)),
                            _p(np.ascontiguousarray(vals, np.int64)),
                            _p(np.ascontiguousarray(ranges, np.int64)), _p(dC), _p(dD), dAp, dmp, dvp,
                            _p(g["g2d"]), _p(g["means"]), _p(g["log_scales"]), _p(g["quats"]),
                            _p(g["opacity_logits"]), _p(g["sh"]), _p(g["pose"]),
                            _p(g["dens_acc"]), _p(g["dens_cnt"]))
    g["g2d"] = g["g2d"][:n_p]
    return g


def image_l1(C, I):
    C, I = _d(C).ravel(), _d(I).ravel()
    grad = np.zeros_like(C)
    loss = lib().oracle_image_l1(C.size, _p(C), _p(I), _p(grad))
    return loss, grad


def ssim(cams, C, I, grad=True):
    """Mean SSIM (reading R17 of the C file) of planar images C against I laid
    out like the renderer's RGB output; returns (mean SSIM, d mean / dC or None)."""
    C, I = _d(C).ravel(), _d(I).ravel()
    g = np.zeros_like(C) if grad else None
    val = lib().oracle_ssim(len(cams), cameras(cams), _p(C), _p(I), _p(g) if grad else None)
    return val, g


def image_loss(cams, C, I, lam):
    """Eq. (6): (1 - lam) mean|C - I| + lam (1 - mean SSIM); returns (loss, dL/dC)."""
    l1, g1 = image_l1(C, I)
    s, gs = ssim(cams, C, I)
    return (1.0 - lam) * l1 + lam * (1.0 - s), (1.0 - lam) * g1 - lam * gs


def kl_normal(m1, s1, m2, s2) -> float:
    return float(lib().oracle_kl_normal(m1, s1, m2, s2))


def depth_loss(P: Params, cams, cfg: Config, depth, alpha, lidar, mode=0, sigma_L=0.05,
               sigma_U=0.05, lam=1.0):
    ca, cc = cameras(cams), cfg.c()
    depth, alpha, lid = _d(depth), _d(alpha), _d(lidar).reshape(-1, 4)
    grad = np.zeros_like(depth)
    nv = ctypes.c_int64(0)
    loss = lib().oracle_depth_loss(len(cams), ca, _p(P.submap_offsets), ctypes.byref(cc),
                                   _p(depth), _p(alpha), lid.shape[0], _p(lid), int(mode),
                                   float(np.float32(sigma_L)), float(np.float32(sigma_U)),
                                   float(np.float32(lam)), _p(grad), ctypes.byref(nv))
    return loss, grad, int(nv.value)


def cov3d(quat, log_scale) -> np.ndarray:
    S = np.zeros(9)
    lib().oracle_cov3d(_p(_d(quat)), _p(_d(log_scale)), _p(S))
    return S.reshape(3, 3)


def sh_basis(deg: int, d) -> np.ndarray:
    Y = np.zeros(16)
    lib().oracle_sh_basis(int(deg), _p(_d(d)), _p(Y))
    return Y[:(deg + 1) ** 2]


def forward(P: Params, cams, cfg: Config):
    """project -> bin -> tiled forward. Returns (rec, keys, vals, ranges, out)."""
    rec = project(P, cams, cfg)
    keys, vals, ranges = bin(P, cams, cfg, rec)
    out = render_fwd(P, cams, cfg, rec, vals, ranges)
    return rec, keys, vals, ranges, out


def linear_loss(P: Params, cams, cfg: Config, wC, wD, wA):
    """sum(wC*C) + sum(wD*D) + sum(wA*A): a linear functional of the images whose
    gradient w.r.t. (C, D, A) is (wC, wD, wA)."""
    rec, keys, vals, ranges, out = forward(P, cams, cfg)
    L = float(np.dot(wC, out["rgb"]) + np.dot(wD, out["depth"]) + np.dot(wA, out["alpha"]))
    return L, out
