"""Seeded synthetic inputs for the multi-view Gaussian-splatting hot path.

This module only draws inputs: Gaussian parameters, camera rigs, LiDAR returns
and target images. It holds none of the renderer's arithmetic, and both the
CUDA path and the FP64 oracle consume what it returns.

The paper evaluates on private apple/pear orchard recordings (Sec. IV) that are
not available, so orchard-shaped scenes stand in for them: rows of trees,
each a thin vertical trunk of elongated Gaussians under a ball-shaped canopy of
small Gaussians, seen by a rig of one forward and two lateral cameras (the
platform of Fig. 2) plus a 32-beam spinning LiDAR. Every array is drawn from
``numpy.random.Generator(PCG64(seed))``.

Conventions shared with the rest of the package:
  * Gaussians: ``means`` [N,3], ``log_scales`` [N,3], ``quats`` [N,4] (w,x,y,z,
    not necessarily unit), ``opacity_logits`` [N], ``sh`` [N,K,3] with
    K=(degree+1)^2, all float32 and C-contiguous.
  * Submaps: ``submap_offsets`` int64 [S+1]; Gaussians of submap s are
    ``offsets[s]:offsets[s+1]``.
  * Cameras: OpenCV axes (x right, y down, z forward); ``T_cw`` is the
    row-major 3x4 world-to-camera transform [R | t].
  * LiDAR: float32 [M,4] rows (u, v, z, view) with (u,v) in pixels of view
    ``view`` and z the camera-frame depth of the return.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# DC basis value of the real spherical harmonics, 1/(2*sqrt(pi)); used only to
# turn the configs' "RGB uniform in [0,1]" into a degree-0 coefficient.
_SH_DC = 0.5 / math.sqrt(math.pi)


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    T_cw: np.ndarray            # float64 [3,4], world -> camera
    submap: int = 0

    def crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """Same camera restricted to the pixel window [x0,x0+w) x [y0,y0+h)."""
        return Camera(w, h, self.fx, self.fy, self.cx - x0, self.cy - y0,
                      self.T_cw.copy(), self.submap)


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    submap_offsets: np.ndarray
    cameras: list
    lidar: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.float32))
    target: np.ndarray | None = None     # planar RGB targets, float32 [sum 3*H*W]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_pix(self) -> int:
        return int(sum(c.width * c.height for c in self.cameras))


# ----------------------------------------------------------------------------
# rigid-body helpers (input construction only)
# ----------------------------------------------------------------------------

def _rot_axis(axis: str, deg: float) -> np.ndarray:
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    if axis == "x":
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], np.float64)
    if axis == "y":
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], np.float64)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], np.float64)


def _so3_exp(w: np.ndarray) -> np.ndarray:
    th = float(np.linalg.norm(w))
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]], np.float64)
    if th < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * (K @ K)


def look_camera(center, forward, width, height, f_ratio=0.9375, submap=0) -> Camera:
    """Pinhole camera at ``center`` looking along world ``forward`` with world +z up.

    f = f_ratio * width (0.9375 is the 300 px / 320 px ratio of the small
    single-camera workload); principal point at the image centre.
    """
    c = np.asarray(center, np.float64)
    zc = np.asarray(forward, np.float64)
    zc = zc / np.linalg.norm(zc)
    up = np.array([0.0, 0.0, 1.0])
    xc = np.cross(zc, up)
    xc /= np.linalg.norm(xc)
    yc = np.cross(zc, xc)
    R_wc = np.stack([xc, yc, zc], axis=1)           # camera axes in world coords
    R_cw = R_wc.T
    T = np.concatenate([R_cw, (-R_cw @ c)[:, None]], axis=1)
    f = f_ratio * width
    return Camera(width, height, f, f, width / 2.0, height / 2.0, T, submap)


def perturb_pose(cam: Camera, rng: np.random.Generator, sigma_t=0.05, sigma_deg=1.0) -> Camera:
    """Left-multiply the pose by exp of seeded SE(3) noise (translation N(0,sigma_t^2)
    per axis in metres, rotation N(0,sigma_deg^2) per axis in degrees)."""
    dt = rng.normal(0.0, sigma_t, 3)
    dw = np.radians(rng.normal(0.0, sigma_deg, 3))
    dR = _so3_exp(dw)
    R = dR @ cam.T_cw[:, :3]
    t = dR @ cam.T_cw[:, 3] + dt
    return Camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                  np.concatenate([R, t[:, None]], axis=1), cam.submap)


def _unit_quats(rng, n) -> np.ndarray:
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


# ----------------------------------------------------------------------------
# workload 1: random box scene, one 320x240 camera
# ----------------------------------------------------------------------------

def random_box_scene(n=10_000, width=320, height=240, f=300.0, seed=0,
                     sh_degree=0, box=((-2, 2), (-1.5, 1.5), (1, 7)),
                     log_scale_mu=-3.0, log_scale_sd=0.5) -> Scene:
    """Means uniform in a box in front of an identity camera, log-scales
    N(mu, sd), unit quaternions from normalised N(0,1)^4, opacity logits N(0,1),
    degree-0 colour uniform in [0,1] (higher degrees: extra coefficients
    N(0,0.2)); random planar RGB target uniform in [0,1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.array([b[0] for b in box], np.float64)
    hi = np.array([b[1] for b in box], np.float64)
    means = lo + (hi - lo) * rng.random((n, 3))
    log_scales = rng.normal(log_scale_mu, log_scale_sd, (n, 3))
    quats = _unit_quats(rng, n)
    opac = rng.normal(0.0, 1.0, n)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    rgb = rng.random((n, 3))
    sh[:, 0, :] = (rgb - 0.5) / _SH_DC
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.2, (n, K - 1, 3))
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0,
                 np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1), 0)
    target = rng.random(3 * width * height).astype(np.float32)
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), opac.astype(np.float32),
                 sh.astype(np.float32), sh_degree,
                 np.array([0, n], np.int64), [cam], target=target,
                 name=f"box{n}_{width}x{height}")


def needle_scene(n=4_000, width=160, height=120, f=150.0, seed=6, long_log_scale=(-2.2, -0.8),
                 thin_log_scale=(-6.0, -5.0)) -> Scene:
    """The box scene with needle-shaped Gaussians: one axis log-uniform in
    `long_log_scale`, the other two in `thin_log_scale` (below the pixel, so
    the image covariance is a long ellipse about as wide as the dilation),
    random orientations.  Their tile rectangles are mostly corners the
    ellipse misses, and their image covariances are badly conditioned."""
    sc = random_box_scene(n, width, height, f, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    ls = np.empty((n, 3))
    ls[:, 0] = rng.uniform(*long_log_scale, n)
    ls[:, 1:] = rng.uniform(*thin_log_scale, (n, 2))
    sc.log_scales = ls.astype(np.float32)
    sc.name = f"needles{n}_{width}x{height}"
    return sc


# ----------------------------------------------------------------------------
# orchard scenes
# ----------------------------------------------------------------------------

TRUNK_PER_TREE = 2_000
CANOPY_PER_TREE = 20_000
TRUNK_RADIUS = 0.08
TRUNK_HEIGHT = 1.0
CANOPY_RADIUS = 1.2
CANOPY_CENTER_Z = 2.2
ROW_SPACING = 3.5
TREE_SPACING = 1.5
RIG_HEIGHT = 1.2
LIDAR_HEIGHT = 1.5


def orchard_trees(n_rows: int, trees_per_row: int, x0=0.0, y0=None):
    """Tree base positions: rows along +x, ROW_SPACING apart, centred on y=0."""
    if y0 is None:
        y0 = -ROW_SPACING * (n_rows - 1) / 2.0
    xs = x0 + TREE_SPACING * np.arange(trees_per_row)
    ys = y0 + ROW_SPACING * np.arange(n_rows)
    return np.array([(x, y) for y in ys for x in xs], np.float64)


def orchard_gaussians(rng, trees: np.ndarray, n_total: int, sh_degree=3,
                      canopy_ratio=CANOPY_PER_TREE / TRUNK_PER_TREE):
    """Trunk cylinders of elongated axis-aligned Gaussians plus canopy balls of
    small randomly oriented Gaussians; per-tree counts keep the trunk:canopy
    ratio and are scaled so the total is exactly ``n_total`` (remainder to the
    last tree)."""
    n_trees = len(trees)
    per_tree = n_total // n_trees
    counts = np.full(n_trees, per_tree, np.int64)
    counts[-1] += n_total - per_tree * n_trees
    means, ls, qs = [], [], []
    for (tx, ty), cnt in zip(trees, counts):
        n_trunk = int(round(cnt / (1.0 + canopy_ratio)))
        n_can = int(cnt) - n_trunk
        ang = rng.random(n_trunk) * 2 * math.pi
        h = rng.random(n_trunk) * TRUNK_HEIGHT
        means.append(np.stack([tx + TRUNK_RADIUS * np.cos(ang),
                               ty + TRUNK_RADIUS * np.sin(ang), h], 1))
        ls.append(np.array([-4.5, -4.5, -2.5]) + rng.normal(0.0, 0.2, (n_trunk, 3)))
        qs.append(np.tile([1.0, 0.0, 0.0, 0.0], (n_trunk, 1)))
        d = rng.normal(0.0, 1.0, (n_can, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        r = CANOPY_RADIUS * rng.random(n_can) ** (1.0 / 3.0)
        means.append(np.array([tx, ty, CANOPY_CENTER_Z]) + d * r[:, None])
        ls.append(rng.normal(-4.0, 0.6, (n_can, 3)))
        qs.append(_unit_quats(rng, n_can))
    means = np.concatenate(means)
    K = (sh_degree + 1) ** 2
    return dict(means=means, log_scales=np.concatenate(ls), quats=np.concatenate(qs),
                opacity_logits=rng.normal(0.0, 1.0, n_total),
                sh=rng.normal(0.0, 0.2, (n_total, K, 3)))


def rig_cameras(x, y, width, height, rear=False, submap=0, z=RIG_HEIGHT):
    """One forward (+x) and two lateral (+y, -y) cameras at (x, y, z); optionally
    a rear (-x) camera."""
    cams = [look_camera((x, y, z), (1, 0, 0), width, height, submap=submap),
            look_camera((x, y, z), (0, 1, 0), width, height, submap=submap),
            look_camera((x, y, z), (0, -1, 0), width, height, submap=submap)]
    if rear:
        cams.append(look_camera((x, y, z), (-1, 0, 0), width, height, submap=submap))
    return cams


def _ray_hits(origin, dirs, trees):
    """Nearest analytic hit of each ray with the trunk cylinders and canopy balls
    (inf where nothing is hit). Returns distances along the unit rays."""
    best = np.full(len(dirs), np.inf)
    o = np.asarray(origin, np.float64)
    for tx, ty in trees:
        # canopy ball
        c = np.array([tx, ty, CANOPY_CENTER_Z])
        oc = o - c
        b = dirs @ oc
        cc = oc @ oc - CANOPY_RADIUS ** 2
        disc = b * b - cc
        ok = disc >= 0
        s = np.sqrt(np.where(ok, disc, 0.0))
        t = -b - s
        t = np.where(t > 1e-6, t, -b + s)
        hit = ok & (t > 1e-6)
        best = np.where(hit & (t < best), t, best)
        # vertical trunk cylinder, z in [0, TRUNK_HEIGHT]
        dx, dy = dirs[:, 0], dirs[:, 1]
        ox, oy = o[0] - tx, o[1] - ty
        A = dx * dx + dy * dy
        B = 2 * (ox * dx + oy * dy)
        C = ox * ox + oy * oy - TRUNK_RADIUS ** 2
        disc = B * B - 4 * A * C
        ok = (disc >= 0) & (A > 1e-12)
        s = np.sqrt(np.where(ok, disc, 0.0))
        t = (-B - s) / np.where(A > 1e-12, 2 * A, 1.0)
        zc = o[2] + t * dirs[:, 2]
        hit = ok & (t > 1e-6) & (zc >= 0) & (zc <= TRUNK_HEIGHT)
        best = np.where(hit & (t < best), t, best)
    return best


def _scan_hits(origin, dirs, n_beams, az, trees):
    """_ray_hits over a beams x azimuths grid of rays (row-major), testing each
    tree only against the azimuths that can reach it: a tree's trunk and
    canopy lie inside the vertical cylinder of radius CANOPY_RADIUS about its
    axis, which a ray from ``origin`` meets only within asin(R / d) of the
    tree's bearing (d the horizontal distance; every azimuth when d <= R).
    The window is widened by 1e-3 rad, so every ray that hits the tree is
    tested, and the nearest hit of each ray is the same as testing all trees."""
    n_az = len(az)
    best = np.full(len(dirs), np.inf)
    o = np.asarray(origin, np.float64)
    step = 2 * math.pi / n_az
    beam_base = (np.arange(n_beams) * n_az)[:, None]
    for tree in trees:
        dx, dy = tree[0] - o[0], tree[1] - o[1]
        d = math.hypot(dx, dy)
        if d <= CANOPY_RADIUS + 1e-6:
            sel = np.arange(len(dirs))
        else:
            half = math.asin(CANOPY_RADIUS / d) + 1e-3
            c = math.atan2(dy, dx)
            k0 = int(math.floor((c - half) / step))
            k1 = int(math.ceil((c + half) / step))
            ks = np.unique(np.arange(k0, k1 + 1) % n_az)
            sel = (beam_base + ks[None, :]).ravel()
        t = _ray_hits(o, dirs[sel], np.asarray([tree]))
        best[sel] = np.minimum(best[sel], t)
    return best


def lidar_scan(rng, origin, trees, cameras, per_view, n_beams=32,
               elev=(-25.0, 15.0), n_az=2048, max_az=65536, near=0.2):
    """32-beam spinning scan from ``origin`` ray-cast against the trunk
    cylinders and canopy balls; the returns are expressed in each camera and
    ``per_view`` of those falling inside the image are kept (seeded sample).
    The azimuth resolution doubles until every view has ``per_view`` returns or
    ``max_az`` is reached; the count actually kept per view is recorded."""
    elevs = np.radians(np.linspace(elev[0], elev[1], n_beams))
    # only trees within LiDAR range matter
    rel = trees - np.asarray(origin[:2])
    near_trees = trees[np.hypot(rel[:, 0], rel[:, 1]) < 40.0]
    while True:
        az = np.linspace(0, 2 * math.pi, n_az, endpoint=False)
        E, Az = np.meshgrid(elevs, az, indexing="ij")
        dirs = np.stack([np.cos(E) * np.cos(Az), np.cos(E) * np.sin(Az), np.sin(E)], -1).reshape(-1, 3)
        dist = _scan_hits(origin, dirs, n_beams, az, near_trees)
        ok = np.isfinite(dist)
        pts = np.asarray(origin)[None, :] + dirs[ok] * dist[ok, None]
        per_cam = []
        for v, cam in enumerate(cameras):
            pc = pts @ cam.T_cw[:, :3].T + cam.T_cw[:, 3]
            z = pc[:, 2]
            front = z > near
            u = cam.fx * pc[front, 0] / z[front] + cam.cx
            vv = cam.fy * pc[front, 1] / z[front] + cam.cy
            inside = (u >= 0) & (u < cam.width) & (vv >= 0) & (vv < cam.height)
            per_cam.append(np.stack([u[inside], vv[inside], z[front][inside],
                                     np.full(int(inside.sum()), v, np.float64)], 1))
        if min(len(p) for p in per_cam) >= per_view or n_az >= max_az:
            break
        n_az *= 2
    out, kept = [], []
    for p in per_cam:
        k = min(per_view, len(p))
        sel = rng.choice(len(p), size=k, replace=False) if k < len(p) else np.arange(len(p))
        out.append(p[np.sort(sel)])
        kept.append(int(k))
    return np.concatenate(out).astype(np.float32), dict(n_az=n_az, kept=kept)


def _pack(parts: list, sh_degree: int, cameras, offsets, rng, lidar, name, meta) -> Scene:
    cat = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    n_pix3 = 3 * sum(c.width * c.height for c in cameras)
    return Scene(cat["means"].astype(np.float32), cat["log_scales"].astype(np.float32),
                 cat["quats"].astype(np.float32), cat["opacity_logits"].astype(np.float32),
                 cat["sh"].astype(np.float32), sh_degree,
                 np.asarray(offsets, np.int64), cameras, lidar=lidar,
                 target=rng.random(n_pix3, dtype=np.float32), name=name, meta=meta)


def orchard_scene(n_total=500_000, n_rows=3, trees_per_row=8, width=1280, height=720,
                  rear=False, lanes=1, lidar_per_view=20_000, pose_noise=False,
                  sh_degree=3, seed=0, name=None) -> Scene:
    """Orchard workload: ``n_rows`` rows of ``trees_per_row`` trees, ``n_total``
    Gaussians, a 3-camera rig (4 with ``rear``) per lane at mid-row, LiDAR
    returns per view from a 32-beam scan at each rig."""
    rng = np.random.Generator(np.random.PCG64(seed))
    trees = orchard_trees(n_rows, trees_per_row)
    g = orchard_gaussians(rng, trees, n_total, sh_degree)
    x_mid = TREE_SPACING * (trees_per_row - 1) / 2.0
    row_ys = sorted(set(trees[:, 1]))
    lane_ys = [(row_ys[i] + row_ys[i + 1]) / 2 for i in range(len(row_ys) - 1)]
    mid = len(lane_ys) // 2
    lane_sel = lane_ys[mid:mid + lanes] if lanes <= len(lane_ys) - mid else lane_ys[:lanes]
    cams, lid, meta = [], [], dict(lanes=lane_sel, lidar=[])
    for ly in lane_sel:
        rig = rig_cameras(x_mid, ly, width, height, rear=rear)
        if pose_noise:
            rig = [perturb_pose(c, rng) for c in rig]
        base = len(cams)
        cams += rig
        if lidar_per_view:
            pts, info = lidar_scan(rng, (x_mid, ly, LIDAR_HEIGHT), trees, rig, lidar_per_view)
            pts[:, 3] += base
            lid.append(pts)
            meta["lidar"].append(info)
    lidar = np.concatenate(lid) if lid else np.zeros((0, 4), np.float32)
    return _pack([g], sh_degree, cams, [0, n_total], rng, lidar,
                 name or f"orchard{n_total}_{len(cams)}x{width}x{height}", meta)


def uneven_submaps(n_submaps=8, n_lo=50_000, n_hi=2_000_000, lidar_per_view=0,
                   sh_degree=3, seed=0, scale=1.0,
                   resolutions=((640, 480), (1280, 720), (1920, 1080))) -> Scene:
    """Several submaps with log-uniform Gaussian counts, each an orchard chunk of
    3 rows whose length grows with its count, each seen by its own 3-camera rig
    with a resolution drawn from ``resolutions``. ``scale`` shrinks counts and
    resolutions together for small test cases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_submaps)) * scale).astype(np.int64)
    counts = np.maximum(counts, 1)
    parts, cams, offs, x0, lid = [], [], [0], 0.0, []
    for s, cnt in enumerate(counts):
        tpr = int(max(2, round(cnt / (3 * (TRUNK_PER_TREE + CANOPY_PER_TREE)))))
        trees = orchard_trees(3, tpr, x0=x0)
        parts.append(orchard_gaussians(rng, trees, int(cnt), sh_degree))
        W, H = resolutions[rng.integers(len(resolutions))]
        W, H = max(16, int(round(W * math.sqrt(scale)))), max(16, int(round(H * math.sqrt(scale))))
        x_mid = x0 + TREE_SPACING * (tpr - 1) / 2.0
        rig = rig_cameras(x_mid, ROW_SPACING / 2.0, W, H, submap=s)
        if lidar_per_view:
            pts, _ = lidar_scan(rng, (x_mid, ROW_SPACING / 2.0, LIDAR_HEIGHT), trees, rig, lidar_per_view)
            pts[:, 3] += len(cams)
            lid.append(pts)
        cams += rig
        offs.append(offs[-1] + int(cnt))
        x0 += TREE_SPACING * tpr + 10.0
    lidar = np.concatenate(lid) if lid else np.zeros((0, 4), np.float32)
    return _pack(parts, sh_degree, cams, offs, rng, lidar, f"submaps{n_submaps}_{offs[-1]}",
                 dict(counts=counts.tolist()))


# ----------------------------------------------------------------------------
# named workloads (the five sizes the benchmark and tests are built around)
# ----------------------------------------------------------------------------

def workload(name: str, seed: int = 0, lidar: bool = True) -> Scene:
    """The named workloads; ``lidar=False`` skips the LiDAR scan (tests that
    only check rendering)."""
    L = lambda k: k if lidar else 0
    if name == "box10k":            # single 320x240 camera, 10k Gaussians, SH 0
        return random_box_scene(10_000, seed=seed)
    if name == "orchard500k":       # 3 rows x 8 trees, 3 x 1280x720, SH 3, 20k LiDAR/view
        return orchard_scene(500_000, 3, 8, 1280, 720, lidar_per_view=L(20_000), seed=seed, name=name)
    if name == "orchard1m_pose":    # 3 rows x 16 trees, 4 x 1440x1080, perturbed poses
        return orchard_scene(1_000_000, 3, 16, 1440, 1080, rear=True, pose_noise=True,
                             lidar_per_view=L(20_000), seed=seed, name=name)
    if name == "submaps8":          # 8 submaps log-U[50k,2M], 24 views of mixed size
        return uneven_submaps(8, seed=seed, lidar_per_view=L(20_000))
    if name == "orchard4m":         # 9 rows x 27 trees, 6 x 1920x1200, 100k LiDAR/view
        return orchard_scene(4_000_000, 9, 27, 1920, 1200, lanes=2,
                             lidar_per_view=L(100_000), seed=seed, name=name)
    raise KeyError(name)


WORKLOADS = ("box10k", "orchard500k", "orchard1m_pose", "submaps8", "orchard4m")
