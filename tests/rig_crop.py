"""The pose-refinement workload (1M Gaussians, four perturbed 1440x1080
cameras) restricted to a 64x48 window of every camera, for checks whose
FP64 side composites every pixel.  Each window is the 64x48 cell of the
camera's image where the most Gaussian means project, so that every crop
sees trees (the forward and rear cameras look down an empty lane at their
principal point)."""
from __future__ import annotations

import copy

import numpy as np

from paper_2510_26358_gb300 import scenes as S

CROP_W, CROP_H = 64, 48


def busiest_window(sc, cam, w=CROP_W, h=CROP_H):
    """(x0, y0) of the w x h cell (on a grid of such cells) holding the most
    projected Gaussian means in front of the camera."""
    T = np.asarray(cam.T_cw, np.float64)
    p = sc.means.astype(np.float64) @ T[:, :3].T + T[:, 3]
    front = p[:, 2] > 0.5
    u = cam.fx * p[front, 0] / p[front, 2] + cam.cx
    v = cam.fy * p[front, 1] / p[front, 2] + cam.cy
    inside = (u >= 0) & (u < cam.width) & (v >= 0) & (v < cam.height)
    gx, gy = cam.width // w, cam.height // h
    cell = (np.minimum(v[inside] // h, gy - 1).astype(np.int64) * gx +
            np.minimum(u[inside] // w, gx - 1).astype(np.int64))
    best = int(np.argmax(np.bincount(cell, minlength=gx * gy)))
    return (best % gx) * w, (best // gx) * h


def pose_rig_crop(lidar=False):
    """orchard1m_pose with every camera cropped to its busiest 64x48 window."""
    sc = S.workload("orchard1m_pose", lidar=lidar)
    out = copy.copy(sc)
    out.cameras = [c.crop(*busiest_window(sc, c), CROP_W, CROP_H) for c in sc.cameras]
    rng = np.random.Generator(np.random.PCG64(31))
    out.target = rng.random(3 * out.n_pix, dtype=np.float32)
    out.lidar = np.zeros((0, 4), np.float32)
    out.name = "orchard1m_pose_crop64x48"
    return out


def visible_subset(sc, gauss):
    """The scene restricted to the Gaussians `gauss` (sorted indices of one
    submap scene), same cameras."""
    g = np.asarray(gauss, np.int64)
    out = copy.copy(sc)
    out.means, out.log_scales, out.quats = sc.means[g], sc.log_scales[g], sc.quats[g]
    out.opacity_logits, out.sh = sc.opacity_logits[g], sc.sh[g]
    out.submap_offsets = np.array([0, len(g)], np.int64)
    return out
