"""Pose refinement at its own workload (Sec. III-C: the pose is refined by
gradients back-propagated through the projection): the 1M-Gaussian orchard
seen by four 1440x1080 cameras, each pose perturbed by seeded SE(3) noise
(0.05 m, 1 degree), every camera cropped to a 64x48 window on both sides.
The CUDA path's gradients of every Gaussian parameter and of all 24 pose
twists against the FP64 oracle's analytic adjoint, at 1e-4 relative L2 per
tensor; the binning stage bit for bit; images within 1e-5."""
import os

import numpy as np
import pytest

import oracle as O
from tests.gpu_helpers import check_binning_stage, pixel_weights, rel_l2, run_gpu, run_oracle
from tests.rig_crop import pose_rig_crop

pytestmark = pytest.mark.gpu

MARGIN = 1e-4


@pytest.fixture(scope="module")
def rig():
    sc = pose_rig_crop()
    ocfg = O.Config()
    prev = O.set_threads(os.cpu_count() or 1)
    try:
        P, cams, rec, keys, vals, ranges, out = run_oracle(sc, ocfg)
        keep = out["margin"] > MARGIN
        rng = np.random.default_rng(13)
        rgbmask, pmask = pixel_weights(sc, keep)
        gC = rng.normal(size=3 * sc.n_pix) * rgbmask
        gD = 0.1 * rng.normal(size=sc.n_pix) * pmask
        gA = rng.normal(size=sc.n_pix) * pmask
        g = run_gpu(sc, ocfg, gC, gD, gA)
        go = O.render_bwd(P, cams, ocfg, rec, vals, ranges, gC, gD, gA)
    finally:
        O.set_threads(prev)
    yield dict(sc=sc, ocfg=ocfg, P=P, cams=cams, rec=rec, out=out, keep=keep, g=g, go=go)
    g["renderer"].close()


def test_pose_rig_images_and_binning(rig):
    sc, g, out, keep = rig["sc"], rig["g"], rig["out"], rig["keep"]
    assert g["status"] == 0 and g["n_vis"] > 10_000
    n_dec, n_band = check_binning_stage(sc, rig["ocfg"], g, rig["P"], rig["cams"])
    rgbmask, pmask = pixel_weights(sc, keep)
    e_rgb = np.abs(g["rgb"].astype(np.float64) - out["rgb"])[rgbmask].max()
    e_d = np.abs(g["depth"].astype(np.float64) - out["depth"])[pmask].max()
    e_a = np.abs(g["alpha"].astype(np.float64) - out["alpha"])[pmask].max()
    print(f"pose rig crop: {g['n_vis']} visible pairs, {n_band} of {n_dec} tile decisions in the float band; "
          f"excluded pixels {(~keep).sum()}; rgb {e_rgb:.2e} depth {e_d:.2e} alpha {e_a:.2e}")
    assert e_rgb <= 1e-5 and e_d <= 1e-5 and e_a <= 1e-5


def test_pose_rig_gradients(rig):
    g, go = rig["g"], rig["go"]
    res = {k: rel_l2(g["g_" + k], go[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose")}
    print("pose rig crop gradients: " + " ".join(f"{k} {v:.1e}" for k, v in res.items()))
    assert g["g_pose"].shape == (4, 6) and np.all(np.abs(go["pose"]) > 0)
    for k, v in res.items():
        assert v <= 1e-4, (k, v)
    # every twist component on its own, relative to its camera's twist
    for v in range(4):
        gv, ov = g["g_pose"][v].astype(np.float64), go["pose"][v]
        assert np.linalg.norm(gv - ov) <= 1e-4 * np.linalg.norm(ov), (v, gv, ov)
