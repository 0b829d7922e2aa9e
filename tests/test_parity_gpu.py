"""CUDA path vs the FP64 oracle, element by element, on seeded scenes.

Tolerances (from the benchmark spec of the method's bar):
  * sort keys, instance order and tile ranges: bit-exact;
  * forward images: within 1e-5 absolute;
  * gradients: within 1e-4 relative (per-tensor L2).
Pixels where the oracle sees a discrete decision (alpha >= 1/255, the T stop)
within MARGIN of its threshold are left out of the image comparison and
counted; their upstream gradients are zeroed on both sides.  The binning is
checked as a stage: the oracle bins the CUDA path's own float32 projection
outputs, so that keys, instance order and ranges compare bit for bit (tile
decisions within a few float ulps of their threshold take the CUDA path's
side, and are counted).
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_26358_gb300 import scenes as S
from tests.gpu_helpers import (check_binning_stage, decode_records, end_to_end_key_mismatch, pixel_weights, rel_l2,
                               run_gpu, run_oracle)

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
GRAD_TOL = 1e-4
MARGIN = 1e-4


def _overlap_scene(n=8_000, deg=3, seed=3):
    """Box scene seen by three cameras with overlapping frusta (the first
    camera and two seeded perturbations of it), so that many Gaussians are
    seen by several views."""
    sc = S.random_box_scene(n, 160, 120, 150.0, seed=seed, sh_degree=deg)
    rng = np.random.default_rng(seed)
    cam0 = sc.cameras[0]
    sc.cameras = [cam0] + [S.perturb_pose(cam0, rng, sigma_t=0.15, sigma_deg=4.0) for _ in range(2)]
    sc.target = rng.random(3 * sum(c.width * c.height for c in sc.cameras)).astype(np.float32)
    sc.name = f"box_overlap_deg{deg}"
    return sc


def _scenes():
    return {
        "box_overlap": _overlap_scene(),
        # the other SH degrees of the projection and SH adjoint kernels
        "box_overlap_deg1": _overlap_scene(3_000, 1, 4),
        "box_overlap_deg2": _overlap_scene(3_000, 2, 5),
        "box10k": S.random_box_scene(10_000, 320, 240, 300.0, seed=0),
        "orchard_rig": S.orchard_scene(40_000, 3, 4, 200, 120, rear=True, pose_noise=True,
                                       lidar_per_view=3000, seed=1, name="orchard_rig"),
        "submaps": S.uneven_submaps(4, 3000, 30000, seed=2, scale=1.0,
                                    resolutions=((96, 64), (160, 96), (128, 128))),
        # long thin ellipses: most rectangle tiles dropped, badly conditioned covariances
        "needles": S.needle_scene(),
    }


SCENES = _scenes()

# Known precision gaps (none at present): (test name, scene) -> reason, run
# as strict xfails so that a fix shows as a pass.
KNOWN_GAPS = {}


def _known_gap(request, case):
    reason = KNOWN_GAPS.get((request.node.originalname, case["name"]))
    if reason:
        request.node.add_marker(pytest.mark.xfail(strict=True, reason=reason))


@pytest.fixture(scope="module", params=list(SCENES))
def case(request):
    sc = SCENES[request.param]
    ocfg = O.Config()
    P, cams, rec, keys, vals, ranges, out = run_oracle(sc, ocfg)
    keep = out["margin"] > MARGIN
    rng = np.random.default_rng(7)
    rgbmask, pmask = pixel_weights(sc, keep)
    gC = rng.normal(size=3 * sc.n_pix) * rgbmask
    gD = 0.1 * rng.normal(size=sc.n_pix) * pmask
    gA = rng.normal(size=sc.n_pix) * pmask
    g = run_gpu(sc, ocfg, gC, gD, gA)
    go = O.render_bwd(P, cams, ocfg, rec, vals, ranges, gC, gD, gA)
    yield dict(name=request.param, sc=sc, ocfg=ocfg, rec=rec, keys=keys, vals=vals, ranges=ranges,
               out=out, keep=keep, gpu=g, go=go)
    g["renderer"].close()


def test_status_ok(case):
    g = case["gpu"]
    assert g["status"] == 0
    vis_g = g["pkey"] != 0xFFFFFFFF
    assert g["n_vis"] == int(vis_g.sum())
    # the oracle's visibility agrees outside its rectangle band
    rec = case["rec"]
    amb = rec[:, O.C_RECT_AMBIG] > 0
    assert np.array_equal((rec[:, O.C_VIS] > 0)[~amb], vis_g[~amb])
    assert g["n_inst"] > 0


def test_projection(case, request):
    _known_gap(request, case)
    rec, g = case["rec"], case["gpu"]
    amb = rec[:, O.C_RECT_AMBIG] > 0
    vis_o = rec[:, O.C_VIS] > 0
    vis_g = g["pkey"] != 0xFFFFFFFF
    assert np.array_equal(vis_o[~amb], vis_g[~amb]), "visibility differs"
    both = vis_o & vis_g
    d = decode_records(g["rec"][both])
    r = rec[both]
    # depth keys: bit-exact
    z32_o = r[:, O.C_Z32].astype(np.float32)
    assert np.array_equal(d["z"].view(np.uint32), z32_o.view(np.uint32))
    assert np.array_equal(g["pkey"][both], z32_o.view(np.uint32))
    # pixel mean
    assert np.abs(d["u"] - r[:, O.C_U]).max() < 1e-6 * (1 + np.abs(r[:, O.C_U]).max())
    assert np.abs(d["v"] - r[:, O.C_V]).max() < 1e-6 * (1 + np.abs(r[:, O.C_V]).max())
    # conic, each entry relative to its own scale: the record holds the
    # Cholesky factor of Q, which fixes qa and qc to their own relative
    # precision, and |qb| <= sqrt(qa qc) for a positive definite Q
    sqa, sqc = r[:, O.C_QA], r[:, O.C_QC]
    for k, c, sc in (("qa", O.C_QA, sqa), ("qb", O.C_QB, np.sqrt(sqa * sqc)), ("qc", O.C_QC, sqc)):
        assert (np.abs(d[k] - r[:, c]) / sc).max() < 1e-5, k
    assert np.abs(d["log2o"] - np.log2(r[:, O.C_OPA])).max() < 2e-6
    assert np.abs(d["rgb"] - r[:, O.C_R:O.C_B + 1]).max() < 2e-6
    # tile rectangles, except pairs in the ambiguity band
    ok = both & ~amb
    rect_o = rec[ok][:, [O.C_TX0, O.C_TY0, O.C_TX1, O.C_TY1]].astype(np.int64)
    assert np.array_equal(g["rect"][ok].astype(np.int64), rect_o)
    print(f"[{case['name']}] visible {both.sum()}, ambiguous rects {amb.sum()}")


def test_keys_and_ranges_bit_exact(case):
    """Binning stage alone: the oracle bins the CUDA path's own float32
    projection outputs; keys, instance order and ranges bit for bit."""
    g, sc, ocfg = case["gpu"], case["sc"], case["ocfg"]
    n_dec, n_band = check_binning_stage(sc, ocfg, g)
    T = case["ranges"].shape[0]
    mism = end_to_end_key_mismatch(g, case["keys"], case["vals"], T)
    # end to end (the FP64 projection upstream), instances may differ only
    # for pairs whose rectangle or tile decisions lie in the oracle's band
    amb = np.nonzero(case["rec"][:, O.C_RECT_AMBIG] > 0)[0]
    gp = g["inst_pair"].astype(np.int64)
    keep_g, keep_o = ~np.isin(gp, amb), ~np.isin(case["vals"], amb)
    assert np.array_equal(gp[keep_g], case["vals"][keep_o])
    print(f"[{case['name']}] {len(gp)} listed instances, {n_dec} rectangle tiles, {n_band} decisions in the "
          f"float band; end to end vs the FP64 projection: {mism} instances differ ({len(amb)} pairs in its band)")


def test_forward_images(case):
    out, g, keep = case["out"], case["gpu"], case["keep"]
    rgbmask, pmask = pixel_weights(case["sc"], keep)
    e_rgb = np.abs(g["rgb"].astype(np.float64) - out["rgb"])[rgbmask].max()
    e_d = np.abs(g["depth"].astype(np.float64) - out["depth"])[pmask].max()
    e_a = np.abs(g["alpha"].astype(np.float64) - out["alpha"])[pmask].max()
    e_t = np.abs(g["tfin"].astype(np.float64) - out["T"])[pmask].max()
    print(f"[{case['name']}] excluded pixels {(~keep).sum()} of {keep.size}; max err rgb {e_rgb:.2e} "
          f"depth {e_d:.2e} alpha {e_a:.2e} T {e_t:.2e}")
    assert e_rgb <= FWD_TOL and e_a <= FWD_TOL and e_t <= FWD_TOL and e_d <= FWD_TOL
    assert (~keep).sum() <= 0.01 * keep.size


def test_gradients(case):
    g, go = case["gpu"], case["go"]
    res = {}
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose", "dens_acc"):
        gk = "g_densify_acc" if k == "dens_acc" else "g_" + k
        res[k] = rel_l2(g[gk], go[k])
    vis = case["rec"][:, O.C_VIS] > 0
    res["g2d"] = rel_l2(g["g2d"][vis], go["g2d"][vis])
    cnt = g["g_densify_cnt"].astype(np.float64)
    print(f"[{case['name']}] " + " ".join(f"{k} {v:.1e}" for k, v in res.items()))
    # the count is the number of views where the pair is visible: exactly the
    # CUDA path's own visibility, and the oracle's for every Gaussian without
    # a pair in the oracle's rectangle band
    rec = case["rec"]
    gauss = rec[:, O.C_GAUSS].astype(np.int64)
    vis_g = g["pkey"] != 0xFFFFFFFF
    assert np.array_equal(cnt, np.bincount(gauss[vis_g], minlength=cnt.size))
    touched = np.zeros(cnt.size, bool)
    touched[gauss[rec[:, O.C_RECT_AMBIG] > 0]] = True
    assert np.array_equal(cnt[~touched], go["dens_cnt"][~touched])
    for k, v in res.items():
        assert v <= GRAD_TOL, (k, v)


def test_scenes_reach_the_colour_clamp_and_shared_gaussians():
    """The gradient parity above covers two paths of the projection adjoint:
    colour channels clamped at 0 (the forward marks them, the SH adjoint must
    give them no gradient) and Gaussians seen by several views (one lane walks
    their views and accumulates their gradients).  Both occur in the scenes."""
    clamped = shared = 0
    for sc in SCENES.values():
        P = O.Params.from_scene(sc)
        rec = O.project(P, O.as_float32_cameras(sc.cameras), O.Config())
        r = rec[rec[:, O.C_VIS] > 0]
        clamped += int((r[:, O.C_CLR:O.C_CLB + 1] > 0).sum())
        shared += int((np.bincount(r[:, O.C_GAUSS].astype(np.int64)) > 1).sum())
    print(f"clamped channels {clamped}, Gaussians seen by several views {shared}")
    assert clamped > 0 and shared > 0
