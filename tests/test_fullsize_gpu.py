"""Parity at the benchmark's full size, in the benchmark's launch configuration
(orchard, 500k Gaussians, three 1280x720 views, SH degree 3, 16x16 tiles,
batch depth 256): every projected pair is compared, and the binning stage
bit for bit (keys, instance order, ranges) on the CUDA path's projection; the
images on 20k sampled pixels (the oracle composites those pixels one by one);
the gradients with upstream gradients non-zero only on those sampled pixels
(the oracle's adjoint skips the others)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_26358_gb300 import scenes as S
from tests.gpu_helpers import (check_binning_stage, decode_records, end_to_end_key_mismatch, pixel_weights,
                               rel_l2, run_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    sc = S.workload("orchard500k")
    ocfg = O.Config()
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    rec = O.project(P, cams, ocfg)
    keys, vals, ranges = O.bin(P, cams, ocfg, rec)
    rng = np.random.default_rng(0)
    pix = np.sort(rng.choice(sc.n_pix, 20_000, replace=False))
    o = O.render_fwd_pixels(P, cams, ocfg, rec, vals, ranges, pix)
    keep = o["margin"] > 1e-4
    w = np.zeros(sc.n_pix)
    w[pix[keep]] = 1.0
    rgbw, pw = pixel_weights(sc, w > 0)
    gC = rng.normal(size=3 * sc.n_pix) * rgbw
    gD = 0.1 * rng.normal(size=sc.n_pix) * pw
    g = run_gpu(sc, ocfg, gC, gD, None, inst_capacity=4 << 20)
    go = O.render_bwd(P, cams, ocfg, rec, vals, ranges, gC, gD, None)
    yield dict(sc=sc, rec=rec, keys=keys, vals=vals, ranges=ranges, pix=pix, o=o, keep=keep, g=g, go=go)
    g["renderer"].close()


def test_fullsize_projection_and_keys(full):
    rec, g = full["rec"], full["g"]
    assert g["status"] == 0
    amb = rec[:, O.C_RECT_AMBIG] > 0
    vis_o, vis_g = rec[:, O.C_VIS] > 0, g["pkey"] != 0xFFFFFFFF
    assert np.array_equal(vis_o[~amb], vis_g[~amb])
    both = vis_o & vis_g
    d = decode_records(g["rec"][both])
    assert np.array_equal(g["pkey"][both], rec[both, O.C_Z32].astype(np.float32).view(np.uint32))
    assert np.abs(d["u"] - rec[both, O.C_U]).max() < 2e-6 * 1280
    # the binning stage, bit for bit on the CUDA path's own projection outputs
    n_dec, n_band = check_binning_stage(full["sc"], O.Config(), g)
    mism = end_to_end_key_mismatch(g, full["keys"], full["vals"], full["ranges"].shape[0])
    print(f"full size: {both.sum()} visible pairs, {len(g['inst_pair'])} listed instances of {n_dec} rectangle "
          f"tiles, {n_band} decisions in the float band; end to end {mism} instances differ "
          f"({amb.sum()} pairs in the FP64 band)")
    assert n_band <= 1e-4 * n_dec


def test_fullsize_sampled_pixels(full):
    sc, g, o, pix, keep = full["sc"], full["g"], full["o"], full["pix"], full["keep"]
    npx = sc.n_pix
    # planar rgb index of each sampled pixel's channels
    offs = np.cumsum([0] + [c.width * c.height for c in sc.cameras])
    view = np.searchsorted(offs, pix, side="right") - 1
    hw = np.array([c.width * c.height for c in sc.cameras])[view]
    base = 3 * offs[view] + (pix - offs[view])
    rgb_g = np.stack([g["rgb"][base + ch * hw] for ch in range(3)], 1).astype(np.float64)
    e_rgb = np.abs(rgb_g - o["rgb"])[keep].max()
    e_a = np.abs(g["alpha"][pix].astype(np.float64) - o["alpha"])[keep].max()
    e_d = np.abs(g["depth"][pix].astype(np.float64) - o["depth"])[keep].max()
    print(f"sampled 20000 px, excluded {(~keep).sum()}: rgb {e_rgb:.2e} alpha {e_a:.2e} depth {e_d:.2e}")
    assert e_rgb <= 1e-5 and e_a <= 1e-5 and e_d <= 1e-5
    assert npx == 2_764_800


def test_fullsize_gradients(full):
    g, go = full["g"], full["go"]
    res = {k: rel_l2(g["g_" + k], go[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose")}
    print("full size gradients: " + " ".join(f"{k} {v:.1e}" for k, v in res.items()))
    for k, v in res.items():
        assert v <= 1e-4, (k, v)
