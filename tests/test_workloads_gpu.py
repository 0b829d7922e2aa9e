"""The larger workloads at full size: the pose-refinement rig (1M Gaussians,
four perturbed 1440x1080 cameras), the uneven batch (8 submaps with
log-uniform Gaussian counts, 24 views of mixed resolution) and the large
keyframe map (4M Gaussians, six 1920x1200 views).  Every projected pair is
compared with the oracle, the binning stage bit for bit on the CUDA path's own
projection outputs, and 2000 sampled pixels are composited by the oracle one
by one."""
import numpy as np
import pytest

import oracle as O
from paper_2510_26358_gb300 import scenes as S
from tests.gpu_helpers import check_binning_stage, decode_records, end_to_end_key_mismatch, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["orchard1m_pose", "submaps8", "orchard4m"])
def test_workload_full_size(name):
    sc = S.workload(name, lidar=False)
    ocfg = O.Config()
    g = run_gpu(sc, ocfg, inst_capacity=1 << 26, depth=128)
    try:
        assert g["status"] == 0
        P = O.Params.from_scene(sc)
        cams = O.as_float32_cameras(sc.cameras)
        rec = O.project(P, cams, ocfg)
        keys, vals, ranges = O.bin(P, cams, ocfg, rec)
        amb = rec[:, O.C_RECT_AMBIG] > 0
        vis_o, vis_g = rec[:, O.C_VIS] > 0, g["pkey"] != 0xFFFFFFFF
        assert np.array_equal(vis_o[~amb], vis_g[~amb])
        both = vis_o & vis_g
        assert np.array_equal(g["pkey"][both], rec[both, O.C_Z32].astype(np.float32).view(np.uint32))
        d = decode_records(g["rec"][both])
        assert np.abs(d["u"] - rec[both, O.C_U]).max() < 1e-6 * 2048
        n_dec, n_band = check_binning_stage(sc, ocfg, g, P, cams)
        assert n_band <= 1e-4 * n_dec
        mism = end_to_end_key_mismatch(g, keys, vals, ranges.shape[0])
        rng = np.random.default_rng(2)
        pix = np.sort(rng.choice(sc.n_pix, 2000, replace=False))
        o = O.render_fwd_pixels(P, cams, ocfg, rec, vals, ranges, pix)
        keep = o["margin"] > 1e-4
        offs = np.cumsum([0] + [c.width * c.height for c in sc.cameras])
        view = np.searchsorted(offs, pix, side="right") - 1
        hw = np.array([c.width * c.height for c in sc.cameras])[view]
        base = 3 * offs[view] + (pix - offs[view])
        rgb = np.stack([g["rgb"][base + ch * hw] for ch in range(3)], 1).astype(np.float64)
        e_rgb = np.abs(rgb - o["rgb"])[keep].max()
        e_a = np.abs(g["alpha"][pix] - o["alpha"])[keep].max()
        e_d = np.abs(g["depth"][pix] - o["depth"])[keep].max()
        print(f"{name}: {both.sum()} visible, {len(g['inst_pair'])} instances, {n_band} of {n_dec} tile decisions "
              f"in the float band, {mism} differ end to end ({amb.sum()} pairs in the FP64 band); "
              f"rgb {e_rgb:.2e} alpha {e_a:.2e} depth {e_d:.2e}")
        assert e_rgb <= 1e-5 and e_a <= 1e-5 and e_d <= 1e-5
    finally:
        g["renderer"].close()
