"""The seeded input generators that both the CUDA path and the oracle take
their inputs from: deterministic for a seed, and shaped like the recipes the
benchmark workloads are quoted on (Gaussian counts, cameras, SH degree, LiDAR
returns, submaps, parameter distributions)."""
import numpy as np
import pytest

from paper_2510_26358_gb300 import scenes as S

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh", "submap_offsets", "lidar", "target")


def _same(a, b):
    for k in FIELDS:
        x, y = getattr(a, k), getattr(b, k)
        if x is None or y is None:
            assert x is None and y is None, k
        elif not np.array_equal(x, y):
            return False
    return [(c.width, c.height, c.fx, c.cx, c.T_cw.tobytes()) for c in a.cameras] == \
           [(c.width, c.height, c.fx, c.cx, c.T_cw.tobytes()) for c in b.cameras]


@pytest.mark.parametrize("name", ["box10k", "orchard500k"])
def test_generators_are_deterministic(name):
    assert _same(S.workload(name, seed=0), S.workload(name, seed=0))
    assert not _same(S.workload(name, seed=0), S.workload(name, seed=1))


def test_orchard500k_recipe():
    sc = S.workload("orchard500k")
    assert sc.n == 500_000 and sc.sh_degree == 3 and list(sc.submap_offsets) == [0, 500_000]
    assert [(c.width, c.height) for c in sc.cameras] == [(1280, 720)] * 3
    assert sc.lidar.shape == (60_000, 4)  # 20k returns a view
    assert sc.target is not None and sc.target.size == 3 * sc.n_pix
    # canopy Gaussians: log-scales N(-4, 0.6), random orientations; trunk ones
    # elongated along z (axis-aligned): 1 trunk to 10 canopy Gaussians a tree
    trunk = np.all(sc.quats == np.array([1, 0, 0, 0], np.float32), axis=1)
    assert abs(trunk.mean() - 1 / 11) < 0.01
    can = sc.log_scales[~trunk].astype(np.float64)
    assert abs(can.mean() + 4.0) < 0.01 and abs(can.std() - 0.6) < 0.01
    assert np.all(sc.log_scales[trunk][:, 2] > sc.log_scales[trunk][:, :2].max(axis=1))
    # SH coefficients N(0, 0.2); opacity logits N(0, 1)
    assert abs(sc.sh.std() - 0.2) < 0.002 and abs(sc.opacity_logits.std() - 1.0) < 0.01


@pytest.mark.parametrize("name,n,cams,submaps", [
    ("box10k", 10_000, {(320, 240)}, 1),
    ("orchard1m_pose", 1_000_000, {(1440, 1080)}, 1),
    ("submaps8", None, {(640, 480), (1280, 720), (1920, 1080)}, 8),
    ("orchard4m", 4_000_000, {(1920, 1200)}, 1),
])
def test_workload_shapes(name, n, cams, submaps):
    sc = S.workload(name, lidar=False)
    if n is not None:
        assert sc.n == n
    assert {(c.width, c.height) for c in sc.cameras} == cams
    off = np.asarray(sc.submap_offsets)
    assert len(off) == submaps + 1 and off[0] == 0 and off[-1] == sc.n and np.all(np.diff(off) >= 0)
    # every camera belongs to an existing submap
    assert all(0 <= c.submap < submaps for c in sc.cameras)
    if name == "submaps8":
        sizes = np.diff(off)
        assert len(sc.cameras) == 24 and sizes.min() >= 50_000 and sizes.max() <= 2_000_000
    if name == "orchard4m":
        assert len(sc.cameras) == 6


def test_needle_scene_axes():
    sc = S.needle_scene()
    ls = sc.log_scales.astype(np.float64)
    assert np.all((ls[:, 0] >= -2.2) & (ls[:, 0] <= -0.8))
    assert np.all((ls[:, 1:] >= -6.0) & (ls[:, 1:] <= -5.0))
    # the rest of the box scene is kept
    base = S.random_box_scene(4_000, 160, 120, 150.0, seed=6)
    assert np.array_equal(sc.means, base.means) and np.array_equal(sc.quats, base.quats)
