"""The tile / batch-depth autotuner: choice, cache, and (on a GPU) a real
tuning run whose choice renders the same images as the default tiles."""
import numpy as np
import pytest

from paper_2510_26358_gb300 import autotune as A
from paper_2510_26358_gb300 import scenes as S


def test_tuner_picks_the_fastest_and_caches(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def measure(tw, th, d):
        calls.append((tw, th, d))
        return {(16, 16, 128): 1.0}.get((tw, th, d), 2.0 + d / 1000)
    r = A.tune(measure, key="rig", cache_path=path)
    assert (r["tile_w"], r["tile_h"], r["batch_depth"]) == (16, 16, 128) and not r["cached"]
    assert len(calls) == len(A.CANDIDATES) == 9
    r2 = A.tune(lambda *a: 0.0, key="rig", cache_path=path)
    assert r2["cached"] and r2["batch_depth"] == 128
    r3 = A.tune(lambda *a: 0.0, key="rig", cache_path=path, refresh=True)
    assert not r3["cached"]


def test_signature_separates_rigs():
    sc = S.random_box_scene(100, 64, 48, 60.0)
    a = A.signature(sc.cameras, sc.n, 0, sc.submap_offsets)
    b = A.signature(sc.cameras, sc.n, 3, sc.submap_offsets)
    c = A.signature([sc.cameras[0].crop(0, 0, 32, 48)], sc.n, 0, sc.submap_offsets)
    assert len({a, b, c}) == 3


@pytest.mark.gpu
def test_tuning_run_on_gpu(tmp_path):
    import torch
    from tests.gpu_helpers import params_to_dev
    sc = S.orchard_scene(20_000, 3, 4, 160, 96, lidar_per_view=0, seed=5, name="tune")
    P = params_to_dev(sc)
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(0)
    up = [torch.from_numpy(rng.normal(size=n).astype(np.float32)).to(dev)
          for n in (3 * sc.n_pix, sc.n_pix, sc.n_pix)]
    meas = A.renderer_measure(sc.cameras, sc.submap_offsets, sc.sh_degree, P, up, steps=2, warmup=1,
                              inst_capacity=1 << 21)
    r = A.tune(meas, key=None, candidates=[(16, 16, 128), (8, 8, 64), (16, 32, 256)])
    assert set(r["timings"]) == {"16x16/128", "8x8/64", "16x32/256"}
    assert all(np.isfinite(v) and v > 0 for v in r["timings"].values())
    from paper_2510_26358_gb300 import gsraster as G
    imgs = []
    for tw, th, d in [(16, 16, 256), (r["tile_w"], r["tile_h"], r["batch_depth"])]:
        rr = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree,
                        config=G.gs_config_default(tile_w=tw, tile_h=th, batch_depth=d), inst_capacity=1 << 21)
        imgs.append(rr.forward(*P)[0].cpu().numpy())
        rr.close()
    assert np.array_equal(imgs[0], imgs[1])
