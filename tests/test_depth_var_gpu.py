"""Rendered depth distribution and Eq. (7) with a predicted variance: the CUDA
forward with the depth mean and variance, the variance KL and the matching
backward against the FP64 oracle, element by element, through the C ABI.

Tolerances: images, mean and variance within 1e-5 of the value's own scale
(|gpu - oracle| <= 1e-5 (1 + |oracle|): depth is in m and the variance in
m^2, not in [0, 1]); losses within 1e-5 relative; gradients within 1e-4
relative (per tensor L2).  Pixels near a discrete decision of the oracle are left out as in
the plain parity tests, and LiDAR returns that land on them are dropped on
both sides.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_26358_gb300 import scenes as S
from tests.gpu_helpers import pixel_weights, rel_l2, run_gpu, run_oracle, torch_dev

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
LOSS_TOL = 1e-5
GRAD_TOL = 1e-4
MARGIN = 1e-4
SIG = dict(sigma_L=0.05, sigma_U=0.03, lam=0.8)


def _scenes():
    return {
        "box10k": S.random_box_scene(10_000, 320, 240, 300.0, seed=0),
        "orchard_rig": S.orchard_scene(40_000, 3, 4, 200, 120, rear=True, pose_noise=True,
                                       lidar_per_view=3000, seed=1, name="orchard_rig"),
        "submaps": S.uneven_submaps(4, 3000, 30000, seed=2, scale=1.0, lidar_per_view=2000,
                                    resolutions=((96, 64), (160, 96), (128, 128))),
    }


SCENES = _scenes()


def _scaled_err(a, b):
    a = np.asarray(a, np.float64)
    return float(np.max(np.abs(a - b) / (1.0 + np.abs(b)))) if a.size else 0.0


def _lidar_kept(sc, keep):
    """LiDAR rows whose pixel is inside, in front and not near a decision."""
    lid = np.asarray(sc.lidar, np.float32).reshape(-1, 4)
    if lid.shape[0] == 0:
        return lid
    offs = np.cumsum([0] + [c.width * c.height for c in sc.cameras])
    ok = np.zeros(lid.shape[0], bool)
    for i, (u, v, z, vw) in enumerate(lid):
        c = sc.cameras[int(vw)]
        if 0 <= u < c.width and 0 <= v < c.height:
            ok[i] = keep[offs[int(vw)] + int(v) * c.width + int(u)]
    return np.ascontiguousarray(lid[ok])


@pytest.fixture(scope="module", params=list(SCENES))
def case(request):
    sc = SCENES[request.param]
    ocfg = O.Config()
    P, cams, rec, keys, vals, ranges, out = run_oracle(sc, ocfg)
    mean, var = O.render_depth_dist(P, cams, ocfg, rec, vals, ranges)
    keep = out["margin"] > MARGIN
    rng = np.random.default_rng(17)
    rgbmask, pmask = pixel_weights(sc, keep)
    up = dict(gC=rng.normal(size=3 * sc.n_pix) * rgbmask, gD=0.1 * rng.normal(size=sc.n_pix) * pmask,
              gA=rng.normal(size=sc.n_pix) * pmask, gmean=rng.normal(size=sc.n_pix) * pmask,
              gvar=3.0 * rng.normal(size=sc.n_pix) * pmask)
    g = run_gpu(sc, ocfg, var=True, **up)
    go = O.render_bwd(P, cams, ocfg, rec, vals, ranges, up["gC"], up["gD"], up["gA"], up["gmean"], up["gvar"])
    yield dict(name=request.param, sc=sc, ocfg=ocfg, P=P, cams=cams, rec=rec, vals=vals, ranges=ranges,
               out=out, mean=mean, var=var, keep=keep, gpu=g, go=go)
    g["renderer"].close()


def test_moment_forward(case):
    g, out, keep = case["gpu"], case["out"], case["keep"]
    assert g["status"] == 0
    rgbmask, pmask = pixel_weights(case["sc"], keep)
    e = dict(rgb=_scaled_err(g["rgb"][rgbmask], out["rgb"][rgbmask]),
             depth=_scaled_err(g["depth"][pmask], out["depth"][pmask]),
             alpha=_scaled_err(g["alpha"][pmask], out["alpha"][pmask]),
             mean=_scaled_err(g["mean"][pmask], case["mean"][pmask]),
             var=_scaled_err(g["var"][pmask], case["var"][pmask]))
    hit = pmask & (out["alpha"] > 0)
    # the record the backward reads: (mean, var, 1/W)
    vs = g["vstat"][hit]
    e["vstat"] = max(_scaled_err(vs[:, 0], case["mean"][hit]), _scaled_err(vs[:, 1], case["var"][hit]),
                     float(np.max(np.abs(vs[:, 2] * out["alpha"][hit] - 1.0))))
    var_o = case["var"][hit]
    print(f"[{case['name']}] " + " ".join(f"{k} {v:.1e}" for k, v in e.items()) +
          f"; pixels with spread > 1 cm: {(var_o > 1e-4).sum()}")
    for k, v in e.items():
        assert v <= FWD_TOL, (k, v)
    assert (var_o > 1e-4).sum() > 100


def test_moment_backward(case):
    g, go = case["gpu"], case["go"]
    res = {k: rel_l2(g["g_" + k], go[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose")}
    vis = case["rec"][:, O.C_VIS] > 0
    res["g2d"] = rel_l2(g["g2d"][vis], go["g2d"][vis])
    print(f"[{case['name']}] " + " ".join(f"{k} {v:.1e}" for k, v in res.items()))
    for k, v in res.items():
        assert v <= GRAD_TOL, (k, v)


def test_variance_kl_loss(case):
    # the loss kernel alone, on the oracle's own images cast to float
    torch, dev = torch_dev()
    sc, out, keep = case["sc"], case["out"], case["keep"]
    lid = _lidar_kept(sc, keep)
    if lid.shape[0] == 0:
        pytest.skip("scene has no LiDAR")
    f32 = lambda a: np.asarray(a, np.float32)
    ins = [f32(out["alpha"]), f32(case["mean"]), f32(case["var"])]
    lo, gmo, gvo, nv = O.depth_loss_var(case["P"], case["cams"], case["ocfg"], *ins, lid, **SIG)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    grads = [torch.zeros(sc.n_pix, device=dev) for _ in range(2)]
    from paper_2510_26358_gb300 import gsraster as G
    from tests.gpu_helpers import gpu_config
    r2 = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree,
                    config=gpu_config(G, case["ocfg"], sigma_L=SIG["sigma_L"], sigma_U=SIG["sigma_U"],
                                      lambda_L=SIG["lam"]), inst_capacity=1 << 16)
    loss = r2.depth_loss_var(*[t(a) for a in ins], t(lid), grads=grads)
    torch.cuda.synchronize()
    lg = float(loss.cpu()[0])
    res = {k: rel_l2(a.cpu().numpy(), b) for k, a, b in zip(("dmean", "dvar"), grads, (gmo, gvo))}
    print(f"[{case['name']}] valid {nv} loss {lg:.6g} vs {lo:.6g}; " + " ".join(f"{k} {v:.1e}" for k, v in res.items()))
    r2.close()
    assert nv > 100
    assert abs(lg - lo) <= LOSS_TOL * abs(lo)
    for k, v in res.items():
        assert v <= GRAD_TOL, (k, v)


def test_variance_kl_end_to_end(case):
    # render with the depth mean and variance -> variance KL -> backward, on
    # both sides
    torch, dev = torch_dev()
    sc, keep = case["sc"], case["keep"]
    lid = _lidar_kept(sc, keep)
    if lid.shape[0] == 0:
        pytest.skip("scene has no LiDAR")
    P, cams, ocfg = case["P"], case["cams"], case["ocfg"]
    out = case["out"]
    lo, gmo, gvo, nv = O.depth_loss_var(P, cams, ocfg, out["alpha"], case["mean"], case["var"], lid, **SIG)
    go = O.render_bwd(P, cams, ocfg, case["rec"], case["vals"], case["ranges"], np.zeros(3 * sc.n_pix),
                      np.zeros(sc.n_pix), None, gmo, gvo)

    from paper_2510_26358_gb300 import gsraster as G
    from tests.gpu_helpers import gpu_config, params_to_dev
    r = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree,
                   config=gpu_config(G, ocfg, sigma_L=SIG["sigma_L"], sigma_U=SIG["sigma_U"], lambda_L=SIG["lam"]),
                   inst_capacity=1 << 22)
    Pd = params_to_dev(sc)
    rgb, dep, alp, mean, var = r.forward(*Pd, var=True)
    gl = [torch.zeros(sc.n_pix, device=dev) for _ in range(2)]
    loss = r.depth_loss_var(alp, mean, var, torch.from_numpy(lid).to(dev), grads=gl)
    grads = r.backward(*Pd, torch.zeros(3 * sc.n_pix, device=dev), None, None, var=True, dL_dmean=gl[0],
                       dL_dvar=gl[1])
    torch.cuda.synchronize()
    lg = float(loss.cpu()[0])
    res = {k: rel_l2(grads[k].cpu().numpy(), go[k])
           for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose")}
    print(f"[{case['name']}] loss {lg:.6g} vs {lo:.6g}; " + " ".join(f"{k} {v:.1e}" for k, v in res.items()))
    r.close()
    assert abs(lg - lo) <= LOSS_TOL * abs(lo)
    for k, v in res.items():
        assert v <= GRAD_TOL, (k, v)


def test_var_backward_needs_var_forward():
    torch, dev = torch_dev()
    from paper_2510_26358_gb300 import gsraster as G
    from tests.gpu_helpers import params_to_dev
    sc = S.random_box_scene(500, 64, 48, 60.0, seed=3)
    r = G.Renderer(sc.cameras, sc.submap_offsets, 0, inst_capacity=1 << 16)
    Pd = params_to_dev(sc)
    r.forward(*Pd)
    z = torch.zeros(3 * sc.n_pix, device=dev)
    with pytest.raises(G.GsError) as ei:
        r.backward(*Pd, z, z[:sc.n_pix], var=True)
    assert ei.value.status == G.GS_ERR_STATE
    # after a variance forward both backwards are accepted
    r.forward(*Pd, var=True)
    r.backward(*Pd, z, z[:sc.n_pix], var=True)
    r.backward(*Pd, z, z[:sc.n_pix])
    torch.cuda.synchronize()
    r.close()


def test_var_empty_and_single_fragment():
    # one fragment per pixel: var = 0 exactly while depth and alpha are not;
    # no visible Gaussian: all zero and a zero loss with no gradient
    torch, dev = torch_dev()
    from paper_2510_26358_gb300 import gsraster as G
    from tests.gpu_helpers import params_to_dev
    sc = S.random_box_scene(1, 40, 32, 50.0, seed=0)
    sc.means[:] = [[0.0, 0.0, 2.0]]
    sc.log_scales[:] = np.log(0.05)
    sc.opacity_logits[:] = 2.0
    r = G.Renderer(sc.cameras, sc.submap_offsets, 0, inst_capacity=1 << 12)
    Pd = params_to_dev(sc)
    rgb, dep, alp, mean, var = r.forward(*Pd, var=True)
    torch.cuda.synchronize()
    hit = alp > 0
    assert hit.sum().item() > 20
    assert torch.count_nonzero(var).item() == 0
    # a single fragment's mean is its own depth, exactly
    assert torch.all(mean[hit] == mean[hit][0]).item() and abs(float(mean[hit][0]) - 2.0) < 1e-6
    Pd[0][:, 2] = -5.0  # behind the camera
    rgb, dep, alp, mean, var = r.forward(*Pd, var=True)
    lid = torch.tensor([[20.5, 16.5, 2.0, 0.0]], device=dev)
    gl = [torch.zeros(sc.n_pix, device=dev) for _ in range(2)]
    loss = r.depth_loss_var(alp, mean, var, lid, grads=gl)
    torch.cuda.synchronize()
    assert float(loss.cpu()[0]) == 0.0 and all(torch.count_nonzero(x).item() == 0 for x in gl)
    assert torch.count_nonzero(alp).item() == 0 and torch.count_nonzero(mean).item() == 0
    r.close()


def test_var_tile_size_and_batch_depth_invariance():
    """The variance rasterisers at every tile shape (their pixels per thread
    differ) give the 16x16 images, depth mean and variance bitwise, and its
    gradients up to the order of float atomics."""
    sc = SCENES["orchard_rig"]
    rng = np.random.default_rng(23)
    n = sc.n_pix
    up = dict(gC=rng.normal(size=3 * n), gD=0.1 * rng.normal(size=n), gA=rng.normal(size=n),
              gmean=rng.normal(size=n), gvar=3.0 * rng.normal(size=n))
    runs = {}
    for (tw, th, depth) in [(16, 16, 256), (8, 8, 64), (16, 32, 128), (32, 16, 256)]:
        g = run_gpu(sc, O.Config(tile_w=tw, tile_h=th), depth=depth, var=True, **up)
        assert g["status"] == 0
        runs[(tw, th, depth)] = g
        g["renderer"].close()
    ref = runs[(16, 16, 256)]
    for key, g in runs.items():
        for k in ("rgb", "depth", "alpha", "tfin", "mean", "var"):
            assert np.array_equal(g[k], ref[k]), (key, k)
        for k in ("g_means", "g_log_scales", "g_quats", "g_opacity_logits", "g_sh", "g_pose"):
            assert rel_l2(g[k], ref[k]) < 1e-5, (key, k)
