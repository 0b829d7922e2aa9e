"""GPU behaviour beyond element-wise parity: tile-size and batch-depth
invariance, CUDA-graph replay, batched vs per-view rendering, the two losses
against the oracle, and the edge cases of the C ABI (empty and fully culled
scenes, a single Gaussian, capacity overflow, invalid arguments, call order)."""
import ctypes
import math
from copy import copy

import numpy as np
import pytest

import oracle as O
from paper_2510_26358_gb300 import scenes as S
from tests.gpu_helpers import params_to_dev, rel_l2, run_gpu, run_oracle, torch_dev

pytestmark = pytest.mark.gpu


def _G():
    from paper_2510_26358_gb300 import gsraster as G
    return G


def _scene():
    return S.orchard_scene(30_000, 3, 4, 160, 96, rear=True, pose_noise=True, lidar_per_view=2000,
                           seed=11, name="orchard_small")


def _upstream(sc, seed=3):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=3 * sc.n_pix), 0.1 * rng.normal(size=sc.n_pix), rng.normal(size=sc.n_pix))


# ---------------------------------------------------------------------------
# invariance, graphs, batching
# ---------------------------------------------------------------------------

def test_tile_size_and_batch_depth_invariance():
    sc = _scene()
    gC, gD, gA = _upstream(sc)
    runs = {}
    for (tw, th, depth) in [(16, 16, 256), (8, 8, 64), (16, 32, 128), (32, 16, 256), (16, 16, 32)]:
        g = run_gpu(sc, O.Config(tile_w=tw, tile_h=th), gC, gD, gA, depth=depth)
        assert g["status"] == 0
        runs[(tw, th, depth)] = g
        g["renderer"].close()
    ref = runs[(16, 16, 256)]
    for key, g in runs.items():
        for k in ("rgb", "depth", "alpha", "tfin"):
            assert np.array_equal(g[k], ref[k]), (key, k)
        # gradient sums differ only in the order of float atomics
        for k in ("g_means", "g_log_scales", "g_quats", "g_opacity_logits", "g_sh", "g_pose"):
            assert rel_l2(g[k], ref[k]) < 1e-5, (key, k)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_plain_forward_matches_scalar_variance_forward_bitwise(tile):
    """The plain forward works its pixels in packed f32x2 pairs, the variance
    forward one pixel at a time; both must give the same images, final
    transmittance and list counts bit for bit (one and two pairs a thread)."""
    sc = _scene()
    cfg = O.Config(tile_w=tile[0], tile_h=tile[1])
    g0 = run_gpu(sc, cfg, depth=64)
    g1 = run_gpu(sc, cfg, depth=64, var=True)
    try:
        assert g0["status"] == 0 and g1["status"] == 0
        for k in ("rgb", "depth", "tfin", "last"):
            assert np.array_equal(g0[k].view(np.uint32), g1[k].view(np.uint32)), k
        assert (g0["last"] > 0).mean() > 0.3
    finally:
        g0["renderer"].close()
        g1["renderer"].close()


def test_graph_replay_matches_eager():
    torch, dev = torch_dev()
    G = _G()
    sc = _scene()
    P = params_to_dev(sc)
    r = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree, inst_capacity=1 << 21)
    gC, gD, gA = (torch.from_numpy(x.astype(np.float32)).to(dev) for x in _upstream(sc))
    outs = [torch.empty(3 * r.n_pix, device=dev), torch.empty(r.n_pix, device=dev),
            torch.empty(r.n_pix, device=dev)]
    grads = dict(means=torch.zeros_like(P[0]), log_scales=torch.zeros_like(P[1]), quats=torch.zeros_like(P[2]),
                 opacity_logits=torch.zeros_like(P[3]), sh=torch.zeros_like(P[4]),
                 pose=torch.zeros(len(sc.cameras), 6, device=dev))

    def step():
        for v in grads.values():
            v.zero_()
        r.forward(*P, outputs=outs)
        r.backward(*P, gC, gD, gA, grads=grads)

    step()
    torch.cuda.synchronize()
    eager = [o.clone() for o in outs] + [grads[k].clone() for k in grads]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        for o in outs:
            o.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip(outs, eager[:3]):
            assert torch.equal(a, b)
        for k, b in zip(grads, eager[3:]):
            assert rel_l2(grads[k].cpu().numpy(), b.cpu().numpy()) < 1e-5, k
    assert r.status()[0] == G.GS_OK
    r.close()


def test_batched_equals_per_view():
    sc = _scene()
    gC, gD, gA = _upstream(sc)
    ocfg = O.Config()
    full = run_gpu(sc, ocfg, gC, gD, gA)
    full["renderer"].close()
    off = 0
    sum_grads = {k: np.zeros_like(full["g_" + k]) for k in ("means", "sh", "opacity_logits")}
    for v, c in enumerate(sc.cameras):
        sub = copy(sc)
        sub.cameras = [c]
        hw = c.width * c.height
        sl = slice(off, off + hw)
        one = run_gpu(sub, ocfg, gC[3 * off: 3 * (off + hw)], gD[sl], gA[sl])
        one["renderer"].close()
        assert np.array_equal(one["rgb"], full["rgb"][3 * off: 3 * (off + hw)])
        assert np.array_equal(one["depth"], full["depth"][sl])
        assert np.array_equal(one["alpha"], full["alpha"][sl])
        assert rel_l2(one["g_pose"][0], full["g_pose"][v]) < 1e-5
        for k in sum_grads:
            sum_grads[k] += one["g_" + k]
        off += hw
    for k, v in sum_grads.items():
        assert rel_l2(v, full["g_" + k]) < 1e-5, k


# ---------------------------------------------------------------------------
# losses
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [0, 1])
def test_depth_loss_parity(mode):
    torch, dev = torch_dev()
    G = _G()
    cams = [S.Camera(64, 48, 60.0, 60.0, 32.0, 24.0, np.eye(3, 4), 0),
            S.Camera(40, 30, 40.0, 40.0, 20.0, 15.0, np.eye(3, 4), 0)]
    rng = np.random.default_rng(5 + mode)
    npx = 64 * 48 + 40 * 30
    depth = rng.uniform(0.5, 8.0, npx).astype(np.float32)
    alpha = rng.uniform(0, 1, npx).astype(np.float32)
    alpha[rng.random(npx) < 0.15] = 0.0
    m = 5000
    lid = np.stack([rng.uniform(-5, 70, m), rng.uniform(-5, 55, m), rng.uniform(0.05, 9, m),
                    rng.integers(-1, 3, m)], 1).astype(np.float32)
    cfg = G.gs_config_default(depth_mode=mode, sigma_L=0.04, sigma_U=0.07, lambda_L=0.8)
    r = G.Renderer(cams, [0, 1], 0, config=cfg, inst_capacity=1024)
    t = lambda a: torch.from_numpy(a).to(dev)
    grad = torch.zeros(npx, device=dev)
    loss = r.depth_loss(t(depth), t(alpha), t(lid), grad)
    torch.cuda.synchronize()
    P = O.Params(np.zeros((1, 3)), np.zeros((1, 3)), np.ones((1, 4)), np.zeros(1), np.zeros((1, 1, 3)), 0,
                 np.array([0, 1]))
    lo, go, nv = O.depth_loss(P, O.as_float32_cameras(cams), O.Config(), depth, alpha, lid, mode=mode,
                              sigma_L=0.04, sigma_U=0.07, lam=0.8)
    assert nv > 500
    assert loss.item() == pytest.approx(lo, rel=1e-6)
    gg = grad.cpu().numpy().astype(np.float64)
    assert np.abs(gg - go).max() <= 1e-6 * np.abs(go).max()
    r.close()


def test_depth_loss_without_valid_points():
    torch, dev = torch_dev()
    G = _G()
    cams = [S.Camera(16, 16, 20.0, 20.0, 8.0, 8.0, np.eye(3, 4), 0)]
    r = G.Renderer(cams, [0, 1], 0, inst_capacity=1024)
    d, a = torch.ones(256, device=dev), torch.zeros(256, device=dev)
    lid = torch.tensor([[3.0, 3.0, 2.0, 0.0], [100.0, 3.0, 2.0, 0.0]], device=dev)
    grad = torch.zeros(256, device=dev)
    loss = r.depth_loss(d, a, lid, grad)
    torch.cuda.synchronize()
    assert loss.item() == 0.0 and grad.abs().max().item() == 0.0
    r.close()


def test_image_l1_parity():
    torch, dev = torch_dev()
    G = _G()
    cams = [S.Camera(50, 30, 50.0, 50.0, 25.0, 15.0, np.eye(3, 4), 0)]
    r = G.Renderer(cams, [0, 1], 0, inst_capacity=1024)
    rng = np.random.default_rng(1)
    C = rng.random(4500).astype(np.float32)
    I = rng.random(4500).astype(np.float32)
    I[:10] = C[:10]  # exact ties: zero gradient
    grad = torch.zeros(4500, device=dev)
    loss = r.image_l1(torch.from_numpy(C).to(dev), torch.from_numpy(I).to(dev), grad)
    torch.cuda.synchronize()
    lo, go = O.image_l1(C, I)
    assert loss.item() == pytest.approx(lo, rel=1e-6)
    assert np.abs(grad.cpu().numpy() - go).max() <= 1e-7 * np.abs(go).max()
    r.close()


def test_image_l1_with_8bit_targets():
    """gs_image_l1_u8 equals gs_image_l1 on the float targets t / 255 bit for
    bit (loss and accumulated gradient, ragged size so the scalar tail runs),
    and both match the oracle; ties give zero gradient."""
    torch, dev = torch_dev()
    G = _G()
    cams = [S.Camera(51, 31, 50.0, 50.0, 25.0, 15.0, np.eye(3, 4), 0)]
    r = G.Renderer(cams, [0, 1], 0, inst_capacity=1024)
    n = 3 * 51 * 31
    rng = np.random.default_rng(2)
    T8 = rng.integers(0, 256, n).astype(np.uint8)
    Tf = T8.astype(np.float32) / np.float32(255.0)  # float32 division, as the kernel divides
    C = rng.random(n).astype(np.float32)
    C[:20] = Tf[:20]  # exact ties
    Cd = torch.from_numpy(C).to(dev)
    g8 = torch.full((n,), 0.25, device=dev)  # accumulation onto existing values
    gf = g8.clone()
    l8 = r.image_l1(Cd, torch.from_numpy(T8).to(dev), g8)
    lf = r.image_l1(Cd, torch.from_numpy(Tf).to(dev), gf)
    torch.cuda.synchronize()
    assert l8.item() == lf.item()
    assert torch.equal(g8, gf)
    lo, go = O.image_l1(C, Tf)
    assert l8.item() == pytest.approx(lo, rel=1e-6)
    # the gradient was added onto 0.25 in float32: one rounding at 0.25's ulp
    assert np.abs(g8.cpu().numpy().astype(np.float64) - 0.25 - go).max() <= float(np.spacing(np.float32(0.25)))
    r.close()


# ---------------------------------------------------------------------------
# edge cases of the C ABI
# ---------------------------------------------------------------------------

def test_empty_and_culled_scenes():
    torch, dev = torch_dev()
    G = _G()
    cam = S.Camera(48, 32, 40.0, 40.0, 24.0, 16.0, np.eye(3, 4), 0)
    # no Gaussians at all
    empty = S.random_box_scene(0, 48, 32, 40.0, seed=0)
    empty.cameras = [cam]
    g = run_gpu(empty, O.Config(), np.ones(3 * 48 * 32), np.ones(48 * 32), None)
    assert g["status"] == 0 and g["n_vis"] == 0 and g["n_inst"] == 0
    assert not g["rgb"].any() and not g["alpha"].any() and not g["depth"].any()
    assert not g["g_pose"].any()
    g["renderer"].close()
    # every Gaussian behind the camera
    sc = S.random_box_scene(500, 48, 32, 40.0, seed=1, box=((-1, 1), (-1, 1), (-5, -1)))
    g = run_gpu(sc, O.Config(), np.ones(3 * 48 * 32), np.ones(48 * 32), None)
    assert g["status"] == 0 and g["n_vis"] == 0
    assert not g["alpha"].any() and not g["g_means"].any() and not g["g_pose"].any()
    g["renderer"].close()


def test_single_gaussian_matches_oracle():
    sc = S.random_box_scene(1, 40, 32, 50.0, seed=0, box=((-0.05, 0.05), (-0.05, 0.05), (1.5, 1.6)),
                            log_scale_mu=-3.0, log_scale_sd=0.01, sh_degree=2)
    gC, gD, gA = _upstream(sc)
    ocfg = O.Config()
    P, cams, rec, keys, vals, ranges, out = run_oracle(sc, ocfg)
    g = run_gpu(sc, ocfg, gC, gD, gA)
    assert g["n_vis"] == 1 and (out["alpha"] > 0).sum() > 10
    assert np.abs(g["rgb"] - out["rgb"]).max() < 1e-5
    go = O.render_bwd(P, cams, ocfg, rec, vals, ranges, gC, gD, gA)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose"):
        assert rel_l2(g["g_" + k], go[k]) < 1e-4, k
    g["renderer"].close()


def test_capacity_overflow_is_reported_not_trapped():
    torch, dev = torch_dev()
    G = _G()
    sc = S.random_box_scene(2000, 96, 64, 90.0, seed=2)
    g = run_gpu(sc, O.Config(), np.ones(3 * sc.n_pix), np.ones(sc.n_pix), None, inst_capacity=100)
    assert g["status"] == G.GS_ERR_CAPACITY
    assert g["n_inst"] > 100
    assert not g["alpha"].any() and not g["g_means"].any()
    need = g["n_inst"]
    g["renderer"].close()
    g2 = run_gpu(sc, O.Config(), np.ones(3 * sc.n_pix), np.ones(sc.n_pix), None, inst_capacity=need)
    assert g2["status"] == G.GS_OK and g2["alpha"].any()
    g2["renderer"].close()


def test_invalid_arguments_and_call_order():
    torch, dev = torch_dev()
    G = _G()
    L = G.lib()
    cams = G.camera_structs([S.Camera(32, 32, 30.0, 30.0, 16.0, 16.0, np.eye(3, 4), 0)])
    offs = (ctypes.c_int64 * 2)(0, 10)
    out = ctypes.c_void_p()
    bad = G.gs_config_default(tile_w=12, tile_h=12)
    assert L.gs_workspace_create(cams, 1, offs, 1, 0, ctypes.byref(bad), 1000, ctypes.byref(out)) == \
        G.GS_ERR_INVALID_ARG
    cfg = G.gs_config_default(batch_depth=100)
    assert L.gs_workspace_create(cams, 1, offs, 1, 0, ctypes.byref(cfg), 1000, ctypes.byref(out)) == \
        G.GS_ERR_INVALID_ARG
    cfg = G.gs_config_default()
    assert L.gs_workspace_create(cams, 1, offs, 1, 4, ctypes.byref(cfg), 1000, ctypes.byref(out)) == \
        G.GS_ERR_INVALID_ARG
    assert L.gs_workspace_create(cams, 1, offs, 1, 0, ctypes.byref(cfg), 1000, ctypes.byref(out)) == G.GS_OK
    ws = out
    buf = torch.zeros(3 * 1024, device=dev)
    p = ctypes.c_void_p(buf.data_ptr())
    s = G._stream()
    # rendering before projecting / binning
    assert L.gs_render_fwd(ws, p, p, p, s) == G.GS_ERR_STATE
    assert L.gs_bin_sort(ws, s) == G.GS_ERR_STATE
    # NULL outputs and a Gaussian count that differs from the workspace's
    assert L.gs_render_fwd(ws, None, p, p, s) == G.GS_ERR_INVALID_ARG
    params = torch.zeros(10 * 48, device=dev)
    gg = G.GsGaussians(params.data_ptr(), params.data_ptr(), params.data_ptr(), params.data_ptr(),
                       params.data_ptr(), 9)
    assert L.gs_project(ws, ctypes.byref(gg), p, s) == G.GS_ERR_INVALID_ARG
    # misaligned LiDAR array
    mis = ctypes.c_void_p(buf.data_ptr() + 4)
    assert L.gs_depth_loss(ws, p, p, mis, 1, p, None, s) == G.GS_ERR_INVALID_ARG
    assert "aligned" in G.last_error()
    L.gs_workspace_destroy(ws)


def test_capacity_flag_clears_on_the_next_binning():
    # an overflow blanks that frame only: the next gs_bin_sort that fits renders
    # normally on the same workspace, identical to a fresh one
    torch, dev = torch_dev()
    G = _G()
    from tests.gpu_helpers import params_to_dev
    sc = S.random_box_scene(2000, 96, 64, 90.0, seed=2)
    P = params_to_dev(sc)
    r = G.Renderer(sc.cameras, sc.submap_offsets, 0, inst_capacity=600)
    r.forward(*P)
    st, need, _ = r.status()
    assert st == G.GS_ERR_CAPACITY and need > 600
    P_small = [p.clone() for p in P]
    P_small[0][100:, 2] = -5.0  # all but 100 Gaussians behind the camera
    rgb, dep, alp = [t.clone() for t in r.forward(*P_small)]
    st, need2, _ = r.status()
    assert st == G.GS_OK and need2 <= 600 and bool(alp.any())
    fresh = G.Renderer(sc.cameras, sc.submap_offsets, 0, inst_capacity=600)
    rgb2, dep2, alp2 = fresh.forward(*P_small)
    torch.cuda.synchronize()
    assert torch.equal(rgb, rgb2) and torch.equal(alp, alp2)
    r.close()
    fresh.close()


def test_device_wait_timeout_is_reported():
    # the bounded wait of the TMA staging, run out on purpose on a barrier no
    # copy completes: a status, not a hang or a fault; cleared by the next binning
    torch, dev = torch_dev()
    G = _G()
    from tests.gpu_helpers import params_to_dev
    sc = S.random_box_scene(500, 64, 48, 60.0, seed=3)
    P = params_to_dev(sc)
    r = G.Renderer(sc.cameras, sc.submap_offsets, 0, inst_capacity=1 << 16)
    r.forward(*P)
    assert r.status()[0] == G.GS_OK
    res = torch.zeros(1, dtype=torch.int32, device=dev)
    assert G.lib().gs_selftest_wait_timeout(r.ws, 50_000_000, G._ptr(res), G._stream()) == G.GS_OK
    torch.cuda.synchronize()
    assert int(res.item()) == 1
    with pytest.raises(G.GsError) as ei:
        st = r.status()
    assert ei.value.status == G.GS_ERR_TIMEOUT
    r.forward(*P)
    assert r.status()[0] == G.GS_OK
    r.close()


def test_zero_buffers():
    # many buffers, odd sizes, unaligned starts, empty ones: exactly the given bytes become 0
    torch, dev = torch_dev()
    G = _G()
    base = torch.full((1 << 20,), 7, dtype=torch.uint8, device=dev)
    views = [base[3:3 + 1001], base[5000:5000 + 64 * 1024 + 5], base[200000:200000], base[300001:300001 + 7],
             base[400000:400000 + 900000 - 400000]]
    G.gs_zero_buffers(views)
    torch.cuda.synchronize()
    ref = torch.full_like(base, 7)
    for a, b in ((3, 1004), (5000, 5000 + 64 * 1024 + 5), (300001, 300008), (400000, 900000)):
        ref[a:b] = 0
    assert torch.equal(base, ref)
    f = torch.ones(12345, 7, device=dev)
    G.gs_zero_buffers([f])
    assert int(torch.count_nonzero(f)) == 0
    with pytest.raises(G.GsError):
        G.gs_zero_buffers([torch.ones(4, device=dev)] * 17)


def test_written_gradients_equal_accumulated_onto_zero():
    """gs_grads.overwrite = 1 writes every output (zeros for the Gaussians no
    view sees) and equals accumulating onto zeroed buffers, up to the order
    of the raster backward's float atomics (each call sums its image-space
    gradients in its own order); with overwrite = 0 the outputs are added onto
    what the buffers held.  The three backwards follow one projection: the
    first adds into the image-space rows the projection cleared, the later
    ones clear the rows themselves (else they would add onto the first's)."""
    torch, dev = torch_dev()
    G = _G()
    sc = _scene()
    gC, gD, gA = _upstream(sc)
    P = params_to_dev(sc)
    r = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree, inst_capacity=1 << 22)
    try:
        r.forward(*P)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        up = (t(gC), t(gD), t(gA))
        keys = ("means", "log_scales", "quats", "opacity_logits", "sh", "pose", "densify_acc", "densify_cnt")
        zeros = r.backward(*P, *up, overwrite=False)  # allocated zeroed, accumulated
        poison = {k: (torch.full_like(v, float("nan")) if v.dtype == torch.float32 else torch.full_like(v, -7))
                  for k, v in zeros.items()}
        written = r.backward(*P, *up, grads=poison, overwrite=True)
        base = {k: (torch.randn_like(v) if v.dtype == torch.float32 else torch.full_like(v, 3)) for k, v in zeros.items()}
        summed = r.backward(*P, *up, grads={k: v.clone() for k, v in base.items()}, overwrite=False)
        torch.cuda.synchronize()
        seen = zeros["densify_cnt"] > 0
        assert 0 < int(seen.sum()) < sc.n  # both kinds of rows occur
        close = lambda a, b: float((a.double() - b.double()).abs().max()) <= 1e-5 * float(b.double().abs().max())
        for k in keys:
            assert not torch.isnan(written[k].float()).any(), k  # every row written
            assert close(written[k], zeros[k]), k
            # the unseen Gaussians' rows are exactly zero
            if k not in ("pose",):
                assert torch.all(written[k][~seen] == 0), k
        assert torch.equal(written["densify_cnt"], zeros["densify_cnt"])
        for k in ("means", "log_scales", "quats", "sh", "opacity_logits", "pose", "densify_acc"):
            assert close(summed[k] - base[k], zeros[k]), k  # added onto what the buffers held
        assert torch.equal(summed["densify_cnt"], base["densify_cnt"] + zeros["densify_cnt"])
        # an invalid mode is refused
        gg = G.GsGrads(*(zeros[k].data_ptr() for k in keys), 2, 0)
        st = G.lib().gs_render_bwd(r.ws, r.gaussians(*P), G._ptr(r.cams_dev), G._ptr(up[0]), G._ptr(up[1]),
                                   None, ctypes.byref(gg), G._stream())
        assert st == G.GS_ERR_INVALID_ARG
    finally:
        r.close()


def test_projection_with_unaligned_sh_rows_matches_aligned():
    """The projection reads each SH row in 16-byte pieces when the SH array
    starts on a 16-byte boundary and one coefficient at a time otherwise, in
    the same order: the images are bitwise equal.  The SH adjoint clears the
    unseen Gaussians' gradient rows in 16-byte pieces only when the caller's
    gradient array is aligned: with SH values and SH gradients both one float
    past a boundary the gradients equal the aligned ones, the unseen rows are
    zeros, and the densification counts are equal."""
    torch, dev = torch_dev()
    G = _G()
    sc = _scene()
    gC, gD, gA = _upstream(sc)
    P = params_to_dev(sc)
    r = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree, inst_capacity=1 << 22)
    try:
        ref = [x.clone() for x in r.forward(*P)]
        buf = torch.empty(P[4].numel() + 1, device=dev)
        sh_u = buf[1:].view_as(P[4])
        sh_u.copy_(P[4])
        assert sh_u.data_ptr() % 16 != 0
        out = r.forward(*P[:4], sh_u)
        torch.cuda.synchronize()
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        r.forward(*P)
        g_a = r.backward(*P, t(gC), t(gD), t(gA))
        r.forward(*P[:4], sh_u)
        g_buf = torch.full((P[4].numel() + 1,), float("nan"), device=dev)
        grads = {k: torch.empty_like(v) for k, v in g_a.items()}
        grads["sh"] = g_buf[1:].view_as(g_a["sh"])
        assert grads["sh"].data_ptr() % 16 != 0
        g_u = r.backward(*P[:4], sh_u, t(gC), t(gD), t(gA), grads=grads, overwrite=True)
        torch.cuda.synchronize()
        assert torch.equal(g_u["densify_cnt"], g_a["densify_cnt"])
        assert not torch.isnan(g_u["sh"]).any()
        unseen = g_a["densify_cnt"] == 0
        assert int(unseen.sum()) > 0 and torch.all(g_u["sh"][unseen] == 0)
        scale = float(g_a["sh"].double().abs().max())
        assert float((g_u["sh"].double() - g_a["sh"].double()).abs().max()) <= 1e-5 * scale
    finally:
        r.close()
