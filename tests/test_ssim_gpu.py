"""SSIM term of Eq. (6) on the GPU against the FP64 oracle, through the C ABI.

Both sides get the same float32 images (the CUDA renderer's output and a
target), so the comparison isolates the loss.  Bars: the three loss values
within 1e-5 relative; dL/drgb within 1e-4 relative (L2 over the tensor).
Targets: the scenes' uniform random targets (large local variance) and a
smooth perturbation of the rendering itself (SSIM near 1, the regime where
the variance terms cancel most).
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_26358_gb300 import scenes as S
from tests.gpu_helpers import rel_l2, torch_dev

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4
LAM = 0.2


def _ragged_scene():
    # views smaller than the window (5x3), and sizes that are no multiple of
    # the 32x16 tiles
    sc = S.random_box_scene(3000, 64, 48, 60.0, seed=5)
    T = sc.cameras[0].T_cw
    sc.cameras = [S.Camera(37, 23, 35.0, 35.0, 18.5, 11.5, T, 0), S.Camera(5, 3, 5.0, 5.0, 2.5, 1.5, T, 0),
                  S.Camera(100, 41, 90.0, 90.0, 50.0, 20.5, T, 0)]
    rng = np.random.default_rng(9)
    sc.target = rng.random(3 * sum(c.width * c.height for c in sc.cameras)).astype(np.float32)
    return sc


def _scenes():
    return {
        "box10k": S.random_box_scene(10_000, 320, 240, 300.0, seed=0),
        "orchard_rig": S.orchard_scene(40_000, 3, 4, 200, 120, rear=True, pose_noise=True,
                                       lidar_per_view=0, seed=1, name="orchard_rig"),
        "ragged": _ragged_scene(),
    }


SCENES = _scenes()


def _render(sc):
    from paper_2510_26358_gb300 import gsraster as G
    from tests.gpu_helpers import params_to_dev
    r = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree, inst_capacity=1 << 22)
    rgb = r.forward(*params_to_dev(sc))[0]
    return r, rgb


def _smooth_target(sc, rgb_np, seed):
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    out, off = np.empty_like(rgb_np), 0
    for c in sc.cameras:
        for _ in range(3):
            n = c.width * c.height
            noise = gaussian_filter(rng.normal(size=(c.height, c.width)), 2.0) * 0.05
            out[off:off + n] = np.clip(rgb_np[off:off + n] + noise.ravel(), 0, 1)
            off += n
    return out.astype(np.float32)


@pytest.fixture(scope="module", params=list(SCENES))
def scene(request):
    sc = SCENES[request.param]
    r, rgb = _render(sc)
    yield request.param, sc, r, rgb
    r.close()


@pytest.mark.parametrize("target_kind", ["random", "smooth"])
def test_image_loss_matches_oracle(scene, target_kind):
    torch, dev = torch_dev()
    name, sc, r, rgb = scene
    rgb_np = rgb.cpu().numpy()
    tgt = sc.target.astype(np.float32) if target_kind == "random" else _smooth_target(sc, rgb_np, 3)
    tgt_d = torch.from_numpy(tgt).to(dev)
    grad = torch.zeros_like(rgb)
    loss = r.image_loss(rgb, tgt_d, LAM, dL_drgb=grad)
    torch.cuda.synchronize()
    lg = loss.cpu().numpy().astype(np.float64)
    cams = O.as_float32_cameras(sc.cameras)
    Lo, go = O.image_loss(cams, rgb_np, tgt, LAM)
    l1o = np.abs(rgb_np.astype(np.float64) - tgt).mean()
    so, _ = O.ssim(cams, rgb_np, tgt, grad=False)
    e_loss = [abs(lg[0] - Lo) / Lo, abs(lg[1] - l1o) / l1o, abs(lg[2] - (1 - so)) / (1 - so)]
    e_grad = rel_l2(grad.cpu().numpy(), go)
    print(f"[{name}/{target_kind}] 1-SSIM {1 - so:.4f}; loss errors {['%.1e' % e for e in e_loss]}; grad {e_grad:.1e}")
    assert max(e_loss) <= LOSS_TOL
    assert e_grad <= GRAD_TOL


def test_lambda_ends_and_identity():
    torch, dev = torch_dev()
    from paper_2510_26358_gb300 import gsraster as G
    sc = SCENES["orchard_rig"]
    r, rgb = _render(sc)
    tgt = torch.from_numpy(sc.target.astype(np.float32)).to(dev)
    # lambda = 0 is the L1 term alone, gradient included
    g0, g1 = torch.zeros_like(rgb), torch.zeros_like(rgb)
    l0 = r.image_loss(rgb, tgt, 0.0, dL_drgb=g0)
    l1 = r.image_l1(rgb, tgt, dL_drgb=g1)
    torch.cuda.synchronize()
    assert abs(float(l0[0]) - float(l1[0])) <= 1e-7 * float(l1[0])
    assert torch.equal(g0, g1)
    # lambda = 1 is 1 - SSIM alone
    l_one = r.image_loss(rgb, tgt, 1.0)
    torch.cuda.synchronize()
    assert float(l_one[0]) == pytest.approx(float(l_one[2]), rel=1e-6)
    # identical images: SSIM 1, gradient of the SSIM term ~0
    gi = torch.zeros_like(rgb)
    li = r.image_loss(rgb, rgb.clone(), 1.0, dL_drgb=gi)
    torch.cuda.synchronize()
    assert abs(float(li[2])) < 1e-6 and float(gi.abs().max()) < 1e-7
    # lambda outside [0, 1] is an argument error
    with pytest.raises(G.GsError) as ei:
        r.image_loss(rgb, tgt, 1.5)
    assert ei.value.status == G.GS_ERR_INVALID_ARG
    r.close()


def test_full_size_orchard500k():
    # the bench workload's three 1280x720 views against its random target
    torch, dev = torch_dev()
    sc = S.workload("orchard500k", lidar=False)
    r, rgb = _render(sc)
    rgb_np = rgb.cpu().numpy()
    tgt = sc.target.astype(np.float32)
    grad = torch.zeros_like(rgb)
    loss = r.image_loss(rgb, torch.from_numpy(tgt).to(dev), LAM, dL_drgb=grad)
    torch.cuda.synchronize()
    Lo, go = O.image_loss(O.as_float32_cameras(sc.cameras), rgb_np, tgt, LAM)
    e_grad = rel_l2(grad.cpu().numpy(), go)
    print(f"[orchard500k] loss {float(loss[0]):.6f} vs {Lo:.6f}; grad {e_grad:.1e}")
    assert abs(float(loss[0]) - Lo) <= LOSS_TOL * Lo
    assert e_grad <= GRAD_TOL
    r.close()
