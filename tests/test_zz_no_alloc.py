"""gs_image_l1_noalloc against gs_image_l1.

The no-allocation variant serves callers that may not call cudaMalloc (a
real-time loop with memory fixed at start-up, or code that only receives
its buffers); its scratch is a static device array instead of a workspace.
Both calls go through the C ABI; the variant must give the workspace
version's loss (within the double-precision reduction's rounding) and the
same gradient, on two calls in a row (the array keeps the previous call's
contents), and must reject sizes beyond its static scratch.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_image_l1_noalloc_matches_workspace_call():
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    from paper_2510_26358_gb300 import scenes as S

    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    cams = [S.Camera(320, 240, 300.0, 300.0, 160.0, 120.0, np.eye(3, 4), 0),
            S.Camera(200, 100, 180.0, 180.0, 100.0, 50.0, np.eye(3, 4), 0)]
    r = G.Renderer(cams, [0, 1], 0, inst_capacity=1 << 10)
    n = 3 * r.n_pix
    stream = G._stream()
    ptr = G._ptr
    try:
        for seed in (0, 1):
            gen = torch.Generator(device="cpu").manual_seed(seed)
            rgb = torch.rand(n, generator=gen).to(dev)
            target = torch.rand(n, generator=gen).to(dev)
            loss_ws, grad_ws = torch.zeros(1, device=dev), torch.zeros(n, device=dev)
            G.gs_image_l1(r.ws, ptr(rgb), ptr(target), ptr(loss_ws), ptr(grad_ws), stream)
            for call in range(2):
                loss_na, grad_na = torch.full((1,), -1.0, device=dev), torch.zeros(n, device=dev)
                G.gs_image_l1_noalloc(ptr(rgb), ptr(target), n, ptr(loss_na), ptr(grad_na), stream)
                torch.cuda.synchronize()
                ref = loss_ws.item()
                assert abs(loss_na.item() - ref) <= 1e-6 * abs(ref), (seed, call, loss_na.item(), ref)
                assert torch.equal(grad_na, grad_ws), (seed, call)
        # a size beyond the static scratch is refused before anything runs
        big = G.IMAGE_L1_NOALLOC_MAX + 1
        st = G.lib().gs_image_l1_noalloc(ptr(rgb), ptr(target), ctypes.c_int64(big), ptr(loss_na), None,
                                         stream)
        assert st == G.GS_ERR_INVALID_ARG
        assert "static scratch" in G.last_error()
        # n = 0 gives a zero loss
        loss0 = torch.full((1,), 5.0, device=dev)
        G.gs_image_l1_noalloc(ptr(rgb), ptr(target), 0, ptr(loss0), None, stream)
        torch.cuda.synchronize()
        assert loss0.item() == 0.0
    finally:
        r.close()
