"""CPU-side checks of the boundary: the library loads without a GPU and
exports every function include/gs.h declares; argument errors are returned
before any CUDA call; the bench's replica aggregation over ranks."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    from paper_2510_26358_gb300 import build
    build.build()
    from paper_2510_26358_gb300 import gsraster
    return gsraster


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gs_project", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_depth_loss"):
        assert must in names


def test_library_exports_every_declared_function(G):
    L = G.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(G.EXPORTED) == set(declared_functions())


def test_defaults_and_status_strings(G):
    c = G.gs_config_default()
    assert (c.tile_w, c.tile_h, c.batch_depth) == (16, 16, 256)
    assert c.alpha_min == pytest.approx(1 / 255) and c.alpha_max == pytest.approx(0.99)
    assert c.t_min == pytest.approx(1e-4) and c.dilation == pytest.approx(0.3)
    assert G.status_string(G.GS_ERR_CAPACITY) == "instance capacity exceeded"


def test_argument_errors_before_any_cuda_call(G):
    L = G.lib()
    from paper_2510_26358_gb300 import scenes as S
    cams = G.camera_structs([S.Camera(32, 32, 30.0, 30.0, 16.0, 16.0, np.eye(3, 4), 0)])
    offs = (ctypes.c_int64 * 2)(0, 10)
    out = ctypes.c_void_p()
    cfg = G.gs_config_default()
    E = G.GS_ERR_INVALID_ARG
    assert L.gs_workspace_create(cams, 0, offs, 1, 0, ctypes.byref(cfg), 1000, ctypes.byref(out)) == E
    assert L.gs_workspace_create(cams, 1, offs, 0, 0, ctypes.byref(cfg), 1000, ctypes.byref(out)) == E
    assert L.gs_workspace_create(cams, 1, offs, 1, 0, ctypes.byref(cfg), 0, ctypes.byref(out)) == E
    bad_offs = (ctypes.c_int64 * 2)(5, 10)
    assert L.gs_workspace_create(cams, 1, bad_offs, 1, 0, ctypes.byref(cfg), 10, ctypes.byref(out)) == E
    cams[0].submap = 3
    assert L.gs_workspace_create(cams, 1, offs, 1, 0, ctypes.byref(cfg), 10, ctypes.byref(out)) == E
    assert "submap" in G.last_error()
    assert L.gs_project(None, None, None, None) == E
    assert L.gs_image_l1_noalloc(None, None, 10, None, None, None) == E
    assert L.gs_image_l1_u8(None, None, None, None, None, None) == E


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms = bench.max_over_ranks(1.0 + rank, "cpu")
    q.put((rank, ms, bench.job_throughput(1_000_000, ms, world)))
    dist.destroy_process_group()


def test_replica_aggregation_takes_the_slowest_rank():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    for rank, ms, value in res:
        assert ms == 2.0                       # max over ranks
        assert value == pytest.approx(1_000_000 * 2 / 2e-3 / 1e6)
