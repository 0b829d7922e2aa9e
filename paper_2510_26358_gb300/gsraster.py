"""Thin Python binding of libgsraster (include/gs.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  The functions below carry the C names and raise ``GsError`` on
a non-OK status.  ``Renderer`` holds a workspace plus the device copy of the
cameras and passes torch tensors' device pointers and the current CUDA
stream; ``GSRender`` wraps forward and backward as a torch.autograd.Function.

There is no fallback: if ``libgsraster.so`` has not been built, loading fails
with an error that says so.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgsraster.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_STATE, GS_ERR_TIMEOUT = range(6)
GS_MAX_VIEWS = 64
GS_MAX_SUBMAPS = 64
# gs_workspace_copy buffer ids
(BUF_RECORDS, BUF_PAIR_KEYS, BUF_RECTS, BUF_INST_TILES, BUF_INST_PAIRS, BUF_RANGES, BUF_LAST, BUF_TFIN, BUF_G2D,
 BUF_VSTAT) = range(10)

EXPORTED = ("gs_config_default", "gs_workspace_create", "gs_workspace_destroy", "gs_project",
            "gs_bin_sort", "gs_render_fwd", "gs_render_fwd_var", "gs_depth_loss", "gs_depth_loss_var",
            "gs_image_l1", "gs_image_l1_u8", "gs_image_loss", "gs_render_bwd", "gs_render_bwd_var",
            "gs_workspace_status", "gs_workspace_info", "gs_workspace_copy", "gs_workspace_set_profiling",
            "gs_workspace_stage_ms", "gs_image_l1_noalloc", "gs_status_string", "gs_last_error",
            "gs_lifecycle_create", "gs_lifecycle_destroy", "gs_lifecycle_run", "gs_lifecycle_status", "gs_adam_step",
            "gs_voxel_keys", "gs_voxel_create", "gs_voxel_destroy", "gs_voxel_insert", "gs_voxel_status",
            "gs_active_select", "gs_partition", "gs_selftest_wait_timeout", "gs_zero_buffers", "gs_alu_probe",
            "gs_workspace_fragment_counts")
GS_LC_PRUNE, GS_LC_DENSIFY, GS_LC_RESET = 1, 2, 4
PARAM_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")
IMAGE_L1_NOALLOC_MAX = 1024 * 65536  # GS_IMAGE_L1_NOALLOC_BLOCKS * GS_IMAGE_L1_NOALLOC_CHUNK
STAGES = ("project", "compact", "depth_sort", "emit", "tile_sort", "ranges", "raster_fwd", "image_l1",
          "depth_loss", "zero_grad", "raster_bwd", "project_bwd", "image_ssim")


class GsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})" + (f": {detail}" if detail else ""))


class GsCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("submap", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("T_cw", ctypes.c_float * 12)]


class GsConfig(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("batch_depth", ctypes.c_int32),
                ("depth_mode", ctypes.c_int32), ("near_z", ctypes.c_float), ("dilation", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float), ("t_min", ctypes.c_float),
                ("jac_clamp", ctypes.c_float), ("ext_rel_pad", ctypes.c_float),
                ("ext_abs_pad", ctypes.c_float), ("sigma_L", ctypes.c_float), ("sigma_U", ctypes.c_float),
                ("lambda_L", ctypes.c_float), ("reserved", ctypes.c_float)]


class GsGaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("n", ctypes.c_int64)]


class GsGrads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("pose", ctypes.c_void_p),
                ("densify_acc", ctypes.c_void_p), ("densify_cnt", ctypes.c_void_p), ("overwrite", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class GsParamArrays(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]


class GsLifecycleParams(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_int32)] + [(k, ctypes.c_float) for k in (
        "prune_opacity", "prune_scale_max", "prune_scale_min", "densify_grad", "split_scale", "clone_scale",
        "split_shrink", "reset_opacity", "reset_scale_min", "reset_scale_max")]


class GsAdamParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 5), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", ctypes.c_int32)]


class GsInsertParams(ctypes.Structure):
    _fields_ = [("voxel", ctypes.c_float), ("s_init", ctypes.c_float), ("o_init", ctypes.c_float),
                ("frame", ctypes.c_int32)]


assert ctypes.sizeof(GsCamera) == 80 and ctypes.sizeof(GsConfig) == 64

_lib = None


def lib() -> ctypes.CDLL:
    """Load libgsraster.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                           "g.build()'` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.gs_config_default.argtypes = [ctypes.POINTER(GsConfig)]
    L.gs_config_default.restype = None
    L.gs_workspace_create.argtypes = [ctypes.POINTER(GsCamera), i32, ctypes.POINTER(ctypes.c_int64), i32, i32,
                                      ctypes.POINTER(GsConfig), i64, ctypes.POINTER(ctypes.c_void_p)]
    L.gs_workspace_destroy.argtypes = [P]
    L.gs_workspace_destroy.restype = None
    L.gs_project.argtypes = [P, ctypes.POINTER(GsGaussians), P, P]
    L.gs_bin_sort.argtypes = [P, P]
    L.gs_render_fwd.argtypes = [P, P, P, P, P]
    L.gs_render_fwd_var.argtypes = [P, P, P, P, P, P, P]
    L.gs_depth_loss.argtypes = [P, P, P, P, i64, P, P, P]
    L.gs_depth_loss_var.argtypes = [P, P, P, P, P, i64, P, P, P, P]
    L.gs_image_l1.argtypes = [P, P, P, P, P, P]
    L.gs_image_l1_u8.argtypes = [P, P, P, P, P, P]
    L.gs_image_loss.argtypes = [P, P, P, ctypes.c_float, P, P, P]
    L.gs_render_bwd.argtypes = [P, ctypes.POINTER(GsGaussians), P, P, P, P, ctypes.POINTER(GsGrads), P]
    L.gs_render_bwd_var.argtypes = [P, ctypes.POINTER(GsGaussians), P, P, P, P, P, P, ctypes.POINTER(GsGrads), P]
    L.gs_workspace_status.argtypes = [P, P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.gs_workspace_info.argtypes = [P, ctypes.POINTER(ctypes.c_int64), i32]
    L.gs_workspace_copy.argtypes = [P, i32, P, ctypes.POINTER(ctypes.c_int64), P]
    L.gs_image_l1_noalloc.argtypes = [P, P, i64, P, P, P]
    L.gs_workspace_set_profiling.argtypes = [P, i32]
    L.gs_workspace_stage_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float), i32]
    PA = ctypes.POINTER(GsParamArrays)
    L.gs_lifecycle_create.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_void_p)]
    L.gs_lifecycle_destroy.argtypes = [P]
    L.gs_lifecycle_destroy.restype = None
    L.gs_lifecycle_run.argtypes = [P, ctypes.POINTER(GsLifecycleParams), i32, i64, i32, P, PA, PA, PA, P, P, P, PA,
                                   PA, PA, i64, P, P, P]
    L.gs_lifecycle_status.argtypes = [P, P, ctypes.POINTER(ctypes.c_int64)]
    L.gs_adam_step.argtypes = [PA, PA, PA, PA, i64, i32, ctypes.POINTER(GsAdamParams), P]
    L.gs_voxel_keys.argtypes = [P, i64, i32, ctypes.c_float, P, P]
    L.gs_voxel_create.argtypes = [i64, i64, ctypes.POINTER(ctypes.c_void_p)]
    L.gs_voxel_destroy.argtypes = [P]
    L.gs_voxel_destroy.restype = None
    L.gs_voxel_insert.argtypes = [P, ctypes.POINTER(GsInsertParams), P, i64, P, P, i64, P, P, i64, i32, PA, P, i64,
                                  P, P]
    L.gs_voxel_status.argtypes = [P, P, ctypes.POINTER(ctypes.c_int64)]
    L.gs_active_select.argtypes = [P, P, i64, i64, P, P]
    L.gs_partition.argtypes = [P, P, i64, i32, PA, P, P, PA, P, P, PA, P, P, P, P]
    L.gs_selftest_wait_timeout.argtypes = [P, i64, P, P]
    L.gs_zero_buffers.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64), i32, P]
    L.gs_alu_probe.argtypes = [i32, i32, i32, P, P]
    L.gs_workspace_fragment_counts.argtypes = [P, ctypes.POINTER(ctypes.c_int64), P]
    L.gs_status_string.argtypes = [i32]
    L.gs_status_string.restype = ctypes.c_char_p
    L.gs_last_error.argtypes = []
    L.gs_last_error.restype = ctypes.c_char_p
    for name in ("gs_workspace_create", "gs_project", "gs_bin_sort", "gs_render_fwd", "gs_render_fwd_var",
                 "gs_depth_loss", "gs_depth_loss_var", "gs_image_l1", "gs_image_l1_u8", "gs_image_loss", "gs_render_bwd",
                 "gs_render_bwd_var",
                 "gs_workspace_status", "gs_workspace_info",
                 "gs_workspace_copy", "gs_workspace_set_profiling", "gs_workspace_stage_ms",
                 "gs_image_l1_noalloc", "gs_lifecycle_create", "gs_lifecycle_run", "gs_lifecycle_status",
                 "gs_adam_step", "gs_voxel_keys", "gs_voxel_create", "gs_voxel_insert", "gs_voxel_status",
                 "gs_active_select", "gs_partition", "gs_selftest_wait_timeout", "gs_zero_buffers", "gs_alu_probe",
                 "gs_workspace_fragment_counts"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def param_arrays(d) -> GsParamArrays | None:
    """GsParamArrays from a dict of tensors keyed by PARAM_FIELDS (None stays None)."""
    if d is None:
        return None
    return GsParamArrays(*(d[k].data_ptr() for k in PARAM_FIELDS))


def _pa(x):
    return ctypes.byref(x) if x is not None else None


def gs_lifecycle_create(max_in, max_submaps):
    out = ctypes.c_void_p()
    _check(lib().gs_lifecycle_create(int(max_in), int(max_submaps), ctypes.byref(out)), "gs_lifecycle_create")
    return out


def gs_lifecycle_destroy(lc):
    lib().gs_lifecycle_destroy(lc)


def gs_lifecycle_run(lc, params: GsLifecycleParams, sh_degree, n_in, n_submaps, offs_in, pin, pin_m, pin_v, acc, cnt,
                     normals, pout, pout_m, pout_v, out_capacity, offs_out, n_out, stream):
    _check(lib().gs_lifecycle_run(lc, ctypes.byref(params), int(sh_degree), int(n_in), int(n_submaps), offs_in,
                                  _pa(pin), _pa(pin_m), _pa(pin_v), acc, cnt, normals, _pa(pout), _pa(pout_m),
                                  _pa(pout_v), int(out_capacity), offs_out, n_out, stream), "gs_lifecycle_run")


def gs_lifecycle_status(lc, stream):
    """Returns (status, outputs needed); does not raise on capacity."""
    n = ctypes.c_int64(0)
    st = lib().gs_lifecycle_status(lc, stream, ctypes.byref(n))
    if st not in (GS_OK, GS_ERR_CAPACITY):
        _check(st, "gs_lifecycle_status")
    return st, int(n.value)


def gs_adam_step(param, grad, m, v, n, sh_degree, params: GsAdamParams, stream):
    _check(lib().gs_adam_step(_pa(param), _pa(grad), _pa(m), _pa(v), int(n), int(sh_degree), ctypes.byref(params),
                              stream), "gs_adam_step")


def lifecycle_params(ops, **kw) -> GsLifecycleParams:
    """GsLifecycleParams with the paper's pruning thresholds and the given rest."""
    d = dict(prune_opacity=0.01, prune_scale_max=0.3, prune_scale_min=5e-5, densify_grad=2e-4, split_scale=0.02,
             clone_scale=0.01, split_shrink=1.6, reset_opacity=0.1, reset_scale_min=1e-4, reset_scale_max=0.25)
    d.update(kw)
    return GsLifecycleParams(int(ops), *(float(d[k]) for k in (
        "prune_opacity", "prune_scale_max", "prune_scale_min", "densify_grad", "split_scale", "clone_scale",
        "split_shrink", "reset_opacity", "reset_scale_min", "reset_scale_max")))


class Lifecycle:
    """Lifecycle scratch plus the torch marshalling of one pass."""

    def __init__(self, max_in, max_submaps, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.lc = gs_lifecycle_create(max_in, max_submaps)

    def close(self):
        if getattr(self, "lc", None):
            gs_lifecycle_destroy(self.lc)
            self.lc = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, params: dict, submap_offsets, sh_degree, lc_params: GsLifecycleParams, densify_acc=None,
            densify_cnt=None, split_normals=None, moments=None, capacity=None, stream=None):
        """One pass; returns (params_out, moments_out or None, submap_offsets_out [S+1] int64, n_out).
        Raises GsError(GS_ERR_CAPACITY) if the outputs exceed ``capacity`` (default 2 n)."""
        torch = self.torch
        n = params["means"].shape[0]
        cap = 2 * n if capacity is None else int(capacity)
        offs = torch.as_tensor(submap_offsets, dtype=torch.int64, device=self.device)
        alloc = lambda: {k: torch.empty((max(cap, 1),) + tuple(params[k].shape[1:]), device=self.device)
                         for k in PARAM_FIELDS}
        out = alloc()
        mom_out = (alloc(), alloc()) if moments is not None else None
        offs_out = torch.empty(offs.numel(), dtype=torch.int64, device=self.device)
        n_out = torch.empty(1, dtype=torch.int64, device=self.device)
        s = _stream(stream)
        gs_lifecycle_run(self.lc, lc_params, sh_degree, n, offs.numel() - 1, _ptr(offs), param_arrays(params),
                         param_arrays(moments[0]) if moments else None, param_arrays(moments[1]) if moments else None,
                         _ptr(densify_acc), _ptr(densify_cnt), _ptr(split_normals), param_arrays(out),
                         param_arrays(mom_out[0]) if moments else None, param_arrays(mom_out[1]) if moments else None,
                         cap, _ptr(offs_out), _ptr(n_out), s)
        st, need = gs_lifecycle_status(self.lc, s)
        if st == GS_ERR_CAPACITY:
            raise GsError(st, "gs_lifecycle_run", f"{need} outputs needed, capacity {cap}")
        trim = lambda d: {k: v[:need] for k, v in d.items()}
        return trim(out), (tuple(trim(d) for d in mom_out) if moments else None), offs_out, need


def adam_step(params: dict, grads: dict, m: dict, v: dict, sh_degree, step, lr, beta1=0.9, beta2=0.999, eps=1e-15,
              stream=None):
    """Adam on the five parameter tensors in place; ``lr`` a float or five floats."""
    lrs = [float(lr)] * 5 if isinstance(lr, (int, float)) else [float(x) for x in lr]
    p = GsAdamParams((ctypes.c_float * 5)(*lrs), float(beta1), float(beta2), float(eps), int(step))
    gs_adam_step(param_arrays(params), param_arrays(grads), param_arrays(m), param_arrays(v),
                 params["means"].shape[0], sh_degree, p, _stream(stream))


def gs_voxel_keys(xyz, n, stride, voxel, keys, stream):
    _check(lib().gs_voxel_keys(xyz, int(n), int(stride), float(voxel), keys, stream), "gs_voxel_keys")


class VoxelMap:
    """Scratch of the voxel-hash insertion and the active-set operations, with
    torch marshalling.  Keys are int64 tensors holding the unsigned 64-bit keys'
    bits; last_used, reload and flags are int32 tensors."""

    def __init__(self, max_points, max_items, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        out = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().gs_voxel_create(int(max_points), int(max_items), ctypes.byref(out)), "gs_voxel_create")
        self.vx = out

    def close(self):
        if getattr(self, "vx", None):
            lib().gs_voxel_destroy(self.vx)
            self.vx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def keys(self, xyz, voxel, stream=None):
        """Eq. (5) keys of the rows of xyz ([n, >= 3] float32)."""
        keys = self.torch.empty(xyz.shape[0], dtype=self.torch.int64, device=self.device)
        gs_voxel_keys(_ptr(xyz), xyz.shape[0], xyz.stride(0), voxel, _ptr(keys), _stream(stream))
        return keys

    def insert(self, points, splat_keys, last_used, host_keys, sh_degree, voxel, s_init, o_init, frame,
               capacity=None, stream=None):
        """Returns (reload int32 [n_host], new params dict, new keys, n_new); updates last_used in place."""
        torch = self.torch
        n_pts = points.shape[0]
        cap = n_pts if capacity is None else int(capacity)
        K = (sh_degree + 1) ** 2
        new = dict(means=torch.empty(max(cap, 1), 3, device=self.device),
                   log_scales=torch.empty(max(cap, 1), 3, device=self.device),
                   quats=torch.empty(max(cap, 1), 4, device=self.device),
                   opacity_logits=torch.empty(max(cap, 1), device=self.device),
                   sh=torch.empty(max(cap, 1), K, 3, device=self.device))
        new_keys = torch.empty(max(cap, 1), dtype=torch.int64, device=self.device)
        reload = torch.empty(host_keys.shape[0], dtype=torch.int32, device=self.device)
        p = GsInsertParams(float(voxel), float(s_init), float(o_init), int(frame))
        s = _stream(stream)
        _check(lib().gs_voxel_insert(self.vx, ctypes.byref(p), _ptr(points), n_pts, _ptr(splat_keys),
                                     _ptr(last_used), splat_keys.shape[0], _ptr(host_keys), _ptr(reload),
                                     host_keys.shape[0], int(sh_degree), ctypes.byref(param_arrays(new)),
                                     _ptr(new_keys), cap, None, s), "gs_voxel_insert")
        n = ctypes.c_int64(0)
        st = lib().gs_voxel_status(self.vx, s, ctypes.byref(n))
        if st != GS_OK:
            raise GsError(st, "gs_voxel_insert", f"{n.value} new splats, capacity {cap}")
        n = int(n.value)
        return reload, {k: v[:n] for k, v in new.items()}, new_keys[:n], n

    def select(self, last_used, tau, stream=None):
        flags = self.torch.empty(last_used.shape[0], dtype=self.torch.int32, device=self.device)
        _check(lib().gs_active_select(self.vx, _ptr(last_used), last_used.shape[0], int(tau), _ptr(flags),
                                      _stream(stream)), "gs_active_select")
        return flags

    def partition(self, flags, sh_degree, params, keys, last_used, kept, kept_keys, kept_lu, moved, moved_keys,
                  moved_lu, stream=None):
        """Stable partition into caller-allocated outputs (device or pinned host tensors)."""
        counts = self.torch.empty(2, dtype=self.torch.int64, device=self.device)
        _check(lib().gs_partition(self.vx, _ptr(flags), flags.shape[0], int(sh_degree),
                                  ctypes.byref(param_arrays(params)), _ptr(keys), _ptr(last_used),
                                  ctypes.byref(param_arrays(kept)), _ptr(kept_keys), _ptr(kept_lu),
                                  ctypes.byref(param_arrays(moved)), _ptr(moved_keys), _ptr(moved_lu),
                                  _ptr(counts), _stream(stream)), "gs_partition")
        return counts


def gs_zero_buffers(tensors, stream=None):
    """Zero up to 16 device tensors in one library launch."""
    ts = [t for t in tensors if t is not None and t.numel() > 0]
    ptrs = (ctypes.c_void_p * max(1, len(ts)))(*[t.data_ptr() for t in ts])
    sizes = (ctypes.c_int64 * max(1, len(ts)))(*[t.numel() * t.element_size() for t in ts])
    _check(lib().gs_zero_buffers(ptrs, sizes, len(ts), _stream(stream)), "gs_zero_buffers")


# operations per lane and round of gs_alu_probe's kinds (FMA = 2 FLOP) and
# their names
ALU_PROBE_KINDS = {0: ("fp32_fma", 2 * 8), 1: ("fp32x2_fma", 4 * 8), 2: ("mufu_ex2", 8), 3: ("mufu_rcp", 8)}


def gs_alu_probe(kind: int, blocks: int, iters: int, sink, stream=None):
    """One launch of the arithmetic-rate probe (see include/gs.h)."""
    _check(lib().gs_alu_probe(int(kind), int(blocks), int(iters), _ptr(sink), _stream(stream)), "gs_alu_probe")


def gs_workspace_fragment_counts(ws, stream=None) -> dict:
    """(pixel, entry) pairs walked and blended, (tile, entry) pairs walked and
    with a blend, for the last forward (synchronises)."""
    c = (ctypes.c_int64 * 4)()
    _check(lib().gs_workspace_fragment_counts(ws, c, _stream(stream)), "gs_workspace_fragment_counts")
    return dict(pixel_entries=int(c[0]), pixel_blends=int(c[1]), tile_entries=int(c[2]), tile_active=int(c[3]))


def status_string(s: int) -> str:
    return lib().gs_status_string(int(s)).decode()


def last_error() -> str:
    return lib().gs_last_error().decode()


def _check(st: int, where: str):
    if st != GS_OK:
        raise GsError(st, where, last_error())


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------

def gs_config_default(**overrides) -> GsConfig:
    c = GsConfig()
    lib().gs_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def gs_workspace_create(cams, n_views, submap_offsets, n_submaps, sh_degree, cfg, inst_capacity):
    out = ctypes.c_void_p()
    offs = (ctypes.c_int64 * (n_submaps + 1))(*[int(x) for x in submap_offsets])
    _check(lib().gs_workspace_create(cams, n_views, offs, n_submaps, sh_degree, ctypes.byref(cfg),
                                     int(inst_capacity), ctypes.byref(out)), "gs_workspace_create")
    return out


def gs_workspace_destroy(ws):
    lib().gs_workspace_destroy(ws)


def gs_project(ws, g: GsGaussians, cams_dev, stream):
    _check(lib().gs_project(ws, ctypes.byref(g), cams_dev, stream), "gs_project")


def gs_bin_sort(ws, stream):
    _check(lib().gs_bin_sort(ws, stream), "gs_bin_sort")


def gs_render_fwd(ws, rgb, depth, alpha, stream):
    _check(lib().gs_render_fwd(ws, rgb, depth, alpha, stream), "gs_render_fwd")


def gs_render_fwd_var(ws, rgb, depth, alpha, depth_mean, depth_var, stream):
    _check(lib().gs_render_fwd_var(ws, rgb, depth, alpha, depth_mean, depth_var, stream), "gs_render_fwd_var")


def gs_depth_loss(ws, depth, alpha, lidar, n_pts, loss, dL_ddepth, stream):
    _check(lib().gs_depth_loss(ws, depth, alpha, lidar, int(n_pts), loss, dL_ddepth, stream), "gs_depth_loss")


def gs_depth_loss_var(ws, alpha, depth_mean, depth_var, lidar, n_pts, loss, dL_dmean, dL_dvar, stream):
    _check(lib().gs_depth_loss_var(ws, alpha, depth_mean, depth_var, lidar, int(n_pts), loss, dL_dmean, dL_dvar,
                                   stream), "gs_depth_loss_var")


def gs_image_l1(ws, rgb, target, loss, dL_drgb, stream):
    _check(lib().gs_image_l1(ws, rgb, target, loss, dL_drgb, stream), "gs_image_l1")


def gs_image_l1_u8(ws, rgb, target_u8, loss, dL_drgb, stream):
    _check(lib().gs_image_l1_u8(ws, rgb, target_u8, loss, dL_drgb, stream), "gs_image_l1_u8")


def gs_image_loss(ws, rgb, target, lam, loss, dL_drgb, stream):
    _check(lib().gs_image_loss(ws, rgb, target, float(lam), loss, dL_drgb, stream), "gs_image_loss")


def gs_image_l1_noalloc(rgb, target, n, loss, dL_drgb, stream):
    """L1 image loss without a workspace; see include/gs.h for its static scratch."""
    _check(lib().gs_image_l1_noalloc(rgb, target, int(n), loss, dL_drgb, stream), "gs_image_l1_noalloc")


def gs_render_bwd(ws, g: GsGaussians, cams_dev, dL_drgb, dL_ddepth, dL_dalpha, grads: GsGrads, stream):
    _check(lib().gs_render_bwd(ws, ctypes.byref(g), cams_dev, dL_drgb, dL_ddepth, dL_dalpha,
                               ctypes.byref(grads), stream), "gs_render_bwd")


def gs_render_bwd_var(ws, g: GsGaussians, cams_dev, dL_drgb, dL_ddepth, dL_dalpha, dL_dmean, dL_dvar,
                      grads: GsGrads, stream):
    _check(lib().gs_render_bwd_var(ws, ctypes.byref(g), cams_dev, dL_drgb, dL_ddepth, dL_dalpha, dL_dmean, dL_dvar,
                                   ctypes.byref(grads), stream), "gs_render_bwd_var")


def gs_workspace_status(ws, stream):
    """Returns (status, n_instances_needed, n_visible); does not raise on capacity."""
    ni, nv = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib().gs_workspace_status(ws, stream, ctypes.byref(ni), ctypes.byref(nv))
    if st not in (GS_OK, GS_ERR_CAPACITY):
        _check(st, "gs_workspace_status")
    return st, int(ni.value), int(nv.value)


def gs_workspace_info(ws) -> dict:
    v = (ctypes.c_int64 * 8)()
    _check(lib().gs_workspace_info(ws, v, 8), "gs_workspace_info")
    keys = ("n_pairs", "n_tiles", "n_pix", "inst_capacity", "n_views", "n", "bytes", "kernel_launches")
    return dict(zip(keys, [int(x) for x in v]))


def gs_workspace_copy(ws, which, dst, nbytes, stream):
    b = ctypes.c_int64(nbytes)
    _check(lib().gs_workspace_copy(ws, int(which), dst, ctypes.byref(b), stream), "gs_workspace_copy")
    return b.value


def gs_workspace_set_profiling(ws, on: bool):
    _check(lib().gs_workspace_set_profiling(ws, 1 if on else 0), "gs_workspace_set_profiling")


def gs_workspace_stage_ms(ws) -> dict:
    """Last duration (ms) of each stage; stages that did not run are omitted."""
    v = (ctypes.c_float * len(STAGES))()
    _check(lib().gs_workspace_stage_ms(ws, v, len(STAGES)), "gs_workspace_stage_ms")
    return {n: float(x) for n, x in zip(STAGES, v) if x >= 0}


def gs_workspace_buffer_bytes(ws, which) -> int:
    b = ctypes.c_int64(0)
    _check(lib().gs_workspace_copy(ws, int(which), None, ctypes.byref(b), None), "gs_workspace_copy")
    return int(b.value)


# ---------------------------------------------------------------------------
# torch convenience layer (marshalling only)
# ---------------------------------------------------------------------------

def camera_structs(cameras) -> ctypes.Array:
    """ctypes array of GsCamera from objects with width/height/submap/fx/fy/cx/cy/T_cw."""
    arr = (GsCamera * len(cameras))()
    for i, c in enumerate(cameras):
        arr[i].width, arr[i].height, arr[i].submap, arr[i].reserved = int(c.width), int(c.height), int(c.submap), 0
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        T = np.asarray(c.T_cw, np.float64).reshape(12)
        for k in range(12):
            arr[i].T_cw[k] = float(T[k])
    return arr


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Renderer:
    """A workspace for a fixed rig (camera sizes, submap partition, SH degree)
    and the device copy of the cameras.  All tensors are float32 CUDA tensors."""

    def __init__(self, cameras, submap_offsets, sh_degree, config: GsConfig | None = None,
                 inst_capacity: int | None = None, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.cameras = list(cameras)
        self.n_views = len(self.cameras)
        self.submap_offsets = [int(x) for x in submap_offsets]
        self.n = self.submap_offsets[-1]
        self.sh_degree = int(sh_degree)
        self.config = config or gs_config_default()
        cams = camera_structs(self.cameras)
        self.n_pix = sum(c.width * c.height for c in self.cameras)
        if inst_capacity is None:
            inst_capacity = max(1 << 20, 16 * self.n * max(1, self.n_views))
            inst_capacity = min(inst_capacity, (1 << 31) - 1)
        with torch.cuda.device(self.device):
            self.ws = gs_workspace_create(cams, self.n_views, self.submap_offsets, len(self.submap_offsets) - 1,
                                          self.sh_degree, self.config, inst_capacity)
        self.info = gs_workspace_info(self.ws)
        self.cams_dev = torch.empty(ctypes.sizeof(cams), dtype=torch.uint8, device=self.device)
        self.set_cameras(self.cameras)

    def close(self):
        if getattr(self, "ws", None):
            gs_workspace_destroy(self.ws)
            self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_cameras(self, cameras):
        """Upload intrinsics and poses (sizes and submaps must not change)."""
        cams = camera_structs(cameras)
        host = self.torch.frombuffer(bytearray(bytes(cams)), dtype=self.torch.uint8)
        self.cams_dev.copy_(host.to(self.device, non_blocking=False))
        self.cameras = list(cameras)

    @staticmethod
    def gaussians(means, log_scales, quats, opacity_logits, sh) -> GsGaussians:
        return GsGaussians(means.data_ptr(), log_scales.data_ptr(), quats.data_ptr(),
                           opacity_logits.data_ptr(), sh.data_ptr(), means.shape[0])

    def forward(self, means, log_scales, quats, opacity_logits, sh, stream=None, outputs=None, var=False):
        """project -> bin/sort -> rasterise. Returns (rgb [3*N_pix], depth [N_pix], alpha [N_pix]), plus
        the depth mean and variance [N_pix] each when ``var``."""
        torch = self.torch
        s = _stream(stream)
        g = self.gaussians(means, log_scales, quats, opacity_logits, sh)
        if outputs is None:
            outputs = tuple([torch.empty(3 * self.n_pix, device=self.device)] +
                            [torch.empty(self.n_pix, device=self.device) for _ in range(4 if var else 2)])
        gs_project(self.ws, g, _ptr(self.cams_dev), s)
        gs_bin_sort(self.ws, s)
        if var:
            rgb, depth, alpha, mean, dvar = outputs
            gs_render_fwd_var(self.ws, _ptr(rgb), _ptr(depth), _ptr(alpha), _ptr(mean), _ptr(dvar), s)
            return rgb, depth, alpha, mean, dvar
        rgb, depth, alpha = outputs
        gs_render_fwd(self.ws, _ptr(rgb), _ptr(depth), _ptr(alpha), s)
        return rgb, depth, alpha

    def backward(self, means, log_scales, quats, opacity_logits, sh, dL_drgb, dL_ddepth, dL_dalpha=None,
                 grads=None, stream=None, pose=True, densify=True, var=False, dL_dmean=None, dL_dvar=None,
                 overwrite=None):
        """Gradients into ``grads`` (dict of tensors): accumulated, or written when ``overwrite``.  If
        ``grads`` is None they are allocated uninitialised and written (``overwrite`` defaults to
        True then, else to False).  With ``var`` the adjoints of the depth mean and variance are
        taken too (after ``forward(var=True)``)."""
        torch = self.torch
        s = _stream(stream)
        g = self.gaussians(means, log_scales, quats, opacity_logits, sh)
        if overwrite is None:
            overwrite = grads is None
        if grads is None:
            new = torch.empty_like if overwrite else torch.zeros_like
            grads = dict(means=new(means), log_scales=new(log_scales), quats=new(quats),
                         opacity_logits=new(opacity_logits), sh=new(sh))
            if pose:
                grads["pose"] = new(torch.empty(self.n_views, 6, device=self.device))
            if densify:
                grads["densify_acc"] = new(torch.empty(self.n, device=self.device))
                grads["densify_cnt"] = new(torch.empty(self.n, dtype=torch.int32, device=self.device))
        gg = GsGrads(grads["means"].data_ptr(), grads["log_scales"].data_ptr(), grads["quats"].data_ptr(),
                     grads["opacity_logits"].data_ptr(), grads["sh"].data_ptr(),
                     grads["pose"].data_ptr() if "pose" in grads else None,
                     grads["densify_acc"].data_ptr() if "densify_acc" in grads else None,
                     grads["densify_cnt"].data_ptr() if "densify_cnt" in grads else None, int(bool(overwrite)), 0)
        if var:
            gs_render_bwd_var(self.ws, g, _ptr(self.cams_dev), _ptr(dL_drgb), _ptr(dL_ddepth), _ptr(dL_dalpha),
                              _ptr(dL_dmean), _ptr(dL_dvar), gg, s)
        else:
            gs_render_bwd(self.ws, g, _ptr(self.cams_dev), _ptr(dL_drgb), _ptr(dL_ddepth), _ptr(dL_dalpha), gg, s)
        return grads

    def depth_loss(self, depth, alpha, lidar, dL_ddepth=None, stream=None):
        loss = self.torch.zeros(1, device=self.device)
        gs_depth_loss(self.ws, _ptr(depth), _ptr(alpha), _ptr(lidar), lidar.shape[0], _ptr(loss),
                      _ptr(dL_ddepth), _stream(stream))
        return loss

    def depth_loss_var(self, alpha, mean, var, lidar, grads=None, stream=None):
        """Eq. (7) with the rendered variance; ``grads`` = (d_mean, d_var) tensors (each may be None)
        accumulated in place."""
        loss = self.torch.zeros(1, device=self.device)
        gm, gv = grads if grads is not None else (None, None)
        gs_depth_loss_var(self.ws, _ptr(alpha), _ptr(mean), _ptr(var), _ptr(lidar), lidar.shape[0],
                          _ptr(loss), _ptr(gm), _ptr(gv), _stream(stream))
        return loss

    def image_l1(self, rgb, target, dL_drgb=None, stream=None):
        """Mean |rgb - target| (accumulates dL/drgb when given); an 8-bit target
        tensor (torch.uint8) stands for target / 255."""
        loss = self.torch.zeros(1, device=self.device)
        f = gs_image_l1_u8 if target.dtype == self.torch.uint8 else gs_image_l1
        f(self.ws, _ptr(rgb), _ptr(target), _ptr(loss), _ptr(dL_drgb), _stream(stream))
        return loss

    def image_loss(self, rgb, target, lam=0.2, dL_drgb=None, stream=None):
        """Eq. (6): returns a [3] tensor (total, L1, 1 - SSIM); accumulates dL/drgb when given."""
        loss = self.torch.zeros(3, device=self.device)
        gs_image_loss(self.ws, _ptr(rgb), _ptr(target), lam, _ptr(loss), _ptr(dL_drgb), _stream(stream))
        return loss

    def status(self, stream=None):
        return gs_workspace_status(self.ws, _stream(stream))

    def buffer(self, which, dtype):
        torch = self.torch
        nb = gs_workspace_buffer_bytes(self.ws, which)
        out = torch.empty(nb, dtype=torch.uint8, device=self.device)
        gs_workspace_copy(self.ws, which, _ptr(out), nb, _stream())
        return out.view(dtype)


def _make_render_function():
    import torch

    class GSRender(torch.autograd.Function):
        """(rgb, depth, alpha) = GSRender.apply(renderer, means, log_scales, quats, opacity_logits, sh,
        pose_delta).  ``pose_delta`` is a [V, 6] tensor whose gradient is the pose twist gradient
        dL/d(rho, phi) at zero (its value is not used: poses come from the renderer's cameras)."""

        @staticmethod
        def forward(ctx, renderer, means, log_scales, quats, opacity_logits, sh, pose_delta):
            rgb, depth, alpha = renderer.forward(means, log_scales, quats, opacity_logits, sh)
            ctx.renderer = renderer
            ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh)
            return rgb, depth, alpha

        @staticmethod
        def backward(ctx, g_rgb, g_depth, g_alpha):
            means, log_scales, quats, opacity_logits, sh = ctx.saved_tensors
            r = ctx.renderer
            z = lambda t, n: t.contiguous() if t is not None else torch.zeros(n, device=r.device)
            grads = r.backward(means, log_scales, quats, opacity_logits, sh, z(g_rgb, 3 * r.n_pix),
                               z(g_depth, r.n_pix), z(g_alpha, r.n_pix), densify=False)
            return (None, grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"],
                    grads["sh"], grads["pose"])

    return GSRender


_GSRender = None


def GSRender():
    global _GSRender
    if _GSRender is None:
        _GSRender = _make_render_function()
    return _GSRender
