#!/usr/bin/env python3
"""Benchmark of the batched multi-view Gaussian-splatting mapping step.

One step = one mapping iteration of a keyframe (Sec. III-B/C): project every
(view, Gaussian) pair, bin and sort, rasterise RGB + depth + alpha for all
cameras, the L1 photometric loss (Eq. 6, lambda = 0) and the LiDAR depth loss
(Eq. 7), then the full backward to every Gaussian parameter and every camera
pose.  The metric is rendered megapixels per second over the whole step.

Default workload: the large keyframe map, 4M Gaussians over a 9-row x 40 m
orchard (trunk cylinders + canopy balls, SH degree 3) seen by two 3-camera
rigs of 1920x1200, with the KL depth-consistency term of Eq. 7 on 100k LiDAR
returns per view and the per-Gaussian densification statistics accumulated
in the backward.  ``--workload orchard500k --depth-loss l1`` runs the 500k
orchard (3 x 1280x720, 20k returns a view).  Synthetic, seeded.

Arms:
  default            the batched path: one CUDA graph per step covering every
                     kernel of every view; L2 flushed between timed steps.
  --impl reference   the FP64 CPU oracle on a bounded sample of the same
                     workload (this paper ships no code to compare against).

Multi-GPU (--gpus N under torchrun): the path does not exchange anything
between keyframes, so each rank runs an independent replica (weak scaling);
value = pixels of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd rendered Mpix/s (RGB+depth, multi-view batch)"
UNIT = "Mpix/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="orchard4m")
    ap.add_argument("--tile", default="auto", help="WxH, or auto to let the autotuner pick tile and depth")
    ap.add_argument("--depth", type=int, default=256)
    ap.add_argument("--no-per-view", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="crop width (px) of each view in the oracle sample (0: full frames)")
    ap.add_argument("--cpu-views", type=int, default=-1,
                    help="views in the oracle sample (0: all; -1: the workload's default)")
    ap.add_argument("--ssim-lambda", type=float, default=0.0,
                    help="weight lambda of the SSIM term of Eq. 6 (0: L1 image loss only)")
    ap.add_argument("--adam", action="store_true",
                    help="end the step with an Adam update of every Gaussian parameter (inside the timed graph)")
    ap.add_argument("--lifecycle", action="store_true",
                    help="also time one map-lifecycle pass (prune, reset, split / clone) on the workload")
    ap.add_argument("--active-set", action="store_true",
                    help="also time voxel-hash insertion of a point batch, LRU selection and an offload to host memory")
    ap.add_argument("--once", action="store_true",
                    help="run the step twice (sizing, then one more) and exit without timing: a short program "
                         "for profilers, whose launches are exactly one step's after the first")
    ap.add_argument("--depth-loss", default="kl", choices=list(DEPTH_LOSSES),
                    help="depth term of the step: l1, kl (Eq. 7, fixed sigma_u) or kl-var (Eq. 7 with the "
                         "rendered variance: forward and backward with the central depth moment)")
    return ap.parse_args()


DEPTH_LOSSES = {"l1": "L1 depth", "kl": "KL depth (fixed sigma_u)", "kl-var": "KL depth (rendered variance)"}


def loss_label(args) -> str:
    lam = getattr(args, "ssim_lambda", 0.0)
    img = "L1 rgb" if lam == 0 else f"(1 - {lam:g}) L1 + {lam:g} (1 - SSIM) rgb"
    return img + " + " + DEPTH_LOSSES[getattr(args, "depth_loss", "l1")] + (" + Adam" if getattr(args, "adam", False)
                                                                           else "")


# per-array learning rates of the Adam option (means, log-scales, quaternions,
# opacity logits, SH): the usual 3DGS values
ADAM_LR = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)


def workload_config(sc, args, tile=None, depth=None):
    W = sorted({(c.width, c.height) for c in sc.cameras})
    return {"workload": sc.name, "n_gaussians": sc.n, "views": len(sc.cameras),
            "resolutions": [f"{w}x{h}" for w, h in W], "n_pix": sc.n_pix, "sh_degree": sc.sh_degree,
            "lidar_points": int(sc.lidar.shape[0]), "losses": loss_label(args),
            "tile": tile or args.tile, "batch_depth": depth or args.depth,
            "l2": "flushed (512 MiB write) before every timed step", "graph": True,
            "parallelism": "replicas", "seed": 0}


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3], parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i, f in enumerate(r[4]) if f.lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def gpu_uuid(torch):
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        return "GPU-" + str(u)
    except Exception:
        return str(torch.cuda.current_device())


def max_over_ranks(ms: float, device) -> float:
    """Slowest rank's step time (the job's time); no-op without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


# the raster kernels and the binning that makes the instance lists they read
RASTER_SOURCES = ("paper_2510_26358_gb300/csrc/gs_raster.cu", "paper_2510_26358_gb300/csrc/gs_frag.cuh",
                  "paper_2510_26358_gb300/csrc/gs_sort.cu")


def raster_source_hash() -> str:
    """sha1 of the code of RASTER_SOURCES with comments and whitespace removed,
    so that an edit of a comment does not void a recorded measurement."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in RASTER_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload: str, config: str, alg_bytes=None):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summary, if it was captured from the current raster sources with the same
    tile size (the batch depth does not change what the backward stages).  On
    another workload it is scaled by the ratio of algorithmic bytes per launch
    (the kernel's traffic grows with the units it processes), when the record
    holds its own algorithmic bytes; otherwise None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)[kernel]
    except (OSError, KeyError, ValueError):
        return None, "no ncu capture recorded"
    if rec.get("source_sha1") != raster_source_hash():
        return None, "kernel changed since the ncu capture"
    if rec.get("config", "").split("/")[0] != config.split("/")[0]:
        return None, f"ncu capture was on {rec.get('workload')} {rec.get('config')}"
    if rec.get("workload") == workload:
        return int(rec["dram_bytes_per_launch"]), rec.get("command", "")
    if alg_bytes and rec.get("algorithmic_bytes"):
        scaled = int(rec["dram_bytes_per_launch"] * alg_bytes / rec["algorithmic_bytes"])
        return scaled, (f"scaled from the {rec['workload']} capture ({rec['dram_bytes_per_launch']} B for "
                        f"{rec['algorithmic_bytes']} algorithmic B) by algorithmic bytes: {rec.get('command', '')}")
    return None, f"ncu capture was on {rec.get('workload')} {rec.get('config')}"


# FP32 operations of the rasterisers per (pixel, list entry), from their
# steps (an FMA counts 2).  Every entry a pixel walks: offset to the mean 2,
# exponent through the Cholesky factor 8 (then one MUFU ex2 where it blends).
EVAL_FLOPS = 10
# every fragment the backward blends: alpha clamp 1, T recovery 2, weight 1,
# h 8, dL/dalpha 3, suffix sum 2, colour and depth gradients 8, dL/dpw 1,
# opacity gradient 1, conic and mean moments 12 (plus one MUFU rcp)
BWD_BLEND_FLOPS = 39
# extra per blend of the variance backward: dz 1, h 4, dL/dz 4
VAR_BLEND_FLOPS = 9
# every fragment the forward blends: alpha clamp 1, T update 2, weight 1,
# colour and depth sums 8
FWD_BLEND_FLOPS = 12


def measure_alu_peaks(torch, G, dev, n_sm, reps=5):
    """FP32 FMA, packed f32x2 FMA and MUFU ex2 / rcp rates of this GPU from
    the library's probe: 8 blocks of 256 threads per SM, each thread running
    long independent chains of one instruction; best of `reps` launches
    timed with CUDA events.  Returns TFLOP/s (FMA kinds) and T op/s (MUFU)."""
    sink = torch.zeros(1, device=dev)
    blocks = 8 * n_sm
    out = {}
    for kind, (name, ops_per_round) in G.ALU_PROBE_KINDS.items():
        iters = 1 << 15 if kind < 2 else 1 << 13
        G.gs_alu_probe(kind, blocks, 64, sink)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        torch.cuda.synchronize()
        for r in range(reps):
            ev[2 * r].record()
            G.gs_alu_probe(kind, blocks, iters, sink)
            ev[2 * r + 1].record()
        torch.cuda.synchronize()
        best = min(ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(reps))
        out[name] = blocks * 256 * iters * ops_per_round / (best * 1e-3) / 1e12
    out["unit"] = "TFLOP/s (FMA kinds, an FMA = 2), T op/s (MUFU)"
    out["how"] = f"gs_alu_probe: {blocks} blocks x 256 threads, 8 independent chains, best of {reps}"
    return out


def stage_bytes(u, args):
    """Algorithmic (unique) bytes each library stage must move: every array
    read or written once, repeated reads of a record assumed to hit L2, a
    radix sort counted at one pass (read and write key + value)."""
    P = 4 * (3 + 3 + 4 + 1 + 3 * u["sh_coeffs"])
    var = args.depth_loss == "kl-var"
    return {
        # geometry of every Gaussian (44 B), SH of those seen, per pair the
        # depth key and rectangle, per visible pair its 48-byte record and its
        # image-space gradient row cleared (40 B)
        "project": 44 * u["N"] + (P - 44) * u["touched"] + 12 * u["pairs"] + 88 * u["visible"],
        # every pair's key read, the visible (key, pair) written
        "compact": 4 * u["pairs"] + 8 * u["visible"],
        "depth_sort": 16 * u["visible"],
        # per visible pair its id, rectangle and the 32 B of record the tile
        # test reads; per instance (tile, pair) written
        "emit": 44 * u["visible"] + 8 * u["instances"],
        "tile_sort": 16 * u["instances"],
        # tile ids read; ranges and the work order written
        "ranges": 4 * u["instances"] + 12 * u["tiles"],
        # ranges, listed pair ids, records once; rgb, depth, alpha, count, T written
        "raster_fwd": 8 * u["tiles"] + 4 * u["listed"] + 48 * u["visible"] + (28 + (24 if var else 0)) * u["pix"],
        # rgb and (float) target read, gradient read and written
        "image_l1": 48 * u["pix"],
        # returns read, depth and alpha gathered, dL/dD read and written
        "depth_loss": 32 * u["lidar"],
        # (only a second backward of one projection clears the rows itself)
        "zero_grad": 40 * u["visible"],
        # ranges, listed pair ids, records once, per-pixel inputs, image-space gradients written
        "raster_bwd": 8 * u["tiles"] + 4 * u["listed"] + 48 * u["visible"] + (44 if var else 24) * u["pix"]
        + 40 * u["visible"],
        # params of the seen Gaussians read; every Gaussian's gradient row and
        # densification statistic written (the step writes them, zeros for the
        # unseen); per visible pair its image-space gradient and view-direction
        # gradient (written by the SH adjoint, read by the geometric one)
        "project_bwd": P * u["touched"] + (P + 8) * u["N"] + (40 + 32) * u["visible"],
    }


def roofline_report(u, kern, step_ms, hbm_peak, hbm_src, alu, args, tw, th):
    """Per-stage HBM rooflines, the step's, and the raster kernels' FP32
    rooflines against the measured FMA rate."""
    b = stage_bytes(u, args)
    stages = {}
    for k, nbytes in b.items():
        t = kern.get(k)
        if not t or t <= 0:
            continue
        gbs = nbytes / (t * 1e-3) / 1e9
        stages[k] = {"bound": "hbm", "algorithmic_bytes": int(nbytes), "ms": t, "achieved": gbs, "unit": "GB/s",
                     "frac": gbs / hbm_peak}
    # the floor for a whole iteration: each array of the step touched once
    P = 4 * (3 + 3 + 4 + 1 + 3 * u["sh_coeffs"])
    B = (3 * u["touched"] * P + 260 * u["visible"] + 52 * u["instances"] + 88 * u["pix"] + 20 * u["lidar"]
         + 8 * u["touched"])
    step = {"bound": "hbm", "algorithmic_bytes": int(B), "ms": step_ms, "achieved": B / (step_ms * 1e-3) / 1e9,
            "peak": hbm_peak, "unit": "GB/s", "frac": B / (step_ms * 1e-3) / 1e9 / hbm_peak,
            "stage_bytes_sum": int(sum(b.values())),
            "formula": "3 N_touched P + 260 N_vis + 52 N_inst + 88 N_pix + 20 N_L + 8 N_touched"}
    fp32 = max(alu["fp32_fma"], alu["fp32x2_fma"])
    var = args.depth_loss == "kl-var"
    walked, blends = u["pixel_entries"], u["pixel_blends"]
    fl_bwd = walked * EVAL_FLOPS + blends * (BWD_BLEND_FLOPS + (VAR_BLEND_FLOPS if var else 0))
    fl_fwd = walked * EVAL_FLOPS + blends * FWD_BLEND_FLOPS
    for k, fl in (("raster_bwd", fl_bwd), ("raster_fwd", fl_fwd)):
        if k in stages:
            a = fl / (stages[k]["ms"] * 1e-3) / 1e12
            stages[k]["alu"] = {"bound": "alu", "flops": int(fl), "achieved": a, "peak": fp32, "unit": "TFLOP/s",
                                "frac": a / fp32}
    t = kern["raster_bwd"]
    a = fl_bwd / (t * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_raster_bwd", "achieved": a, "peak": fp32, "unit": "TFLOP/s",
                "frac": a / fp32, "ms": t, "flops": int(fl_bwd),
                "work": f"{walked} (pixel, entry) pairs walked x {EVAL_FLOPS} + {blends} blended x "
                        f"{BWD_BLEND_FLOPS + (VAR_BLEND_FLOPS if var else 0)} FP32 operations",
                "peak_source": "measured FP32 FMA rate (gs_alu_probe, the larger of scalar and packed f32x2)"}
    hb = b["raster_bwd"] / (t * 1e-3) / 1e9
    roofline_hbm = {"bound": "hbm", "kernel": "k_raster_bwd", "achieved": hb, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hb / hbm_peak, "algorithmic_bytes": int(b["raster_bwd"]), "ms": t,
                    "peak_source": hbm_src}
    for v in stages.values():
        v["peak"] = hbm_peak
    return {"roofline": roofline, "roofline_hbm": roofline_hbm, "step": step, "stages": stages, "bytes": b}


def lifecycle_timing(torch, G, step, sc, dev, reps=5):
    """One lifecycle pass (prune, opacity reset, split / clone) over the
    workload's Gaussians with the densification statistic of the last step;
    gamma_g is set to the 90th percentile of the mean image-space gradient so
    that about a tenth of the visible splats densify.  CUDA events, mean of
    `reps` passes after one warm-up."""
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    params = dict(zip(keys, step.P))
    acc, cnt = step.grads["densify_acc"], step.grads["densify_cnt"]
    g = acc[cnt > 0] / cnt[cnt > 0].float()
    gamma = float(torch.quantile(g[:1 << 20].float(), 0.9)) if g.numel() else 1.0
    ls_max = step.P[1].max(1).values
    kappa = float(torch.quantile(ls_max[:1 << 20], 0.5).exp())
    lp = G.lifecycle_params(G.GS_LC_PRUNE | G.GS_LC_DENSIFY | G.GS_LC_RESET, densify_grad=gamma,
                            split_scale=kappa, clone_scale=kappa)
    normals = torch.randn(sc.n, 2, 3, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    lc = G.Lifecycle(sc.n, len(sc.submap_offsets) - 1)
    cap = 2 * sc.n
    out = {k: torch.empty((cap,) + tuple(v.shape[1:]), device=dev) for k, v in params.items()}
    offs = torch.as_tensor(sc.submap_offsets, dtype=torch.int64, device=dev)
    offs_out = torch.empty_like(offs)
    s = G._stream()

    def run():
        G.gs_lifecycle_run(lc.lc, lp, sc.sh_degree, sc.n, offs.numel() - 1, G._ptr(offs), G.param_arrays(params),
                           None, None, G._ptr(acc), G._ptr(cnt), G._ptr(normals), G.param_arrays(out), None, None,
                           cap, G._ptr(offs_out), None, s)
    run()
    st, n_out = G.gs_lifecycle_status(lc.lc, s)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        run()
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    lc.close()
    nsh = 3 * (sc.sh_degree + 1) ** 2
    bytes_moved = sc.n * (4 * 11 + 8) + n_out * 4 * (11 + nsh)
    return {"ms": ms, "n_in": sc.n, "n_out": n_out, "status": int(st), "gamma_g": gamma, "kappa": kappa,
            "algorithmic_bytes": int(bytes_moved + sc.n * 4 * nsh),
            "gbs": (bytes_moved + sc.n * 4 * nsh) / (ms * 1e-3) / 1e9}


def active_set_timing(torch, G, step, sc, dev, reps=5):
    """Voxel-hash insertion (Eq. 5) of a keyframe's fused points into the
    workload's map, LRU selection over its splats and the offload of the
    selected ones to pinned host memory, each timed with CUDA events (mean of
    `reps` after one warm-up).  Points: 300k, a fifth on existing splats
    (jittered by 1 mm), the rest uniform in the map's bounding box, with
    colours; host store: 100k keys of random voxels; v = 0.05 m; last_used
    frames uniform in [0, 30); tau = 80 % of the splats."""
    gen = torch.Generator(device=dev).manual_seed(0)
    means = step.P[0]
    n = means.shape[0]
    lo, hi = means.min(0).values, means.max(0).values
    n_pts = 300_000
    on = means[torch.randint(0, n, (n_pts // 5,), device=dev, generator=gen)]
    on = on + 1e-3 * torch.rand(on.shape, device=dev, generator=gen)
    off = lo + (hi - lo) * torch.rand(n_pts - on.shape[0], 3, device=dev, generator=gen)
    pts = torch.cat([torch.cat([on, off]), torch.rand(n_pts, 3, device=dev, generator=gen)], 1).contiguous()
    vm = G.VoxelMap(n_pts, n)
    v = 0.05
    keys = vm.keys(means, v)
    host_keys = torch.randint(0, 2 ** 62, (100_000,), device=dev, generator=gen)
    lu = torch.randint(0, 30, (n,), dtype=torch.int32, device=dev, generator=gen)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    K = (sc.sh_degree + 1) ** 2
    new = dict(means=torch.empty(n_pts, 3, device=dev), log_scales=torch.empty(n_pts, 3, device=dev),
               quats=torch.empty(n_pts, 4, device=dev), opacity_logits=torch.empty(n_pts, device=dev),
               sh=torch.empty(n_pts, K, 3, device=dev))
    new_keys = torch.empty(n_pts, dtype=torch.int64, device=dev)
    reload = torch.empty(host_keys.shape[0], dtype=torch.int32, device=dev)
    ip = G.GsInsertParams(v, 0.02, 0.1, 31)
    s = G._stream()

    def insert():
        G.lib().gs_voxel_insert(vm.vx, ctypes.byref(ip), G._ptr(pts), n_pts, G._ptr(keys), G._ptr(lu), n,
                                G._ptr(host_keys), G._ptr(reload), host_keys.shape[0], sc.sh_degree,
                                ctypes.byref(G.param_arrays(new)), G._ptr(new_keys), n_pts, None, s)
    t_insert = timed(insert)
    n_new = ctypes.c_int64(0)
    G.lib().gs_voxel_status(vm.vx, s, ctypes.byref(n_new))
    tau = int(0.8 * n)
    flags = torch.empty(n, dtype=torch.int32, device=dev)
    t_select = timed(lambda: G.lib().gs_active_select(vm.vx, G._ptr(lu), n, tau, G._ptr(flags), s))
    params = dict(zip(("means", "log_scales", "quats", "opacity_logits", "sh"), step.P))
    kept = {k: torch.empty_like(t) for k, t in params.items()}
    moved = {k: torch.empty(t.shape, dtype=t.dtype).pin_memory() for k, t in params.items()}
    pk, pm = G.param_arrays(kept), G.param_arrays(moved)
    pin = G.param_arrays(params)
    t_part = timed(lambda: G.lib().gs_partition(vm.vx, G._ptr(flags), n, sc.sh_degree, ctypes.byref(pin), None, None,
                                                ctypes.byref(pk), None, None, ctypes.byref(pm), None, None, None, s))
    vm.close()
    row = 4 * (3 + 3 + 4 + 1 + 3 * K)
    moved_bytes = (n - tau) * row
    return {"points": n_pts, "splats": n, "host_keys": int(host_keys.shape[0]), "voxel": v,
            "new_splats": int(n_new.value), "insert_ms": t_insert, "select_ms": t_select, "tau": tau,
            "partition_ms": t_part, "offloaded": n - tau, "offload_gbs_to_host": moved_bytes / (t_part * 1e-3) / 1e9}


def job_throughput(pix_per_rank: int, ms: float, world: int) -> float:
    """Whole-job Mpix/s: every rank renders its own replica in `ms`."""
    return pix_per_rank * world / (ms * 1e-3) / 1e6


# ---------------------------------------------------------------------------
# the step
# ---------------------------------------------------------------------------

class Step:
    """All device buffers of one mapping step plus the calls that make it."""

    def __init__(self, G, torch, sc, cfg, dev, inst_capacity=None, var=False, ssim_lambda=0.0, adam=False):
        self.G, self.torch, self.sc, self.dev = G, torch, sc, dev
        self.var = var
        self.ssim_lambda = ssim_lambda
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        self.P = [t(sc.means), t(sc.log_scales), t(sc.quats), t(sc.opacity_logits), t(sc.sh)]
        self.target = t(sc.target)
        # the same targets as 8-bit camera values (t = round(255 x)), for the
        # end-to-end leg that uploads keyframes as cameras deliver them
        self.target_u8 = t(np.clip(np.rint(np.asarray(sc.target, np.float64) * 255.0), 0, 255).astype(np.uint8))
        self.u8 = False
        self.lidar = t(sc.lidar)
        self.r = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree, config=cfg,
                            inst_capacity=inst_capacity or max(1 << 22, 8 * sc.n))
        npx = self.r.n_pix
        self.rgb = torch.empty(3 * npx, device=dev)
        self.depth = torch.empty(npx, device=dev)
        self.alpha = torch.empty(npx, device=dev)
        self.g_rgb = torch.zeros(3 * npx, device=dev)
        self.g_depth = torch.zeros(npx, device=dev)
        self.grads = dict(means=torch.zeros_like(self.P[0]), log_scales=torch.zeros_like(self.P[1]),
                          quats=torch.zeros_like(self.P[2]), opacity_logits=torch.zeros_like(self.P[3]),
                          sh=torch.zeros_like(self.P[4]), pose=torch.zeros(len(sc.cameras), 6, device=dev),
                          densify_acc=torch.zeros(sc.n, device=dev),
                          densify_cnt=torch.zeros(sc.n, dtype=torch.int32, device=dev))
        self.loss_rgb = torch.zeros(3, device=dev)
        self.loss_depth = torch.zeros(1, device=dev)
        # depth mean and variance and their adjoints (variance KL only)
        self.dist = [torch.empty(npx, device=dev) for _ in range(2)] if var else []
        self.g_var = [torch.zeros(npx, device=dev) for _ in range(2)] if var else []
        # Adam moments (the bias-correction step is a constant of the captured graph)
        self.adam = adam
        if adam:
            self.adam_m = [torch.zeros_like(p) for p in self.P]
            self.adam_v = [torch.zeros_like(p) for p in self.P]

    def zero(self):
        # one library launch for the image-space gradient buffers the losses
        # accumulate into; the backward writes the parameter gradients
        # (gs_grads.overwrite), so those need no clearing
        self.G.gs_zero_buffers([self.g_rgb, self.g_depth, *self.g_var])

    # stage-by-stage so that the breakdown can put events between them
    def stages(self):
        G, r = self.G, self.r
        torch = self.torch

        def project():
            s = G._stream()
            G.gs_project(r.ws, r.gaussians(*self.P), G._ptr(r.cams_dev), s)

        def binsort():
            G.gs_bin_sort(r.ws, G._stream())

        def fwd():
            if self.var:
                G.gs_render_fwd_var(r.ws, G._ptr(self.rgb), G._ptr(self.depth), G._ptr(self.alpha),
                                    G._ptr(self.dist[0]), G._ptr(self.dist[1]), G._stream())
            else:
                G.gs_render_fwd(r.ws, G._ptr(self.rgb), G._ptr(self.depth), G._ptr(self.alpha), G._stream())

        def losses():
            s = G._stream()
            if self.ssim_lambda > 0:
                G.gs_image_loss(r.ws, G._ptr(self.rgb), G._ptr(self.target), self.ssim_lambda, G._ptr(self.loss_rgb),
                                G._ptr(self.g_rgb), s)
            else:
                (G.gs_image_l1_u8 if self.u8 else G.gs_image_l1)(r.ws, G._ptr(self.rgb),
                                                                  G._ptr(self.target_u8 if self.u8 else self.target),
                                                                  G._ptr(self.loss_rgb), G._ptr(self.g_rgb), s)
            if self.var:
                G.gs_depth_loss_var(r.ws, G._ptr(self.alpha), G._ptr(self.dist[0]), G._ptr(self.dist[1]),
                                    G._ptr(self.lidar), self.lidar.shape[0], G._ptr(self.loss_depth),
                                    *(G._ptr(x) for x in self.g_var), s)
            else:
                G.gs_depth_loss(r.ws, G._ptr(self.depth), G._ptr(self.alpha), G._ptr(self.lidar),
                                self.lidar.shape[0], G._ptr(self.loss_depth), G._ptr(self.g_depth), s)

        def bwd():
            gg = self.grads
            grads = G.GsGrads(*(gg[k].data_ptr() for k in ("means", "log_scales", "quats", "opacity_logits", "sh",
                                                            "pose", "densify_acc", "densify_cnt")), 1, 0)
            if self.var:
                G.gs_render_bwd_var(r.ws, r.gaussians(*self.P), G._ptr(r.cams_dev), G._ptr(self.g_rgb),
                                    None, None, *(G._ptr(x) for x in self.g_var), grads, G._stream())
            else:
                G.gs_render_bwd(r.ws, r.gaussians(*self.P), G._ptr(r.cams_dev), G._ptr(self.g_rgb),
                                G._ptr(self.g_depth), None, grads, G._stream())
        def adam():
            keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
            pa = lambda ts: G.GsParamArrays(*(t.data_ptr() for t in ts))
            ap = G.GsAdamParams((ctypes.c_float * 5)(*ADAM_LR), 0.9, 0.999, 1e-15, 10)
            G.gs_adam_step(pa(self.P), pa([self.grads[k] for k in keys]), pa(self.adam_m), pa(self.adam_v),
                           self.P[0].shape[0], self.sc.sh_degree, ap, G._stream())
        st = [("zero", self.zero), ("project", project), ("bin_sort", binsort), ("raster_fwd", fwd),
              ("losses", losses), ("backward", bwd)]
        return st + ([("adam", adam)] if self.adam else [])

    def run(self):
        for _, f in self.stages():
            f()


def make_graph(torch, step):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            step.run()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step.run()
    return g


def time_steps(torch, fn, steps, warmup, flush):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        times.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


def stage_breakdown(torch, step, steps, flush):
    names = [n for n, _ in step.stages()]
    acc = {n: [] for n in names}
    for _ in range(steps):
        flush.zero_()
        evs = []
        for n, f in step.stages():
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            evs.append((n, e0, e1))
        torch.cuda.synchronize()
        for n, a, b in evs:
            acc[n].append(a.elapsed_time(b))
    return {n: float(np.mean(v)) for n, v in acc.items()}


def kernel_breakdown(torch, G, step, steps, flush):
    """Mean CUDA-event duration of every library stage (events recorded by the
    library itself around each kernel group, on the launching stream)."""
    G.gs_workspace_set_profiling(step.r.ws, True)
    acc = {}
    for _ in range(steps):
        flush.zero_()
        step.run()
        for k, v in G.gs_workspace_stage_ms(step.r.ws).items():
            acc.setdefault(k, []).append(v)
    G.gs_workspace_set_profiling(step.r.ws, False)
    return {k: float(np.mean(v)) for k, v in acc.items()}


# ---------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------

# The oracle's sample of each workload: full frames of every view for the
# small box scene and the 500k orchard; one full view of the larger ones (the
# FP64 step over all six 1920x1200 views of the 4M map takes minutes).
ORACLE_VIEWS = {"box10k": 0, "orchard500k": 0, "orchard1m_pose": 1, "submaps8": 1, "orchard4m": 1}


def oracle_sample(sc, crop_w=0, n_views=0):
    """The cameras the oracle renders: the first ``n_views`` views (0: all),
    each cropped to a centred window ``crop_w`` wide of the same aspect ratio
    (0: the full frame).  Same scene, same Gaussians, fewer pixels.  Returns
    (cameras, their view indices in the workload)."""
    idx = list(range(len(sc.cameras) if n_views <= 0 else min(n_views, len(sc.cameras))))
    cams = []
    for v in idx:
        c = sc.cameras[v]
        w = c.width if crop_w <= 0 else min(crop_w, c.width)
        h = c.height if crop_w <= 0 else max(1, int(round(w * c.height / c.width)))
        cams.append(c.crop(int(c.cx) - w // 2, int(c.cy) - h // 2, w, h) if (w, h) != (c.width, c.height) else c)
    return cams, idx


def run_oracle_step(O, P, cams, cfg, lidar_full, sc, depth_loss="l1", ssim_lambda=0.0, adam=False):
    """project -> bin -> forward -> image + depth losses -> backward (-> Adam), in FP64."""
    rec = O.project(P, cams, cfg)
    keys, vals, ranges = O.bin(P, cams, cfg, rec)
    out = O.render_fwd(P, cams, cfg, rec, vals, ranges)
    npx = sum(c.width * c.height for c in cams)
    target = np.zeros(3 * npx)
    if ssim_lambda > 0:
        _, gC = O.image_loss(cams, out["rgb"], target, ssim_lambda)
    else:
        _, gC = O.image_l1(out["rgb"], target)
    if depth_loss == "kl-var":
        mean, var = O.render_depth_dist(P, cams, cfg, rec, vals, ranges)
        _, gm, gv, _ = O.depth_loss_var(P, cams, cfg, out["alpha"], mean, var, lidar_full)
        g = O.render_bwd(P, cams, cfg, rec, vals, ranges, gC, np.zeros(npx), None, gm, gv)
    else:
        _, gD, _ = O.depth_loss(P, cams, cfg, out["depth"], out["alpha"], lidar_full,
                                mode=1 if depth_loss == "kl" else 0)
        g = O.render_bwd(P, cams, cfg, rec, vals, ranges, gC, gD)
    if adam:
        from oracle import lifecycle as OL
        for i, k in enumerate(OL.FIELDS):
            a = getattr(P, k)
            OL.adam(a, g[k], np.zeros_like(a), np.zeros_like(a), 10, ADAM_LR[i])
    return npx


def oracle_threads() -> int:
    """Every host core of the machine (the oracle's loops over pairs and
    pixels run on OpenMP threads)."""
    return os.cpu_count() or 1


def cpu_baseline(sc, args, reps=1, state=None):
    """The FP64 oracle's full step on the sample of ``oracle_sample``, on all
    host cores.  ``state`` (a dict) keeps the widened parameters between calls."""
    import oracle as O
    O.build()
    cores = oracle_threads()
    O.set_threads(cores)
    n_views = args.cpu_views if args.cpu_views >= 0 else ORACLE_VIEWS.get(sc.name, 1)
    sel, idx = oracle_sample(sc, args.cpu_sample, n_views)
    cams = O.as_float32_cameras(sel)
    if state is not None and "P" in state:
        P = state["P"]
    else:
        P = O.Params.from_scene(sc)
        if state is not None:
            state["P"] = P
    # the sample's LiDAR returns, re-expressed in its (cropped) views
    lid_all = sc.lidar.astype(np.float64)
    parts = []
    for j, (v, cc) in enumerate(zip(idx, cams)):
        c = sc.cameras[v]
        m = lid_all[lid_all[:, 3] == v].copy()
        m[:, 0] -= (c.cx - cc.cx)
        m[:, 1] -= (c.cy - cc.cy)
        m[:, 3] = j
        parts.append(m)
    lid = np.concatenate(parts) if parts else np.zeros((0, 4))
    cfg = O.Config()
    t0 = time.perf_counter()
    npx = 0
    for _ in range(reps):
        npx += run_oracle_step(O, P, cams, cfg, lid, sc, args.depth_loss, args.ssim_lambda, args.adam)
    dt = time.perf_counter() - t0
    full = all((c.width, c.height) == (sc.cameras[v].width, sc.cameras[v].height) for v, c in zip(idx, cams))
    frames = "full frames" if full else f"centred {cams[0].width}x{cams[0].height} crops"
    views = "every view" if len(idx) == len(sc.cameras) else f"{len(idx)} of the {len(sc.cameras)} views"
    sample = (f"FP64 oracle on {cores} host threads, full step (project all {sc.n} Gaussians x {len(cams)} "
              f"view(s), bin, forward, {loss_label(args)}, backward) on {frames} of {views}, "
              f"{npx} pixels, {reps} step(s), {dt:.1f} s")
    return {"value": npx / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": dt, "pixels": npx}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2510_26358_gb300 import scenes
    sc = scenes.workload(args.workload)
    # warm-up and timed steps, each a bounded sample of the workload
    cb = None
    state = {}
    for _ in range(args.warmup):
        cpu_baseline(sc, args, state=state)
    vals, secs, pix = [], 0.0, 0
    for _ in range(args.steps):
        cb = cpu_baseline(sc, args, state=state)
        secs += cb["seconds"]
        pix += cb["pixels"]
    value = pix / secs / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(sc, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_26358_gb300 import gsraster as G
    from paper_2510_26358_gb300 import scenes

    sc = scenes.workload(args.workload, seed=rank)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    step_runs = [0]  # steps run while sizing (each launches every kernel of a step once)

    def build_step(tw, th, depth):
        """A Step whose instance capacity fits the scene (sized from a first run)."""
        cfg = G.gs_config_default(tile_w=tw, tile_h=th, batch_depth=depth,
                                  depth_mode=1 if args.depth_loss == "kl" else 0)
        mom = args.depth_loss == "kl-var"
        st_ = Step(G, torch, sc, cfg, dev, var=mom, ssim_lambda=args.ssim_lambda, adam=args.adam)
        st_.run()
        step_runs[0] += 1
        code, need_, _ = st_.r.status()
        if code == G.GS_ERR_CAPACITY or need_ > st_.r.info["inst_capacity"]:
            st_.r.close()
            st_ = Step(G, torch, sc, cfg, dev, inst_capacity=int(need_ * 1.25) + 1024, var=mom,
                       ssim_lambda=args.ssim_lambda, adam=args.adam)
            st_.run()
            step_runs[0] += 1
        return st_

    tuned = None
    if args.tile == "auto":
        from paper_2510_26358_gb300 import autotune

        def measure(tw, th, depth):
            st_ = build_step(tw, th, depth)
            g_ = make_graph(torch, st_)
            t_ = time_steps(torch, g_.replay, 5, 2, flush)
            st_.r.close()
            del g_
            return float(np.mean(t_))
        key = autotune.signature(sc.cameras, sc.n, sc.sh_degree, sc.submap_offsets,
                                 extra="bench-step" + ("" if args.depth_loss == "l1" else "-" + args.depth_loss)
                                 + ("" if args.ssim_lambda == 0 else "-ssim") + ("-adam" if args.adam else ""))
        tuned = autotune.tune(measure, key=key)
        tw, th, args.depth = tuned["tile_w"], tuned["tile_h"], tuned["batch_depth"]
    else:
        tw, th = (int(x) for x in args.tile.split("x"))
    step = build_step(tw, th, args.depth)
    st, need, nvis = step.r.status()
    assert st == G.GS_OK, G.status_string(st)
    if args.once:
        step.run()
        torch.cuda.synchronize()
        assert step.r.status()[0] == G.GS_OK
        step.r.close()
        # a profiler skips this many launches of a kernel to reach the last step's
        print(json.dumps({"once": True, "steps_before_last": step_runs[0]}))
        return 0

    # launches per step, from the library's own counter
    k0 = G.gs_workspace_info(step.r.ws)["kernel_launches"]
    step.run()
    launches_per_step = G.gs_workspace_info(step.r.ws)["kernel_launches"] - k0
    # the gradient zeroing and the Adam step are library kernels outside the workspace
    launches_per_step += 1 + (1 if args.adam else 0)

    graph = make_graph(torch, step)
    # timed region: graph replays, clocks sampled meanwhile
    sampler = ClockSampler(gpu_uuid(torch))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    times = time_steps(torch, graph.replay, args.steps, args.warmup, flush)
    clocks = sampler.stop()
    ms = max_over_ranks(float(np.mean(times)), dev)
    value = job_throughput(sc.n_pix, ms, world)

    # correctness of the timed state (status after the replays)
    st, need2, _ = step.r.status()
    assert st == G.GS_OK

    breakdown = stage_breakdown(torch, step, max(3, args.steps // 2), flush)
    kern = kernel_breakdown(torch, G, step, max(3, args.steps // 2), flush)
    lifecycle = lifecycle_timing(torch, G, step, sc, dev) if args.lifecycle else None
    active_set = active_set_timing(torch, G, step, sc, dev) if args.active_set else None

    # per-view plain version: one workspace per camera, no graph
    per_view = None
    if not args.no_per_view:
        from copy import copy
        pv_steps = []
        for v, c in enumerate(sc.cameras):
            sub = copy(sc)
            c1 = copy(c)
            c1.submap = 0
            s0, s1 = int(sc.submap_offsets[c.submap]), int(sc.submap_offsets[c.submap + 1])
            sub.means, sub.log_scales, sub.quats = sc.means[s0:s1], sc.log_scales[s0:s1], sc.quats[s0:s1]
            sub.opacity_logits, sub.sh = sc.opacity_logits[s0:s1], sc.sh[s0:s1]
            sub.submap_offsets = np.array([0, s1 - s0], np.int64)
            sub.cameras = [c1]
            off = sum(cc.width * cc.height for cc in sc.cameras[:v])
            hw = c.width * c.height
            sub.target = sc.target[3 * off:3 * (off + hw)]
            m = sc.lidar[:, 3] == v
            lid = sc.lidar[m].copy()
            lid[:, 3] = 0
            sub.lidar = lid
            pv_steps.append(Step(G, torch, sub, G.gs_config_default(depth_mode=1 if args.depth_loss == "kl" else 0),
                                 dev, inst_capacity=need + 1024, var=args.depth_loss == "kl-var",
                                 ssim_lambda=args.ssim_lambda, adam=args.adam))
        run_all = lambda: [s.run() for s in pv_steps]
        pv_times = time_steps(torch, run_all, max(3, args.steps // 2), 3, flush)
        pv_ms = float(np.mean(pv_times))
        per_view = {"value": sc.n_pix / (pv_ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": pv_ms,
                    "how": "one workspace and launch sequence per camera, 16x16 tiles, no CUDA graph",
                    "batched_over_per_view": (sc.n_pix / (ms * 1e-3) / 1e6) / (sc.n_pix / (pv_ms * 1e-3) / 1e6)}
        for s in pv_steps:
            s.r.close()

    # end to end through the C ABI with host buffers.  Every step copies its
    # inputs from pinned host memory -- the keyframe batch: target images,
    # LiDAR returns and camera poses -- and reads both losses back.  The map
    # (the Gaussians) is the optimised state, resident on the device across
    # steps as a network's weights are; a second figure also re-uploads it
    # every step.
    e2e = None
    if not args.no_e2e:
        def e2e_run(tensors, g):
            host = [t.cpu().pin_memory() for t in tensors]
            loss_h = torch.empty(2, pin_memory=True)
            h2d = sum(h.numel() * h.element_size() for h in host)

            def e2e_step():
                for h, d in zip(host, tensors):
                    d.copy_(h, non_blocking=True)
                g.replay()
                loss_h[0:1].copy_(step.loss_rgb[0:1], non_blocking=True)
                loss_h[1:2].copy_(step.loss_depth, non_blocking=True)
            e_times = time_steps(torch, e2e_step, max(3, args.steps // 2), 3, flush)
            e_ms = float(np.mean(e_times))
            return {"value": sc.n_pix * world / (e_ms * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": 8, "ms_per_step": e_ms}
        batch = [step.target, step.lidar, step.r.cams_dev]
        if args.ssim_lambda == 0:
            # keyframes as cameras deliver them: 8-bit target images (the step's
            # L1 reads them directly); the float-target figure is kept beside it
            step.u8 = True
            graph_u8 = make_graph(torch, step)
            step.u8 = False
            batch_u8 = [step.target_u8, step.lidar, step.r.cams_dev]
            e2e = e2e_run(batch_u8, graph_u8)
            e2e["inputs"] = ("keyframe batch: 8-bit target images, LiDAR returns, cameras (map resident); "
                             "gs_image_l1_u8")
            e2e["with_map_upload"] = e2e_run(list(step.P) + batch_u8, graph_u8)
            e2e["float_targets"] = e2e_run(batch, graph)
        else:
            e2e = e2e_run(batch, graph)
            e2e["inputs"] = "keyframe batch: target images, LiDAR returns, cameras (map resident)"
            e2e["with_map_upload"] = e2e_run(list(step.P) + batch, graph)

    # rooflines: every library stage against its bound, the dominant kernel
    # (the raster backward) against the measured FP32 rate
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s"
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu = measure_alu_peaks(torch, G, dev, n_sm)
    frag = G.gs_workspace_fragment_counts(step.r.ws)
    rng = step.r.buffer(G.BUF_RANGES, torch.int32).view(-1, 2).to(torch.int64)
    units = dict(N=sc.n, views=len(sc.cameras), pairs=step.r.info["n_pairs"], visible=nvis, instances=need,
                 listed=int((rng[:, 1] - rng[:, 0]).sum().item()), tiles=step.r.info["n_tiles"], pix=sc.n_pix,
                 lidar=int(sc.lidar.shape[0]), touched=int((step.grads["densify_cnt"] > 0).sum().item()),
                 sh_coeffs=(sc.sh_degree + 1) ** 2, **frag)
    rep = roofline_report(units, kern, ms, hbm_peak, hbm_src, alu, args, tw, th)
    roofline, roofline_hbm = rep["roofline"], rep["roofline_hbm"]
    if args.depth_loss == "kl-var":
        traffic, traffic_note = None, "the ncu capture covers the kernel without the depth variance"
    else:
        traffic, traffic_note = measured_traffic("k_raster_bwd", sc.name, f"{tw}x{th}/{args.depth}",
                                                 rep["bytes"]["raster_bwd"])
    for r_ in (roofline, roofline_hbm):
        r_["traffic"], r_["traffic_source"] = traffic, traffic_note

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            # (value is from the mean step time; the median, for a median-based reading)
            "ms_per_step_median": float(np.median(times)),
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(sc, args, f"{tw}x{th}", args.depth),
                           autotune=None if tuned is None else {"chosen": f"{tw}x{th}/{args.depth}",
                                                                "cached": tuned.get("cached"),
                                                                "ms": tuned["timings"]}),
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches_per_step * args.steps),
            "launches_per_step": int(launches_per_step), "roofline": roofline, "roofline_hbm": roofline_hbm,
            "step_roofline": rep["step"], "kernel_rooflines": rep["stages"], "alu_peaks": alu,
            "per_view": per_view, "breakdown_ms": breakdown, "kernel_ms": kern, "lifecycle": lifecycle,
            "active_set": active_set, "counts": units}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(sc, args, reps=2).items()
                                if k not in ("seconds", "pixels")}
    elif rank == 0:
        line["cpu_baseline"] = None
    step.r.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
