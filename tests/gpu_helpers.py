"""Shared helpers for the GPU parity tests: run a scene through the CUDA path
(via the C ABI) and through the FP64 oracle, and compare."""
from __future__ import annotations

import math

import numpy as np

import oracle as O

S2 = math.log2(math.e) / 2.0   # square of the Cholesky scale used by the records


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def params_to_dev(sc):
    torch, dev = torch_dev()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return [t(sc.means), t(sc.log_scales), t(sc.quats), t(sc.opacity_logits), t(sc.sh)]


def oracle_config(**kw) -> O.Config:
    return O.Config(**kw)


def gpu_config(G, ocfg: O.Config, **kw):
    return G.gs_config_default(tile_w=ocfg.tile_w, tile_h=ocfg.tile_h, near_z=ocfg.near_z,
                               dilation=ocfg.dilation, alpha_min=ocfg.alpha_min, alpha_max=ocfg.alpha_max,
                               t_min=ocfg.t_min, jac_clamp=ocfg.jac_clamp, ext_rel_pad=ocfg.ext_rel_pad,
                               ext_abs_pad=ocfg.ext_abs_pad, **kw)


def run_gpu(sc, ocfg: O.Config, gC=None, gD=None, gA=None, depth=256, inst_capacity=None, var=False,
            gmean=None, gvar=None, **kw):
    """Forward (and backward when upstream gradients are given) on cuda:0.
    With ``var`` the forward and backward with the depth mean and variance
    are used (upstream gmean, gvar for the latter).  Returns a dict of numpy
    arrays."""
    from paper_2510_26358_gb300 import gsraster as G
    torch, dev = torch_dev()
    cfg = gpu_config(G, ocfg, batch_depth=depth, **kw)
    r = G.Renderer(sc.cameras, sc.submap_offsets, sc.sh_degree, config=cfg,
                   inst_capacity=inst_capacity or (1 << 22))
    P = params_to_dev(sc)
    fw = r.forward(*P, var=var)
    rgb, dep, alp = fw[:3]
    st, n_inst, n_vis = r.status()
    out = dict(status=st, n_inst=n_inst, n_vis=n_vis, rgb=rgb.cpu().numpy(), depth=dep.cpu().numpy(),
               alpha=alp.cpu().numpy())
    if var:
        out["mean"], out["var"] = fw[3].cpu().numpy(), fw[4].cpu().numpy()
        out["vstat"] = r.buffer(G.BUF_VSTAT, torch.float32).cpu().numpy().reshape(-1, 4)
    out["rec"] = r.buffer(G.BUF_RECORDS, torch.float32).cpu().numpy().reshape(-1, 12)
    out["pkey"] = r.buffer(G.BUF_PAIR_KEYS, torch.int32).cpu().numpy().view(np.uint32)
    out["rect"] = r.buffer(G.BUF_RECTS, torch.int16).cpu().numpy().reshape(-1, 4)
    m = min(n_inst, r.info["inst_capacity"]) if st == G.GS_OK else 0
    tiles = r.buffer(G.BUF_INST_TILES, torch.int32).cpu().numpy().view(np.uint32)[:m]
    pairs = r.buffer(G.BUF_INST_PAIRS, torch.int32).cpu().numpy().view(np.uint32)[:m]
    # the rectangle tiles that the ellipse misses carry tile id 0xFFFFFFFF and
    # sort after every real tile: the lists proper are the prefix
    kept = int(np.count_nonzero(tiles != 0xFFFFFFFF))
    assert np.all(tiles[kept:] == 0xFFFFFFFF), "dropped instances not sorted last"
    out["inst_tile"], out["inst_pair"] = tiles[:kept], pairs[:kept]
    out["dropped_pair"] = pairs[kept:]
    out["ranges"] = r.buffer(G.BUF_RANGES, torch.int32).cpu().numpy().view(np.uint32).reshape(-1, 2)
    out["last"] = r.buffer(G.BUF_LAST, torch.int32).cpu().numpy().view(np.uint32)
    out["tfin"] = r.buffer(G.BUF_TFIN, torch.float32).cpu().numpy()
    if gC is not None:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        o = lambda a: t(a) if a is not None else None
        grads = r.backward(*P, t(gC), t(gD), o(gA), var=var, dL_dmean=o(gmean), dL_dvar=o(gvar))
        torch.cuda.synchronize()
        for k, v in grads.items():
            out["g_" + k] = v.cpu().numpy()
        out["g2d"] = r.buffer(G.BUF_G2D, torch.float32).cpu().numpy().reshape(-1, 10)
    out["renderer"] = r
    out["params"] = P
    return out


def run_oracle(sc, ocfg: O.Config):
    P = O.Params.from_scene(sc)
    cams = O.as_float32_cameras(sc.cameras)
    rec, keys, vals, ranges, out = O.forward(P, cams, ocfg)
    return P, cams, rec, keys, vals, ranges, out


def decode_records(rec_gpu: np.ndarray):
    """u, v, Q (qa, qb, qc), log2 o, rgb, z from the GPU records."""
    r = rec_gpu.astype(np.float64)
    u = r[:, 0] + 0.5 - r[:, 2]
    v = r[:, 1] + 0.5 - r[:, 3]
    l11, l12, l22 = r[:, 4], r[:, 5], r[:, 6]
    qa = l11 * l11 / S2
    qb = l11 * l12 / S2
    qc = (l12 * l12 + l22 * l22) / S2
    return dict(u=u, v=v, qa=qa, qb=qb, qc=qc, log2o=r[:, 7], rgb=r[:, 8:11], z=rec_gpu[:, 11])


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def pixel_weights(sc, keep: np.ndarray):
    """keep mask per pixel -> (mask for planar rgb, mask per pixel)."""
    npx = keep.size
    rgbmask = np.empty(3 * npx, bool)
    off = 0
    for c in sc.cameras:
        hw = c.width * c.height
        for ch in range(3):
            rgbmask[3 * off + ch * hw: 3 * off + (ch + 1) * hw] = keep[off:off + hw]
        off += hw
    return rgbmask, keep
