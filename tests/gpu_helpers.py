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


# A float32 evaluation of the tile test (tile_reached in the binning kernel)
# rounds its box edges, products and threshold: its value of (threshold -
# minimum) is off from the exact one on the same float inputs by at most
# about 16 float ulps of the scale oracle.tile_decisions32 divides by.  Four
# times that is the band inside which either decision is correct.
TILE_BAND = 64 * 2.0 ** -24


def rect_tile_codes(sc, ocfg: O.Config, rect, pkey):
    """(pair, global tile) of every rectangle tile of every visible pair, in
    the emission order of oracle.tile_decisions32, as pair * n_tiles + tile."""
    rect = np.asarray(rect, np.int64).reshape(-1, 4)
    ng = [int(sc.submap_offsets[c.submap + 1] - sc.submap_offsets[c.submap]) for c in sc.cameras]
    pair_view = np.repeat(np.arange(len(sc.cameras)), ng)
    ntx = np.array([-(-c.width // ocfg.tile_w) for c in sc.cameras], np.int64)
    nty = np.array([-(-c.height // ocfg.tile_h) for c in sc.cameras], np.int64)
    toff = np.concatenate([[0], np.cumsum(ntx * nty)])
    T = int(toff[-1])
    vis = (np.asarray(pkey) != 0xFFFFFFFF) & (rect[:, 2] >= rect[:, 0]) & (rect[:, 3] >= rect[:, 1])
    p = np.nonzero(vis)[0]
    w = rect[p, 2] - rect[p, 0] + 1
    area = w * (rect[p, 3] - rect[p, 1] + 1)
    rp = np.repeat(p, area)
    j = np.arange(int(area.sum())) - np.repeat(np.cumsum(area) - area, area)
    ww = np.repeat(w, area)
    ty = np.repeat(rect[p, 1], area) + j // ww
    tx = np.repeat(rect[p, 0], area) + j % ww
    v = pair_view[rp]
    return rp * T + toff[v] + ty * ntx[v] + tx, T


def check_binning_stage(sc, ocfg: O.Config, g, P=None, cams=None):
    """The binning stage against the oracle, bit for bit: the oracle takes
    the CUDA path's own float32 projection outputs (records, rectangles,
    depth keys), decides every rectangle tile exactly (R6b) and sorts.  Tile
    decisions must agree except inside TILE_BAND, where the CUDA path's
    decision is taken; then the sorted keys, instance order and per-tile
    ranges must be identical.  Returns (decisions, decisions in the band)."""
    P = P if P is not None else O.Params.from_scene(sc)
    cams = cams if cams is not None else O.as_float32_cameras(sc.cameras)
    dec, margin = O.tile_decisions32(P, cams, ocfg, g["rec"], g["rect"], g["pkey"])
    codes, T = rect_tile_codes(sc, ocfg, g["rect"], g["pkey"])
    assert codes.shape == dec.shape
    gp = g["inst_pair"].astype(np.int64)
    gdec = np.isin(codes, gp * T + g["inst_tile"].astype(np.int64))
    band = np.abs(margin) < TILE_BAND
    bad = (gdec != dec.astype(bool)) & ~band
    assert not bad.any(), f"{int(bad.sum())} tile decisions differ outside the band"
    resolved = np.where(band, gdec, dec.astype(bool)).astype(np.int8)
    keys, vals, ranges = O.bin_decided(P, cams, ocfg, g["rect"], g["pkey"], resolved)
    gkeys = (g["inst_tile"].astype(np.uint64) << np.uint64(32)) | g["pkey"][gp].astype(np.uint64)
    assert np.array_equal(gkeys, keys), "sorted keys differ"
    assert np.array_equal(gp, vals), "instance order differs"
    assert np.array_equal(g["ranges"].astype(np.int64), ranges), "tile ranges differ"
    # every rectangle tile is emitted once, listed or dropped
    drop = np.bincount(g["dropped_pair"].astype(np.int64), minlength=len(g["pkey"]))
    assert drop.sum() + len(gp) == len(dec)
    return int(len(dec)), int(band.sum())


def end_to_end_key_mismatch(g, keys, vals, T):
    """Instances on one side only, against the FP64 oracle's own projection
    and binning: (pair, tile) pairs in the symmetric difference."""
    a = g["inst_pair"].astype(np.int64) * T + g["inst_tile"].astype(np.int64)
    b = vals.astype(np.int64) * T + (keys >> np.uint64(32)).astype(np.int64)
    return int(np.setxor1d(a, b).size)


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
