"""Map lifecycle and optimiser step of the Gaussian map, plain numpy (TEST
INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s CPU legs; the
product library never imports it).

Readings of the paper's lifecycle operations (Sec. III-B, "Gaussian Splats
Lifecycle Operations"; the paper gives tau_opa = 0.01 and the size bounds
0.3 and 5e-5, and leaves gamma_g, kappa, s_init, tau_reset, s_min, s_max and
the split rule open):

  R18  size s_j = the largest of the three axis scales exp(log_scale).
       Every decision is taken on the stored float32 values against float32
       thresholds moved to the logit / log domain on the host:
       o < tau  <=>  omega < logit(tau),   s > t  <=>  max log_scale > ln(t),
       so that both implementations decide bit for bit alike.
  R19  per splat, in order: prune (o < tau_opa, s > s_prune_max or
       s < s_prune_min) drops it; otherwise the opacity reset (tau_opa < o <
       tau_reset and s_min < s < s_max) sets o = tau_reset; then, with the
       mean image-space gradient g = acc / cnt (float32; 0 if cnt = 0) and
       g > gamma_g, a splat with s > kappa is split into two children, one
       with s <= clone_scale (= 2 s_init) is cloned, others are kept.
  R20  split child k of splat j: mean mu_j + R(q_j) diag(exp(log_scale_j)) z_jk
       (a sample of N(mu_j, Sigma_j); the standard-normal z_jk are inputs),
       log_scale_j - ln(split_shrink) on every axis, quaternion, opacity and
       SH copied.  A clone is an exact copy placed right after the original.
       Output order: the input order with children / copies in place of /
       after their splat, so every submap stays contiguous; the new submap
       offsets are the output positions of each submap's first splat.
  R21  optimiser state (Adam first and second moments): survivors keep
       theirs, clone copies and split children start at zero.
  R22  Adam (the paper names no optimiser): m = b1 m + (1 - b1) g,
       v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parity status: pinned (tests/test_oracle_pins.py): counts and order against
independent per-rule filters, Mahalanobis distance of split children equal
to |z|^2, scale ratio, reset value, moments; Adam against torch.optim.Adam.
"""
from __future__ import annotations

import math

import numpy as np

PRUNE, DENSIFY, RESET = 1, 2, 4
FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _f32(x) -> np.float32:
    return np.float32(x)


def thresholds(p: dict) -> dict:
    """The paper's thresholds moved to the logit / log domain, as float32 (R18).
    The parameters themselves are float32 values (as the C ABI holds them)."""
    p = {k: float(np.float32(v)) for k, v in p.items()}
    logit = lambda t: _f32(math.log(t / (1.0 - t)))
    return dict(opa=logit(p["prune_opacity"]), smax=_f32(math.log(p["prune_scale_max"])),
                smin=_f32(math.log(p["prune_scale_min"])), grad=_f32(p["densify_grad"]),
                split=_f32(math.log(p["split_scale"])), clone=_f32(math.log(p["clone_scale"])),
                reset=logit(p["reset_opacity"]), rmin=_f32(math.log(p["reset_scale_min"])),
                rmax=_f32(math.log(p["reset_scale_max"])), shrink=math.log(p["split_shrink"]))


def quat_to_rot(q) -> np.ndarray:
    """Rotation matrix of the normalised quaternion (w, x, y, z)."""
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(np.asarray(q, np.float64))
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def lifecycle(params: dict, moments: tuple | None, submap_offsets, densify_acc, densify_cnt, split_normals,
              p: dict, ops: int):
    """One pass of R18-R21 over every splat in order.

    params: dict of float32 arrays (FIELDS); moments: (m, v) dicts of the same
    shapes or None; densify_acc float32 [N], densify_cnt int32 [N];
    split_normals float32 [N][2][3].  Returns (params_out, moments_out,
    submap_offsets_out, actions) with float64 outputs and actions[j] in
    {"prune", "keep", "clone", "split"}."""
    t = thresholds(p)
    N = params["means"].shape[0]
    out = {k: [] for k in FIELDS}
    mom = None if moments is None else ({k: [] for k in FIELDS}, {k: [] for k in FIELDS})
    actions = []
    first_out = []  # output position of each splat's first output (or of the next)

    def emit(src_j, mean=None, log_scale=None, omega=None, zero_moments=False):
        for k in FIELDS:
            v = np.asarray(params[k][src_j], np.float64).copy()
            if k == "means" and mean is not None:
                v = mean
            if k == "log_scales" and log_scale is not None:
                v = log_scale
            if k == "opacity_logits" and omega is not None:
                v = np.float64(omega)
            out[k].append(v)
            if mom is not None:
                for a in range(2):
                    mom[a][k].append(np.zeros_like(v) if zero_moments
                                     else np.asarray(moments[a][k][src_j], np.float64).copy())

    for j in range(N):
        first_out.append(len(out["means"]))
        ls = params["log_scales"][j]
        smax = np.max(ls)  # float32 (R18)
        om = params["opacity_logits"][j]
        if (ops & PRUNE) and (om < t["opa"] or smax > t["smax"] or smax < t["smin"]):
            actions.append("prune")
            continue
        omega = None
        if (ops & RESET) and t["opa"] < om < t["reset"] and t["rmin"] < smax < t["rmax"]:
            omega = t["reset"]
        g = _f32(densify_acc[j]) / _f32(densify_cnt[j]) if densify_cnt[j] > 0 else _f32(0.0)
        if (ops & DENSIFY) and g > t["grad"] and smax > t["split"]:
            R = quat_to_rot(params["quats"][j])
            S = np.exp(np.asarray(ls, np.float64))
            mu = np.asarray(params["means"][j], np.float64)
            for k in range(2):
                z = np.asarray(split_normals[j][k], np.float64)
                emit(j, mean=mu + R @ (S * z), log_scale=np.asarray(ls, np.float64) - t["shrink"], omega=omega,
                     zero_moments=True)
            actions.append("split")
        elif (ops & DENSIFY) and g > t["grad"] and smax <= t["clone"]:
            emit(j, omega=omega)
            emit(j, omega=omega, zero_moments=True)
            actions.append("clone")
        else:
            emit(j, omega=omega)
            actions.append("keep")
    first_out.append(len(out["means"]))
    offs = np.array([first_out[o] for o in np.asarray(submap_offsets, np.int64)], np.int64)
    P = {k: (np.array(v, np.float64).reshape((-1,) + params[k].shape[1:]) if v else
             np.zeros((0,) + params[k].shape[1:])) for k, v in out.items()}
    M = None
    if mom is not None:
        M = tuple({k: (np.array(v, np.float64).reshape((-1,) + params[k].shape[1:]) if v else
                       np.zeros((0,) + params[k].shape[1:])) for k, v in mm.items()} for mm in mom)
    return P, M, offs, actions


def adam(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step (R22) in float64; returns (param, m, v)."""
    param, grad = np.asarray(param, np.float64), np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v
