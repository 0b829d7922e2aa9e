"""Voxel-hash insertion and the LRU active set of the incremental Gaussian
map, plain Python / numpy (TEST INFRASTRUCTURE ONLY: imported by ``tests/``;
the product library never imports it).

Readings of Sec. III-B ("Incremental Gaussian Mapping", "Memory Management";
Eq. 5 gives the key, the paper gives neither the primes nor v):

  R23  key k = floor(x/v) P1 + floor(y/v) P2 + floor(z/v) P3 in unsigned
       64-bit arithmetic (two's complement of negative cells, wrap-around),
       with Teschner et al.'s primes P1 = 73856093, P2 = 19349663,
       P3 = 83492791; x/v is divided in float32 (the stored precision) before
       the floor, on both implementations.  A splat's key is that of its mean.
       The all-ones key (which marks empty hash slots) is folded onto
       all-ones minus one.
  R24  inserting a batch of points (x, y, z, r, g, b) at frame f: every
       device splat whose key equals some point's key gets last_used = f;
       every host-resident splat whose key equals some point's key is flagged
       for reload; every key matched by neither creates one new splat, from
       the first point (in input order) with that key: mean = the point,
       isotropic log-scale ln(s_init), identity rotation, opacity o_init,
       SH DC = (rgb - 1/2) / Y00 (so that it renders the point's colour) and
       zero higher coefficients; new splats are ordered by that first point.
  R25  active set: with more than tau device splats, the (n - tau) least
       recently used ones, ordered by (last_used, index), are offloaded;
       partitions (offload, reload) keep the input order on both sides.

Parity status: pinned (tests/test_voxel_oracle.py): keys against an
independent integer formula (Python big integers reduced mod 2^64) and
against the voxel cells of points placed by construction; insertion against
brute force over all (point, splat) pairs; LRU against numpy's lexsort.
"""
from __future__ import annotations

import math

import numpy as np

P1, P2, P3 = 73856093, 19349663, 83492791
MASK = (1 << 64) - 1
Y00 = 0.28209479177387814


def cell(x, v) -> int:
    """floor(x / v) with the division in float32 (R23)."""
    return int(math.floor(float(np.float32(x) / np.float32(v))))


def key(p, v) -> int:
    """Eq. (5) (R23); the all-ones key is folded onto its predecessor, which
    the GPU table reserves for empty slots."""
    k = (cell(p[0], v) * P1 + cell(p[1], v) * P2 + cell(p[2], v) * P3) & MASK
    return k if k != MASK else MASK - 1


def keys(xyz, v) -> np.ndarray:
    return np.array([key(p, v) for p in np.asarray(xyz, np.float32).reshape(-1, 3)], np.uint64)


def insert(splat_keys, last_used, host_keys, points, v, frame, s_init, o_init, sh_degree):
    """R24.  Returns (last_used_out, reload_flags, new_params (dict, float64),
    new_keys)."""
    splat_keys = [int(k) for k in np.asarray(splat_keys, np.uint64)]
    host_keys = [int(k) for k in np.asarray(host_keys, np.uint64)]
    pts = np.asarray(points, np.float32).reshape(-1, 6)
    pkeys = [key(p[:3], v) for p in pts]
    pset = set(pkeys)
    lu = np.array(last_used, np.int32).copy()
    for j, k in enumerate(splat_keys):
        if k in pset:
            lu[j] = frame
    reload = np.array([1 if k in pset else 0 for k in host_keys], np.int32)
    known = set(splat_keys) | set(host_keys)
    first = {}
    for i, k in enumerate(pkeys):
        if k not in known and k not in first:
            first[k] = i
    order = sorted(first.values())
    K = (sh_degree + 1) ** 2
    n = len(order)
    new = dict(means=np.zeros((n, 3)), log_scales=np.full((n, 3), math.log(float(np.float32(s_init)))),
               quats=np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)),
               opacity_logits=np.full(n, math.log(float(np.float32(o_init)) / (1 - float(np.float32(o_init))))),
               sh=np.zeros((n, K, 3)))
    for r, i in enumerate(order):
        new["means"][r] = pts[i, :3].astype(np.float64)
        new["sh"][r, 0] = (pts[i, 3:6].astype(np.float64) - 0.5) / Y00
    new_keys = np.array([pkeys[i] for i in order], np.uint64)
    return lu, reload, new, new_keys


def lru_offload(last_used, tau) -> np.ndarray:
    """R25: flags of the splats to offload."""
    lu = np.asarray(last_used)
    n = lu.shape[0]
    flags = np.zeros(n, np.int32)
    if n <= tau:
        return flags
    order = sorted(range(n), key=lambda j: (int(lu[j]), j))
    for j in order[:n - tau]:
        flags[j] = 1
    return flags


def partition(arrays: dict, flags):
    """Stable partition by flags: (kept, moved), each a dict of the same keys."""
    f = np.asarray(flags).astype(bool)
    return {k: np.asarray(a)[~f] for k, a in arrays.items()}, {k: np.asarray(a)[f] for k, a in arrays.items()}
