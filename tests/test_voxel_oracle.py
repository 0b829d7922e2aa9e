"""Pins for the voxel-hash / active-set oracle (oracle/voxel.py): keys
against numpy's wrapping int64 arithmetic and cells placed by construction;
insertion against a vectorised np.isin / np.unique formulation; LRU against
np.lexsort; new splats render their point's colour."""
import numpy as np
import pytest

import oracle as O
from oracle import voxel as V


def _np_keys(xyz, v):
    c = np.floor(np.asarray(xyz, np.float32) / np.float32(v)).astype(np.int64)
    with np.errstate(over="ignore"):
        k = c[:, 0] * np.int64(V.P1) + c[:, 1] * np.int64(V.P2) + c[:, 2] * np.int64(V.P3)
    return k.view(np.uint64)


def test_keys_match_wrapping_int64_and_cells():
    rng = np.random.default_rng(0)
    v = 0.05
    xyz = rng.uniform(-1e4, 1e4, (2000, 3)).astype(np.float32)
    assert np.array_equal(V.keys(xyz, v), _np_keys(xyz, v))
    # cell centres: the cell index is the construction index exactly
    idx = rng.integers(-5000, 5000, (500, 3))
    centres = ((idx + 0.5) * v).astype(np.float32)
    for (i, j, k), p in zip(idx, centres):
        assert V.cell(p[0], v) == i and V.cell(p[1], v) == j and V.cell(p[2], v) == k
    # distinct nearby cells give distinct keys
    g = np.stack(np.meshgrid(*[np.arange(-20, 21)] * 3, indexing="ij"), -1).reshape(-1, 3)
    ks = V.keys(((g + 0.5) * v).astype(np.float32), v)
    assert len(np.unique(ks)) == len(g)


def _scene(rng, n_splats=3000, n_host=800, n_pts=5000, v=0.1):
    sp = rng.uniform(-3, 3, (n_splats, 3)).astype(np.float32)
    hp = rng.uniform(-3, 3, (n_host, 3)).astype(np.float32)
    pts = np.concatenate([rng.uniform(-4, 4, (n_pts, 3)), rng.random((n_pts, 3))], 1).astype(np.float32)
    # some points fall exactly into splat / host voxels
    pts[:500, :3] = sp[rng.integers(0, n_splats, 500)] + rng.uniform(-1e-3, 1e-3, (500, 3))
    pts[500:700, :3] = hp[rng.integers(0, n_host, 200)] + rng.uniform(-1e-3, 1e-3, (200, 3))
    return sp, hp, pts, v


def test_insert_matches_vectorised_rules():
    rng = np.random.default_rng(1)
    sp, hp, pts, v = _scene(rng)
    sk, hk, pk = _np_keys(sp, v), _np_keys(hp, v), _np_keys(pts[:, :3], v)
    lu0 = rng.integers(0, 5, len(sp)).astype(np.int32)
    lu, reload, new, new_keys = V.insert(sk, lu0, hk, pts, v, 9, 0.02, 0.1, 1)
    act = np.isin(sk, pk)
    assert np.array_equal(lu, np.where(act, 9, lu0))
    assert np.array_equal(reload.astype(bool), np.isin(hk, pk))
    unmatched = ~np.isin(pk, np.concatenate([sk, hk]))
    uk, first = np.unique(pk[unmatched], return_index=True)
    first_pts = np.nonzero(unmatched)[0][first]
    order = np.argsort(first_pts)
    assert np.array_equal(new_keys, uk[order])
    assert np.array_equal(new["means"], pts[first_pts[order], :3].astype(np.float64))
    assert act.sum() > 50 and reload.sum() > 50 and len(new_keys) > 1000
    # a new splat renders its point's colour: 0.5 + Y00 * DC
    rgb = 0.5 + V.Y00 * new["sh"][:, 0]
    assert np.allclose(rgb, pts[first_pts[order], 3:6], atol=1e-12)
    assert np.allclose(O.sh_basis(0, np.array([0.0, 0.0, 1.0]))[0], V.Y00, rtol=1e-15)
    # isotropic scale and identity rotation
    assert np.allclose(np.exp(new["log_scales"]), np.float32(0.02), rtol=1e-15)
    assert np.all(new["quats"] == [1, 0, 0, 0])


def test_lru_matches_lexsort():
    rng = np.random.default_rng(2)
    lu = rng.integers(0, 30, 5000).astype(np.int32)
    for tau in (5000, 4999, 3000, 0):
        flags = V.lru_offload(lu, tau)
        n_off = max(0, len(lu) - tau)
        ref = np.zeros(len(lu), np.int32)
        ref[np.lexsort((np.arange(len(lu)), lu))[:n_off]] = 1
        assert np.array_equal(flags, ref), tau
        assert flags.sum() == n_off


def test_partition_is_stable():
    rng = np.random.default_rng(3)
    a = {"x": np.arange(100), "y": rng.random((100, 3))}
    f = rng.integers(0, 2, 100)
    kept, moved = V.partition(a, f)
    assert list(kept["x"]) == [i for i in range(100) if not f[i]]
    assert list(moved["x"]) == [i for i in range(100) if f[i]]
