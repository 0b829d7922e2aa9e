"""Voxel-hash insertion (Eq. 5) and the LRU active set on the GPU against the
oracle (oracle/voxel.py), through the C ABI.

Keys, last_used, reload flags, the set and order of new splats, LRU flags and
partitions are integer results: bit-exact.  New splats' means and quaternions
are copies (exact); log-scale, opacity logit and SH DC (float32 against
float64 arithmetic) within 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import voxel as V
from tests.test_voxel_oracle import _scene

pytestmark = pytest.mark.gpu


def _t(torch, a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda() if dtype is None else \
        torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def test_keys_bit_exact():
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(0)
    xyz = np.concatenate([rng.uniform(-1e4, 1e4, (20000, 3)), rng.uniform(-2, 2, (20000, 3))]).astype(np.float32)
    vm = G.VoxelMap(16, 16)
    for v in (0.05, 0.1, 0.37):
        k = vm.keys(_t(torch, xyz), v)
        assert np.array_equal(_u64(k), V.keys(xyz, v)), v
    # strided rows (points with colour)
    pts = np.concatenate([xyz[:1000], rng.random((1000, 3)).astype(np.float32)], 1)
    k = vm.keys(_t(torch, pts), 0.1)
    assert np.array_equal(_u64(k), V.keys(pts[:, :3], 0.1))
    vm.close()


@pytest.mark.parametrize("n_pts", [5000, 60000])
def test_insert_matches_oracle(n_pts):
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(n_pts)
    sp, hp, pts, v = _scene(rng, n_pts=n_pts)
    sk, hk = V.keys(sp, v), V.keys(hp, v)
    lu0 = rng.integers(0, 5, len(sp)).astype(np.int32)
    lu_o, reload_o, new_o, nk_o = V.insert(sk, lu0, hk, pts, v, 9, 0.02, 0.1, 2)
    vm = G.VoxelMap(n_pts, 16)
    lu = _t(torch, lu0)
    reload, new, nk, n = vm.insert(_t(torch, pts), _t(torch, sk.view(np.int64)), lu, _t(torch, hk.view(np.int64)),
                                   2, v, 0.02, 0.1, 9)
    torch.cuda.synchronize()
    assert np.array_equal(lu.cpu().numpy(), lu_o)
    assert np.array_equal(reload.cpu().numpy(), reload_o)
    assert n == len(nk_o) and np.array_equal(_u64(nk), nk_o)
    assert np.array_equal(new["means"].cpu().numpy().astype(np.float64), new_o["means"])
    assert np.array_equal(new["quats"].cpu().numpy().astype(np.float64), new_o["quats"])
    for k in ("log_scales", "opacity_logits", "sh"):
        g, o = new[k].cpu().numpy().astype(np.float64), new_o[k]
        assert (np.abs(g - o) / (1 + np.abs(o))).max() <= 1e-6, k
    print(f"[{n_pts} points] active {(lu_o == 9).sum()}, reload {reload_o.sum()}, new {n}")
    vm.close()


def test_insert_edges():
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(3)
    sp, hp, pts, v = _scene(rng, n_pts=3000)
    sk, hk = V.keys(sp, v), V.keys(hp, v)
    vm = G.VoxelMap(3000, 16)
    lu = torch.zeros(len(sp), dtype=torch.int32, device="cuda")
    # capacity one short of the new splats: capacity error, nothing written
    _, _, _, n_needed = vm.insert(_t(torch, pts), _t(torch, sk.view(np.int64)), lu, _t(torch, hk.view(np.int64)),
                                  0, v, 0.02, 0.1, 1)
    with pytest.raises(G.GsError) as ei:
        vm.insert(_t(torch, pts), _t(torch, sk.view(np.int64)), lu, _t(torch, hk.view(np.int64)), 0, v, 0.02, 0.1, 1,
                  capacity=n_needed - 1)
    assert ei.value.status == G.GS_ERR_CAPACITY
    # empty batch: nothing changes
    lu2 = torch.full((len(sp),), 4, dtype=torch.int32, device="cuda")
    reload, new, nk, n = vm.insert(torch.zeros(0, 6, device="cuda"), _t(torch, sk.view(np.int64)), lu2,
                                   _t(torch, hk.view(np.int64)), 0, v, 0.02, 0.1, 7)
    assert n == 0 and int(lu2.min()) == 4 and int(reload.sum()) == 0
    # a batch of points all in one new voxel: one splat, from the first point
    one = np.tile(np.array([[100.01, 100.02, 100.03, 0.2, 0.4, 0.6]], np.float32), (50, 1))
    one[1:, :3] += rng.uniform(0, 1e-3, (49, 3)).astype(np.float32)
    reload, new, nk, n = vm.insert(_t(torch, one), _t(torch, sk.view(np.int64)), lu2, _t(torch, hk.view(np.int64)),
                                   0, 0.1, 0.02, 0.1, 8)
    assert n == 1 and np.array_equal(new["means"].cpu().numpy()[0], one[0, :3])
    vm.close()


@pytest.mark.parametrize("tau", [100_000, 99_999, 70_000, 31_337, 0])
def test_lru_select_matches_oracle(tau):
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(4)
    lu = rng.integers(-3, 40, 100_000).astype(np.int32)  # many ties, negative frames too
    vm = G.VoxelMap(16, 100_000)
    flags = vm.select(_t(torch, lu), tau)
    torch.cuda.synchronize()
    assert np.array_equal(flags.cpu().numpy(), V.lru_offload(lu, tau))
    vm.close()


def test_offload_and_reload_through_host_memory():
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(5)
    n, deg, tau = 30_000, 3, 21_000
    K = (deg + 1) ** 2
    params = dict(means=rng.normal(size=(n, 3)), log_scales=rng.normal(size=(n, 3)), quats=rng.normal(size=(n, 4)),
                  opacity_logits=rng.normal(size=n), sh=rng.normal(size=(n, K, 3)))
    params = {k: v.astype(np.float32) for k, v in params.items()}
    keys = rng.integers(0, 2 ** 63, n).astype(np.int64)
    lu = rng.integers(0, 20, n).astype(np.int32)
    vm = G.VoxelMap(16, n)
    pd = {k: _t(torch, v) for k, v in params.items()}
    flags = vm.select(_t(torch, lu), tau)
    f = flags.cpu().numpy()
    assert f.sum() == n - tau
    dev_out = {k: torch.empty_like(v) for k, v in pd.items()}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in pd.items()}
    kk, km = torch.empty(n, dtype=torch.int64, device="cuda"), torch.empty(n, dtype=torch.int64).pin_memory()
    lk, lm = torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32).pin_memory()
    counts = vm.partition(flags, deg, pd, _t(torch, keys), _t(torch, lu), dev_out, kk, lk, host_out, km, lm)
    torch.cuda.synchronize()
    nk, nm = counts.cpu().tolist()
    assert (nk, nm) == (tau, n - tau)
    kept_o, moved_o = V.partition(dict(params, keys=keys, lu=lu), f)
    for k in params:
        assert np.array_equal(dev_out[k][:nk].cpu().numpy(), kept_o[k]), k
        assert np.array_equal(host_out[k][:nm].numpy(), moved_o[k]), k
    assert np.array_equal(kk[:nk].cpu().numpy(), kept_o["keys"]) and np.array_equal(km[:nm].numpy(), moved_o["keys"])
    assert np.array_equal(lk[:nk].cpu().numpy(), kept_o["lu"]) and np.array_equal(lm[:nm].numpy(), moved_o["lu"])
    # reload every other offloaded splat from host memory back to the device
    rf = np.zeros(nm, np.int32)
    rf[::2] = 1
    hk_in = {k: v[:nm] for k, v in host_out.items()}
    stay = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in hk_in.items()}
    back = {k: torch.empty_like(v).cuda() for k, v in hk_in.items()}
    c2 = vm.partition(_t(torch, rf), deg, hk_in, None, None, stay, None, None, back, None, None)
    torch.cuda.synchronize()
    assert c2.cpu().tolist() == [nm - rf.sum(), rf.sum()]
    for k in params:
        assert np.array_equal(back[k][:rf.sum()].cpu().numpy(), moved_o[k][rf.astype(bool)]), k
        assert np.array_equal(stay[k][:nm - rf.sum()].numpy(), moved_o[k][~rf.astype(bool)]), k
    vm.close()
