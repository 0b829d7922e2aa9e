"""Map lifecycle and Adam on the GPU against the numpy oracle
(oracle/lifecycle.py), through the C ABI.

Bars: which splats survive, are cloned or split, the output count and the new
submap offsets are integer results and must match exactly; copied rows,
opacity resets and moments are bit-exact; split children (float32 against
float64 arithmetic) within 1e-6 relative; Adam within 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import lifecycle as L
from tests.test_lifecycle_oracle import P, random_map

pytestmark = pytest.mark.gpu

FIELDS = L.FIELDS


def _dev(torch, d):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


def _run_gpu(G, torch, params, offs, acc, cnt, z, ops, moments=None, deg=1, capacity=None):
    lc = G.Lifecycle(params["means"].shape[0] + 1, len(offs) - 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out, mom, offs_out, n = lc.run(_dev(torch, params), offs, deg, G.lifecycle_params(ops, **P), t(acc), t(cnt),
                                   t(z), moments=None if moments is None else tuple(_dev(torch, m) for m in moments),
                                   capacity=capacity)
    torch.cuda.synchronize()
    lc.close()
    np_ = lambda d: {k: v.cpu().numpy() for k, v in d.items()}
    return np_(out), (None if mom is None else tuple(np_(m) for m in mom)), offs_out.cpu().numpy(), n


def _compare(params, out_g, out_o, actions, mom_g=None, mom_o=None):
    n = out_o["means"].shape[0]
    assert out_g["means"].shape[0] == n
    split_rows = []
    pos = 0
    for a in actions:
        c = {"prune": 0, "keep": 1, "clone": 2, "split": 2}[a]
        if a == "split":
            split_rows += [pos, pos + 1]
        pos += c
    exact = np.ones(n, bool)
    exact[split_rows] = False
    for k in ("quats", "opacity_logits", "sh"):
        assert np.array_equal(out_g[k].astype(np.float64), out_o[k]), k
    for k in ("means", "log_scales"):
        assert np.array_equal(out_g[k][exact].astype(np.float64), out_o[k][exact]), k
        if split_rows:
            err = np.abs(out_g[k][split_rows] - out_o[k][split_rows]) / (1.0 + np.abs(out_o[k][split_rows]))
            assert err.max() <= 1e-6, (k, err.max())
    if mom_o is not None:
        for a in range(2):
            for k in FIELDS:
                assert np.array_equal(mom_g[a][k].astype(np.float64), mom_o[a][k]), (a, k)
    return len(split_rows) // 2


@pytest.mark.parametrize("ops", [L.PRUNE, L.DENSIFY, L.RESET, L.PRUNE | L.DENSIFY | L.RESET])
def test_lifecycle_matches_oracle(ops):
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(100 + ops)
    params, acc, cnt, z, offs = random_map(rng, 5000, submaps=(0, 1200, 1200, 4000, 5000))
    out_o, _, offs_o, actions = L.lifecycle(params, None, offs, acc, cnt, z, P, ops)
    out_g, _, offs_g, n = _run_gpu(G, torch, params, offs, acc, cnt, z, ops)
    assert n == out_o["means"].shape[0]
    assert np.array_equal(offs_g, offs_o)
    nsplit = _compare(params, out_g, out_o, actions)
    print(f"[ops {ops}] {len(actions)} -> {n}; " +
          " ".join(f"{a} {actions.count(a)}" for a in ("prune", "keep", "clone", "split")))
    if ops & L.DENSIFY:
        assert nsplit > 10


def test_lifecycle_moments_and_chunks():
    # several scatter blocks (2048 splats each) and submaps crossing them
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(7)
    n = 9000
    params, acc, cnt, z, offs = random_map(rng, n, deg=3, submaps=(0, 2047, 2048, 2049, 6000, 9000))
    m = {k: rng.normal(size=v.shape).astype(np.float32) for k, v in params.items()}
    v = {k: rng.random(size=vv.shape).astype(np.float32) for k, vv in params.items()}
    ops = L.PRUNE | L.DENSIFY | L.RESET
    out_o, mom_o, offs_o, actions = L.lifecycle(params, (m, v), offs, acc, cnt, z, P, ops)
    out_g, mom_g, offs_g, nout = _run_gpu(G, torch, params, offs, acc, cnt, z, ops, moments=(m, v), deg=3)
    assert nout == out_o["means"].shape[0] and np.array_equal(offs_g, offs_o)
    _compare(params, out_g, out_o, actions, mom_g, mom_o)


def test_lifecycle_full_size():
    # a 500k-splat map in 8 uneven submaps, every operation
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(8)
    n = 500_000
    cuts = np.sort(rng.choice(np.arange(1, n), 7, replace=False))
    offs = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    params, acc, cnt, z, _ = random_map(rng, n, deg=3, submaps=offs)
    ops = L.PRUNE | L.DENSIFY | L.RESET
    out_o, _, offs_o, actions = L.lifecycle(params, None, offs, acc, cnt, z, P, ops)
    out_g, _, offs_g, nout = _run_gpu(G, torch, params, offs, acc, cnt, z, ops, deg=3)
    assert nout == out_o["means"].shape[0] and np.array_equal(offs_g, offs_o)
    _compare(params, out_g, out_o, actions)


def test_lifecycle_edges():
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(9)
    params, acc, cnt, z, offs = random_map(rng, 3000, submaps=(0, 1000, 3000))
    ops = L.PRUNE | L.DENSIFY
    out_o, _, offs_o, _ = L.lifecycle(params, None, offs, acc, cnt, z, P, ops)
    need = out_o["means"].shape[0]
    # capacity one short: GS_ERR_CAPACITY, nothing written
    with pytest.raises(G.GsError) as ei:
        _run_gpu(G, torch, params, offs, acc, cnt, z, ops, capacity=need - 1)
    assert ei.value.status == G.GS_ERR_CAPACITY
    # exactly enough
    out_g, _, offs_g, n = _run_gpu(G, torch, params, offs, acc, cnt, z, ops, capacity=need)
    assert n == need and np.array_equal(offs_g, offs_o)
    # everything pruned: empty output, all offsets 0
    dead = dict(params)
    dead["opacity_logits"] = np.full_like(params["opacity_logits"], -20.0)
    out_g, _, offs_g, n = _run_gpu(G, torch, dead, offs, acc, cnt, z, L.PRUNE)
    assert n == 0 and not offs_g.any()
    # nothing to do: outputs equal inputs bitwise
    out_g, _, offs_g, n = _run_gpu(G, torch, params, offs, acc, cnt, z, 0)
    assert n == 3000 and np.array_equal(offs_g, offs)
    for k in FIELDS:
        assert np.array_equal(out_g[k], params[k])
    # empty input
    lc = G.Lifecycle(16, 2)
    empty = {k: torch.zeros((0,) + v.shape[1:], device="cuda") for k, v in params.items()}
    out, _, offs_e, n = lc.run(empty, [0, 0, 0], 1, G.lifecycle_params(L.PRUNE))
    assert n == 0 and offs_e.cpu().tolist() == [0, 0, 0]
    lc.close()


def test_adam_matches_oracle():
    import torch
    from paper_2510_26358_gb300 import gsraster as G
    rng = np.random.default_rng(10)
    n = 20_000
    params, _, _, _, _ = random_map(rng, n, deg=2, submaps=(0, n))
    lr = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    pd = _dev(torch, params)
    md = {k: torch.zeros_like(v) for k, v in pd.items()}
    vd = {k: torch.zeros_like(v) for k, v in pd.items()}
    po = {k: v.astype(np.float64) for k, v in params.items()}
    mo = {k: np.zeros_like(v) for k, v in po.items()}
    vo = {k: np.zeros_like(v) for k, v in po.items()}
    for step in range(1, 4):
        grads = {k: (rng.normal(size=v.shape) * 1e-3).astype(np.float32) for k, v in params.items()}
        G.adam_step(pd, _dev(torch, grads), md, vd, 2, step, lr)
        for i, k in enumerate(FIELDS):
            po[k], mo[k], vo[k] = L.adam(po[k], grads[k], mo[k], vo[k], step, lr[i])
    torch.cuda.synchronize()
    for k in FIELDS:
        g = pd[k].cpu().numpy().astype(np.float64)
        step_size = np.abs(params[k].astype(np.float64) - po[k]).max()
        err = np.abs(g - po[k]).max()
        # float32 parameters carry their own rounding (ulp of the value); the update must be right to 1e-4 of its size
        ulp = np.abs(po[k]).max() * 2 ** -23
        assert err <= 1e-4 * step_size + 2 * ulp, (k, err, step_size)
