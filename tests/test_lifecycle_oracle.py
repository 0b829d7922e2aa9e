"""Pins for the map-lifecycle and optimiser oracle (oracle/lifecycle.py)
against facts that do not come from its per-splat loop: vectorised rules in
the real (not logit) domain on values kept away from the thresholds, the
covariance of the C oracle (Mahalanobis distance of split children), exact
scale ratios, and torch.optim.Adam."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lifecycle as L

P = dict(prune_opacity=0.01, prune_scale_max=0.3, prune_scale_min=5e-5, densify_grad=2e-4,
         split_scale=0.02, clone_scale=0.01, split_shrink=1.6, reset_opacity=0.1,
         reset_scale_min=1e-4, reset_scale_max=0.25)


def random_map(rng, n, deg=1, submaps=(0, 300, 301, 700)):
    """Values drawn so that none lies within 1e-3 (relative) of a threshold."""
    def away(x, edges):
        x = x.copy()
        for e in edges:
            near = np.abs(x - e) < 1e-3 * max(1.0, abs(e))
            x[near] += 3e-3 * max(1.0, abs(e))
        return x
    logit = lambda t: math.log(t / (1 - t))
    om = away(rng.normal(-2.0, 2.0, n), [logit(0.01), logit(0.1)])
    ls = rng.normal(-4.5, 1.5, (n, 3))
    mx = ls.max(1)
    fix = away(mx, [math.log(x) for x in (0.3, 5e-5, 0.02, 0.01, 1e-4, 0.25)]) - mx
    ls += fix[:, None]
    acc = np.abs(rng.normal(0, 3e-4, n)) * rng.integers(1, 5, n)
    cnt = rng.integers(0, 5, n).astype(np.int32)
    g = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0)
    acc = np.where(np.abs(g - 2e-4) < 2e-7, acc * 1.01, acc)
    params = dict(means=rng.normal(0, 2, (n, 3)).astype(np.float32), log_scales=ls.astype(np.float32),
                  quats=rng.normal(0, 1, (n, 4)).astype(np.float32), opacity_logits=om.astype(np.float32),
                  sh=rng.normal(0, 0.3, (n, (deg + 1) ** 2, 3)).astype(np.float32))
    z = rng.normal(0, 1, (n, 2, 3)).astype(np.float32)
    return params, acc.astype(np.float32), cnt, z, np.array(submaps, np.int64)


def real_domain_actions(params, acc, cnt, ops):
    o = 1 / (1 + np.exp(-params["opacity_logits"].astype(np.float64)))
    s = np.exp(params["log_scales"].astype(np.float64)).max(1)
    g = np.where(cnt > 0, acc.astype(np.float64) / np.maximum(cnt, 1), 0.0)
    prune = (ops & L.PRUNE) > 0 and 1 or 0
    pr = prune * ((o < 0.01) | (s > 0.3) | (s < 5e-5))
    dens = ((ops & L.DENSIFY) > 0) & (g > 2e-4) & ~pr.astype(bool)
    split = dens & (s > 0.02)
    clone = dens & ~split & (s <= 0.01)
    act = np.where(pr.astype(bool), "prune", np.where(split, "split", np.where(clone, "clone", "keep")))
    reset = ((ops & L.RESET) > 0) & ~pr.astype(bool) & (o > 0.01) & (o < 0.1) & (s > 1e-4) & (s < 0.25)
    return act, reset


@pytest.mark.parametrize("ops", [L.PRUNE, L.DENSIFY, L.RESET, L.PRUNE | L.DENSIFY | L.RESET])
def test_actions_counts_and_offsets(ops):
    rng = np.random.default_rng(ops)
    params, acc, cnt, z, offs = random_map(rng, 700)
    out, mom, offs_out, actions = L.lifecycle(params, None, offs, acc, cnt, z, P, ops)
    act, reset = real_domain_actions(params, acc, cnt, ops)
    assert list(actions) == list(act)
    per = {"prune": 0, "keep": 1, "clone": 2, "split": 2}
    n_out = sum(per[a] for a in act)
    assert out["means"].shape[0] == n_out
    # submap offsets: prefix counts at each submap's first splat
    c = np.concatenate([[0], np.cumsum([per[a] for a in act])])
    assert np.array_equal(offs_out, c[offs])
    # every (kept or cloned) row equals its source exactly, resets aside
    pos = 0
    for j, a in enumerate(act):
        if a in ("keep", "clone"):
            for r in range(1 if a == "keep" else 2):
                for k in ("means", "log_scales", "quats", "sh"):
                    assert np.array_equal(out[k][pos + r], params[k][j].astype(np.float64))
                if reset[j]:
                    o = 1 / (1 + math.exp(-out["opacity_logits"][pos + r]))
                    assert o == pytest.approx(0.1, rel=1e-6)
                else:
                    assert out["opacity_logits"][pos + r] == params["opacity_logits"][j]
        pos += per[a]
    if ops & L.DENSIFY:
        assert (act == "split").sum() > 5 and (act == "clone").sum() > 5
    if ops & L.PRUNE:
        assert (act == "prune").sum() > 20
    if ops & L.RESET:
        assert reset.sum() > 5


def test_split_children_are_covariance_samples():
    rng = np.random.default_rng(5)
    params, acc, cnt, z, offs = random_map(rng, 400, submaps=(0, 400))
    out, _, _, actions = L.lifecycle(params, None, offs, acc, cnt, z, P, L.DENSIFY)
    pos, checked = 0, 0
    for j, a in enumerate(actions):
        if a == "split":
            Sig = O.cov3d(params["quats"][j].astype(np.float64), params["log_scales"][j].astype(np.float64))
            Si = np.linalg.inv(Sig)
            for k in range(2):
                d = out["means"][pos + k] - params["means"][j]
                zz = z[j, k].astype(np.float64)
                assert d @ Si @ d == pytest.approx(float(zz @ zz), rel=1e-9)
                assert np.allclose(np.exp(out["log_scales"][pos + k]) * float(np.float32(1.6)),
                                   np.exp(params["log_scales"][j].astype(np.float64)), rtol=1e-12)
                assert np.array_equal(out["quats"][pos + k], params["quats"][j].astype(np.float64))
            checked += 1
        pos += {"prune": 0, "keep": 1, "clone": 2, "split": 2}[a]
    assert checked > 5
    # children differ from each other (two independent samples)


def test_moments_follow_their_splats():
    rng = np.random.default_rng(6)
    params, acc, cnt, z, offs = random_map(rng, 500, submaps=(0, 250, 500))
    m = {k: rng.normal(size=v.shape).astype(np.float32) for k, v in params.items()}
    v = {k: rng.random(size=vv.shape).astype(np.float32) for k, vv in params.items()}
    out, (mo, vo), _, actions = L.lifecycle(params, (m, v), offs, acc, cnt, z, P, L.PRUNE | L.DENSIFY)
    pos = 0
    for j, a in enumerate(actions):
        n = {"prune": 0, "keep": 1, "clone": 2, "split": 2}[a]
        for r in range(n):
            fresh = a == "split" or (a == "clone" and r == 1)
            for k in L.FIELDS:
                if fresh:
                    assert not mo[k][pos + r].any() and not vo[k][pos + r].any()
                else:
                    assert np.array_equal(mo[k][pos + r], m[k][j].astype(np.float64))
                    assert np.array_equal(vo[k][pos + r], v[k][j].astype(np.float64))
        pos += n


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    p0 = rng.normal(size=(50, 3))
    grads = [rng.normal(size=(50, 3)) for _ in range(4)]
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for step, g in enumerate(grads, 1):
        t.grad = torch.tensor(g)
        opt.step()
        p, m, v = L.adam(p, g, m, v, step, 1e-2)
    assert np.allclose(p, t.detach().numpy(), rtol=1e-13, atol=1e-15)
