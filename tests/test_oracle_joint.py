"""Pins of the oracle's joint LP of Alg. 1 Step 1 (Eq. (WeightedD2) under the
constraints of Eq. (D2opt)), each against a value fixed without the LP
library: closed forms for one member and for one support, the exact
breakpoint search for two supports, the transshipment form for two members
(solved by the oracle's own transportation simplex), and the per-member
decomposition at the returned weights."""
import numpy as np
import pytest

from paper_1302_0435_gb300 import synth

pytest.importorskip("scipy")


def _cluster(seed, n_mem, s, t_lo=3, t_hi=9, d=3):
    rng = np.random.default_rng(seed)
    z = rng.normal(0, 2.0, size=(s, d))
    xs = [rng.normal(0, 2.0, size=(int(t), d)) for t in rng.integers(t_lo, t_hi, size=n_mem)]
    qs = [rng.dirichlet(np.full(x.shape[0], 0.7)) for x in xs]
    om = rng.uniform(0.5, 2.0, size=n_mem)
    return z, xs, qs, om


def _costs(o, z, xs):
    return [o.cost(z, x) for x in xs]


def test_one_member_sends_each_point_to_its_nearest_support(oracle_mod):
    z, xs, qs, om = _cluster(1, 1, 5)
    c = _costs(oracle_mod, z, xs)[0]
    eps, p = oracle_mod.joint_lp([c], qs, om)
    near = c.argmin(axis=0)
    assert eps == pytest.approx(om[0] * float((qs[0] * c.min(axis=0)).sum()), rel=1e-10)
    assert np.allclose(p, np.bincount(near, weights=qs[0], minlength=5), atol=1e-9)


def test_one_support_is_the_weighted_mean_cost(oracle_mod):
    z, xs, qs, om = _cluster(2, 7, 1)
    cs = _costs(oracle_mod, z, xs)
    eps, p = oracle_mod.joint_lp(cs, qs, om)
    want = sum(w * float((q * c[0]).sum()) for c, q, w in zip(cs, qs, om))
    assert eps == pytest.approx(want, rel=1e-10) and p == pytest.approx([1.0])


def _knapsack_value(c, q, p0):
    """W(p) for two supports at p = (p0, 1 - p0): send the mass with the
    smallest c[0] - c[1] to support 0 first (fractional knapsack)."""
    order = np.argsort(c[0] - c[1], kind="stable")
    left, val = p0, float((q * c[1]).sum())
    for a in order:
        take = min(q[a], left)
        val += take * (c[0, a] - c[1, a])
        left -= take
        if left <= 0:
            break
    return val


def test_two_supports_by_breakpoint_search(oracle_mod):
    """F(p0) is convex piecewise linear with kinks at each member's partial
    sums of q in knapsack order: its minimum is at one of them or an end."""
    for seed in (3, 4, 5):
        z, xs, qs, om = _cluster(seed, 6, 2)
        cs = _costs(oracle_mod, z, xs)
        cand = {0.0, 1.0}
        for c, q in zip(cs, qs):
            cand.update(np.cumsum(q[np.argsort(c[0] - c[1], kind="stable")]).tolist())
        F = lambda p0: sum(w * _knapsack_value(c, q, min(max(p0, 0.0), 1.0))
                           for c, q, w in zip(cs, qs, om))
        best = min(F(p0) for p0 in cand)
        eps, p = oracle_mod.joint_lp(cs, qs, om)
        assert eps == pytest.approx(best, rel=1e-9)
        assert F(p[0]) == pytest.approx(best, rel=1e-9)


def test_two_members_reduce_to_transshipment(oracle_mod):
    """With two members the shared weights p are an intermediate layer:
    mass goes from member 1's supports through z to member 2's, so the
    optimum is a transportation LP between q1 and q2 whose cost is the
    cheapest route, min_r (omega_1 c1[r, a] + omega_2 c2[r, b])."""
    for seed in (6, 7):
        z, xs, qs, om = _cluster(seed, 2, 6)
        c1, c2 = _costs(oracle_mod, z, xs)
        route = (om[0] * c1[:, :, None] + om[1] * c2[:, None, :]).min(axis=0)
        want, _, _, _, _ = oracle_mod.transport(route, qs[0], qs[1])
        eps, _ = oracle_mod.joint_lp([c1, c2], qs, om)
        assert eps == pytest.approx(want, rel=1e-9)


def test_decomposition_and_bounds(oracle_mod):
    """At the returned p the members' own transportation LPs (the oracle's
    simplex) add up to epsilon; epsilon lies between the relaxation that
    lets every member pick its own p and the value at uniform weights."""
    z, xs, qs, om = _cluster(8, 12, 6)
    cs = _costs(oracle_mod, z, xs)
    eps, p = oracle_mod.joint_lp(cs, qs, om)
    assert p.sum() == pytest.approx(1.0, abs=1e-9)
    at_p = sum(w * oracle_mod.transport(c, p / p.sum(), q)[0] for c, q, w in zip(cs, qs, om))
    assert at_p == pytest.approx(eps, rel=1e-9)
    relax = sum(w * float((q * c.min(axis=0)).sum()) for c, q, w in zip(cs, qs, om))
    unif = sum(w * oracle_mod.transport(c, np.full(6, 1 / 6), q)[0] for c, q, w in zip(cs, qs, om))
    assert relax <= eps * (1 + 1e-12) and eps <= unif * (1 + 1e-12)


def test_update_weights_per_cluster(oracle_mod):
    objs, cents = synth.image_like(N=60, K=4, seed=9)
    lab, _ = oracle_mod.assign(objs, cents)
    lab[lab == 3] = 2                      # cluster 3 empty: keeps its weights
    w, eps = oracle_mod.update_weights(objs, None, lab, cents)
    off = cents.off
    assert eps[3] == 0.0 and np.array_equal(w[off[3]:off[4]], cents.w[off[3]:off[4]].astype(float))
    for j in range(3):
        assert w[off[j]:off[j + 1]].sum() == pytest.approx(1.0, abs=1e-9)
        mem = np.nonzero(lab == j)[0]
        pj = w[off[j]:off[j + 1]]
        z = np.asarray(cents.loc[off[j]:off[j + 1]], dtype=float)
        tot = 0.0
        for i in mem:
            x, wx = oracle_mod.bag(objs, i)
            tot += oracle_mod.transport(oracle_mod.cost(z, x), pj / pj.sum(), wx / wx.sum())[0]
        assert tot == pytest.approx(eps[j], rel=1e-9)


def test_hand_derived_optima(oracle_mod):
    """Hand-derived values of the joint LP (tests/golden/joint_hand.json),
    including a face of optimal weights."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "joint_hand.json")) as f:
        g = json.load(f)
    z = np.asarray(g["z"], dtype=float)[:, None]
    for case in g["cases"]:
        cs, qs = [], []
        for xs, ws in case["bags"]:
            cs.append(oracle_mod.cost(z, np.asarray(xs, dtype=float)[:, None]))
            qs.append(np.asarray(ws, dtype=float) / np.sum(ws))
        eps, p = oracle_mod.joint_lp(cs, qs, np.asarray(case["omega"], dtype=float))
        assert eps == pytest.approx(case["eps"], rel=1e-12), case["name"]
        lo, hi = case["p0_range"]
        assert lo - 1e-9 <= p[0] <= hi + 1e-9, case["name"]
        assert p.sum() == pytest.approx(1.0, abs=1e-12)
