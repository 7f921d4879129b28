"""Pins for the oracle's location update (Eq. (UpdateZ), Eq. (WeightedUpdate)),
label merge (Eq. (UpdateLabel), Eq. (UpdateGlobalLabel)), weight propagation
and level loop (Alg. 3 with Alg. 2 inside segments)."""
import json
import os

import numpy as np
import pytest

from paper_1302_0435_gb300.synth import Bags

HERE = os.path.dirname(os.path.abspath(__file__))


def _bags(list_of_xw):
    locs = [np.asarray(x, dtype=np.float64).reshape(len(w), -1) for x, w in list_of_xw]
    ws = [np.asarray(w, dtype=np.float64) for _, w in list_of_xw]
    off = np.concatenate([[0], np.cumsum([len(w) for w in ws])]).astype(np.int64)
    return Bags(np.concatenate(locs), np.concatenate(ws), off)


def _monotone_flows_1d(x, p, y, q):
    """Flows of the monotone coupling in 1-D, from the quantile intervals."""
    ix, iy = np.argsort(x, kind="stable"), np.argsort(y, kind="stable")
    p = p / p.sum()
    q = q / q.sum()
    Fx, Fy = np.cumsum(p[ix]), np.cumsum(q[iy])
    Fx[-1] = Fy[-1] = 1.0
    bps = np.unique(np.concatenate([[0.0], Fx, Fy]))
    W = np.zeros((x.size, y.size))
    for lo, hi in zip(bps[:-1], bps[1:]):
        mid = 0.5 * (lo + hi)
        a = ix[min(int(np.searchsorted(Fx, mid)), x.size - 1)]
        r = iy[min(int(np.searchsorted(Fy, mid)), y.size - 1)]
        W[a, r] += hi - lo
    return W


def _coo(W, i):
    a, r = np.nonzero(W)
    return np.full(a.size, i), a, r, W[a, r]


def test_update_golden(oracle_mod):
    with open(os.path.join(HERE, "golden", "hand_examples.json")) as f:
        ex = json.load(f)["update"][0]
    objs = _bags([(ex["x"], ex["wx"])])
    cents = _bags([(ex["y"], ex["wy"])])
    lab = np.array([0])
    fo, fa, fr, fw = oracle_mod.assigned_flows(objs, cents, lab)
    new = oracle_mod.update_locations(objs, None, lab, fo, fa, fr, fw, cents)
    assert np.allclose(new, np.asarray(ex["y_new"]), rtol=0, atol=1e-15)


def test_update_one_dimensional_monotone(oracle_mod):
    rng = np.random.default_rng(21)
    for _ in range(20):
        m, n = int(rng.integers(1, 15)), int(rng.integers(1, 15))
        x, p = rng.normal(size=m), rng.dirichlet(np.ones(m))
        y, q = rng.normal(size=n), np.full(n, 1.0 / n)
        objs = _bags([(x[:, None], p)])
        cents = _bags([(y[:, None], q)])
        lab = np.array([0])
        fo, fa, fr, fw = oracle_mod.assigned_flows(objs, cents, lab)
        new = oracle_mod.update_locations(objs, None, lab, fo, fa, fr, fw, cents)[:, 0]
        W = _monotone_flows_1d(x, p, y, q)
        col = W.sum(axis=0)
        expect = np.where(col > 0, (W * x[:, None]).sum(axis=0) / np.where(col > 0, col, 1), y)
        assert np.allclose(new, expect, rtol=1e-12, atol=1e-12)


def test_update_fixed_point(oracle_mod):
    rng = np.random.default_rng(22)
    y = rng.normal(size=(6, 3))
    q = np.full(6, 1.0 / 6)
    objs = _bags([(y, q), (y, q * 7.0)])
    cents = _bags([(y, q)])
    lab = np.array([0, 0])
    fo, fa, fr, fw = oracle_mod.assigned_flows(objs, cents, lab)
    new = oracle_mod.update_locations(objs, np.array([2.0, 0.5]), lab, fo, fa, fr, fw, cents)
    assert np.allclose(new, y, rtol=0, atol=1e-14)


def test_update_weights_common_scale_and_single_weight(oracle_mod):
    rng = np.random.default_rng(23)
    objs = _bags([(rng.normal(size=(m, 2)), rng.dirichlet(np.ones(m))) for m in (3, 5, 4)])
    cents = _bags([(rng.normal(size=(4, 2)), np.full(4, 0.25))])
    lab = np.zeros(3, dtype=np.int64)
    fo, fa, fr, fw = oracle_mod.assigned_flows(objs, cents, lab)
    om = np.array([1.0, 2.0, 3.0])
    a = oracle_mod.update_locations(objs, om, lab, fo, fa, fr, fw, cents)
    b = oracle_mod.update_locations(objs, om * 17.0, lab, fo, fa, fr, fw, cents)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-13)
    # all weight on object 1: its barycentric projection alone
    c = oracle_mod.update_locations(objs, np.array([0.0, 1.0, 0.0]), lab, fo, fa, fr, fw, cents)
    x1 = objs.loc[3:8]
    W = np.zeros((5, 4))
    sel = fo == 1
    W[fa[sel], fr[sel]] = fw[sel]
    assert np.allclose(c, (W.T @ x1) / W.sum(axis=0)[:, None], rtol=1e-13, atol=1e-13)


def test_update_empty_cluster_and_zero_mass_support_keep_location(oracle_mod):
    cents = _bags([([[0.0], [5.0]], [0.5, 0.5]), ([[9.0], [9.5]], [0.5, 0.5])])
    objs = _bags([([[1.0], [4.0]], [0.5, 0.5])])
    lab = np.array([0])
    # synthetic flows: only support 0 of centroid 0 receives mass
    new = oracle_mod.update_locations(objs, None, lab, np.array([0]), np.array([1]), np.array([0]),
                                      np.array([1.0]), cents)
    assert np.allclose(new[:, 0], [4.0, 5.0, 9.0, 9.5])


def test_label_merge_hand_maps(oracle_mod):
    seg = [np.array([0, 1, 1]), np.array([1, 0])]
    C_tilde = np.concatenate(oracle_mod.update_label(seg, [2, 2]))
    assert C_tilde.tolist() == [0, 1, 1, 3, 2]
    assert oracle_mod.update_global_label(np.array([4, 0, 2]), C_tilde).tolist() == [2, 0, 1]
    w = oracle_mod.propagate_weights(C_tilde, np.ones(5), 4)
    assert w.tolist() == [1.0, 2.0, 1.0, 1.0]
    # three segments with unequal centroid counts
    seg = [np.array([2, 0]), np.array([0]), np.array([1, 1, 0])]
    assert np.concatenate(oracle_mod.update_label(seg, [3, 1, 2])).tolist() == [2, 0, 3, 5, 5, 4]


def _cluster_data(rng, N, d, centers, m_range=(3, 6)):
    sizes = rng.integers(*m_range, size=N)
    comp = rng.integers(0, len(centers), size=N)
    loc = np.concatenate([centers[c] + 0.3 * rng.normal(size=(s, d)) for c, s in zip(comp, sizes)])
    w = np.concatenate([rng.dirichlet(np.ones(s)) for s in sizes])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return Bags(loc, w, off), comp


def test_level_single_segment_is_alg2(oracle_mod):
    rng = np.random.default_rng(24)
    centers = np.array([[-4.0, 0.0], [4.0, 0.0], [0.0, 5.0]])
    objs, _ = _cluster_data(rng, 30, 2, centers)
    init = _bags([(centers[k] + rng.normal(size=(3, 2)), np.full(3, 1 / 3)) for k in range(3)])
    cl, cw, lab = oracle_mod.cluster_level(objs, None, init, 3, 100, 3)
    # the same loop written out: assign, flows, update, three times
    cents = init
    for _ in range(3):
        l2, _ = oracle_mod.assign(objs, cents)
        fo, fa, fr, fw = oracle_mod.assigned_flows(objs, cents, l2)
        cents = Bags(oracle_mod.update_locations(objs, None, l2, fo, fa, fr, fw, cents), cents.w, cents.off)
    assert lab.tolist() == l2.tolist()
    assert np.allclose(cl, cents.loc, rtol=0, atol=0)
    assert cw.sum() == pytest.approx(30.0)


def test_level_two_levels_weights_and_labels(oracle_mod):
    rng = np.random.default_rng(25)
    centers = np.array([[-6.0, 0.0], [6.0, 0.0]])
    objs, comp = _cluster_data(rng, 40, 2, centers)
    init = _bags([(centers[k] + 0.5 * rng.normal(size=(3, 2)), np.full(3, 1 / 3)) for k in range(2)])
    om = rng.uniform(0.5, 2.0, size=40)
    cl, cw, lab = oracle_mod.cluster_level(objs, om, init, 2, 12, 2)
    assert cw.sum() == pytest.approx(om.sum(), rel=1e-12)       # weights conserved across levels
    assert set(np.unique(lab)) <= {0, 1}
    # well separated groups end in different clusters, members agree
    for c in range(2):
        assert len(set(lab[comp == c].tolist())) == 1
    assert lab[comp == 0][0] != lab[comp == 1][0]
    for k in range(2):
        assert cw[k] == pytest.approx(om[lab == k].sum(), rel=1e-12)
