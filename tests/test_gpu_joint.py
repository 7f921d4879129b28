"""Centroid weights of Alg. 1 Step 1 (the joint LP of Eq. (WeightedD2)) on
the GPU against the oracle's LP.  The optimal value is unique, the optimal
weights need not be: the test compares the objective, and checks that the
GPU's weights are a distribution that attains it (re-evaluated by the
oracle's own transportation LPs)."""
import time

import numpy as np
import pytest

from paper_1302_0435_gb300 import synth

pytestmark = pytest.mark.gpu
pytest.importorskip("scipy")


@pytest.fixture(scope="module")
def d2():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_0435_gb300 import build, d2 as mod
    build.build()
    mod.load()
    return mod


def _weights(d2, objs, cents, lab, omega=None, max_iter=1500, tol=1e-11, table=None, cold=False):
    ctx = d2.Context(0, joint_cold_start=cold)
    if table is not None:
        d2.d2_set_cost_table(ctx, table)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents))
    K = cents.count
    eps = np.zeros(K)
    its = np.zeros(K, dtype=np.int32)
    rc = d2.d2_update_weights(ctx, d2.bags_from_synth(objs), np.ascontiguousarray(lab, np.int32),
                              max_iter=max_iter, tol=tol, omega=omega, eps=eps, iters=its)
    w = np.zeros(int(cents.off[-1]))
    d2.load().d2_get_centroids(ctx.h, None, w.ctypes.data, None, None, None)
    ctx.close()
    return rc, w, eps, its


def _F(oracle_mod, objs, cents, lab, omega, w, j, table=None):
    """Eq. (WeightedD2) of cluster j at weights w, by the oracle's LPs."""
    off = cents.off
    z = np.asarray(cents.loc[off[j]:off[j + 1]], dtype=float)
    p = w[off[j]:off[j + 1]]
    tot = 0.0
    for i in np.nonzero(lab == j)[0]:
        x, wx = oracle_mod.bag(objs, i)
        if table is None:
            c = oracle_mod.cost(z, x)
        else:
            c = table[np.ix_(x[:, 0].astype(int), z[:, 0].astype(int))].T
        tot += (1.0 if omega is None else omega[i]) * oracle_mod.transport(c, p, wx / wx.sum())[0]
    return tot


def _check(d2, oracle_mod, objs, cents, lab, omega, rc, w, eps, its, table=None, ref=None):
    assert rc == d2.D2_OK
    off = cents.off
    if ref is None:
        ref = oracle_mod.update_weights(objs, omega, lab, cents)[1] if table is None else None
    for j in range(cents.count):
        pj = w[off[j]:off[j + 1]]
        assert (pj >= 0).all() and pj.sum() == pytest.approx(1.0, abs=1e-12)
        if not (lab == j).any():
            assert its[j] == 0 and eps[j] == 0.0
            continue
        Fj = _F(oracle_mod, objs, cents, lab, omega, w, j, table)
        assert Fj == pytest.approx(eps[j], rel=1e-9)          # the weights attain eps
        if ref is not None:
            assert eps[j] == pytest.approx(ref[j], rel=1e-7)  # and eps is the LP optimum


def test_joint_weights_match_oracle(d2, oracle_mod):
    objs, cents = synth.image_like(N=360, K=6, seed=91)
    lab, _ = oracle_mod.assign(objs, cents, nthreads=8)
    rc, w, eps, its = _weights(d2, objs, cents, lab)
    _check(d2, oracle_mod, objs, cents, lab, None, rc, w, eps, its)
    print("rounds per cluster:", its.tolist())


def test_joint_weights_weighted_uneven(d2, oracle_mod):
    objs, cents = synth.uneven(N=240, K=4, seed=92)   # supports up to 64 x 32
    lab, _ = oracle_mod.assign(objs, cents, nthreads=8)
    om = np.random.default_rng(3).uniform(0.2, 4.0, objs.count)
    rc, w, eps, its = _weights(d2, objs, cents, lab, omega=om)
    _check(d2, oracle_mod, objs, cents, lab, om, rc, w, eps, its)


def test_one_support_and_empty_cluster(d2, oracle_mod):
    objs, _ = synth.image_like(N=80, K=3, seed=93)
    rng = np.random.default_rng(4)
    cents = synth._pack(np.array([1, 1, 4], dtype=np.int64), rng.normal(0, 2, (6, objs.dim)).astype(np.float32),
                        np.array([1, 1, .1, .2, .3, .4], np.float32), "f32", "f32")
    lab = rng.integers(0, 2, objs.count).astype(np.int32)   # cluster 2 stays empty
    rc, w, eps, its = _weights(d2, objs, cents, lab)
    assert rc == d2.D2_OK and its[2] == 0
    assert np.allclose(w[2:], [.1, .2, .3, .4], rtol=1e-6)  # kept
    for j in range(2):
        assert w[j] == 1.0 and its[j] == 1
        assert eps[j] == pytest.approx(_F(oracle_mod, objs, cents, lab, None, w, j), rel=1e-12)


def test_symbol_table_weights(d2, oracle_mod):
    objs, cents, table = synth.sequence_like(N=150, K=4, seed=94)
    lab, _, _ = oracle_mod.assign_table(objs, cents, table)
    rc, w, eps, its = _weights(d2, objs, cents, lab, table=table)
    ref = np.zeros(cents.count)
    off = cents.off
    for j in range(cents.count):
        mem = np.nonzero(lab == j)[0]
        if mem.size == 0:
            continue
        zs = np.asarray(cents.loc[off[j]:off[j + 1]], dtype=float)[:, 0].astype(int)
        cs, qs = [], []
        for i in mem:
            x, wx = oracle_mod.bag(objs, i)
            cs.append(table[np.ix_(x[:, 0].astype(int), zs)].T)
            qs.append(wx / wx.sum())
        ref[j] = oracle_mod.joint_lp(cs, qs, np.ones(mem.size))[0]
    _check(d2, oracle_mod, objs, cents, lab, None, rc, w, eps, its, table=table, ref=ref)


def test_alg1_step2_does_not_increase_the_objective(d2, oracle_mod):
    """Alg. 1: after Step 1 (weights) Step 2 moves the supports to the
    flow-weighted means of the joint optimum's flows, which cannot raise
    Eq. (WeightedD2)."""
    objs, cents = synth.image_like(N=300, K=5, seed=95)
    lab, _ = oracle_mod.assign(objs, cents, nthreads=8)
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents))
    ob = d2.bags_from_synth(objs)
    eps = np.zeros(5)
    lab32 = lab.astype(np.int32)
    assert d2.d2_update_weights(ctx, ob, lab32, max_iter=1500, tol=1e-11, eps=eps) == d2.D2_OK
    d2.d2_update_locations(ctx, ob, lab32)
    loc = np.zeros((int(cents.off[-1]), objs.dim))
    w = np.zeros(int(cents.off[-1]))
    d2.load().d2_get_centroids(ctx.h, loc.ctypes.data, w.ctypes.data, None, None, None)
    ctx.close()
    moved = synth._pack(np.diff(cents.off), loc, w, "f64", "f64")
    for j in range(5):
        assert _F(oracle_mod, objs, moved, lab, None, w, j) <= eps[j] * (1 + 1e-9)


def test_update_weights_errors(d2):
    objs, cents = synth.image_like(N=30, K=3, seed=96)
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents))
    lab = np.zeros(objs.count, dtype=np.int32)
    ob = d2.bags_from_synth(objs)
    for kw in (dict(max_iter=0), dict(tol=-1.0), dict(max_iter=5000)):
        with pytest.raises(d2.D2Error) as e:
            d2.d2_update_weights(ctx, ob, lab, **kw)
        assert e.value.code == d2.D2_EINVAL
    # a round cap too small to certify: best weights kept, status reported
    rc = d2.d2_update_weights(ctx, ob, lab, max_iter=2, tol=0.0)
    assert rc == d2.D2_ENOTCONVERGED
    ctx.close()


def test_joint_weights_image_like_full_size(d2, oracle_mod):
    """200,000 image-like bags in 64 clusters (their nearest centroids)."""
    import torch
    objs, cents = synth.image_like()
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    d2.d2_assign(ctx, ob, lab, dist)
    d2.d2_sync(ctx)
    before = float(dist.sum())
    eps = torch.zeros(64, dtype=torch.float64, device="cuda:0")
    its = torch.zeros(64, dtype=torch.int32, device="cuda:0")
    t0 = time.perf_counter()
    rc = d2.d2_update_weights(ctx, ob, lab, max_iter=1000, tol=1e-9, eps=eps, iters=its)
    d2.d2_sync(ctx)
    dt = time.perf_counter() - t0
    w = np.zeros(int(cents.off[-1]))
    d2.load().d2_get_centroids(ctx.h, None, w.ctypes.data, None, None, None)
    ctx.close()
    assert rc == d2.D2_OK
    e = eps.cpu().numpy()
    it = its.cpu().numpy()
    print("joint weights, 200,000 bags x 64 clusters: %.2f s, rounds %d..%d (mean %.0f), "
          "objective %.6g -> %.6g" % (dt, it.min(), it.max(), it.mean(), before, e.sum()))
    assert e.sum() <= before * (1 + 1e-9)
    labn = lab.cpu().numpy()
    for j in (0, 37):                                   # sampled clusters, re-evaluated
        assert _F(oracle_mod, objs, cents, labn, None, w, j) == pytest.approx(e[j], rel=1e-9)


@pytest.mark.parametrize("law", ["image_like", "uneven"])
def test_warm_rounds_match_cold_rounds(d2, oracle_mod, law):
    """Rounds that restart every member from its previous optimal basis
    (dual pivots after the weights moved) reach the same optimum as rounds
    that solve every member cold, with fewer member pivots; the warm weights
    attain eps and eps is the LP optimum (oracle)."""
    if law == "image_like":
        objs, cents = synth.image_like(N=600, K=6, seed=93)
    else:
        objs, cents = synth.uneven(N=500, K=5, seed=94)
    lab, _ = oracle_mod.assign(objs, cents, nthreads=8)
    out = {}
    for cold in (True, False):
        s0 = d2.d2_get_stats()
        rc, w, eps, its = _weights(d2, objs, cents, lab, cold=cold)
        s1 = d2.d2_get_stats()
        out[cold] = (rc, w, eps, its, s1["pivots_exact"] - s0["pivots_exact"],
                     s1["pairs_exact"] - s0["pairs_exact"])
    rc, w, eps, its, piv_w, pairs_w = out[False]
    _check(d2, oracle_mod, objs, cents, lab, None, rc, w, eps, its)
    np.testing.assert_allclose(eps, out[True][2], rtol=1e-9)
    # pivots per member solve: the warm restarts need fewer
    assert piv_w / pairs_w < out[True][4] / out[True][5]
