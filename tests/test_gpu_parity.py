"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Bars: labels bit-exact except at ties within 1e-9 relative (the oracle's
own D^2 values decide what is a tie); D^2 within 1e-6 relative (with an
absolute floor of 1e-12 * the largest cost for D^2 ~ 0); update against the
oracle's update from the GPU's own flows within 1e-12 relative.
"""
import numpy as np
import pytest

from paper_1302_0435_gb300 import synth
from paper_1302_0435_gb300.synth import Bags

pytestmark = pytest.mark.gpu

REL = 1e-6
TIE = 1e-9


@pytest.fixture(scope="module")
def d2():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_0435_gb300 import build, d2 as mod
    build.build()
    mod.load()
    return mod


def make_bags(pairs, dtype=np.float64, wdtype=np.float64):
    locs = [np.asarray(x, dtype=np.float64).reshape(len(w), -1) for x, w in pairs]
    ws = [np.asarray(w, dtype=np.float64) for _, w in pairs]
    off = np.concatenate([[0], np.cumsum([len(w) for w in ws])]).astype(np.int64)
    name = "f64" if dtype == np.float64 else "f32"
    wname = "f64" if wdtype == np.float64 else "f32"
    return Bags(np.concatenate(locs).astype(dtype), np.concatenate(ws).astype(wdtype), off, name, wname)


def rand_pairs(rng, count, mrange, d, alpha=1.0, spread=2.0):
    out = []
    for _ in range(count):
        m = int(rng.integers(*mrange))
        out.append((rng.normal(0, spread, size=(m, d)), rng.dirichlet(np.full(m, alpha))))
    return out


def gpu_pairs(d2, objs, cents, pi, pj, precision=0, group=0, flows=False, start_rule=0):
    import torch
    ctx = d2.Context(0, precision=precision, group_lanes=group, start_rule=start_rule)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    po = torch.as_tensor(np.asarray(pi, dtype=np.int64), device="cuda:0")
    pc = torch.as_tensor(np.asarray(pj, dtype=np.int64), device="cuda:0")
    dist = torch.empty(len(pi), dtype=torch.float64, device="cuda:0")
    st = torch.empty(len(pi), dtype=torch.int32, device="cuda:0")
    fl = None
    if flows:
        stride = 127
        fl = (torch.empty((len(pi), stride), dtype=torch.int32, device="cuda:0"),
              torch.empty((len(pi), stride), dtype=torch.float64, device="cuda:0"))
    rc = d2.d2_mallows_batch(ctx, ob, po, pc, dist, flows=fl, status=st)
    d2.d2_sync(ctx)
    res = dist.cpu().numpy(), st.cpu().numpy(), rc
    if flows:
        res = res + ((fl[0].cpu().numpy(), fl[1].cpu().numpy()),)
    ctx.close()
    return res


def assert_d2_close(gpu, ref, cmax=None, rel=REL):
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    floor = 1e-12 * (np.asarray(cmax) if cmax is not None else 1.0)
    err = np.abs(gpu - ref)
    bad = err > rel * np.abs(ref) + floor
    assert not bad.any(), "max rel err %.3e at %s" % (np.max(err / np.maximum(np.abs(ref), 1e-300)),
                                                       np.nonzero(bad)[0][:10])


def all_pairs(N, K):
    return np.repeat(np.arange(N), K), np.tile(np.arange(K), N)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("seed", [32, 16, 8])
def test_mallows_random_sizes(d2, oracle_mod, precision, seed):
    rng = np.random.default_rng(1000 + precision + seed)
    objs_l = rand_pairs(rng, 40, (1, 65), 5, alpha=0.5)
    cents_l = rand_pairs(rng, 9, (1, 65), 5)
    cents_l.append((cents_l[0][0], np.full(len(cents_l[0][1]), 1.0 / len(cents_l[0][1]))))
    dt = np.float64 if precision == 1 else np.float32
    objs = make_bags(objs_l, dt, dt)
    cents = make_bags(cents_l, dt, dt)
    pi, pj = all_pairs(objs.count, cents.count)
    got, st, rc = gpu_pairs(d2, objs, cents, pi, pj, precision=precision)
    assert rc == 0 and (st == 0).all()
    ref = oracle_mod.mallows_pairs(objs, cents, pi, pj, nthreads=8)
    assert_d2_close(got, ref)


def test_mallows_exhaustive_tiny(d2, oracle_mod):
    rng = np.random.default_rng(77)
    objs_l, cents_l = [], []
    for m in (1, 2, 3):
        for _ in range(30):
            objs_l.append((rng.integers(-2, 3, size=(m, 2)).astype(float),
                           rng.integers(0, 3, size=m).astype(float) + (np.arange(m) == 0)))
    for n in (1, 2, 3):
        for _ in range(4):
            cents_l.append((rng.integers(-2, 3, size=(n, 2)).astype(float), np.full(n, 1.0 / n)))
    objs = make_bags(objs_l)
    cents = make_bags(cents_l)
    pi, pj = all_pairs(objs.count, cents.count)
    for prec in (1, 2):
        o = objs if prec == 1 else make_bags(objs_l, np.float32, np.float32)
        c = cents if prec == 1 else make_bags(cents_l, np.float32, np.float32)
        got, st, rc = gpu_pairs(d2, o, c, pi, pj, precision=prec)
        assert rc == 0
        ref = oracle_mod.mallows_pairs(o, c, pi, pj, nthreads=8)
        # integer lattice points: many exact ties and degenerate bases
        assert_d2_close(got, ref, cmax=32.0)


def test_mallows_edge_cases(d2, oracle_mod):
    rng = np.random.default_rng(5)
    x = rng.normal(size=(7, 3))
    w = rng.dirichlet(np.ones(7))
    w0 = w.copy()
    w0[[1, 4]] = 0.0                       # zero-mass supports
    dup = np.repeat(x[:2], 3, axis=0)      # repeated support locations
    objs_l = [(x, w), (x, w0), (x[:1], [1.0]), (dup, np.full(6, 1 / 6)), (x, w * 1e-30),
              (rng.normal(size=(64, 3)), rng.dirichlet(np.ones(64)))]
    cents_l = [(x, w), (x[:1], [3.0]), (x[::-1], w[::-1]), (rng.normal(size=(64, 3)), np.full(64, 1 / 64))]
    for prec, dt in ((1, np.float64), (2, np.float32)):
        objs = make_bags(objs_l, dt, dt)
        cents = make_bags(cents_l, dt, dt)
        pi, pj = all_pairs(objs.count, cents.count)
        got, st, rc = gpu_pairs(d2, objs, cents, pi, pj, precision=prec)
        assert rc == 0
        ref = oracle_mod.mallows_pairs(objs, cents, pi, pj)
        assert_d2_close(got, ref, cmax=50.0)
        # identical bags: zero distance (object 0 vs centroid 0, object 2 vs centroid 1)
        assert abs(got[0]) <= 1e-12 and abs(got[2 * 4 + 1]) <= 1e-12


def test_flows_are_optimal_plans(d2, oracle_mod):
    rng = np.random.default_rng(8)
    objs = make_bags(rand_pairs(rng, 30, (1, 40), 4), np.float32, np.float32)
    cents = make_bags(rand_pairs(rng, 5, (1, 40), 4), np.float32, np.float32)
    pi, pj = all_pairs(objs.count, cents.count)
    got, st, rc, (cell, w) = gpu_pairs(d2, objs, cents, pi, pj, precision=2, flows=True)
    ref = oracle_mod.mallows_pairs(objs, cents, pi, pj)
    for t in range(len(pi)):
        x, p = oracle_mod.bag(objs, pi[t])
        y, q = oracle_mod.bag(cents, pj[t])
        m, n = len(p), len(q)
        c = cell[t]
        used = c >= 0
        assert used.sum() == m + n - 1
        a, r = c[used] >> 16, c[used] & 0xFFFF
        W = np.zeros((m, n))
        np.add.at(W, (a, r), w[t][used])
        assert (W >= 0).all()
        assert np.allclose(W.sum(1), p / p.sum(), atol=1e-12)
        assert np.allclose(W.sum(0), q / q.sum(), atol=1e-12)
        cost = float(np.sum(W * oracle_mod.cost(x, y)))
        assert cost == pytest.approx(ref[t], rel=REL)
        assert cost == pytest.approx(got[t], rel=1e-12)


def _check_assign(oracle_mod, objs, cents, labels, dist2, nthreads=8):
    lab_o, d_o, allm = oracle_mod.assign(objs, cents, nthreads=nthreads, return_all=True)
    diff = np.nonzero(labels != lab_o)[0]
    for i in diff:  # only ties may differ
        a, b = allm[i, labels[i]], allm[i, lab_o[i]]
        assert abs(a - b) <= TIE * max(a, b, 1e-300), (i, labels[i], lab_o[i], a, b)
    assert_d2_close(dist2, d_o, cmax=1.0)
    return lab_o, d_o


def gpu_assign(d2, objs, cents, omega=None, precision=0, group=0, flows=False, host=False):
    import torch
    ctx = d2.Context(0, precision=precision, group_lanes=group)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    N = objs.count
    if host:
        ob = d2.bags_from_synth(objs)
        lab = np.empty(N, dtype=np.int32)
        dist = np.empty(N)
        eps = np.empty(1)
        om = omega
    else:
        ob = d2.bags_from_synth(objs, device="cuda:0")
        lab = torch.empty(N, dtype=torch.int32, device="cuda:0")
        dist = torch.empty(N, dtype=torch.float64, device="cuda:0")
        eps = torch.empty(1, dtype=torch.float64, device="cuda:0")
        om = None if omega is None else torch.as_tensor(omega, device="cuda:0")
    fl = None
    if flows:
        stride = 127
        fl = (torch.empty((N, stride), dtype=torch.int32, device="cuda:0"),
              torch.empty((N, stride), dtype=torch.float64, device="cuda:0"))
    rc = d2.d2_assign(ctx, ob, lab, dist, omega=om, eps=eps, flows=fl)
    d2.d2_sync(ctx)
    out = dict(rc=rc, ctx=ctx, objs=ob)
    if host:
        out.update(labels=lab, dist2=dist, eps=float(eps[0]))
    else:
        out.update(labels=lab.cpu().numpy(), dist2=dist.cpu().numpy(), eps=float(eps.cpu()[0]))
    if flows:
        out["flows"] = fl
    return out


def test_assign_plain_small_full(d2, oracle_mod):
    objs, cents = synth.plain_small()
    r = gpu_assign(d2, objs, cents)
    assert r["rc"] == 0
    lab_o, d_o = _check_assign(oracle_mod, objs, cents, r["labels"], r["dist2"])
    assert r["eps"] == pytest.approx(float(np.sum(d_o)), rel=1e-9)
    r["ctx"].close()


@pytest.mark.parametrize("gen,kw", [
    (synth.image_like, dict(N=1500, K=64)),
    (synth.uneven, dict(N=1500, K=48)),
    (synth.high_dim, dict(N=60, K=24)),
])
def test_assign_fp32_configs_small(d2, oracle_mod, gen, kw):
    objs, cents = gen(**kw)
    r = gpu_assign(d2, objs, cents)
    assert r["rc"] == 0
    _check_assign(oracle_mod, objs, cents, r["labels"], r["dist2"])
    r["ctx"].close()


def test_assign_host_buffers_match_device(d2, oracle_mod):
    objs, cents = synth.image_like(N=700, K=16)
    a = gpu_assign(d2, objs, cents)
    b = gpu_assign(d2, objs, cents, host=True)
    assert (a["labels"] == b["labels"]).all()
    assert np.array_equal(a["dist2"], b["dist2"])
    a["ctx"].close()
    b["ctx"].close()


def test_assign_ties_choose_smallest_index(d2):
    objs, cents = synth.image_like(N=200, K=8)
    # centroid 5 duplicates centroid 2: 5 may never be chosen
    sel = [0, 1, 2, 3, 4, 2, 6, 7]
    c2 = cents.subset(sel)
    r = gpu_assign(d2, objs, c2)
    assert r["rc"] == 0
    assert not (r["labels"] == 5).any()
    r["ctx"].close()


def test_update_matches_oracle_from_gpu_flows(d2, oracle_mod):
    import torch
    objs, cents = synth.image_like(N=2000, K=16)
    omega = np.random.default_rng(3).uniform(0.5, 2.0, size=objs.count)
    r = gpu_assign(d2, objs, cents, omega=omega, flows=True)
    ctx, ob = r["ctx"], r["objs"]
    lab = torch.as_tensor(r["labels"], device="cuda:0")
    om = torch.as_tensor(omega, device="cuda:0")
    rc = d2.d2_update_locations(ctx, ob, lab, omega=om, flows=r["flows"])
    assert rc == 0
    new_gpu, _, _ = d2.d2_get_centroids(ctx, objs.dim)
    cell, w = (t.cpu().numpy() for t in r["flows"])
    used = cell >= 0
    fo = np.nonzero(used)[0]
    fa, fr = cell[used] >> 16, cell[used] & 0xFFFF
    new_o = oracle_mod.update_locations(objs, omega, r["labels"], fo, fa, fr, w[used], cents)
    new_o = new_o.astype(np.float32).astype(np.float64)   # centroids stored in their FP32 type
    assert np.allclose(new_gpu, new_o, rtol=1e-6, atol=1e-6)
    exact = np.abs(new_gpu - new_o) <= 1e-12 * np.maximum(np.abs(new_o), 1e-300)
    assert exact.mean() > 0.999
    # against the oracle's own optimal flows
    fo2, fa2, fr2, fw2 = oracle_mod.assigned_flows(objs, cents, r["labels"])
    new_o2 = oracle_mod.update_locations(objs, omega, r["labels"], fo2, fa2, fr2, fw2, cents)
    assert np.allclose(new_gpu, new_o2, rtol=1e-5, atol=1e-5)
    # re-solving the flows inside the call gives the same result
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    d2.d2_update_locations(ctx, ob, lab, omega=om, flows=None)
    new_gpu2, _, _ = d2.d2_get_centroids(ctx, objs.dim)
    assert np.array_equal(new_gpu, new_gpu2)
    ctx.close()


def test_cluster_level_matches_oracle(d2, oracle_mod):
    import torch
    objs, cents = synth.image_like(N=900, K=6, seed=4242)
    omega = np.random.default_rng(9).uniform(0.5, 1.5, size=objs.count)
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    K, tau, iters = 6, 200, 3
    out_loc = torch.empty((cents.loc.shape[0], objs.dim), dtype=torch.float64, device="cuda:0")
    out_w = torch.empty(K, dtype=torch.float64, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    rc = d2.d2_cluster_level(ctx, ob, K, tau, iters, out_loc, out_w, lab,
                             omega=torch.as_tensor(omega, device="cuda:0"))
    d2.d2_sync(ctx)
    assert rc == 0
    cl, cw, lo = oracle_mod.cluster_level(objs, omega, cents, K, tau, iters, loc_round=np.float32,
                                          nthreads=8)
    assert (lab.cpu().numpy() == lo).all()
    assert np.allclose(out_loc.cpu().numpy(), cl, rtol=1e-6, atol=1e-6)
    assert np.allclose(out_w.cpu().numpy(), cw, rtol=1e-12)
    assert out_w.sum().item() == pytest.approx(omega.sum(), rel=1e-12)
    ctx.close()


def test_invalid_inputs_are_reported(d2):
    objs, cents = synth.image_like(N=50, K=4)
    bad = Bags(objs.loc.copy(), objs.w.copy(), objs.off.copy(), "f32", "f32")
    bad.w[bad.off[3]] = -1.0
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents))
    lab = np.empty(bad.count, dtype=np.int32)
    dist = np.empty(bad.count)
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign(ctx, d2.bags_from_synth(bad), lab, dist)
    assert e.value.code == d2.D2_EINVAL
    big = synth.uneven(N=20, K=2)[0]
    sizes = np.full(3, 65)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    over = Bags(np.zeros((off[-1], cents.dim), np.float32), np.ones(off[-1], np.float32), off, "f32", "f32")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign(ctx, d2.bags_from_synth(over), np.empty(3, np.int32), np.empty(3))
    assert e.value.code == d2.D2_EUNSUPPORTED
    del big
    ctx.close()


def test_binned_autotuned_assign_is_bitwise_unbinned(d2, oracle_mod):
    """Large ragged batches are split into bins by tree size and each bin's
    launch shape is autotuned; per-object results must not change (labels
    exactly; D^2 to rounding, since a tuned cold-start rule may reach another
    optimal basis of a degenerate pair)."""
    objs, cents = synth.uneven(N=20000, K=32)        # bins: m+32 <= 64 and <= 96
    big = gpu_assign(d2, objs, cents)                 # binned (>= 4096 objects), tuned
    head = objs.subset(np.arange(3000))
    small = gpu_assign(d2, head, cents)               # one unbinned launch
    assert np.array_equal(big["labels"][:3000], small["labels"])
    assert np.allclose(big["dist2"][:3000], small["dist2"], rtol=1e-12, atol=0)
    idx = np.concatenate([np.arange(0, 20000, 97), np.argsort(-objs.sizes())[:5]])
    sub = objs.subset(idx)
    _check_assign(oracle_mod, sub, cents, big["labels"][idx], big["dist2"][idx])
    big["ctx"].close()
    small["ctx"].close()


# ---- cold-start rules on trees of more than one node per lane (m+n > 32) ----

@pytest.mark.parametrize("rule", ["ranked", "vogel"])
def test_mallows_start_rules_large(d2, oracle_mod, rule):
    rng = np.random.default_rng(77 if rule == "vogel" else 78)
    objs_l = rand_pairs(rng, 24, (20, 65), 6, alpha=0.7)
    cents_l = rand_pairs(rng, 6, (20, 65), 6)
    objs = make_bags(objs_l, np.float32, np.float32)
    cents = make_bags(cents_l, np.float32, np.float32)
    pi, pj = all_pairs(objs.count, cents.count)
    r = d2.D2_START_VOGEL if rule == "vogel" else d2.D2_START_RANKED
    got, st, rc, (cell, w) = gpu_pairs(d2, objs, cents, pi, pj, precision=2, flows=True,
                                       start_rule=r)
    assert rc == 0 and (st == 0).all()
    ref = oracle_mod.mallows_pairs(objs, cents, pi, pj, nthreads=8)
    assert_d2_close(got, ref)
    _check_plans(oracle_mod, objs, cents, pi, pj, cell, w, ref)


def _lattice_pairs(rng, count, mrange, d):
    """Integer-lattice supports (many equal costs), weights with equal, zero
    and repeated entries (many equal partial sums and degenerate bases)."""
    out = []
    for t in range(count):
        m = int(rng.integers(*mrange))
        x = rng.integers(0, 3, size=(m, d)).astype(np.float64)
        kind = t % 3
        if kind == 0:
            w = np.full(m, 1.0 / m)
        elif kind == 1:
            w = rng.integers(0, 3, size=m).astype(np.float64)
            if w.sum() == 0:
                w[0] = 1.0
        else:
            w = np.repeat(rng.dirichlet(np.ones((m + 1) // 2)), 2)[:m]
        out.append((x, w))
    return out


def test_vogel_degenerate_lattices(d2, oracle_mod):
    rng = np.random.default_rng(79)
    objs = make_bags(_lattice_pairs(rng, 18, (30, 65), 2), np.float32, np.float32)
    cents = make_bags(_lattice_pairs(rng, 6, (30, 65), 2), np.float32, np.float32)
    pi, pj = all_pairs(objs.count, cents.count)
    got, st, rc, (cell, w) = gpu_pairs(d2, objs, cents, pi, pj, precision=2, flows=True,
                                       start_rule=d2.D2_START_VOGEL)
    assert rc == 0 and (st == 0).all()
    ref = oracle_mod.mallows_pairs(objs, cents, pi, pj, nthreads=8)
    assert_d2_close(got, ref)
    _check_plans(oracle_mod, objs, cents, pi, pj, cell, w, ref)


def _check_plans(oracle_mod, objs, cents, pi, pj, cell, w, ref):
    """Each returned plan meets both marginals within 1e-12 and costs D^2."""
    for t in range(len(pi)):
        x, p = oracle_mod.bag(objs, int(pi[t]))
        y, q = oracle_mod.bag(cents, int(pj[t]))
        p = p / p.sum()
        q = q / q.sum()
        ok = cell[t] >= 0
        a = cell[t][ok] >> 16
        r = cell[t][ok] & 0xFFFF
        f = w[t][ok]
        assert (f >= -1e-15).all()
        assert np.abs(np.bincount(a, weights=f, minlength=len(p)) - p).max() <= 1e-12
        assert np.abs(np.bincount(r, weights=f, minlength=len(q)) - q).max() <= 1e-12
        c = np.sum((x[a] - y[r]) ** 2, axis=1)
        assert abs(float(np.dot(f, c)) - ref[t]) <= 1e-9 * max(ref[t], 1e-12)


def test_assign_start_rules_agree(d2, oracle_mod):
    """The screen's cold start changes the path, not the answer."""
    import torch
    objs, cents = synth.uneven(N=3000, K=24, seed=1203)
    out = {}
    for rule in (d2.D2_START_RANKED, d2.D2_START_VOGEL):
        ctx = d2.Context(0, start_rule=rule)
        d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
        ob = d2.bags_from_synth(objs, device="cuda:0")
        lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
        dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
        assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
        d2.d2_sync(ctx)
        out[rule] = (lab.cpu().numpy(), dist.cpu().numpy())
        ctx.close()
    (la, da), (lb, db) = out[d2.D2_START_RANKED], out[d2.D2_START_VOGEL]
    for i in np.nonzero(la != lb)[0]:
        assert abs(da[i] - db[i]) <= TIE * max(da[i], db[i])
    assert np.allclose(da, db, rtol=1e-12, atol=0)
    idx = np.sort(np.random.default_rng(3).choice(objs.count, size=40, replace=False))
    big = np.argsort(-objs.sizes(), kind="stable")[:8]
    idx = np.unique(np.concatenate([idx, big]))
    lo, do_ = oracle_mod.assign(objs.subset(idx), cents, nthreads=8)
    assert_d2_close(db[idx], do_)
