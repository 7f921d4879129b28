"""Symbol ground costs (the sequence variant of Eq. (D2opt)) on the GPU
against the oracle's table variant."""
import time

import numpy as np
import pytest

from paper_1302_0435_gb300 import synth

pytestmark = pytest.mark.gpu
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


def _ctx(d2, cents, table):
    ctx = d2.Context(0)
    d2.d2_set_cost_table(ctx, table)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    return ctx


def test_table_assign_matches_oracle(d2, oracle_mod):
    import torch
    objs, cents, table = synth.sequence_like(N=400, K=12, seed=61)
    ctx = _ctx(d2, cents, table)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    d2.d2_sync(ctx)
    ctx.close()
    lab_o, d_o, allm = oracle_mod.assign_table(objs, cents, table)
    lg, dg = lab.cpu().numpy(), dist.cpu().numpy()
    for i in np.nonzero(lg != lab_o)[0]:
        a, b = allm[i, lg[i]], allm[i, lab_o[i]]
        assert abs(a - b) <= TIE * max(a, b)
    assert (np.abs(dg - d_o) <= 1e-6 * d_o + 1e-12).all()


def test_table_plans_and_cost_matrix(d2, oracle_mod):
    import torch
    objs, cents, table = synth.sequence_like(N=60, K=5, seed=62)
    ctx = _ctx(d2, cents, table)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    pi = np.repeat(np.arange(objs.count), cents.count)
    pj = np.tile(np.arange(cents.count), objs.count)
    dist = torch.empty(len(pi), dtype=torch.float64, device="cuda:0")
    st = torch.empty(len(pi), dtype=torch.int32, device="cuda:0")
    fl = (torch.empty((len(pi), 63), dtype=torch.int32, device="cuda:0"),
          torch.empty((len(pi), 63), dtype=torch.float64, device="cuda:0"))
    rc = d2.d2_mallows_batch(ctx, ob, torch.as_tensor(pi, device="cuda:0"),
                             torch.as_tensor(pj, device="cuda:0"), dist, flows=fl, status=st)
    d2.d2_sync(ctx)  # device outputs: the call returned without waiting
    assert rc == d2.D2_OK and (st.cpu().numpy() == 0).all()
    cell, w = fl[0].cpu().numpy(), fl[1].cpu().numpy()
    got = dist.cpu().numpy()
    for t in range(len(pi)):
        xs, p = oracle_mod.bag(objs, int(pi[t]))
        ys, q = oracle_mod.bag(cents, int(pj[t]))
        ref = oracle_mod.mallows_table(xs, p, ys, q, table)[0]
        assert abs(got[t] - ref) <= 1e-6 * ref + 1e-12
        ok = cell[t] >= 0
        a, r, f = cell[t][ok] >> 16, cell[t][ok] & 0xFFFF, w[t][ok]
        assert np.abs(np.bincount(a, weights=f, minlength=len(p)) - p / p.sum()).max() <= 1e-12
        assert np.abs(np.bincount(r, weights=f, minlength=len(q)) - q / q.sum()).max() <= 1e-12
        c = table[xs.ravel().astype(int)[a], ys.ravel().astype(int)[r]]
        assert abs(float(np.dot(f, c)) - ref) <= 1e-9 * max(ref, 1e-12)
    # the cost matrix is the table read at the symbol pairs
    xs, _ = oracle_mod.bag(objs, 3)
    ys, _ = oracle_mod.bag(cents, 2)
    C = d2.d2_cost_matrix(ctx, ob, 3, 2, d2.D2_PREC_FP64, len(xs), len(ys))
    assert np.array_equal(C, table[np.ix_(xs.ravel().astype(int), ys.ravel().astype(int))])
    ctx.close()


def test_discrete_metric_gives_total_variation(d2):
    import torch
    objs, cents, _ = synth.sequence_like(N=200, K=6, seed=63)
    table = 1.0 - np.eye(20)
    ctx = _ctx(d2, cents, table)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    pi = np.repeat(np.arange(objs.count), cents.count)
    pj = np.tile(np.arange(cents.count), objs.count)
    dist = torch.empty(len(pi), dtype=torch.float64, device="cuda:0")
    assert d2.d2_mallows_batch(ctx, ob, torch.as_tensor(pi, device="cuda:0"),
                               torch.as_tensor(pj, device="cuda:0"), dist) == d2.D2_OK
    d2.d2_sync(ctx)
    ctx.close()

    def dense(b, i):
        lo, hi = int(b.off[i]), int(b.off[i + 1])
        v = np.zeros(20)
        np.add.at(v, b.loc[lo:hi, 0].astype(int), b.w[lo:hi].astype(np.float64))
        return v / v.sum()
    tv = np.array([1.0 - np.minimum(dense(objs, i), dense(cents, j)).sum() for i, j in zip(pi, pj)])
    assert np.abs(dist.cpu().numpy() - tv).max() <= 1e-9


def test_table_errors(d2):
    import torch
    objs, cents, table = synth.sequence_like(N=20, K=3, seed=64)
    ctx = d2.Context(0)
    with pytest.raises(d2.D2Error) as e:
        d2.d2_set_cost_table(ctx, -table)          # negative costs
    assert e.value.code == d2.D2_EINVAL
    ctx2 = _ctx(d2, cents, table)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_update_locations(ctx2, ob, lab)      # symbolic supports are not moved
    assert e.value.code == d2.D2_EUNSUPPORTED
    bad = synth._pack(np.diff(objs.off).astype(np.int64), objs.loc + np.float32(0.5), objs.w,
                      "f32", "f32")                # not integer symbol ids
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    # device outputs: the call returns without waiting, d2_sync reports
    d2.d2_assign(ctx2, d2.bags_from_synth(bad, device="cuda:0"), lab, dist)
    with pytest.raises(d2.D2Error) as e:
        d2.d2_sync(ctx2)
    assert e.value.code == d2.D2_EINVAL
    # host outputs: the call waits and reports it itself
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign(ctx2, d2.bags_from_synth(bad), np.empty(objs.count, np.int32),
                     np.empty(objs.count))
    assert e.value.code == d2.D2_EINVAL
    ctx.close()
    ctx2.close()


def test_sequence_like_full_size(d2, oracle_mod):
    """100,000 sequence histograms against 64 centroids, sampled parity."""
    import torch
    objs, cents, table = synth.sequence_like()
    ctx = _ctx(d2, cents, table)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    d2.d2_assign(ctx, ob, lab, dist)
    d2.d2_sync(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    d2.d2_sync(ctx)
    dt = time.perf_counter() - t0
    ctx.close()
    print("sequence-like assign: %.3g pairs/s" % (objs.count * cents.count / dt))
    idx = np.sort(np.random.default_rng(7).choice(objs.count, size=60, replace=False))
    sub = objs.subset(idx)
    lab_o, d_o, allm = oracle_mod.assign_table(sub, cents, table)
    lg, dg = lab.cpu().numpy()[idx], dist.cpu().numpy()[idx]
    for k in np.nonzero(lg != lab_o)[0]:
        a, b = allm[k, lg[k]], allm[k, lab_o[k]]
        assert abs(a - b) <= TIE * max(a, b)
    assert (np.abs(dg - d_o) <= 1e-6 * d_o + 1e-12).all()
