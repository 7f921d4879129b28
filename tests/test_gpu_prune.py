"""Pairs that cannot be an object's argmin are skipped (d2_config.no_prune
= 0, the default for assignments without a certificate of every pair):
D^2 >= ||mean_P - mean_Q||^2 and D^2 <= ||mean_P - mean_Q||^2 + var_P +
var_Q, so a centroid whose lower bound exceeds the object's best upper bound
is never solved.  Labels and distances must be bitwise those of solving
every pair, and the oracle's; far fewer pairs are solved."""
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


def _assign(d2, objs, cents, **kw):
    import torch
    ctx = d2.Context(0, **kw)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    d2.d2_assign(ctx, ob, lab, dist)  # tuned shapes settle
    d2.d2_sync(ctx)
    s0 = d2.d2_get_stats()
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    d2.d2_sync(ctx)
    s1 = d2.d2_get_stats()
    ctx.close()
    return lab.cpu().numpy(), dist.cpu().numpy(), s1["pairs_screened"] - s0["pairs_screened"]


@pytest.mark.parametrize("law", ["image_like", "uneven", "serving", "high_dim"])
def test_pruned_assign_is_bitwise_the_full_one(d2, oracle_mod, law):
    if law == "image_like":
        objs, cents = synth.image_like(N=20000, K=64, seed=701)
    elif law == "uneven":
        objs, cents = synth.uneven(N=20000, K=128, seed=702)
    elif law == "serving":
        cents, means = synth.serving_centroids(K=1024, seed=703)
        objs = synth.serving_request(np.random.default_rng(704), means, size=2000)
    else:
        objs, cents = synth.high_dim(N=600, K=64, seed=705)
    lp, dp, sp = _assign(d2, objs, cents)
    lf, df, sf = _assign(d2, objs, cents, no_prune=True)
    assert np.array_equal(lp, lf)
    if law == "image_like":  # one bin, no autotuning: the same launches solve the argmin pairs
        assert np.array_equal(dp, df)
    else:  # each context tunes its own cold start: equal optima, maybe another optimal basis
        assert np.allclose(dp, df, rtol=1e-12, atol=0)
    assert sf == objs.count * cents.count
    # the clustered laws prune most pairs; the high-dimension descriptors all
    # lie close together (no cluster structure), so their bounds prune none
    assert sp <= sf and (law == "high_dim" or sp < 0.2 * sf)
    print("%s: %d of %d pairs solved with pruning" % (law, sp, sf))
    # and the oracle on a sample
    idx = np.sort(np.random.default_rng(7).choice(objs.count, size=min(300, objs.count),
                                                  replace=False))
    sub = objs.subset(idx)
    lab_o, d_o, allm = oracle_mod.assign(sub, cents, nthreads=8, return_all=True)
    for k in np.nonzero(lp[idx] != lab_o)[0]:
        a, b = allm[k, lp[idx][k]], allm[k, lab_o[k]]
        assert abs(a - b) <= TIE * max(a, b)
    assert np.all(np.abs(dp[idx] - d_o) <= 1e-6 * d_o + 1e-12)


def test_pruned_level_matches_oracle(d2, oracle_mod):
    """The level loop with pruning and warm bases: a pair skipped in one
    round has no saved basis and restarts cold when it is solved again."""
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
    s0 = d2.d2_get_stats()
    rc = d2.d2_cluster_level(ctx, ob, K, tau, iters, out_loc, out_w, lab,
                             omega=torch.as_tensor(omega, device="cuda:0"))
    d2.d2_sync(ctx)
    s1 = d2.d2_get_stats()
    assert rc == 0
    cl, cw, lo = oracle_mod.cluster_level(objs, omega, cents, K, tau, iters, loc_round=np.float32,
                                          nthreads=8)
    assert (lab.cpu().numpy() == lo).all()
    assert np.allclose(out_loc.cpu().numpy(), cl, rtol=1e-6, atol=1e-6)
    assert np.allclose(out_w.cpu().numpy(), cw, rtol=1e-12)
    ctx.close()
