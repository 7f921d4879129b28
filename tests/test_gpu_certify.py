"""FP64 certification of every pair (D2_CERTIFY_ALL, d2_mallows_all).

Every (object, centroid) D^2 the call returns must match the FP64 oracle's
Mallows distance within 1e-6 relative (absolute floor 1e-12 * the largest
ground cost, for D^2 ~ 0); labels are bit-exact except where the oracle's
own values tie within 1e-9 relative.  The workload laws run at sizes the
oracle finishes in seconds but that span many launch tiles, several tree
bins and a ragged tail.
"""
import os

import numpy as np
import pytest

from paper_1302_0435_gb300 import synth
from paper_1302_0435_gb300.synth import Bags

pytestmark = pytest.mark.gpu

REL = 1e-6
TIE = 1e-9
CORES = os.cpu_count() or 1


@pytest.fixture(scope="module")
def d2():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_0435_gb300 import build, d2 as mod
    build.build()
    mod.load()
    return mod


def _cmax(objs, cents):
    """Largest ground cost over all pairs (the absolute floor's scale)."""
    x = objs.loc.astype(np.float64)   # for BF16 data: the BF16 values
    y = cents.loc.astype(np.float64)
    nx = (x * x).sum(1)
    ny = (y * y).sum(1)
    return float(nx.max() + ny.max() + 2.0 * np.sqrt(nx.max() * ny.max()))


def _all_pairs_gpu(d2, objs, cents, **ctx_kw):
    import torch
    ctx = d2.Context(0, **ctx_kw)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    N, K = objs.count, cents.count
    allg = torch.empty((N, K), dtype=torch.float64, device="cuda:0")
    lab = torch.empty(N, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(N, dtype=torch.float64, device="cuda:0")
    s0 = d2.d2_get_stats()
    rc = d2.d2_mallows_all(ctx, ob, allg, lab, dist)
    d2.d2_sync(ctx)
    s1 = d2.d2_get_stats()
    ctx.close()
    assert rc == d2.D2_OK
    st = {k: s1[k] - s0[k] for k in s0}
    return allg.cpu().numpy(), lab.cpu().numpy(), dist.cpu().numpy(), st


def _check_all(oracle_mod, objs, cents, allg, lab, dist):
    N, K = objs.count, cents.count
    pi = np.repeat(np.arange(N), K)
    pj = np.tile(np.arange(K), N)
    ref = oracle_mod.mallows_pairs(objs, cents, pi, pj, nthreads=CORES).reshape(N, K)
    floor = 1e-12 * _cmax(objs, cents)
    err = np.abs(allg - ref)
    bad = ~(err <= REL * ref + floor)
    assert not bad.any(), ("pairs off", int(bad.sum()), float(np.nanmax(err / np.maximum(ref, 1e-300))))
    lab_o = np.argmin(ref, axis=1)
    for i in np.nonzero(lab != lab_o)[0]:
        a, b = ref[i, lab[i]], ref[i, lab_o[i]]
        assert abs(a - b) <= TIE * max(a, b), (i, lab[i], lab_o[i], a, b)
    # the argmin's value is the returned pair value of that centroid
    assert np.array_equal(dist, allg[np.arange(N), lab])
    return ref


@pytest.mark.parametrize("law", ["image_like", "uneven", "serving", "plain_small"])
def test_mallows_all_matches_oracle(d2, oracle_mod, law):
    if law == "image_like":
        objs, cents = synth.image_like(N=1500, K=64, seed=501)
    elif law == "uneven":
        objs, cents = synth.uneven(N=1200, K=32, seed=502)   # tree bins of 2 and 3 nodes per lane
    elif law == "serving":
        cents, means = synth.serving_centroids(K=48, seed=503)
        objs = synth.serving_request(np.random.default_rng(504), means, size=300)
    else:
        objs, cents = synth.plain_small(N=1000, K=8)          # FP64 data: solved in FP64 throughout
    allg, lab, dist, st = _all_pairs_gpu(d2, objs, cents)
    _check_all(oracle_mod, objs, cents, allg, lab, dist)
    if law != "plain_small":
        pairs = objs.count * cents.count
        assert st["pairs_screened"] == pairs
        # the certificate clears almost every pair; the rest were solved exactly
        assert st["pairs_certified"] >= 0.99 * pairs, st
        assert st["pairs_exact"] >= pairs - st["pairs_certified"], st


def test_mallows_all_tensor_core_tiles(d2, oracle_mod):
    """BF16 d=128 descriptors: the screen's FP32 tiles come from the tensor
    cores; the certificate's bound carries their error term."""
    objs, cents = synth.high_dim(N=40, K=24, seed=505)
    allg, lab, dist, st = _all_pairs_gpu(d2, objs, cents, cost_tc=2)
    _check_all(oracle_mod, objs, cents, allg, lab, dist)
    assert st["pairs_screened"] == objs.count * cents.count


def test_mallows_all_degenerate_lattice(d2, oracle_mod):
    """Integer lattice supports and weights in small integer ratios: many
    optimal plans and nonbasic cells with zero reduced cost, so the
    certificate must re-price cells in FP64 and still accept optimal bases."""
    rng = np.random.default_rng(506)

    def bags(count, lo, hi):
        locs, ws, sizes = [], [], []
        for _ in range(count):
            m = int(rng.integers(lo, hi + 1))
            locs.append(rng.integers(0, 3, size=(m, 3)).astype(np.float32))
            ws.append(rng.integers(1, 4, size=m).astype(np.float32))
            sizes.append(m)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        return Bags(np.concatenate(locs), np.concatenate(ws), off, "f32", "f32")

    objs = bags(400, 2, 12)
    cents = bags(16, 2, 16)
    allg, lab, dist, st = _all_pairs_gpu(d2, objs, cents)
    _check_all(oracle_mod, objs, cents, allg, lab, dist)
    assert st["cells_checked"] > 0, st


def test_assign_certify_all_agrees_with_default(d2):
    """d2_assign with D2_CERTIFY_ALL gives the labels of the default mode
    (both are the exact argmin) and D^2 within the certificate's 2^-24."""
    import torch
    objs, cents = synth.image_like(N=6000, K=64, seed=507)
    out = []
    for cert in (d2.D2_CERTIFY_CANDIDATES, d2.D2_CERTIFY_ALL):
        ctx = d2.Context(0, certify=cert)
        d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
        ob = d2.bags_from_synth(objs, device="cuda:0")
        lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
        dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
        assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
        d2.d2_sync(ctx)
        out.append((lab.cpu().numpy(), dist.cpu().numpy()))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.all(np.abs(out[1][1] - out[0][1]) <= 2.0 ** -23 * out[0][1] + 1e-12)


def test_cluster_level_certify_all_matches_oracle(d2, oracle_mod):
    import torch
    objs, cents = synth.image_like(N=900, K=6, seed=4242)
    omega = np.random.default_rng(9).uniform(0.5, 1.5, size=objs.count)
    ctx = d2.Context(0, certify=d2.D2_CERTIFY_ALL)
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
    scr = s1["pairs_screened"] - s0["pairs_screened"]
    cert = s1["pairs_certified"] - s0["pairs_certified"]
    assert scr > 0 and cert >= 0.99 * scr
    ctx.close()
