"""One segment of the benchmark's level step at its full shape (Alg. 3 with
Alg. 2 inside the segment): the first 5,000 bags of the image-like workload
against K = 64 centroids of 16 supports, tau = 5,000, every pair certified
(D2_CERTIFY_ALL), rounds after the first warm-started and replayed from a
CUDA graph.

Round 1 is unique (continuous data: one optimal plan per pair with
probability 1), so it is compared with the oracle in full: labels bit-exact
except ties within 1e-9, D^2 within 1e-6, and the location update equal to
the oracle's update from the GPU's own flows.  Two rounds of the level are
compared with the oracle's level loop.  Ten rounds: the invariants (summed
omega, valid labels, member weights) and bitwise repeatability; the plans of
later rounds need not be unique (coincident centroid supports), so their
trajectory is not compared."""
import os

import numpy as np
import pytest

from paper_1302_0435_gb300 import synth

pytestmark = pytest.mark.gpu

TIE = 1e-9
CORES = os.cpu_count() or 1
K, TAU, NSEG = 64, 5000, 5000


@pytest.fixture(scope="module")
def d2():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_0435_gb300 import build, d2 as mod
    build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def segment():
    objs, cents = synth.image_like(N=200_000, K=K)  # the benchmark's workload
    return objs.subset(np.arange(NSEG)), cents


def _ctx(d2, cents):
    ctx = d2.Context(0, certify=d2.D2_CERTIFY_ALL)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    return ctx


def test_round_one_matches_oracle(d2, oracle_mod, segment):
    import torch
    objs, cents = segment
    ctx = _ctx(d2, cents)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(NSEG, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(NSEG, dtype=torch.float64, device="cuda:0")
    stride = 16 + 16 - 1
    fl = (torch.empty((NSEG, stride), dtype=torch.int32, device="cuda:0"),
          torch.empty((NSEG, stride), dtype=torch.float64, device="cuda:0"))
    assert d2.d2_assign(ctx, ob, lab, dist, flows=fl) == d2.D2_OK
    d2.d2_sync(ctx)
    lg, dg = lab.cpu().numpy(), dist.cpu().numpy()
    lab_o, d_o, allm = oracle_mod.assign(objs, cents, nthreads=CORES, return_all=True)
    for i in np.nonzero(lg != lab_o)[0]:
        a, b = allm[i, lg[i]], allm[i, lab_o[i]]
        assert abs(a - b) <= TIE * max(a, b), (i, lg[i], lab_o[i])
    assert np.all(np.abs(dg - d_o) <= 1e-6 * d_o + 1e-12)
    # the update from the GPU's own flows, against the oracle's update
    assert d2.d2_update_locations(ctx, ob, lab, flows=fl) == d2.D2_OK
    new_gpu, _, _ = d2.d2_get_centroids(ctx, objs.dim)
    cell, w = (t.cpu().numpy() for t in fl)
    used = cell >= 0
    fo = np.nonzero(used)[0]
    new_o = oracle_mod.update_locations(objs, None, lg, fo, cell[used] >> 16, cell[used] & 0xFFFF,
                                        w[used], cents)
    new_o = new_o.astype(np.float32).astype(np.float64)  # stored in the centroids' FP32 type
    assert np.allclose(new_gpu, new_o, rtol=1e-6, atol=1e-6)
    assert (np.abs(new_gpu - new_o) <= 1e-12 * np.maximum(np.abs(new_o), 1e-300)).mean() > 0.999
    ctx.close()


def _level(d2, ctx, objs, iters):
    import torch
    T = 64 * 16
    out_loc = torch.empty((T, objs.dim), dtype=torch.float64, device="cuda:0")
    out_w = torch.empty(K, dtype=torch.float64, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    rc = d2.d2_cluster_level(ctx, d2.bags_from_synth(objs, device="cuda:0"), K, TAU, iters,
                             out_loc, out_w, lab)
    d2.d2_sync(ctx)
    assert rc == d2.D2_OK
    return out_loc.cpu().numpy(), out_w.cpu().numpy(), lab.cpu().numpy()


def test_two_rounds_match_oracle_level(d2, oracle_mod, segment):
    """Round 2 starts from round 1's centroids; its plans need not be unique
    any more, so its update is compared with the oracle's update from the
    GPU's own round-2 flows, and its labels and D^2 with the oracle's
    assignment to the same centroids.  The level loop (warm bases, graph
    replay) gives the same labels as the oracle's level loop."""
    import torch
    objs, cents = segment
    ctx = _ctx(d2, cents)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(NSEG, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(NSEG, dtype=torch.float64, device="cuda:0")
    stride = 16 + 16 - 1
    fl = (torch.empty((NSEG, stride), dtype=torch.int32, device="cuda:0"),
          torch.empty((NSEG, stride), dtype=torch.float64, device="cuda:0"))
    d2.d2_assign(ctx, ob, lab, dist, flows=fl)
    d2.d2_update_locations(ctx, ob, lab, flows=fl)            # round 1
    c1, w1, off1 = d2.d2_get_centroids(ctx, objs.dim)
    d2.d2_assign(ctx, ob, lab, dist, flows=fl)                # round 2
    d2.d2_sync(ctx)
    cents1 = synth.Bags(c1, w1, off1, "f64", "f64")
    lg, dg = lab.cpu().numpy(), dist.cpu().numpy()
    lab_o, d_o, allm = oracle_mod.assign(objs, cents1, nthreads=CORES, return_all=True)
    for i in np.nonzero(lg != lab_o)[0]:
        a, b = allm[i, lg[i]], allm[i, lab_o[i]]
        assert abs(a - b) <= TIE * max(a, b), (i, lg[i], lab_o[i])
    assert np.all(np.abs(dg - d_o) <= 1e-6 * d_o + 1e-12)
    d2.d2_update_locations(ctx, ob, lab, flows=fl)
    c2, _, _ = d2.d2_get_centroids(ctx, objs.dim)
    cell, w = (t.cpu().numpy() for t in fl)
    used = cell >= 0
    new_o = oracle_mod.update_locations(objs, None, lg, np.nonzero(used)[0], cell[used] >> 16,
                                        cell[used] & 0xFFFF, w[used], cents1)
    new_o = new_o.astype(np.float32).astype(np.float64)
    assert np.allclose(c2, new_o, rtol=1e-6, atol=1e-6)
    ctx.close()
    # the level loop's labels after two rounds
    ctx = _ctx(d2, cents)
    _, cw, lab2 = _level(d2, ctx, objs, 2)
    ctx.close()
    _, cw_o, lab_o2 = oracle_mod.cluster_level(objs, None, cents, K, TAU, 2, loc_round=np.float32,
                                               nthreads=CORES)
    assert np.array_equal(lab2, lab_o2)
    assert np.allclose(cw, cw_o, rtol=1e-12)


def test_ten_rounds_invariants_and_repeatability(d2, segment):
    objs, cents = segment
    ctx = _ctx(d2, cents)
    a = _level(d2, ctx, objs, 10)
    b = _level(d2, ctx, objs, 10)
    ctx.close()
    loc, cw, lab = a
    assert lab.min() >= 0 and lab.max() < K
    assert cw.sum() == pytest.approx(NSEG, rel=1e-12)  # summed omega (all ones) conserved
    assert np.array_equal(np.bincount(lab, minlength=K).astype(np.float64), cw)
    assert np.isfinite(loc).all()
    for x, y in zip(a, b):  # the graph-replayed warm rounds are deterministic
        assert np.array_equal(x, y)


def test_tree_only_warm_store_is_bitwise_the_full_one(d2, segment):
    """A warm-store budget that holds the bases' trees but not their flows
    (3 of 11 bytes per node) recomputes the flows from the marginals on
    reload: the level's centroids, weights and labels are bitwise those of
    the full store."""
    objs, cents = segment
    out = {}
    # full store: 5,000 x 64 pairs x 32 nodes x 11 B = 113 MB; trees 31 MB
    for mib in (0, 64):
        ctx = d2.Context(0, warm_budget_mib=mib, no_prune=True)
        d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
        out[mib] = _level(d2, ctx, objs, 6)
        ctx.close()
    for a, b in zip(out[0], out[64]):
        assert np.array_equal(a, b)
