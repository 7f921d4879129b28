"""Parity at the workloads' full sizes, in the launch configurations the
benchmark and the library use, checked on sampled objects the FP64 oracle
recomputes one by one (labels bit-exact except ties within 1e-9 relative,
D^2 within 1e-6 relative), plus invariants that hold at any size."""
import os

import numpy as np
import pytest

from paper_1302_0435_gb300 import synth

pytestmark = pytest.mark.gpu

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


def _assign_device(d2, objs, cents):
    import torch
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    rc = d2.d2_assign(ctx, ob, lab, dist)
    d2.d2_sync(ctx)
    ctx.close()
    assert rc == d2.D2_OK
    return lab.cpu().numpy(), dist.cpu().numpy()


def _check_sample(oracle_mod, objs, cents, lab, dist, idx):
    sub = objs.subset(idx)
    lab_o, d_o, allm = oracle_mod.assign(sub, cents, nthreads=CORES, return_all=True)
    lg, dg = lab[idx], dist[idx]
    for k in np.nonzero(lg != lab_o)[0]:
        a, b = allm[k, lg[k]], allm[k, lab_o[k]]
        assert abs(a - b) <= TIE * max(a, b), (idx[k], lg[k], lab_o[k], a, b)
    err = np.abs(dg - d_o)
    assert (err <= 1e-6 * d_o + 1e-12).all(), float(np.max(err / np.maximum(d_o, 1e-300)))


def _sample(rng, objs, count, heavy=0):
    """Random objects plus the `heavy` largest ones (ragged tail)."""
    idx = rng.choice(objs.count, size=count, replace=False)
    if heavy:
        big = np.argsort(-objs.sizes(), kind="stable")[:heavy]
        idx = np.unique(np.concatenate([idx, big]))
    return np.sort(idx)


def test_image_like_full_assign(d2, oracle_mod):
    objs, cents = synth.image_like()                  # 200,000 x 64
    lab, dist = _assign_device(d2, objs, cents)
    assert ((lab >= 0) & (lab < cents.count)).all()
    _check_sample(oracle_mod, objs, cents, lab, dist, _sample(np.random.default_rng(1), objs, 1500, 20))


def test_uneven_full_assign(d2, oracle_mod):
    objs, cents = synth.uneven()                      # 1,000,000 x 256, m ~ m^-2 on 2..64
    lab, dist = _assign_device(d2, objs, cents)
    assert ((lab >= 0) & (lab < cents.count)).all()
    _check_sample(oracle_mod, objs, cents, lab, dist, _sample(np.random.default_rng(2), objs, 400, 12))


def test_high_dim_full_size(d2, oracle_mod):
    objs, cents = synth.high_dim()                    # 100,000 BF16 bags, d=128, K=512 of 64 supports
    lab, dist = _assign_device(d2, objs, cents)       # tensor-core tiles, Vogel start
    assert ((lab >= 0) & (lab < cents.count)).all()
    _check_sample(oracle_mod, objs, cents, lab, dist, _sample(np.random.default_rng(3), objs, 40, 4))


def test_serving_full_k(d2, oracle_mod):
    cents, means = synth.serving_centroids()          # K=1024 resident
    import torch  # noqa: F401
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    srv = d2.Server(ctx, slots=4)
    rng = np.random.default_rng(4)
    reqs = [synth.serving_request(rng, means, size=s) for s in (1, 37, 700, 4096)]
    tickets = [srv.submit(d2.bags_from_synth(r)) for r in reqs]
    for r, t in zip(reqs, tickets):
        rc, lab, dist, _ = srv.poll(t, timeout_ms=600000)
        assert rc == d2.D2_OK
        k = min(r.count, 25)
        _check_sample(oracle_mod, r, cents, lab, dist, _sample(rng, r, k, 2 if r.count > 25 else 0))
    srv.close()
    ctx.close()


def test_image_like_full_level_invariants(d2):
    import torch
    objs, cents = synth.image_like()                  # the benchmark step
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    out_loc = torch.empty((cents.loc.shape[0], objs.dim), dtype=torch.float64, device="cuda:0")
    out_w = torch.empty(64, dtype=torch.float64, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    assert d2.d2_cluster_level(ctx, ob, 64, 5000, 10, out_loc, out_w, lab) == d2.D2_OK
    d2.d2_sync(ctx)
    lab = lab.cpu().numpy()
    w = out_w.cpu().numpy()
    assert ((lab >= 0) & (lab < 64)).all()
    assert w.sum() == pytest.approx(objs.count, rel=1e-12)          # sum of omega = N
    assert np.array_equal(np.bincount(lab, minlength=64).astype(float), w)
    loc = out_loc.cpu().numpy()
    assert np.isfinite(loc).all()
    assert np.array_equal(loc.astype(np.float32).astype(np.float64), loc)  # FP32 centroid type
    # a second run gives bit-identical output (deterministic reductions)
    lab2 = torch.empty_like(torch.as_tensor(lab, device="cuda:0"))
    out2 = torch.empty_like(out_loc)
    w2 = torch.empty_like(out_w)
    d2.d2_cluster_level(ctx, ob, 64, 5000, 10, out2, w2, lab2)
    d2.d2_sync(ctx)
    assert np.array_equal(lab2.cpu().numpy(), lab)
    assert np.array_equal(out2.cpu().numpy(), loc)
    ctx.close()
