"""Combined distance of several bag types (Eq. (imgdist)) on the GPU
against the oracle's assign_multi."""
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


def _run(d2, objs_list, cents_list):
    import torch
    ctxs = []
    for c in cents_list:
        ctx = d2.Context(0)
        d2.d2_set_centroids(ctx, d2.bags_from_synth(c, device="cuda:0"))
        ctxs.append(ctx)
    obs = [d2.bags_from_synth(o, device="cuda:0") for o in objs_list]
    N = objs_list[0].count
    lab = torch.empty(N, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(N, dtype=torch.float64, device="cuda:0")
    rc = d2.d2_assign_multi(ctxs, obs, lab, dist)
    torch.cuda.synchronize()
    for c in ctxs:
        c.close()
    assert rc == d2.D2_OK
    return lab.cpu().numpy(), dist.cpu().numpy()


def _check(lg, dg, lo, do, allm):
    for i in np.nonzero(lg != lo)[0]:
        a, b = allm[i, lg[i]], allm[i, lo[i]]
        assert abs(a - b) <= TIE * max(a, b)
    assert (np.abs(dg - do) <= 1e-6 * do + 1e-12).all()


def test_two_bag_types_match_oracle(d2, oracle_mod):
    objs, cents = synth.image_two_bags(N=500, K=10, seed=81)
    lg, dg = _run(d2, objs, cents)
    lo, do, allm = oracle_mod.assign_multi(objs, cents, nthreads=8)
    _check(lg, dg, lo, do, allm)


def test_one_type_equals_assign(d2, oracle_mod):
    import torch
    objs, cents = synth.image_like(N=400, K=8, seed=82)
    lg, dg = _run(d2, [objs], [cents])
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    d2.d2_assign(ctx, d2.bags_from_synth(objs, device="cuda:0"), lab, dist)
    d2.d2_sync(ctx)
    ctx.close()
    assert np.array_equal(lg, lab.cpu().numpy())
    assert np.allclose(dg, dist.cpu().numpy(), rtol=1e-12, atol=0)


def test_identical_types_double_the_distance(d2):
    objs, cents = synth.image_like(N=300, K=6, seed=83)
    l1, d1 = _run(d2, [objs], [cents])
    l2, d2v = _run(d2, [objs, objs], [cents, cents])
    assert np.array_equal(l1, l2)
    assert np.allclose(d2v, 2.0 * d1, rtol=1e-12, atol=0)


def test_multi_errors(d2):
    import torch
    objs, cents = synth.image_two_bags(N=20, K=4, seed=84)
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents[0], device="cuda:0"))
    obs = [d2.bags_from_synth(o, device="cuda:0") for o in objs]
    lab = torch.empty(20, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(20, dtype=torch.float64, device="cuda:0")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign_multi([ctx, ctx], obs, lab, dist)   # one context per type
    assert e.value.code == d2.D2_EINVAL
    short = synth.image_like(N=10, K=4, seed=85)[0]
    ctx2 = d2.Context(0)
    d2.d2_set_centroids(ctx2, d2.bags_from_synth(cents[1], device="cuda:0"))
    with pytest.raises(d2.D2Error) as e:
        d2.d2_assign_multi([ctx, ctx2], [obs[0], d2.bags_from_synth(short, device="cuda:0")],
                           lab, dist)                     # different object counts
    assert e.value.code == d2.D2_EINVAL
    ctx.close()
    ctx2.close()


def test_two_bag_image_like_full_size(d2, oracle_mod):
    """200,000 images of a colour and a texture bag against 64 centroids."""
    import torch
    objs, cents = synth.image_two_bags()
    ctxs = []
    for c in cents:
        ctx = d2.Context(0)
        d2.d2_set_centroids(ctx, d2.bags_from_synth(c, device="cuda:0"))
        ctxs.append(ctx)
    obs = [d2.bags_from_synth(o, device="cuda:0") for o in objs]
    N = objs[0].count
    lab = torch.empty(N, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(N, dtype=torch.float64, device="cuda:0")
    d2.d2_assign_multi(ctxs, obs, lab, dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert d2.d2_assign_multi(ctxs, obs, lab, dist) == d2.D2_OK
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    print("two-bag assign: %.3g image pairs/s (%.3g LPs/s)" % (N * 64 / dt, 2 * N * 64 / dt))
    idx = np.sort(np.random.default_rng(8).choice(N, size=200, replace=False))
    lo, do, allm = oracle_mod.assign_multi([o.subset(idx) for o in objs], cents, nthreads=16)
    _check(lab.cpu().numpy()[idx], dist.cpu().numpy()[idx], lo, do, allm)
