"""Initial data segmentation (Alg. 3 Step 1) on the GPU against the oracle:
the segment of every bag must be the oracle's (the splits are exact
assignments and FP64 updates, so the partitions agree except where a D^2
comparison ties), and the level driver with constrained segments must match
the oracle's level loop (labels bit-exact, centroids within 1e-6)."""
import time

import numpy as np
import pytest

from paper_1302_0435_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def d2():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_0435_gb300 import build, d2 as mod
    build.build()
    mod.load()
    return mod


@pytest.mark.parametrize("law", ["image_like", "uneven", "plain_small"])
def test_segment_matches_oracle(d2, oracle_mod, law):
    if law == "image_like":
        objs, _ = synth.image_like(N=420, K=2, seed=31)
    elif law == "uneven":
        objs, _ = synth.uneven(N=360, K=2, seed=32)  # supports up to 64: larger trees
    else:
        objs, _ = synth.plain_small(N=300, seed=33)    # FP64 bags: FP64 solves throughout
    tau, iters = 45, 5
    ctx = d2.Context(0)
    seg, M = d2.d2_segment(ctx, d2.bags_from_synth(objs), tau, iters)
    ctx.close()
    ref, Mo = oracle_mod.segment(objs, None, tau, iters, nthreads=8)
    assert M == Mo
    assert np.array_equal(seg, ref)
    assert np.bincount(seg).max() <= tau


def test_segment_weighted_device_buffers(d2, oracle_mod):
    import torch
    objs, _ = synth.image_like(N=300, K=2, seed=34)
    omega = np.random.default_rng(6).uniform(0.2, 3.0, objs.count)
    ctx = d2.Context(0)
    out = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    _, M = d2.d2_segment(ctx, d2.bags_from_synth(objs, device="cuda:0"), 40, 6,
                         omega=torch.as_tensor(omega, device="cuda:0"), seg_id=out)
    d2.d2_sync(ctx)
    ctx.close()
    ref, Mo = oracle_mod.segment(objs, omega, 40, 6, nthreads=8)
    assert M == Mo and np.array_equal(out.cpu().numpy(), ref)


def _single_support_law(N, K, n, seed):
    """Bags of one support each (mixture of 8 components, d = 4) and K
    centroids of n supports.  With one support per bag every transport plan
    is unique, and at the merge level a bag's supports coincide, so each
    round's update is unique too: the level loop's whole trajectory is
    determined (with several supports, plans can tie -- Eq. (D2opt) fixes
    D^2, not the flows -- and equally valid runs may part ways)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-6, 6, size=(8, 4))
    pts = means[rng.integers(0, 8, size=N)] + rng.normal(0, 1.0, size=(N, 4))
    objs = synth._pack(np.ones(N, dtype=np.int64), pts.astype(np.float32), np.ones(N, np.float32),
                       "f32", "f32")
    cl = means[rng.integers(0, 8, size=K * n)] + rng.normal(0, 1.0, size=(K * n, 4))
    cents = synth._pack(np.full(K, n, dtype=np.int64), cl.astype(np.float32),
                        np.full(K * n, 1.0 / n, np.float32), "f32", "f32")
    return objs, cents


def _level(d2, objs, cents, K, tau, iters, si, omega):
    import torch
    ctx = d2.Context(0, segmentation=d2.D2_SEG_CONSTRAINED, split_iters=si)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    out_loc = torch.empty((cents.loc.shape[0], objs.dim), dtype=torch.float64, device="cuda:0")
    out_w = torch.empty(K, dtype=torch.float64, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    rc = d2.d2_cluster_level(ctx, ob, K, tau, iters, out_loc, out_w, lab,
                             omega=torch.as_tensor(omega, device="cuda:0"))
    d2.d2_sync(ctx)
    ctx.close()
    assert rc == 0
    return out_loc.cpu().numpy(), out_w.cpu().numpy(), lab.cpu().numpy()


def test_cluster_level_constrained_matches_oracle(d2, oracle_mod):
    objs, cents = _single_support_law(800, 6, 4, 4244)
    omega = np.random.default_rng(10).uniform(0.5, 1.5, size=objs.count)
    K, tau, iters, si = 6, 150, 3, 5
    loc, w, lab = _level(d2, objs, cents, K, tau, iters, si, omega)
    cl, cw, lo = oracle_mod.cluster_level(objs, omega, cents, K, tau, iters, loc_round=np.float32,
                                          nthreads=8, segmentation="constrained", split_iters=si)
    assert (lab == lo).all()
    assert np.allclose(loc, cl, rtol=1e-6, atol=1e-6)
    assert np.allclose(w, cw, rtol=1e-12)


def test_cluster_level_constrained_invariants(d2):
    """Multi-support bags: weights conserved and equal to the members'
    omega, labels in range, and the run is bitwise repeatable."""
    objs, cents = synth.image_like(N=700, K=6, seed=4243)
    omega = np.random.default_rng(10).uniform(0.5, 1.5, size=objs.count)
    a = _level(d2, objs, cents, 6, 150, 3, 5, omega)
    b = _level(d2, objs, cents, 6, 150, 3, 5, omega)
    loc, w, lab = a
    assert lab.min() >= 0 and lab.max() < 6
    assert w.sum() == pytest.approx(omega.sum(), rel=1e-12)
    assert np.allclose(np.bincount(lab, weights=omega, minlength=6), w, rtol=1e-12)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_segment_image_like_full_size(d2):
    """The benchmark's 200,000 bags into segments of at most 5,000."""
    objs, _ = synth.image_like()
    ctx = d2.Context(0)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    t0 = time.perf_counter()
    seg, M = d2.d2_segment(ctx, ob, 5000, 10)
    dt = time.perf_counter() - t0
    ctx.close()
    counts = np.bincount(seg, minlength=M)
    assert M >= 40 and counts.max() <= 5000 and counts.min() >= 1 and counts.sum() == objs.count
    first = [int(np.argmax(seg == s)) for s in range(M)]
    assert first == sorted(first)
    print("segmentation of 200,000 bags: %d segments in %.2f s" % (M, dt))
