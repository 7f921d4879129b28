"""d2_cluster_level_ex with Alg. 1 updates (D2_UPDATE_ALG1: the weighted
D2-clustering of Alg. 3 Step 2, support weights by the joint LP each round)
against the oracle's level loop with update="alg1"."""
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


def _single_support(N, K, n, seed):
    # one support per bag: every member's transport is forced, the weight LP
    # is linear in p with a unique vertex optimum, so the trajectory is unique
    rng = np.random.default_rng(seed)
    means = rng.uniform(-6, 6, size=(8, 4))
    pts = means[rng.integers(0, 8, size=N)] + rng.normal(0, 1.0, size=(N, 4))
    objs = synth._pack(np.ones(N, dtype=np.int64), pts.astype(np.float32), np.ones(N, np.float32),
                       "f32", "f32")
    cl = means[rng.integers(0, 8, size=K * n)] + rng.normal(0, 1.0, size=(K * n, 4))
    cents = synth._pack(np.full(K, n, dtype=np.int64), cl.astype(np.float32),
                        np.full(K * n, 1.0 / n, np.float32), "f32", "f32")
    return objs, cents


def _level(d2, objs, cents, K, tau, iters, omega=None, update=None, jmax=1000):
    import torch
    upd = d2.D2_UPDATE_ALG1 if update is None else update
    ctx = d2.Context(0, centroid_update=upd, joint_max_iter=jmax, joint_tol=1e-10)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    T = cents.loc.shape[0]
    out_loc = torch.empty((T, objs.dim), dtype=torch.float64, device="cuda:0")
    out_sw = torch.empty(T, dtype=torch.float64, device="cuda:0")
    out_w = torch.empty(K, dtype=torch.float64, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    om = None if omega is None else torch.as_tensor(omega, device="cuda:0")
    rc = d2.d2_cluster_level_ex(ctx, ob, K, tau, iters, out_loc, out_sw, out_w, lab, omega=om)
    d2.d2_sync(ctx)
    ctx.close()
    return rc, out_loc.cpu().numpy(), out_sw.cpu().numpy(), out_w.cpu().numpy(), lab.cpu().numpy()


def test_alg1_level_matches_oracle(d2, oracle_mod):
    objs, cents = _single_support(900, 4, 3, 501)
    omega = np.random.default_rng(11).uniform(0.5, 1.5, size=objs.count)
    K, tau, iters = 4, 300, 3
    rc, loc, sw, w, lab = _level(d2, objs, cents, K, tau, iters, omega)
    assert rc == d2.D2_OK
    cl, cw, lo, csw = oracle_mod.cluster_level(objs, omega, cents, K, tau, iters,
                                               loc_round=np.float32, nthreads=8, update="alg1",
                                               return_support_weights=True)
    assert (lab == lo).all()
    assert np.allclose(sw, csw, atol=1e-9)
    assert np.allclose(loc, cl, rtol=1e-6, atol=1e-6)
    assert np.allclose(w, cw, rtol=1e-12)


def test_alg1_level_invariants(d2):
    """Multi-support bags (the weight LP may have several optima): support
    weights are distributions, the level conserves omega, results repeat
    bitwise, and the weights differ from the constrained run's."""
    objs, cents = synth.image_like(N=1200, K=4, seed=502)
    omega = np.random.default_rng(12).uniform(0.5, 1.5, size=objs.count)
    a = _level(d2, objs, cents, 4, 400, 2, omega)
    b = _level(d2, objs, cents, 4, 400, 2, omega)
    rc, loc, sw, w, lab = a
    assert rc == d2.D2_OK
    assert all(np.array_equal(x, y) for x, y in zip(a[1:], b[1:]))
    off = cents.off
    for j in range(4):
        assert (sw[off[j]:off[j + 1]] >= 0).all()
        assert sw[off[j]:off[j + 1]].sum() == pytest.approx(1.0, abs=1e-12)
    assert w.sum() == pytest.approx(omega.sum(), rel=1e-12)
    c = _level(d2, objs, cents, 4, 400, 2, omega, update=d2.D2_UPDATE_CONSTRAINED)
    assert c[0] == d2.D2_OK
    assert np.allclose(c[2], 1.0 / 16)          # constrained: the resident uniform weights
    assert not np.allclose(sw, c[2])


def test_alg1_with_constrained_segmentation(d2):
    """Alg. 1 updates inside segments formed by the binary constrained D2
    splits: the level conserves omega, weights stay distributions, runs
    repeat bitwise."""
    import torch
    objs, cents = synth.image_like(N=900, K=3, seed=503)

    def run():
        ctx = d2.Context(0, centroid_update=d2.D2_UPDATE_ALG1, segmentation=d2.D2_SEG_CONSTRAINED,
                         split_iters=4, joint_max_iter=1000)
        d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
        ob = d2.bags_from_synth(objs, device="cuda:0")
        T = cents.loc.shape[0]
        loc = torch.empty((T, objs.dim), dtype=torch.float64, device="cuda:0")
        sw = torch.empty(T, dtype=torch.float64, device="cuda:0")
        w = torch.empty(3, dtype=torch.float64, device="cuda:0")
        lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
        rc = d2.d2_cluster_level_ex(ctx, ob, 3, 300, 2, loc, sw, w, lab)
        d2.d2_sync(ctx)
        ctx.close()
        return rc, loc.cpu().numpy(), sw.cpu().numpy(), w.cpu().numpy(), lab.cpu().numpy()

    a, b = run(), run()
    assert a[0] == d2.D2_OK
    assert all(np.array_equal(x, y) for x, y in zip(a[1:], b[1:]))
    off = cents.off
    for j in range(3):
        assert a[2][off[j]:off[j + 1]].sum() == pytest.approx(1.0, abs=1e-12)
    assert a[3].sum() == pytest.approx(objs.count, rel=1e-12)
    assert a[4].min() >= 0 and a[4].max() < 3
