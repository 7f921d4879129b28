"""d2_cluster_level with eps_tol ("until epsilon converges", Alg. 2 Step 4)
against the oracle's level loop with the same stopping rule."""
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


def _single_support(N, K, n, seed):
    # one support per bag: unique plans, so the level trajectory is determined
    rng = np.random.default_rng(seed)
    means = rng.uniform(-6, 6, size=(8, 4))
    pts = means[rng.integers(0, 8, size=N)] + rng.normal(0, 1.0, size=(N, 4))
    objs = synth._pack(np.ones(N, dtype=np.int64), pts.astype(np.float32), np.ones(N, np.float32),
                       "f32", "f32")
    cl = means[rng.integers(0, 8, size=K * n)] + rng.normal(0, 1.0, size=(K * n, 4))
    cents = synth._pack(np.full(K, n, dtype=np.int64), cl.astype(np.float32),
                        np.full(K * n, 1.0 / n, np.float32), "f32", "f32")
    return objs, cents


def _level(d2, objs, cents, K, tau, iters, eps_tol):
    import torch
    ctx = d2.Context(0, eps_tol=eps_tol)
    st = torch.cuda.Stream()
    d2.d2_set_stream(ctx, st)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    out_loc = torch.empty((cents.loc.shape[0], objs.dim), dtype=torch.float64, device="cuda:0")
    out_w = torch.empty(K, dtype=torch.float64, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    s0 = d2.d2_get_stats()
    assert d2.d2_cluster_level(ctx, ob, K, tau, iters, out_loc, out_w, lab) == 0
    d2.d2_sync(ctx)
    launches = d2.d2_get_stats()["kernel_launches"] - s0["kernel_launches"]
    ctx.close()
    return out_loc.cpu().numpy(), out_w.cpu().numpy(), lab.cpu().numpy(), launches


def test_level_eps_tol_matches_oracle(d2, oracle_mod):
    objs, cents = _single_support(900, 5, 3, 77)
    K, tau, iters = 5, 300, 40
    loc, w, lab, n_early = _level(d2, objs, cents, K, tau, iters, 1e-12)
    cl, cw, lo = oracle_mod.cluster_level(objs, None, cents, K, tau, iters, loc_round=np.float32,
                                          nthreads=8, eps_tol=1e-12)
    assert (lab == lo).all()
    assert np.allclose(loc, cl, rtol=1e-6, atol=1e-6)
    assert np.allclose(w, cw, rtol=1e-12)
    _, _, lab_full, n_full = _level(d2, objs, cents, K, tau, iters, 0.0)
    assert (lab_full == lab).all()          # the fixed point: more rounds change nothing
    assert n_early < n_full                 # and the rounds did stop early
