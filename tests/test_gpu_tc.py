"""Tensor-core ground costs (BF16 operands, FP32 accumulation) for the FP32
screen at high support dimension.

The tile is checked cell by cell against the FP64 oracle's cost of
Eq. (D2opt) within the stated bound, and the assignment that screens with it
must give the same FP64-exact labels and distances as the SIMT screen and
the oracle (labels bit-exact except ties within 1e-9 relative, D^2 within
1e-6 relative).
"""
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


def _bf16(a):
    return synth.bf16_bits_to_f32(synth.f32_to_bf16_bits(np.asarray(a, dtype=np.float32)))


def tc_bound(x, y):
    """The per-cell bound the screen adds for a tensor-core tile, evaluated
    in FP64 from the pair's supports: d*2^-22 + (d+3)*2^-24 relative to the
    largest squared norms (accumulation, norms, final FMA) plus the move from
    the BF16-rounded centroid y^ back to y."""
    d = x.shape[1]
    yh = _bf16(y).astype(np.float64)
    nxm = float(np.max(np.sum(x * x, axis=1)))
    cn = float(np.max(np.sum(yh * yh, axis=1)))
    cd = float(np.max(np.linalg.norm(y - yh, axis=1)))
    rel = d * 2.0 ** -22 + (d + 3) * 2.0 ** -24
    return (rel * (nxm + cn) + (2 * (np.sqrt(nxm) + np.sqrt(cn)) + 2 * cd) * cd) * (1 + 2.0 ** -10)


def _cost_tiles(d2, objs, cents, pairs):
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    out = []
    for i, j in pairs:
        m = int(objs.off[i + 1] - objs.off[i])
        n = int(cents.off[j + 1] - cents.off[j])
        out.append((d2.d2_cost_matrix(ctx, ob, i, j, d2.D2_PREC_TC, m, n),
                    d2.d2_cost_matrix(ctx, ob, i, j, d2.D2_PREC_FP64, m, n)))
    ctx.close()
    return out


def test_tc_tile_within_bound_bf16_centroids(d2, oracle_mod):
    objs, cents = synth.high_dim(N=24, K=40)
    rng = np.random.default_rng(11)
    pairs = [(int(rng.integers(objs.count)), int(rng.integers(cents.count))) for _ in range(12)]
    pairs += [(0, 0), (objs.count - 1, cents.count - 1), (3, 39)]   # last column tile too
    worst = 0.0
    nonzero = 0.0
    for (i, j), (ctc, c64) in zip(pairs, _cost_tiles(d2, objs, cents, pairs)):
        x, _ = oracle_mod.bag(objs, i)
        y, _ = oracle_mod.bag(cents, j)
        ref = oracle_mod.cost(x, y)
        assert np.array_equal(c64, ref) or np.allclose(c64, ref, rtol=1e-13, atol=1e-15)
        err = np.abs(ctc - ref)
        b = tc_bound(x, y)
        assert err.max() <= b, (i, j, err.max(), b)
        assert (ctc >= 0).all()
        worst = max(worst, err.max() / b)
        nonzero = max(nonzero, err.max())
    assert nonzero > 0  # the tile is the FP32 contraction, not the FP64 one
    print("max |C_tc - C_fp64| / bound = %.3g" % worst)


def test_tc_tile_within_bound_rounded_centroids(d2, oracle_mod):
    # FP32 centroids that BF16 does not represent: the bound's rounding term
    objs, _ = synth.high_dim(N=16, K=8)
    rng = np.random.default_rng(12)
    K, n, d = 6, 48, 128
    loc = np.abs(rng.standard_normal((K * n, d))).astype(np.float32)
    loc /= np.linalg.norm(loc, axis=1, keepdims=True)
    cents = synth._pack(np.full(K, n, dtype=np.int64), loc.astype(np.float32),
                        np.full(K * n, 1.0 / n, np.float32), "f32", "f32")
    pairs = [(i, j) for i in (0, 5, 15) for j in range(K)]
    for (i, j), (ctc, _) in zip(pairs, _cost_tiles(d2, objs, cents, pairs)):
        x, _ = oracle_mod.bag(objs, i)
        y, _ = oracle_mod.bag(cents, j)
        ref = oracle_mod.cost(x, y)
        assert np.abs(ctc - ref).max() <= tc_bound(x, y)


def test_tc_rejects_non_bf16_objects(d2):
    objs, cents = synth.image_like(N=8, K=2)
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_cost_matrix(ctx, ob, 0, 0, d2.D2_PREC_TC, int(objs.off[1]), int(cents.off[1]))
    assert e.value.code == d2.D2_EUNSUPPORTED
    ctx.close()


def _assign(d2, objs, cents, **cfg):
    import torch
    ctx = d2.Context(0, **cfg)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    s0 = d2.d2_get_stats()
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    d2.d2_sync(ctx)
    s1 = d2.d2_get_stats()
    ctx.close()
    exact = (s1["pairs_exact"] - s0["pairs_exact"]) / objs.count
    return lab.cpu().numpy(), dist.cpu().numpy(), exact


def _check_vs(oracle_mod, objs, cents, lab, dist, idx):
    sub = objs.subset(idx)
    lab_o, d_o, allm = oracle_mod.assign(sub, cents, nthreads=8, return_all=True)
    lg, dg = lab[idx], dist[idx]
    for k in np.nonzero(lg != lab_o)[0]:
        a, b = allm[k, lg[k]], allm[k, lab_o[k]]
        assert abs(a - b) <= TIE * max(a, b)
    assert (np.abs(dg - d_o) <= 1e-6 * d_o + 1e-12).all()


def test_tc_assign_binned_chunked_matches_simt_and_oracle(d2, oracle_mod):
    # 4,500 objects (two node bins), 16 centroids; an 8 MiB tile budget
    # forces dozens of chunks per bin
    objs, cents = synth.high_dim(N=4500, K=16, seed=2024)
    lab_t, d_t, ex_t = _assign(d2, objs, cents, tile_budget_mib=8)
    lab_s, d_s, ex_s = _assign(d2, objs, cents, cost_tc=d2.D2_TC_OFF)
    assert ((lab_t >= 0) & (lab_t < cents.count)).all()
    diff = np.nonzero(lab_t != lab_s)[0]
    for i in diff:  # only FP64 ties may differ
        assert abs(d_t[i] - d_s[i]) <= TIE * max(d_t[i], d_s[i])
    assert np.allclose(d_t, d_s, rtol=1e-12, atol=0)
    print("exact solves per object: tensor-core screen %.3f, SIMT screen %.3f" % (ex_t, ex_s))
    idx = np.sort(np.random.default_rng(5).choice(objs.count, size=40, replace=False))
    _check_vs(oracle_mod, objs, cents, lab_t, d_t, idx)


def test_tc_assign_after_update_uses_new_centroids(d2, oracle_mod):
    """The BF16 copy is rebuilt after d2_update_locations moves the resident
    set; FP32 centroids hold the means unrounded, so the rounding term of
    the bound is nonzero on the second assign."""
    import torch
    objs, c16 = synth.high_dim(N=300, K=12, seed=77)
    cents = synth._pack(np.diff(c16.off).astype(np.int64), c16.loc.astype(np.float32), c16.w,
                        "f32", "f32")
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    assert d2.d2_update_locations(ctx, ob, lab) == d2.D2_OK
    loc, _, off = d2.d2_get_centroids(ctx, objs.dim)
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    d2.d2_sync(ctx)
    ctx.close()
    moved = synth._pack(np.diff(off).astype(np.int64), loc.astype(np.float32), cents.w,
                        "f32", "f32")
    assert not np.array_equal(_bf16(moved.loc), moved.loc)  # not BF16-exact any more
    _check_vs(oracle_mod, objs, moved, lab.cpu().numpy(), dist.cpu().numpy(),
              np.arange(objs.count))


def test_tc_completion_wait_runs_out_and_is_reported(d2, oracle_mod):
    """The contraction's bounded wait on its MMA-completion barrier: the
    diagnostic probe makes the first wait poll a barrier that nothing
    arrives on, so it runs out with MMAs in flight.  The kernel must then
    raise the timeout (D2_ETIMEOUT), wait (bounded) for its issued MMAs, free
    its tensor memory and return; the context and the GPU stay usable."""
    objs, cents = synth.high_dim(N=6, K=4, seed=131)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    m = int(objs.off[1] - objs.off[0])
    n = int(cents.off[1] - cents.off[0])
    ctx = d2.Context(0, tc_wait_probe=256)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    for _ in range(2):  # twice: the first expiry left nothing behind
        with pytest.raises(d2.D2Error) as e:
            d2.d2_cost_matrix(ctx, ob, 0, 0, d2.D2_PREC_TC, m, n)
        assert e.value.code == d2.D2_ETIMEOUT
    # the same context still computes: FP64 tile against the oracle's cost
    x, _ = oracle_mod.bag(objs, 0)
    y, _ = oracle_mod.bag(cents, 0)
    c64 = d2.d2_cost_matrix(ctx, ob, 0, 0, d2.D2_PREC_FP64, m, n)
    assert np.allclose(c64, oracle_mod.cost(x, y), rtol=1e-12, atol=1e-12)
    ctx.close()
    # and a context without the probe gets its tensor-core tile within the bound
    ctx2 = d2.Context(0)
    d2.d2_set_centroids(ctx2, d2.bags_from_synth(cents, device="cuda:0"))
    ctc = d2.d2_cost_matrix(ctx2, ob, 0, 0, d2.D2_PREC_TC, m, n)
    assert np.abs(ctc - oracle_mod.cost(x, y)).max() <= tc_bound(x, y)
    ctx2.close()
