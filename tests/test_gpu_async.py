"""The C-ABI's asynchronous calls: with device outputs and declared bag
bounds (d2_bags.max_support), d2_assign, d2_mallows_all, d2_mallows_batch
and d2_update_locations enqueue their kernels and return at once; their
errors are raised on the device and reported by d2_sync (or by the next
call that waits)."""
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


def _ctx(d2, torch, cents, stream=None, **kw):
    ctx = d2.Context(0, **kw)
    if stream is not None:
        d2.d2_set_stream(ctx, stream)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    return ctx


def test_device_calls_return_before_their_kernels(d2):
    import torch
    objs, cents = synth.image_like(N=200_000, K=64, seed=901)
    stream = torch.cuda.Stream()  # the context's stream, so that the event follows its work
    ctx = _ctx(d2, torch, cents, stream=stream)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    torch.cuda.synchronize()  # inputs written on the default stream, read on `stream`
    assert ob.s.max_support == 16
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    d2.d2_assign(ctx, ob, lab, dist)  # first call: buffers grow, shapes settle
    d2.d2_sync(ctx)
    ref_lab, ref_dist = lab.clone(), dist.clone()
    with torch.cuda.stream(stream):
        lab.fill_(-7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    t_call = time.perf_counter() - t0
    ev = torch.cuda.Event()
    ev.record(stream)
    pending = not ev.query()
    d2.d2_sync(ctx)
    t_all = time.perf_counter() - t0
    # 12.8 M pair LPs take >100 ms on the GPU; the call itself only enqueues
    assert pending, "the kernels had already finished when the call returned"
    assert t_call < 0.2 * t_all, (t_call, t_all)
    assert torch.equal(lab, ref_lab) and torch.equal(dist, ref_dist)
    ctx.close()


def test_one_pair_calls_do_not_wait(d2):
    """The plain one-pair-per-launch form costs launches, not round trips."""
    import torch
    cents, means = synth.serving_centroids(K=64, seed=902)
    one = synth.serving_request(np.random.default_rng(903), means, size=64)
    ctx = _ctx(d2, torch, cents)
    ob = d2.bags_from_synth(one, device="cuda:0")
    po = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    pc = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    dd = torch.empty(1, dtype=torch.float64, device="cuda:0")
    d2.d2_mallows_batch(ctx, ob, po, pc, dd)
    d2.d2_sync(ctx)
    calls = 200
    t0 = time.perf_counter()
    for _ in range(calls):
        d2.d2_mallows_batch(ctx, ob, po, pc, dd)
    t_enq = (time.perf_counter() - t0) / calls
    d2.d2_sync(ctx)
    assert t_enq < 2e-4, t_enq  # about the cost of a few kernel launches
    ctx.close()


def test_errors_are_reported_by_sync_and_cleared(d2):
    import torch
    objs, cents = synth.image_like(N=500, K=8, seed=904)
    ctx = _ctx(d2, torch, cents)
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    bad = synth.Bags(objs.loc.copy(), objs.w.copy(), objs.off.copy(), "f32", "f32")
    bad.w[bad.off[7]] = -1.0  # a negative weight
    assert d2.d2_assign(ctx, d2.bags_from_synth(bad, device="cuda:0"), lab, dist) == d2.D2_OK
    with pytest.raises(d2.D2Error) as e:
        d2.d2_sync(ctx)
    assert e.value.code == d2.D2_EINVAL
    d2.d2_sync(ctx)  # reported once, then cleared
    # a bag above the declared bound
    ob = d2.bags_from_synth(objs, device="cuda:0")
    ob.s.max_support = 10
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    with pytest.raises(d2.D2Error) as e:
        d2.d2_sync(ctx)
    assert e.value.code == d2.D2_EINVAL
    # a pending error is returned by the next call that waits, which does
    # nothing else; the context stays usable
    assert d2.d2_assign(ctx, d2.bags_from_synth(bad, device="cuda:0"), lab, dist) == d2.D2_OK
    with pytest.raises(d2.D2Error) as e:
        d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    assert e.value.code == d2.D2_EINVAL
    ob.s.max_support = 16
    assert d2.d2_assign(ctx, ob, lab, dist) == d2.D2_OK
    d2.d2_sync(ctx)
    h_lab = np.empty(objs.count, np.int32)
    h_dist = np.empty(objs.count)
    assert d2.d2_assign(ctx, d2.bags_from_synth(objs), h_lab, h_dist) == d2.D2_OK
    assert np.array_equal(lab.cpu().numpy(), h_lab) and np.array_equal(dist.cpu().numpy(), h_dist)
    ctx.close()


def test_binned_assign_without_host_counts_matches(d2):
    """Bins whose counts stay on the device (no autotuning: group_lanes
    fixed) give the results of the waiting, host-counted path."""
    import torch
    objs, cents = synth.uneven(N=30000, K=32, seed=905)
    out = []
    for lanes in (32, 0):
        ctx = _ctx(d2, torch, cents, group_lanes=lanes)
        ob = d2.bags_from_synth(objs, device="cuda:0")
        lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
        dist = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
        d2.d2_assign(ctx, ob, lab, dist)
        d2.d2_sync(ctx)
        out.append((lab.cpu().numpy(), dist.cpu().numpy()))
        ctx.close()
    # the tuned shape may pick another cold start: same optima
    assert np.array_equal(out[0][0], out[1][0])
    assert np.allclose(out[0][1], out[1][1], rtol=1e-12, atol=0)


def test_all_pairs_step_replays_from_a_cuda_graph(d2):
    """Once its launch shapes are tuned, the certified all-pairs call and
    the location update only enqueue kernels, so a caller can capture them
    into a CUDA graph: bins, screen, merge, exact pass and update replay
    with the eager results."""
    import torch
    objs, cents = synth.uneven(N=40000, K=64, seed=906)
    stream = torch.cuda.Stream()
    ctx = _ctx(d2, torch, cents, stream=stream, certify=d2.D2_CERTIFY_ALL)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    torch.cuda.synchronize()  # inputs written on the default stream, read on `stream`
    N, K = objs.count, cents.count
    allg = torch.empty((N, K), dtype=torch.float64, device="cuda:0")
    lab = torch.empty(N, dtype=torch.int32, device="cuda:0")
    dd = torch.empty(N, dtype=torch.float64, device="cuda:0")
    d2.d2_mallows_all(ctx, ob, allg, lab, dd)  # tunes the bins' launch shapes
    d2.d2_update_locations(ctx, ob, lab)
    d2.d2_sync(ctx)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    d2.d2_mallows_all(ctx, ob, allg, lab, dd)  # eager reference at the initial centroids
    d2.d2_sync(ctx)
    ref = (allg.clone(), lab.clone(), dd.clone())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
        d2.d2_mallows_all(ctx, ob, allg, lab, dd)
    d2.d2_sync(ctx)
    allg.zero_()
    lab.fill_(-1)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    d2.d2_sync(ctx)
    assert torch.equal(allg, ref[0]) and torch.equal(lab, ref[1]) and torch.equal(dd, ref[2])
    ctx.close()
