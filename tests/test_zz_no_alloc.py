"""d2_update_locations_noalloc: the location update for callers that cannot
call cudaMalloc during the call (a framework that owns all device memory
through its own allocator and budget, or a latency-critical loop that must
not pay for allocator synchronisation).  It must give the same centroids as
d2_update_locations, call after call, while using only its fixed scratch
array.  Collected last on purpose: if it fails, every other test has run.
"""
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


def _assign(d2, torch, ctx, ob, N, stride):
    lab = torch.empty(N, dtype=torch.int32, device="cuda:0")
    dist = torch.empty(N, dtype=torch.float64, device="cuda:0")
    flows = (torch.empty((N, stride), dtype=torch.int32, device="cuda:0"),
             torch.empty((N, stride), dtype=torch.float64, device="cuda:0"))
    assert d2.d2_assign(ctx, ob, lab, dist, flows=flows) == d2.D2_OK
    return lab, flows


@pytest.mark.parametrize("N", [3000, 20000])
def test_noalloc_matches_update_locations_two_calls(d2, N):
    """N = 3000 <= 512*K: both entry points sum every centroid in one block,
    so the centroids are identical.  N = 20000 > 512*K: d2_update_locations
    splits each cluster over several blocks (another FP64 summation order),
    so the two agree within one unit in the last place of the FP32
    centroid type they are rounded to."""
    import torch
    K = 16
    objs, cents = synth.image_like(N=N, K=K, seed=77)
    split = N > 512 * K
    dim = objs.dim
    omega = torch.as_tensor(np.random.default_rng(5).uniform(0.5, 2.0, objs.count), device="cuda:0")
    ctx = d2.Context(0)
    stream = torch.cuda.current_stream()
    d2.d2_set_stream(ctx, stream)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    loc0, _, off0 = d2.d2_get_centroids(ctx, dim)
    # caller-owned centroid arrays for the allocation-free variant
    c64 = torch.as_tensor(loc0, device="cuda:0").contiguous()
    c32 = c64.float().contiguous()
    coff = torch.as_tensor(off0, device="cuda:0")
    stride = 16 + 16 - 1
    for call in range(2):
        lab, flows = _assign(d2, torch, ctx, ob, objs.count, stride)
        d2.d2_sync(ctx)
        # the existing entry point updates the resident set ...
        assert d2.d2_update_locations(ctx, ob, lab, omega=omega, flows=flows) == d2.D2_OK
        ref, _, _ = d2.d2_get_centroids(ctx, dim)
        # ... the variant updates the caller's copy from the same inputs
        d2.d2_update_locations_noalloc(ob, lab, flows, cents.count, coff, d2.D2_F32, c64, c32,
                                       omega=omega, stream=stream)
        torch.cuda.synchronize()
        got = c64.cpu().numpy()
        if split:
            ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(got - ref) <= ulp), (call, float(np.max(np.abs(got - ref))))
        else:
            assert np.array_equal(got, ref), (call, float(np.max(np.abs(got - ref))))
        assert np.array_equal(c32.cpu().numpy(), got.astype(np.float32))
        assert not np.allclose(ref, loc0)  # the centroids did move
    ctx.close()


def test_noalloc_rejects_bad_bag_offsets(d2):
    """The bag offsets are checked on the device before the update runs: a
    bag with no support or with more than 64 is refused with D2_EINVAL."""
    import torch
    objs, cents = synth.image_like(N=64, K=4, seed=79)
    lab = torch.zeros(objs.count, dtype=torch.int32, device="cuda:0")
    flows = (torch.full((objs.count, 31), -1, dtype=torch.int32, device="cuda:0"),
             torch.zeros((objs.count, 31), dtype=torch.float64, device="cuda:0"))
    coff = torch.arange(0, 16 * 5, 16, dtype=torch.int64, device="cuda:0")
    c64 = torch.zeros((16 * 4, objs.dim), dtype=torch.float64, device="cuda:0")
    c32 = torch.zeros((16 * 4, objs.dim), dtype=torch.float32, device="cuda:0")
    for bad in ("empty", "wide"):
        off = objs.off.astype(np.int64).copy()
        if bad == "empty":
            off[5] = off[4]  # bag 4 has no support
        else:
            off[1:] += 70  # bag 0 has 70 + m supports
        ob = d2.bags_from_synth(objs, device="cuda:0")
        ob.off.copy_(torch.as_tensor(off))
        with pytest.raises(d2.D2Error) as e:
            d2.d2_update_locations_noalloc(ob, lab, flows, 4, coff, d2.D2_F32, c64, c32)
        assert e.value.code == d2.D2_EINVAL
        assert not c64.any()  # nothing was written


def test_noalloc_rejects_oversize_and_host_buffers(d2):
    import torch
    objs, cents = synth.image_like(N=64, K=4, seed=78)
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.zeros(objs.count, dtype=torch.int32, device="cuda:0")
    flows = (torch.full((objs.count, 31), -1, dtype=torch.int32, device="cuda:0"),
             torch.zeros((objs.count, 31), dtype=torch.float64, device="cuda:0"))
    K = 2000  # beyond the 1,024-centroid limit
    coff = torch.arange(0, 16 * (K + 1), 16, dtype=torch.int64, device="cuda:0")
    c64 = torch.zeros((16 * K, objs.dim), dtype=torch.float64, device="cuda:0")
    c32 = torch.zeros((16 * K, objs.dim), dtype=torch.float32, device="cuda:0")
    with pytest.raises(d2.D2Error) as e:
        d2.d2_update_locations_noalloc(ob, lab, flows, K, coff, d2.D2_F32, c64, c32)
    assert e.value.code == d2.D2_EUNSUPPORTED
    hb = d2.bags_from_synth(objs)  # host arrays
    with pytest.raises(d2.D2Error) as e:
        d2.d2_update_locations_noalloc(hb, lab, flows, 4, coff[:5], d2.D2_F32, c64, c32)
    assert e.value.code == d2.D2_EINVAL
