"""The Python usage example of the README, at a small size."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_readme_example():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_0435_gb300 import build, d2, synth
    build.build()
    objs, cents = synth.image_like(N=2000, K=64)
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dist2 = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    assert d2.d2_assign(ctx, ob, lab, dist2) == d2.D2_OK
    assert d2.d2_update_weights(ctx, ob, lab) == d2.D2_OK
    assert d2.d2_update_locations(ctx, ob, lab) == d2.D2_OK
    d2.d2_sync(ctx)
    loc, w, off = d2.d2_get_centroids(ctx, objs.dim)
    ctx.close()
    assert loc.shape == (int(off[-1]), objs.dim) and np.isfinite(loc).all()
    for j in range(64):
        assert w[off[j]:off[j + 1]].sum() == pytest.approx(1.0, abs=1e-12)
    lab = lab.cpu().numpy()
    assert lab.min() >= 0 and lab.max() < 64
