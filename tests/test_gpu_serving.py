"""Serving (continuous batching): requests that arrive while others are on
the GPU are admitted into free slots and overlap on the device; every
request's labels and distances are bitwise the same alone (d2_assign) and
in the mix."""
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


def test_results_identical_alone_and_in_the_mix(d2, oracle_mod):
    cents, means = synth.serving_centroids(K=48)
    rng = np.random.default_rng(21)
    reqs = [synth.serving_request(rng, means, size=int(s))
            for s in np.exp(rng.uniform(0, np.log(400), size=24)).astype(int) + 1]
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    alone = []
    for r in reqs:
        lab = np.empty(r.count, dtype=np.int32)
        dist = np.empty(r.count)
        assert d2.d2_assign(ctx, d2.bags_from_synth(r), lab, dist) == d2.D2_OK
        alone.append((lab, dist))
    srv = d2.Server(ctx, slots=4)
    refs = [d2.bags_from_synth(r) for r in reqs]
    tickets = [srv.submit(b) for b in refs]          # all arrive while the first run
    for t, (lab_a, d_a) in zip(tickets, alone):
        rc, lab, dist, lat = srv.poll(t, timeout_ms=120000)
        assert rc == d2.D2_OK
        assert np.array_equal(lab, lab_a)
        assert np.array_equal(dist, d_a)              # bitwise
        assert lat >= 0.0
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["peak_inflight"] > 1
    # spot check against the FP64 oracle
    lab_o, d_o = oracle_mod.assign(reqs[0], cents, nthreads=8)
    assert np.array_equal(alone[0][0], lab_o) or np.allclose(alone[0][1], d_o, rtol=1e-9)
    assert np.allclose(alone[0][1], d_o, rtol=1e-6)
    srv.close()
    ctx.close()


def test_poll_timeout_and_memory_admission(d2):
    cents, means = synth.serving_centroids(K=32)
    rng = np.random.default_rng(22)
    ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    # a budget smaller than one request: requests are admitted one at a time
    srv = d2.Server(ctx, slots=4, mem_budget=1)
    reqs = [d2.bags_from_synth(synth.serving_request(rng, means, size=200)) for _ in range(5)]
    tickets = [srv.submit(b) for b in reqs]
    rc0, _, _, _ = srv.poll(tickets[-1], timeout_ms=0)
    assert rc0 in (d2.D2_ETIMEOUT, d2.D2_OK)
    if rc0 == d2.D2_OK:
        tickets = tickets[:-1]
    for t in tickets:
        rc, lab, dist, lat = srv.poll(t, timeout_ms=120000)
        assert rc == d2.D2_OK and (lab >= 0).all()
    assert srv.stats()["peak_inflight"] == 1
    srv.close()
    ctx.close()
