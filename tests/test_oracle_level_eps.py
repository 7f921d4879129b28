"""Pin of the oracle's level loop with "until epsilon converges" (Alg. 2
Step 4): once a level reaches a fixed point (labels repeat, so the update
returns the same centroids), further rounds change nothing, so stopping
early must give exactly what running every round gives; and with no
tolerance the loop runs every round."""
import numpy as np

from paper_1302_0435_gb300 import synth


def test_early_stop_equals_the_fixed_point(oracle_mod):
    objs, cents = synth.image_like(N=240, K=3, seed=41)
    full = oracle_mod.cluster_level(objs, None, cents, 3, 120, 60)
    early = oracle_mod.cluster_level(objs, None, cents, 3, 120, 60, eps_tol=1e-12)
    assert np.array_equal(full[2], early[2])
    assert np.array_equal(full[0], early[0]) and np.array_equal(full[1], early[1])


def test_loose_tolerance_stops_after_two_rounds(oracle_mod):
    """A tolerance of 1 accepts any change: the level stops after round 1
    (the second), which is what two fixed rounds give."""
    objs, cents = synth.image_like(N=200, K=3, seed=42)
    two = oracle_mod.cluster_level(objs, None, cents, 3, 100, 2)
    loose = oracle_mod.cluster_level(objs, None, cents, 3, 100, 30, eps_tol=1.0)
    assert all(np.array_equal(a, b) for a, b in zip(two, loose))


def test_alg1_with_one_support_equals_the_constrained_update(oracle_mod):
    """With one support per centroid the weight LP has the single feasible
    point p = [1]: Alg. 1 and the constrained update coincide."""
    objs, _ = synth.image_like(N=160, K=3, seed=43)
    rng = np.random.default_rng(5)
    cents = synth._pack(np.ones(3, dtype=np.int64), rng.normal(0, 3, (3, objs.dim)),
                        np.ones(3), "f64", "f64")
    a = oracle_mod.cluster_level(objs, None, cents, 3, 80, 3, return_support_weights=True)
    b = oracle_mod.cluster_level(objs, None, cents, 3, 80, 3, update="alg1",
                                 return_support_weights=True)
    assert np.array_equal(a[2], b[2])
    assert np.allclose(a[0], b[0], rtol=1e-12, atol=1e-12) and np.allclose(a[3], b[3])


def test_alg1_weights_are_distributions_and_help(oracle_mod):
    """Alg. 1 moves the support weights away from the uniform start, and
    each centroid's weights stay a distribution."""
    objs, cents = synth.image_like(N=120, K=2, seed=44)
    loc, w, lab, sw = oracle_mod.cluster_level(objs, None, cents, 2, 200, 1, update="alg1",
                                               return_support_weights=True)
    off = np.asarray(cents.off)
    for j in range(2):
        assert abs(sw[off[j]:off[j + 1]].sum() - 1.0) < 1e-9 and (sw >= 0).all()
    assert not np.allclose(sw, np.asarray(cents.w, dtype=float))
