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
