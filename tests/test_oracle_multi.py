"""Pins of the oracle's combined distance of several bag types
(Eq. (imgdist)), reduced to the single-type assignment."""
import numpy as np

from paper_1302_0435_gb300 import synth


def test_identical_types_double_the_distance(oracle_mod):
    objs, cents = synth.image_like(N=40, K=5, seed=71)
    lab1, d1 = oracle_mod.assign(objs, cents)
    lab2, d2, _ = oracle_mod.assign_multi([objs, objs], [cents, cents])
    assert np.array_equal(lab1, lab2)
    assert np.allclose(d2, 2.0 * d1, rtol=1e-15, atol=0)


def test_constant_second_type_reduces_to_the_first(oracle_mod):
    objs, cents = synth.image_like(N=40, K=5, seed=72)
    n, k = objs.count, cents.count
    one = synth._pack(np.ones(n, dtype=np.int64), np.zeros((n, 2)), np.ones(n), "f64", "f64")
    onec = synth._pack(np.ones(k, dtype=np.int64), np.zeros((k, 2)), np.ones(k), "f64", "f64")
    lab1, d1 = oracle_mod.assign(objs, cents)
    lab2, d2, _ = oracle_mod.assign_multi([objs, one], [cents, onec])
    assert np.array_equal(lab1, lab2) and np.array_equal(d1, d2)


def test_combined_labels_minimise_the_sum(oracle_mod):
    objs, cents = synth.image_two_bags(N=30, K=6, seed=73)
    lab, d, tot = oracle_mod.assign_multi(objs, cents)
    _, _, a = oracle_mod.assign(objs[0], cents[0], return_all=True)
    _, _, b = oracle_mod.assign(objs[1], cents[1], return_all=True)
    assert np.array_equal(tot, a + b)
    assert (d <= (a + b).min(axis=1) + 0.0).all() and np.array_equal(lab, np.argmin(a + b, axis=1))
