"""Pins of the oracle's initial data segmentation (Alg. 3 Step 1: binary
splits by constrained D2-clustering, Alg. 2 with Step 3* and k = 2), and of
the level loop that uses it."""
import numpy as np

from paper_1302_0435_gb300 import synth


def _bags_1d(points):
    """One single-support bag per point (d = 1)."""
    n = len(points)
    return synth._pack(np.ones(n, dtype=np.int64), np.asarray(points, dtype=np.float64).reshape(n, 1),
                       np.ones(n), "f64", "f64")


def test_identical_bags_fall_back_to_halves(oracle_mod):
    # every split is degenerate (z_2 = z_1, all labels 0): halves by member
    # order.  Hand-derived for N=10, tau=3: [0..9] -> [0..4] | [5..9];
    # tie between the two sizes-5 goes to the earlier one: [0,1] | [2,3,4];
    # then [5..9] -> [5,6] | [7,8,9]; ids by smallest member.
    pts = np.zeros(10)
    seg, M = oracle_mod.segment(_bags_1d(pts), None, 3, 5)
    assert M == 4
    assert seg.tolist() == [0, 0, 1, 1, 1, 2, 2, 3, 3, 3]


def test_split_is_two_means_for_single_supports(oracle_mod):
    # single-support bags: D^2 is the squared distance and the constrained
    # update is the weighted mean, so a split is 2-means from the
    # farthest-point start: z1 = 0, z2 = 12 -> {0,1,2} | {10,11,12}
    objs = _bags_1d([0.0, 10.0, 1.0, 11.0, 2.0, 12.0])
    a, b = oracle_mod.split_binary(objs, None, np.arange(6), 5)
    assert a.tolist() == [0, 2, 4] and b.tolist() == [1, 3, 5]


def test_split_weighted_mean_moves_the_boundary(oracle_mod):
    # weights pull the first centroid: points 0, 4, 5 and 10 with omega
    # 1, 1, 9, 1.  Start z1 = 0, z2 = 10: 4 -> z1, 5 -> z2 (|5-0| = |5-10|,
    # ties to the first centroid: 5 -> z1).  Update: z1 = (0 + 4 + 45)/11,
    # z2 = 10; then 5 stays with z1 and the split is {0, 4, 5} | {10}.
    objs = _bags_1d([0.0, 4.0, 5.0, 10.0])
    a, b = oracle_mod.split_binary(objs, np.array([1.0, 1.0, 9.0, 1.0]), np.arange(4), 5)
    assert a.tolist() == [0, 1, 2] and b.tolist() == [3]


def test_well_separated_groups_are_recovered(oracle_mod):
    # groups of 10 tight bags around (0,0), (100,0), (1000,0), (1100,0):
    # the first split's start pair lies in different halves {0,100} and
    # {1000,1100} (the farthest bag from any bag is in the far half), every
    # midpoint between the centroids falls between groups, so the split is
    # {0,100} | {1000,1100}; each half then splits into its two groups the
    # same way.  tau = 10 stops there.
    rng = np.random.default_rng(5)
    centres = np.array([[0.0, 0.0], [100.0, 0.0], [1000.0, 0.0], [1100.0, 0.0]])
    sizes = rng.integers(3, 7, size=40)
    grp = np.repeat(np.arange(4), 10)
    rng.shuffle(grp)
    locs = np.concatenate([centres[g] + rng.normal(0, 1.0, size=(m, 2)) for g, m in zip(grp, sizes)])
    w = np.concatenate([rng.dirichlet(np.ones(m)) for m in sizes])
    objs = synth._pack(sizes.astype(np.int64), locs, w, "f64", "f64")
    seg, M = oracle_mod.segment(objs, None, 10, 10)
    assert M == 4
    for s in range(M):  # each segment is exactly one group
        assert len(set(grp[seg == s])) == 1 and (seg == s).sum() == 10


def test_segments_partition_and_respect_tau(oracle_mod):
    objs, _ = synth.image_like(N=300, K=4, seed=17)
    seg, M = oracle_mod.segment(objs, None, 40, 4)
    assert seg.shape == (300,) and seg.min() == 0 and seg.max() == M - 1
    counts = np.bincount(seg, minlength=M)
    assert (counts >= 1).all() and (counts <= 40).all() and M >= 8
    first = [np.nonzero(seg == s)[0][0] for s in range(M)]
    assert first == sorted(first)  # numbered by smallest member


def test_constrained_level_equals_slices_when_one_segment(oracle_mod):
    objs, cents = synth.image_like(N=60, K=4, seed=18)
    a = oracle_mod.cluster_level(objs, None, cents, 4, 100, 3)
    b = oracle_mod.cluster_level(objs, None, cents, 4, 100, 3, segmentation="constrained")
    assert np.array_equal(a[2], b[2]) and np.allclose(a[0], b[0], rtol=0, atol=0)


def test_constrained_level_conserves_weight_and_labels_members(oracle_mod):
    objs, cents = synth.image_like(N=240, K=4, seed=19)
    omega = np.random.default_rng(2).uniform(0.5, 2.0, objs.count)
    loc, w, C = oracle_mod.cluster_level(objs, omega, cents, 4, 50, 3, segmentation="constrained",
                                         split_iters=4)
    assert abs(w.sum() - omega.sum()) <= 1e-9 * omega.sum()
    assert C.min() >= 0 and C.max() < 4
    assert np.allclose(np.bincount(C, weights=omega, minlength=4), w)


def test_split_order_does_not_change_the_partition(oracle_mod):
    """A split depends only on its own members, so splitting every segment
    above tau generation by generation (as the device batches them) gives
    the partition of largest-first splitting."""
    objs, _ = synth.image_like(N=260, K=2, seed=37)
    tau, iters = 40, 4
    ref, M = oracle_mod.segment(objs, None, tau, iters)
    segs = [np.arange(objs.count, dtype=np.int64)]
    while any(len(s) > tau for s in segs):
        nxt = []
        for s in segs:
            if len(s) > tau:
                a, b = oracle_mod.split_binary(objs, None, s, iters)
                nxt += [a, b]
            else:
                nxt.append(s)
        segs = nxt
    got = np.empty(objs.count, dtype=np.int64)
    for new_id, s in enumerate(sorted(segs, key=lambda s: int(s[0]))):
        got[s] = new_id
    assert len(segs) == M and np.array_equal(got, ref)
