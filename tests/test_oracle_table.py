"""Pins of the oracle's custom-cost variant (symbolic supports with a
pairwise symbol distance in place of the squared Euclidean cost)."""
import numpy as np


def _hist(rng, A, kmin=1):
    k = int(rng.integers(kmin, A + 1))
    s = np.sort(rng.choice(A, size=k, replace=False))
    return s, rng.dirichlet(np.full(k, 0.8))


def test_embedded_table_equals_euclidean(oracle_mod):
    # table = squared distances of an embedding: the same LP as the
    # Euclidean oracle on the embedded supports
    rng = np.random.default_rng(1)
    A = 12
    e = rng.normal(size=(A, 3))
    table = ((e[:, None, :] - e[None, :, :]) ** 2).sum(-1)
    for _ in range(30):
        xs, p = _hist(rng, A)
        ys, q = _hist(rng, A)
        v, _ = oracle_mod.mallows_table(xs, p, ys, q, table)
        ref = oracle_mod.mallows(e[xs], p, e[ys], q)[0]
        assert abs(v - ref) <= 1e-12 * max(1.0, ref)


def test_discrete_metric_is_total_variation(oracle_mod):
    # 0 on the diagonal, 1 elsewhere: D^2 = 1 - sum_s min(p_s, q_s)
    rng = np.random.default_rng(2)
    A = 20
    table = 1.0 - np.eye(A)
    for _ in range(40):
        xs, p = _hist(rng, A)
        ys, q = _hist(rng, A)
        P = np.zeros(A); P[xs] = p / p.sum()
        Q = np.zeros(A); Q[ys] = q / q.sum()
        v, _ = oracle_mod.mallows_table(xs, p, ys, q, table)
        assert abs(v - (1.0 - np.minimum(P, Q).sum())) <= 1e-12


def test_line_table_is_quantile_form(oracle_mod):
    # table (i - j)^2 on symbols 0..A-1: the 1-D closed form
    # D^2 = int_0^1 (F^-1(u) - G^-1(u))^2 du over the merged breakpoints
    rng = np.random.default_rng(3)
    A = 15
    idx = np.arange(A, dtype=float)
    table = (idx[:, None] - idx[None, :]) ** 2
    for _ in range(30):
        xs, p = _hist(rng, A)
        ys, q = _hist(rng, A)
        p = p / p.sum(); q = q / q.sum()
        cp, cq = np.cumsum(p), np.cumsum(q)
        u = np.unique(np.concatenate([[0.0], cp, cq]))
        u = u[u <= 1.0]
        ref = 0.0
        for lo, hi in zip(u[:-1], u[1:]):
            mid = 0.5 * (lo + hi)
            a = xs[min(np.searchsorted(cp, mid), len(xs) - 1)]
            b = ys[min(np.searchsorted(cq, mid), len(ys) - 1)]
            ref += (hi - lo) * (a - b) ** 2
        v, _ = oracle_mod.mallows_table(xs, p, ys, q, table)
        assert abs(v - ref) <= 1e-10 * max(1.0, ref)


def test_assign_table_ties_and_self(oracle_mod):
    from paper_1302_0435_gb300 import synth
    A = 6
    table = 1.0 - np.eye(A)
    # each bag's own histogram as a centroid: D^2 = 0 to itself
    sizes = np.array([2, 3, 1], dtype=np.int64)
    syms = np.array([0, 3, 1, 2, 5, 4], dtype=np.float32).reshape(-1, 1)
    w = np.array([0.5, 0.5, 0.2, 0.3, 0.5, 1.0], dtype=np.float32)
    objs = synth._pack(sizes, syms, w, "f32", "f32")
    lab, d2, allm = oracle_mod.assign_table(objs, objs, table)
    assert lab.tolist() == [0, 1, 2] and np.allclose(d2, 0.0)
    assert np.allclose(allm, allm.T)
