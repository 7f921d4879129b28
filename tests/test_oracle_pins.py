"""Pins for the FP64 oracle's Mallows distance (Eq. (D2opt) with z fixed).

Each pin is independent of the oracle's own code: brute-force enumeration of
the LP's vertices, the 1-D quantile closed form, the assignment form for
uniform weights, an LP library solver (HiGHS) as an outside referee, hand-
derived values, LP duality, and metric / geometric invariants.  A dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of these.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_bag(rng, m, d, alpha=1.0, spread=2.0):
    x = rng.normal(0.0, spread, size=(m, d))
    w = rng.dirichlet(np.full(m, alpha))
    return x, w


def _cost_by_hand(x, y):
    # squared Euclidean ground cost written out independently of the oracle
    m, n = x.shape[0], y.shape[0]
    C = np.zeros((m, n))
    for a in range(m):
        for r in range(n):
            C[a, r] = float(np.sum((x[a] - y[r]) ** 2))
    return C


def brute_force_vertices(C, p, q):
    """Minimum of the transportation LP over all its vertices.  A vertex is a
    basic solution: m+n-1 cells forming a spanning tree of the bipartite
    row/column graph, whose flows are then fixed by the marginals."""
    m, n = C.shape
    cells = [(a, r) for a in range(m) for r in range(n)]
    b = np.concatenate([p, q])
    best = math.inf
    for subset in itertools.combinations(range(m * n), m + n - 1):
        parent = list(range(m + n))

        def find(z):
            while parent[z] != z:
                parent[z] = parent[parent[z]]
                z = parent[z]
            return z
        tree = True
        for t in subset:
            a, r = cells[t]
            ra, rb = find(a), find(m + r)
            if ra == rb:
                tree = False
                break
            parent[ra] = rb
        if not tree:
            continue
        A = np.zeros((m + n, m + n - 1))
        for k, t in enumerate(subset):
            a, r = cells[t]
            A[a, k] = 1.0
            A[m + r, k] = 1.0
        w, *_ = np.linalg.lstsq(A, b, rcond=None)
        if np.max(np.abs(A @ w - b)) > 1e-12 or np.min(w) < -1e-13:
            continue
        val = sum(w[k] * C[cells[t]] for k, t in enumerate(subset))
        best = min(best, val)
    return best


def quantile_closed_form(x, p, y, q):
    """1-D: D^2 = int_0^1 (F^-1(u) - G^-1(u))^2 du with F, G the CDFs."""
    ix, iy = np.argsort(x, kind="stable"), np.argsort(y, kind="stable")
    x, p = x[ix], p[ix] / p.sum()
    y, q = y[iy], q[iy] / q.sum()
    Fx, Fy = np.cumsum(p), np.cumsum(q)
    Fx[-1] = Fy[-1] = 1.0
    bps = np.unique(np.concatenate([[0.0], Fx, Fy]))
    total = 0.0
    for lo, hi in zip(bps[:-1], bps[1:]):
        mid = 0.5 * (lo + hi)
        a = min(int(np.searchsorted(Fx, mid)), x.size - 1)
        r = min(int(np.searchsorted(Fy, mid)), y.size - 1)
        total += (hi - lo) * (x[a] - y[r]) ** 2
    return total


# ---------------------------------------------------------------- golden --

def test_hand_examples(oracle_mod):
    with open(os.path.join(HERE, "golden", "hand_examples.json")) as f:
        g = json.load(f)
    for ex in g["mallows"]:
        d2 = oracle_mod.mallows(ex["x"], ex["wx"], ex["y"], ex["wy"])[0]
        assert d2 == pytest.approx(ex["d2"], rel=1e-14, abs=1e-14), ex["name"]


# ------------------------------------------------------------ brute force --

@pytest.mark.parametrize("m,n", [(1, 1), (1, 3), (2, 2), (2, 3), (3, 2), (3, 3)])
def test_vertex_enumeration_small(oracle_mod, m, n):
    rng = np.random.default_rng(100 + 10 * m + n)
    for trial in range(40):
        d = int(rng.integers(1, 4))
        x, p = _rand_bag(rng, m, d)
        y, q = _rand_bag(rng, n, d)
        if trial % 5 == 0:  # degenerate weights: equal partial sums, zeros
            q = np.full(n, 1.0 / n)
            p = np.full(m, 1.0 / m)
        if trial % 7 == 0 and m > 1:
            p[0] = 0.0
            p /= p.sum()
        d2 = oracle_mod.mallows(x, p, y, q)[0]
        C = _cost_by_hand(x, y)
        bf = brute_force_vertices(C, p / p.sum(), q / q.sum())
        assert d2 == pytest.approx(bf, rel=1e-12, abs=1e-13)


def test_vertex_enumeration_4x4(oracle_mod):
    rng = np.random.default_rng(44)
    for _ in range(3):
        x, p = _rand_bag(rng, 4, 2)
        y, q = _rand_bag(rng, 4, 2)
        d2 = oracle_mod.mallows(x, p, y, q)[0]
        bf = brute_force_vertices(_cost_by_hand(x, y), p, q)
        assert d2 == pytest.approx(bf, rel=1e-12, abs=1e-13)


# -------------------------------------------------------- 1-D closed form --

def test_one_dimensional_quantile_form(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(60):
        m, n = int(rng.integers(1, 25)), int(rng.integers(1, 25))
        x, p = _rand_bag(rng, m, 1)
        y, q = _rand_bag(rng, n, 1, alpha=0.5)
        d2 = oracle_mod.mallows(x, p, y, q)[0]
        ref = quantile_closed_form(x[:, 0], p, y[:, 0], q)
        assert d2 == pytest.approx(ref, rel=1e-11, abs=1e-13)


# -------------------------------------------- assignment form (uniform) --

def test_uniform_weights_is_best_permutation(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(20):
        k = int(rng.integers(1, 7))
        d = int(rng.integers(1, 5))
        x = rng.normal(size=(k, d))
        y = rng.normal(size=(k, d))
        u = np.full(k, 1.0 / k)
        d2 = oracle_mod.mallows(x, u, y, u)[0]
        C = _cost_by_hand(x, y)
        best = min(sum(C[i, pi[i]] for i in range(k)) for pi in itertools.permutations(range(k))) / k
        assert d2 == pytest.approx(best, rel=1e-12, abs=1e-13)


# --------------------------------------------------------- single support --

def test_single_support_closed_form(oracle_mod):
    rng = np.random.default_rng(12)
    for _ in range(20):
        m, d = int(rng.integers(1, 30)), int(rng.integers(1, 8))
        x, p = _rand_bag(rng, m, d)
        y = rng.normal(size=(1, d))
        d2 = oracle_mod.mallows(x, p, y, [1.0])[0]
        ref = float(np.sum(p * np.sum((x - y) ** 2, axis=1)))
        assert d2 == pytest.approx(ref, rel=1e-13)
        d2t = oracle_mod.mallows(y, [2.5], x, p * 3.0)[0]  # transposed roles
        assert d2t == pytest.approx(ref, rel=1e-13)


# ------------------------------------------------------- outside referee --

def test_against_highs_lp(oracle_mod):
    linprog = pytest.importorskip("scipy.optimize").linprog
    rng = np.random.default_rng(13)
    for _ in range(25):
        m, n = int(rng.integers(1, 14)), int(rng.integers(1, 14))
        d = int(rng.integers(1, 7))
        x, p = _rand_bag(rng, m, d, alpha=0.5)
        y, q = _rand_bag(rng, n, d)
        C = _cost_by_hand(x, y)
        A = np.zeros((m + n, m * n))
        for a in range(m):
            A[a, a * n:(a + 1) * n] = 1.0
        for r in range(n):
            A[m + r, r::n] = 1.0
        b = np.concatenate([p / p.sum(), q / q.sum()])
        res = linprog(C.ravel(), A_eq=A, b_eq=b, bounds=(0, None), method="highs",
                      options={"primal_feasibility_tolerance": 1e-10,
                               "dual_feasibility_tolerance": 1e-10})
        assert res.status == 0
        d2 = oracle_mod.mallows(x, p, y, q)[0]
        assert d2 == pytest.approx(res.fun, rel=1e-8, abs=1e-10)


# ------------------------------------------------ duality certificate --

def test_duality_certificate(oracle_mod):
    rng = np.random.default_rng(14)
    for _ in range(30):
        m, n, d = int(rng.integers(1, 40)), int(rng.integers(1, 40)), int(rng.integers(1, 9))
        x, p = _rand_bag(rng, m, d, alpha=0.5)
        y, q = _rand_bag(rng, n, d)
        d2, w, u, v, _ = oracle_mod.mallows(x, p, y, q)
        C = _cost_by_hand(x, y)
        pn, qn = p / p.sum(), q / q.sum()
        scale = max(1.0, C.max())
        assert np.all(w >= 0.0)
        assert np.allclose(w.sum(axis=1), pn, atol=1e-14)
        assert np.allclose(w.sum(axis=0), qn, atol=1e-14)
        assert np.all(u[:, None] + v[None, :] <= C + 1e-11 * scale)      # dual feasible
        assert float(pn @ u + qn @ v) == pytest.approx(d2, rel=1e-11, abs=1e-12)  # no gap
        assert float(np.sum(w * C)) == pytest.approx(d2, rel=1e-12, abs=1e-13)


# ----------------------------------------------------------- invariants --

def test_metric_axioms(oracle_mod):
    rng = np.random.default_rng(15)
    for _ in range(30):
        d = int(rng.integers(1, 6))
        bags = [_rand_bag(rng, int(rng.integers(1, 12)), d) for _ in range(3)]
        D = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                D[i, j] = math.sqrt(max(0.0, oracle_mod.mallows(*bags[i], *bags[j])[0]))
        assert D[0, 0] == pytest.approx(0.0, abs=1e-7)  # sqrt of ~1e-16
        assert oracle_mod.mallows(*bags[1], *bags[1])[0] == pytest.approx(0.0, abs=1e-13)
        assert np.allclose(D, D.T, rtol=1e-12, atol=1e-12)
        for i, j, k in itertools.permutations(range(3)):
            assert D[i, k] <= D[i, j] + D[j, k] + 1e-12


def test_support_permutation_invariance(oracle_mod):
    rng = np.random.default_rng(16)
    for _ in range(20):
        m, n, d = int(rng.integers(1, 20)), int(rng.integers(1, 20)), 3
        x, p = _rand_bag(rng, m, d)
        y, q = _rand_bag(rng, n, d)
        a = oracle_mod.mallows(x, p, y, q)[0]
        px, py = rng.permutation(m), rng.permutation(n)
        b = oracle_mod.mallows(x[px], p[px], y[py], q[py])[0]
        assert b == pytest.approx(a, rel=1e-12, abs=1e-13)


def test_translation_identity_and_bounds(oracle_mod):
    rng = np.random.default_rng(17)
    for _ in range(30):
        m, n, d = int(rng.integers(1, 20)), int(rng.integers(1, 20)), int(rng.integers(1, 6))
        x, p = _rand_bag(rng, m, d)
        y, q = _rand_bag(rng, n, d)
        t = rng.normal(size=d)
        base = oracle_mod.mallows(x, p, y, q)[0]
        mu_p = (p / p.sum()) @ x
        mu_q = (q / q.sum()) @ y
        shifted = oracle_mod.mallows(x + t, p, y, q)[0]
        assert shifted == pytest.approx(base + t @ t + 2 * t @ (mu_p - mu_q), rel=1e-10, abs=1e-10)
        lower = float(np.sum((mu_p - mu_q) ** 2))
        upper = float((p / p.sum()) @ _cost_by_hand(x, y) @ (q / q.sum()))
        assert lower - 1e-12 <= base <= upper + 1e-12


def test_argmin_smallest_index_on_ties(oracle_mod):
    from paper_1302_0435_gb300.synth import Bags
    rng = np.random.default_rng(18)
    x, p = _rand_bag(rng, 5, 2)
    y0, q0 = _rand_bag(rng, 4, 2)
    y1, q1 = _rand_bag(rng, 4, 2, spread=0.1)
    # centroids 1 and 3 are the same bag; 3 must never win over 1
    cy = np.concatenate([y0, y1, y0 + 10.0, y1])
    cq = np.concatenate([q0, q1, q0, q1])
    cents = Bags(cy, cq, np.array([0, 4, 8, 12, 16]))
    objs = Bags(np.concatenate([x, y1]), np.concatenate([p, q1]), np.array([0, 5, 9]))
    labels, dist2, allm = oracle_mod.assign(objs, cents, return_all=True)
    assert allm[1, 1] == allm[1, 3]
    assert labels[1] == 1 and dist2[1] == pytest.approx(0.0, abs=1e-13)
    for i in range(2):
        assert labels[i] == int(np.argmin(allm[i]))


def test_rejects_bad_weights(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.mallows([[0.0]], [0.0], [[1.0]], [1.0])
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.mallows([[0.0], [1.0]], [0.5, -0.1], [[1.0]], [1.0])
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.mallows([[0.0]], [float("nan")], [[1.0]], [1.0])
