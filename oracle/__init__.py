"""FP64 CPU oracle for the D2-clustering assignment step (arXiv 1302.0435).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import this package.  It shares no code
with paper_1302_0435_gb300/ and never imports it; inputs come from the
seeded generators, which hold none of the method's arithmetic.

Contents (each function cites the passage it follows):
  mallows            Eq. (D2opt) with z fixed: exact transportation LP (C).
  mallows_pairs      the same over a list of (object, centroid) pairs (C).
  assign             Alg. 2 Step 2, nearest centroid, ties to smallest j (C).
  update_locations   Eq. (WeightedUpdate) / Eq. (UpdateZ), numpy.
  update_label, update_global_label, propagate_weights
                     Eq. (UpdateLabel), Eq. (UpdateGlobalLabel) and the
                     weight rule of the weighted D2-clustering section.
  cluster_level      Alg. 3 levels with the segment-wise Alg. 2 loop.
  joint_lp, update_weights
                     Alg. 1 Step 1: the LP of Eq. (WeightedD2) over the
                     centroid weights and all flows of a cluster (HiGHS).

Bags are passed as any object with attributes ``loc`` ([T, d] array),
``w`` ([T]) and ``off`` ([N+1] int64, bag b = rows off[b]:off[b+1]).
Every function converts to float64 first.

Parity pins for every function live in tests/test_oracle_*.py (the joint
LP of Alg. 1 Step 1 in tests/test_oracle_joint.py); no function here is
"parity unpinned".
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None

OK = 0
EINVAL = -1
ENOMEM = -2
ENOTCONVERGED = -3


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.d2o_normalise.argtypes = [dp, ctypes.c_int64, dp]
        lib.d2o_cost.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64, ctypes.c_int32, dp]
        lib.d2o_cost.restype = None
        lib.d2o_transport.argtypes = [dp, dp, ctypes.c_int64, dp, ctypes.c_int64, dp, dp, dp, dp, ip]
        lib.d2o_mallows.argtypes = [dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int64, ctypes.c_int32,
                                    dp, dp, dp, dp, ip]
        lib.d2o_mallows_pairs.argtypes = [dp, dp, ip, dp, dp, ip, ctypes.c_int32, ip, ip,
                                          ctypes.c_int64, ctypes.c_int32, dp, i32p, ip]
        lib.d2o_assign.argtypes = [dp, dp, ip, ctypes.c_int64, dp, dp, ip, ctypes.c_int64,
                                   ctypes.c_int32, ctypes.c_int32, i32p, dp, dp]
        _LIB = lib
    return _LIB


def _p(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != OK:
        raise OracleError("%s failed with status %d" % (what, st))


def normalise(w):
    """Equal-mass rule of Eq. (D2opt): divide a bag's weights by their sum."""
    w = _f64(w)
    out = np.empty_like(w)
    _check(_lib().d2o_normalise(_p(w), w.size, _p(out)), "normalise")
    return out


def cost(x, y):
    """Ground cost of Eq. (D2opt): c[a, r] = ||x_a - y_r||^2 by explicit differences."""
    x = _f64(x)
    y = _f64(y)
    if x.ndim == 1:
        x = x[:, None]
    if y.ndim == 1:
        y = y[:, None]
    m, d = x.shape
    n = y.shape[0]
    C = np.empty((m, n))
    _lib().d2o_cost(_p(x), m, _p(y), n, d, _p(C))
    return C


def transport(C, p, q):
    """Exact transportation LP of Eq. (D2opt) with z fixed, for given cost and
    marginals (already normalised).  Returns (value, flow, u, v, pivots)."""
    C = _f64(C)
    p = _f64(p)
    q = _f64(q)
    m, n = C.shape
    w = np.empty((m, n))
    u = np.empty(m)
    v = np.empty(n)
    obj = np.empty(1)
    piv = np.zeros(1, dtype=np.int64)
    st = _lib().d2o_transport(_p(C), _p(p), m, _p(q), n, _p(w), _p(u), _p(v), _p(obj),
                              _p(piv, ctypes.c_int64))
    _check(st, "transport")
    return float(obj[0]), w, u, v, int(piv[0])


def mallows(x, wx, y, wy):
    """Mallows distance D^2 between bags (x, wx) and (y, wy): Eq. (D2opt) with
    z fixed.  Weights are normalised first.  Returns (D2, flow, u, v, pivots)."""
    x = _f64(x)
    y = _f64(y)
    if x.ndim == 1:
        x = x[:, None]
    if y.ndim == 1:
        y = y[:, None]
    wx = _f64(wx)
    wy = _f64(wy)
    m, d = x.shape
    n = y.shape[0]
    if y.shape[1] != d:
        raise ValueError("dimension mismatch")
    w = np.empty((m, n))
    u = np.empty(m)
    v = np.empty(n)
    d2 = np.empty(1)
    piv = np.zeros(1, dtype=np.int64)
    st = _lib().d2o_mallows(_p(x), _p(wx), m, _p(y), _p(wy), n, d, _p(d2), _p(w), _p(u), _p(v),
                            _p(piv, ctypes.c_int64))
    _check(st, "mallows")
    return float(d2[0]), w, u, v, int(piv[0])


def _bag_arrays(b):
    loc = _f64(b.loc)
    if loc.ndim == 1:
        loc = loc[:, None]
    return loc, _f64(b.w), _i64(b.off)


def mallows_table(xs, wx, ys, wy, table):
    """Mallows distance with a custom ground cost between symbols (the
    sequence variant of Eq. (D2opt): the squared Euclidean distance between
    supports is replaced by a pairwise symbol distance, here any
    nonnegative table[A][A]).  xs, ys: integer symbol ids of the supports.
    Weights are normalised first.  Returns (D2, flow)."""
    xs = np.asarray(xs, dtype=np.int64).ravel()
    ys = np.asarray(ys, dtype=np.int64).ravel()
    C = _f64(table)[np.ix_(xs, ys)]
    p = normalise(wx)
    q = normalise(wy)
    v, w, _, _, _ = transport(C, p, q)
    return v, w


def assign_table(objs, cents, table):
    """Alg. 2 Step 2 with the symbol cost table: labels (ties to the smallest
    j) and D^2 of every bag; supports are symbol ids (dim 1)."""
    N = len(objs.off) - 1
    K = len(cents.off) - 1
    allm = np.empty((N, K))
    for i in range(N):
        x, wx = bag(objs, i)
        for j in range(K):
            y, wy = bag(cents, j)
            allm[i, j] = mallows_table(x, wx, y, wy, table)[0]
    lab = np.argmin(allm, axis=1)  # first minimum
    return lab.astype(np.int32), allm[np.arange(N), lab], allm


def assign_multi(objs_list, cents_list, nthreads=1):
    """Alg. 2 Step 2 with the combined distance of several bag types
    (Eq. (imgdist)): D^2(I_i, Z_j) = sum_b D^2(U_i^b, Z_j^b); labels with
    ties to the smallest j.  objs_list[b] / cents_list[b] hold bag type b of
    every object / centroid.  Returns (labels, summed D^2, summed matrix)."""
    tot = None
    for objs, cents in zip(objs_list, cents_list):
        _, _, allm = assign(objs, cents, nthreads=nthreads, return_all=True)
        tot = allm if tot is None else tot + allm
    lab = np.argmin(tot, axis=1)
    return lab.astype(np.int32), tot[np.arange(tot.shape[0]), lab], tot


def bag(b, i):
    """Rows of bag i as (loc [m, d], w [m]) in float64."""
    lo, hi = int(b.off[i]), int(b.off[i + 1])
    loc = np.asarray(b.loc[lo:hi], dtype=np.float64)
    if loc.ndim == 1:
        loc = loc[:, None]
    return loc, np.asarray(b.w[lo:hi], dtype=np.float64)


def mallows_pairs(objs, cents, pair_obj, pair_cen, nthreads=1, return_pivots=False):
    """D^2 of Eq. (D2opt) for each listed (object, centroid) pair (and, if
    asked, the simplex pivot count of each pair)."""
    xl, xw, xo = _bag_arrays(objs)
    yl, yw, yo = _bag_arrays(cents)
    pi = _i64(pair_obj)
    pj = _i64(pair_cen)
    out = np.empty(pi.size)
    st = np.zeros(pi.size, dtype=np.int32)
    piv = np.zeros(pi.size, dtype=np.int64)
    rc = _lib().d2o_mallows_pairs(_p(xl), _p(xw), _p(xo, ctypes.c_int64), _p(yl), _p(yw),
                                  _p(yo, ctypes.c_int64), xl.shape[1], _p(pi, ctypes.c_int64),
                                  _p(pj, ctypes.c_int64), pi.size, nthreads, _p(out),
                                  _p(st, ctypes.c_int32), _p(piv, ctypes.c_int64))
    _check(rc, "mallows_pairs")
    if return_pivots:
        return out, piv
    return out


def assign(objs, cents, nthreads=1, return_all=False):
    """Alg. 2 Step 2: C(i) = argmin_j D(v_i, z_j), ties to the smallest j.
    Returns (labels int32 [N], dist2 [N]) and, if asked, the [N, K] D^2 matrix."""
    xl, xw, xo = _bag_arrays(objs)
    yl, yw, yo = _bag_arrays(cents)
    N = xo.size - 1
    K = yo.size - 1
    labels = np.empty(N, dtype=np.int32)
    dist2 = np.empty(N)
    allm = np.empty((N, K)) if return_all else None
    rc = _lib().d2o_assign(_p(xl), _p(xw), _p(xo, ctypes.c_int64), N, _p(yl), _p(yw),
                           _p(yo, ctypes.c_int64), K, xl.shape[1], nthreads,
                           _p(labels, ctypes.c_int32), _p(dist2), _p(allm) if allm is not None else None)
    _check(rc, "assign")
    if return_all:
        return labels, dist2, allm
    return labels, dist2


def assigned_flows(objs, cents, labels):
    """Optimal flows of each assigned pair (i, C(i)) as COO arrays
    (obj, alpha, r, w), from the oracle's own LP solutions (Eq. (D2opt))."""
    co, ca, cr, cw = [], [], [], []
    N = len(objs.off) - 1
    for i in range(N):
        x, wx = bag(objs, i)
        y, wy = bag(cents, int(labels[i]))
        _, w, _, _, _ = mallows(x, wx, y, wy)
        a, r = np.nonzero(w)
        co.append(np.full(a.size, i, dtype=np.int64))
        ca.append(a.astype(np.int64))
        cr.append(r.astype(np.int64))
        cw.append(w[a, r])
    if N == 0:
        z = np.zeros(0, dtype=np.int64)
        return z, z, z, np.zeros(0)
    return np.concatenate(co), np.concatenate(ca), np.concatenate(cr), np.concatenate(cw)


def update_locations(objs, omega, labels, flow_obj, flow_alpha, flow_r, flow_w, cents):
    """Eq. (WeightedUpdate) (Eq. (UpdateZ) when omega = 1), centroid weights
    held fixed (the constrained form of Alg. 2 Step 3*):

        z_j^(r) = sum_{i: C(i)=j} omega_i sum_a w_ra^(i) v_i^(a)
                  / sum_{i: C(i)=j} omega_i sum_a w_ra^(i)

    with the flows given as COO entries (object i, support a, centroid
    support r, flow w), summed in entry order.  Where the denominator is
    zero (empty cluster, or a support that receives no mass) the previous
    location is kept.  Returns the new [sum n_j, d] float64 locations."""
    xl, _, xo = _bag_arrays(objs)
    yl, _, yo = _bag_arrays(cents)
    N = xo.size - 1
    om = np.ones(N) if omega is None else _f64(omega)
    lab = np.asarray(labels, dtype=np.int64)
    fo = _i64(flow_obj)
    fa = _i64(flow_alpha)
    fr = _i64(flow_r)
    fw = _f64(flow_w)
    rows = yo[lab[fo]] + fr
    src = xo[fo] + fa
    coef = om[fo] * fw
    num = np.zeros_like(yl)
    den = np.zeros(yl.shape[0])
    np.add.at(num, rows, coef[:, None] * xl[src])
    np.add.at(den, rows, coef)
    new = yl.copy()
    ok = den > 0
    new[ok] = num[ok] / den[ok][:, None]
    return new


def update_label(seg_labels, seg_sizes_centroids):
    """Eq. (UpdateLabel): labels of segment mu are offset by the number of
    centroids merged before it, |Z^(mu-1)|.  seg_labels is a list of label
    arrays (one per segment, in segment order) and seg_sizes_centroids the
    number of centroids each segment produced.  Returns the offset labels."""
    out = []
    offset = 0
    for lab, k in zip(seg_labels, seg_sizes_centroids):
        out.append(np.asarray(lab, dtype=np.int64) + offset)
        offset += int(k)
    return out


def update_global_label(C, C_tilde):
    """Eq. (UpdateGlobalLabel): C(i) = C~(C(i)) for every original object."""
    return np.asarray(C_tilde, dtype=np.int64)[np.asarray(C, dtype=np.int64)]


def propagate_weights(C_tilde, omega, k_prime):
    """Weight of a parent point = sum of its children's weights (weighted
    D2-clustering section; Alg. 3 Step 3): omega_i = sum_{a: C~(a)=i} omega'_a."""
    out = np.zeros(int(k_prime))
    np.add.at(out, np.asarray(C_tilde, dtype=np.int64), _f64(omega))
    return out


class _Bags:
    def __init__(self, loc, w, off):
        self.loc = loc
        self.w = w
        self.off = off


def _slice_bags(b, lo, hi):
    o = np.asarray(b.off, dtype=np.int64)
    s, e = int(o[lo]), int(o[hi])
    return _Bags(np.asarray(b.loc[s:e]), np.asarray(b.w[s:e]), o[lo:hi + 1] - s)


def _take_bags(b, idx):
    """Bags idx of b (in the given order), repacked."""
    o = np.asarray(b.off, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    rows = [np.arange(o[i], o[i + 1]) for i in idx]
    rows = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    sizes = o[idx + 1] - o[idx]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return _Bags(np.asarray(b.loc)[rows], np.asarray(b.w)[rows], off)


def _uniform_bag(b, i):
    """Bag i of b as a centroid of the constrained form: its supports with
    uniform weights 1/s (Alg. 2 Step 3*)."""
    x, _ = bag(b, i)
    return _Bags(x.copy(), np.full(len(x), 1.0 / len(x)), np.array([0, len(x)], dtype=np.int64))


def _join_bags(parts):
    locs = np.concatenate([np.asarray(p.loc, dtype=np.float64).reshape(len(p.w), -1) for p in parts])
    ws = np.concatenate([np.asarray(p.w, dtype=np.float64) for p in parts])
    offs = np.concatenate([[0], np.cumsum([len(p.w) for p in parts])]).astype(np.int64)
    return _Bags(locs, ws, offs)


def split_binary(objs, omega, members, iters, nthreads=1):
    """One binary split of the initial data segmentation (Alg. 3 Step 1, the
    constrained D2-clustering of Alg. 2 with Step 3* and k = 2).

    Start: z_1 is the first member's bag and z_2 the member's bag with the
    largest D^2 to z_1 (ties to the earlier member), both with uniform
    weights.  Then assign (Alg. 2 Step 2); up to `iters` times update the
    locations with the weights held fixed (Eq. (WeightedUpdate)) and assign
    again, stopping early when the labels repeat.  Returns the members
    labelled 0 and 1; if one side is empty, the first and second halves.
    """
    members = np.asarray(members, dtype=np.int64)
    sub = _take_bags(objs, members)
    om = np.ones(len(members)) if omega is None else _f64(omega)[members]
    z1 = _uniform_bag(sub, 0)
    _, d1 = assign(sub, z1, nthreads=nthreads)
    i2 = int(np.argmax(d1))  # first index of the largest value
    cents = _join_bags([z1, _uniform_bag(sub, i2)])
    lab, _ = assign(sub, cents, nthreads=nthreads)
    for _ in range(int(iters)):
        fo, fa, fr, fw = assigned_flows(sub, cents, lab)
        cents = _Bags(update_locations(sub, om, lab, fo, fa, fr, fw, cents), cents.w, cents.off)
        new, _ = assign(sub, cents, nthreads=nthreads)
        if np.array_equal(new, lab):
            break
        lab = new
    a, b = members[lab == 0], members[lab == 1]
    if len(a) == 0 or len(b) == 0:
        h = len(members) // 2
        a, b = members[:h], members[h:]
    return a, b


def segment(objs, omega, tau, iters, nthreads=1):
    """Initial data segmentation of Alg. 3 Step 1: repeatedly split the
    segment holding the most objects (ties: the one created first) into two
    with split_binary, until no segment holds more than tau objects.  A split
    keeps the first part in the parent's place and appends the second.
    Returns (segment id per object [N] int64, number of segments); segments
    are numbered in increasing order of their smallest member."""
    N = len(objs.off) - 1
    segs = [np.arange(N, dtype=np.int64)]
    while True:
        big = max(range(len(segs)), key=lambda k: (len(segs[k]), -k))
        if len(segs[big]) <= tau:
            break
        a, b = split_binary(objs, omega, segs[big], iters, nthreads=nthreads)
        segs[big] = a
        segs.append(b)
    order = sorted(range(len(segs)), key=lambda k: int(segs[k][0]))
    seg_id = np.empty(N, dtype=np.int64)
    for new_id, k in enumerate(order):
        seg_id[segs[k]] = new_id
    return seg_id, len(segs)


def joint_lp(costs, qs, omega):
    """Alg. 1 Step 1 for one cluster: with the support locations z^(r) fixed,
    minimise Eq. (WeightedD2), sum_i omega_i sum_{r,a} c^(i)_{ra} w^(i)_{ra},
    over the centroid weights p_z and every member's flows w^(i), under the
    constraints of Eq. (D2opt): sum_r p_r = 1, sum_a w^(i)_{ra} = p_r for
    every member i and support r, sum_r w^(i)_{ra} = q^(i)_a, p, w >= 0.
    The LP is written out whole (variables p first, then each member's
    w^(i) row-major in (r, a)) and handed to a library dual simplex (HiGHS
    through scipy) at tight tolerances.  costs[i]: [s', t_i] array of
    c^(i)_{ra}; qs[i]: member i's normalised weights; omega: [n'].
    Returns (epsilon, p) with p clamped at 0."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    s = costs[0].shape[0]
    nvar = s + sum(c.size for c in costs)
    obj = np.zeros(nvar)
    ri, ci, vals, rhs = [], [], [], []
    row = 0
    ri += [0] * s
    ci += list(range(s))
    vals += [1.0] * s
    rhs.append(1.0)
    row = 1
    col = s
    for c, q, om in zip(costs, qs, omega):
        c = np.asarray(c, dtype=np.float64)
        t = c.shape[1]
        obj[col:col + c.size] = om * c.ravel()
        for r in range(s):                       # sum_a w_ra - p_r = 0
            ri += [row] * (t + 1)
            ci += list(range(col + r * t, col + (r + 1) * t)) + [r]
            vals += [1.0] * t + [-1.0]
            rhs.append(0.0)
            row += 1
        for a in range(t):                       # sum_r w_ra = q_a
            ri += [row] * s
            ci += list(range(col + a, col + c.size, t))
            vals += [1.0] * s
            rhs.append(float(q[a]))
            row += 1
        col += c.size
    A = coo_matrix((vals, (ri, ci)), shape=(row, nvar)).tocsr()
    res = linprog(obj, A_eq=A, b_eq=np.array(rhs), bounds=(0, None), method="highs-ds",
                  options=dict(primal_feasibility_tolerance=1e-10,
                               dual_feasibility_tolerance=1e-10))
    if res.status != 0:
        raise RuntimeError("joint LP: " + res.message)
    return float(res.fun), np.maximum(res.x[:s], 0.0)


def update_weights(objs, omega, labels, cents):
    """Alg. 1 Step 1 for every cluster (Eq. (WeightedD2) under the
    constraints of Eq. (D2opt)): the new centroid weights p_z of each
    centroid j, from its members i with C(i) = j, with the supports of z_j
    fixed.  Empty clusters keep their weights and get epsilon 0.  Returns
    (weights [sum n_j] float64, epsilon [K])."""
    xl, xw, xo = _bag_arrays(objs)
    yl, yw, yo = _bag_arrays(cents)
    N = xo.size - 1
    K = yo.size - 1
    om = np.ones(N) if omega is None else _f64(omega)
    lab = np.asarray(labels, dtype=np.int64)
    wout = yw.copy()
    eps = np.zeros(K)
    for j in range(K):
        mem = np.nonzero(lab == j)[0]
        if mem.size == 0:
            continue
        z = yl[yo[j]:yo[j + 1]]
        cs, qs = [], []
        for i in mem:
            x = xl[xo[i]:xo[i + 1]]
            cs.append(cost(z, x))
            qs.append(normalise(xw[xo[i]:xo[i + 1]]))
        eps[j], wout[yo[j]:yo[j + 1]] = joint_lp(cs, qs, om[mem])
    return wout, eps


def cluster_level(objs, omega, init_cents, K, seg_size, iters, loc_round=None, nthreads=1,
                  segmentation="slices", split_iters=10, eps_tol=0.0, update="constrained",
                  return_support_weights=False):
    """Alg. 3 level loop with the segment-wise weighted D2-clustering of
    Alg. 2 (constrained update, Step 3*) inside each segment.

    Level loop: split the current data into contiguous segments of at most
    seg_size (tau) objects; in each segment start from init_cents and run
    `iters` rounds of (Alg. 2 Step 2 assign, Eq. (WeightedUpdate) update);
    merge labels with Eq. (UpdateLabel) and Eq. (UpdateGlobalLabel); give
    each centroid the summed weight of its members; if more than one segment
    was used, the merged centroids become the next level's weighted data.
    Stops after the level that fits in one segment.  After each update the
    locations are rounded to loc_round (e.g. np.float32) when given, so that
    every level's data keep the input location precision.
    segmentation="constrained" forms each level's segments with the binary
    constrained D2 splits of Alg. 3 Step 1 (segment(), split_iters rounds per
    split) instead of contiguous slices; segment mu's labels are offset by
    mu*K (Eq. (UpdateLabel) with its index list L_mu).
    eps_tol > 0 ends a level's rounds after the first round r >= 1 whose
    level objective eps_r = sum_i omega_i D^2(v_i, z_C(i)) (over all its
    segments, from round r's assignment) is within eps_tol relative of
    eps_{r-1} (Alg. 2 Step 4, "until epsilon converges"); the segments run
    their rounds in step.
    update="alg1" updates each cluster by Alg. 1 (the weighted D2-clustering
    of Alg. 3 Step 2): Step 1 re-solves the support weights by the joint LP
    (update_weights), Step 2 moves the supports with the members' optimal
    flows at those weights; the next level's data carry the weights.
    return_support_weights adds the result's support weights to the tuple.

    Returns (centroid locations [K*n, d] float64, centroid weights [K],
    labels [N] int64)."""
    K = int(K)
    if seg_size <= K:
        raise ValueError("segment size must exceed K for the hierarchy to shrink")
    data = _Bags(np.asarray(objs.loc), np.asarray(objs.w), np.asarray(objs.off, dtype=np.int64))
    N0 = len(data.off) - 1
    om = np.ones(N0) if omega is None else _f64(omega)
    C = np.arange(N0, dtype=np.int64)
    while True:
        n_l = len(data.off) - 1
        if segmentation == "constrained" and n_l > seg_size:
            seg_id, M = segment(data, om, seg_size, split_iters, nthreads=nthreads)
            members = [np.nonzero(seg_id == mu)[0] for mu in range(M)]
        else:
            M = 1 if n_l <= seg_size else int(math.ceil(n_l / seg_size))
            members = [np.arange(mu * seg_size, min((mu + 1) * seg_size, n_l)) for mu in range(M)]
        segs = [_take_bags(data, members[mu]) for mu in range(M)]
        oms = [om[members[mu]] for mu in range(M)]
        seg_cents = [_Bags(_f64(init_cents.loc).copy(), _f64(init_cents.w).copy(),
                           _i64(init_cents.off).copy()) for _ in range(M)]
        seg_labels = [None] * M
        eps_prev = None
        for _ in range(int(iters)):
            eps = 0.0
            for mu in range(M):
                seg, cents = segs[mu], seg_cents[mu]
                lab, dist2 = assign(seg, cents, nthreads=nthreads)
                eps += float(np.sum(oms[mu] * dist2))
                if update == "alg1":
                    wj, _ = update_weights(seg, oms[mu], lab, cents)
                    cents = _Bags(cents.loc, wj, cents.off)
                fo, fa, fr, fw = assigned_flows(seg, cents, lab)
                newloc = update_locations(seg, oms[mu], lab, fo, fa, fr, fw, cents)
                if loc_round is not None:
                    newloc = newloc.astype(loc_round).astype(np.float64)
                seg_cents[mu] = _Bags(newloc, cents.w, cents.off)
                seg_labels[mu] = lab
            if eps_tol > 0 and eps_prev is not None and abs(eps - eps_prev) <= eps_tol * eps:
                break
            eps_prev = eps
        for mu in range(M):
            if seg_labels[mu] is None:
                seg_labels[mu], _ = assign(segs[mu], seg_cents[mu], nthreads=nthreads)
        C_tilde = np.empty(n_l, dtype=np.int64)
        for mu, lab_mu in zip(range(M), update_label(seg_labels, [K] * M)):
            C_tilde[members[mu]] = lab_mu
        C = update_global_label(C, C_tilde)
        w_new = propagate_weights(C_tilde, om, M * K)
        if M == 1:
            c0 = seg_cents[0]
            if return_support_weights:
                return _f64(c0.loc), w_new, C, _f64(c0.w)
            return _f64(c0.loc), w_new, C
        locs = np.concatenate([c.loc for c in seg_cents])
        ws = np.concatenate([c.w for c in seg_cents])
        n_per = [np.diff(c.off) for c in seg_cents]
        offs = np.concatenate([[0], np.cumsum(np.concatenate(n_per))]).astype(np.int64)
        data = _Bags(locs, ws, offs)
        om = w_new
