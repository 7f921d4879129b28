"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CUDA path, the tests and the FP64 oracle's
callers.  It only draws random numbers and packs them into ragged (CSR)
bags: it holds none of the method's arithmetic (no normalisation, no cost,
no LP).  The paper's image, video and sequence datasets are not available,
so these laws stand in for them:

  plain_small   N=1000 bags, 4-8 supports, d=3, 5-component Gaussian mixture
                (sd 1, means uniform in [-5,5]^d), Dirichlet(1) weights, FP64;
                K=8 centroids of 8 supports.
  image_like    N=200k bags, 8-16 supports, d=6 (3 colour + 3 texture
                coordinates as one bag), 32-component mixture,
                Dirichlet(0.5) weights, FP32; K=64 centroids of 16 supports.
  uneven        N=1M bags, support size P(m) ~ m^-2 on 2..64, d=16: N(0, I)
                plus one of 256 cluster offsets drawn from N(0, 9 I),
                Dirichlet(1) weights, FP32; K=256 centroids of 32 supports.
  high_dim      N=100k bags, 16-64 supports, d=128 nonnegative descriptors
                (|N(0,1)| then L2-normalised per vector), BF16 locations,
                Dirichlet(1) FP32 weights; K=512 centroids of 64 supports.
  serving       requests of log-uniform size on [1, 4096] bags, 4-64
                supports, d=32, 32-component mixture, Dirichlet(1), FP32;
                K=1024 resident centroids of 32 supports.

Every object draws one mixture component and all its supports from it, so
objects form clusters.  Centroids draw their supports from the same
location law and carry uniform weights 1/n.  Generator: numpy PCG64 with
seed 1000 + config number unless given.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Bags:
    """Ragged bags of weighted vectors.  Bag b owns rows off[b]:off[b+1] of
    loc ([T, d]) and w ([T]).  loc holds the exact values in a numpy float
    type; for BF16 data, loc holds the float32 values of the BF16 numbers
    and loc_bits their raw 16-bit patterns."""
    loc: np.ndarray
    w: np.ndarray
    off: np.ndarray
    loc_dtype: str = "f64"          # "f64" | "f32" | "bf16"
    w_dtype: str = "f64"            # "f64" | "f32"
    loc_bits: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def count(self) -> int:
        return int(self.off.size - 1)

    @property
    def dim(self) -> int:
        return int(self.loc.shape[1])

    def sizes(self) -> np.ndarray:
        return np.diff(self.off)

    def subset(self, idx) -> "Bags":
        """Bags idx (in the given order), repacked."""
        idx = np.asarray(idx, dtype=np.int64)
        sz = self.sizes()[idx]
        off = np.zeros(idx.size + 1, dtype=np.int64)
        np.cumsum(sz, out=off[1:])
        rows = np.concatenate([np.arange(self.off[i], self.off[i + 1]) for i in idx]) \
            if idx.size else np.zeros(0, dtype=np.int64)
        bits = self.loc_bits[rows] if self.loc_bits is not None else None
        return Bags(self.loc[rows], self.w[rows], off, self.loc_dtype, self.w_dtype, bits)


def f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even); returns bits."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    return ((u + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def _pack(sizes, loc, w, loc_dtype, w_dtype, bits=None) -> Bags:
    off = np.zeros(sizes.size + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return Bags(loc, w, off, loc_dtype, w_dtype, bits)


def _dirichlet_ragged(rng, sizes, alpha, dtype):
    """Dirichlet(alpha) per bag via normalised Gamma draws (sampling only;
    the method's own renormalisation happens in the consumers)."""
    g = rng.gamma(alpha, 1.0, size=int(sizes.sum()))
    seg = np.repeat(np.arange(sizes.size), sizes)
    tot = np.bincount(seg, weights=g, minlength=sizes.size)
    tot[tot == 0] = 1.0
    return (g / tot[seg]).astype(dtype)


def _mixture_bags(rng, sizes, d, ncomp, spread, dtype, comp_means=None):
    means = comp_means if comp_means is not None else rng.uniform(-spread, spread, size=(ncomp, d))
    comp = rng.integers(0, means.shape[0], size=sizes.size)
    rows = np.repeat(comp, sizes)
    loc = means[rows] + rng.standard_normal(size=(rows.size, d))
    return loc.astype(dtype), means


def _uniform_centroids(rng, K, n, d, means, dtype, w_dtype):
    sizes = np.full(K, n, dtype=np.int64)
    comp = rng.integers(0, means.shape[0], size=K)
    loc = means[np.repeat(comp, n)] + rng.standard_normal(size=(K * n, d))
    w = np.full(K * n, 1.0 / n, dtype=w_dtype)
    return _pack(sizes, loc.astype(dtype), w, "f64" if dtype == np.float64 else "f32",
                 "f64" if w_dtype == np.float64 else "f32")


def plain_small(N=1000, K=8, seed=1001):
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(4, 9, size=N).astype(np.int64)
    loc, means = _mixture_bags(rng, sizes, 3, 5, 5.0, np.float64)
    w = _dirichlet_ragged(rng, sizes, 1.0, np.float64)
    objs = _pack(sizes, loc, w, "f64", "f64")
    cents = _uniform_centroids(rng, K, 8, 3, means, np.float64, np.float64)
    return objs, cents


def image_like(N=200_000, K=64, seed=1002, n=16):
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(8, 17, size=N).astype(np.int64)
    loc, means = _mixture_bags(rng, sizes, 6, 32, 5.0, np.float32)
    w = _dirichlet_ragged(rng, sizes, 0.5, np.float32)
    objs = _pack(sizes, loc, w, "f32", "f32")
    cents = _uniform_centroids(rng, K, n, 6, means, np.float32, np.float32)
    return objs, cents


def uneven_sizes(rng, N, lo=2, hi=64, alpha=2.0):
    ms = np.arange(lo, hi + 1)
    p = ms.astype(np.float64) ** (-alpha)
    p /= p.sum()
    return rng.choice(ms, size=N, p=p).astype(np.int64)


def uneven(N=1_000_000, K=256, seed=1003, n=32):
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = uneven_sizes(rng, N)
    d = 16
    offsets = rng.normal(0.0, 3.0, size=(256, d))
    comp = rng.integers(0, 256, size=N)
    loc = (offsets[np.repeat(comp, sizes)]
           + rng.standard_normal(size=(int(sizes.sum()), d))).astype(np.float32)
    w = _dirichlet_ragged(rng, sizes, 1.0, np.float32)
    objs = _pack(sizes, loc, w, "f32", "f32")
    cc = rng.integers(0, 256, size=K)
    cloc = (offsets[np.repeat(cc, n)] + rng.standard_normal(size=(K * n, d))).astype(np.float32)
    cents = _pack(np.full(K, n, dtype=np.int64), cloc, np.full(K * n, 1.0 / n, np.float32),
                  "f32", "f32")
    return objs, cents


def _descriptors(rng, rows, d):
    a = np.abs(rng.standard_normal(size=(rows, d))).astype(np.float32)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    bits = f32_to_bf16_bits(a)
    return bf16_bits_to_f32(bits), bits


def high_dim(N=100_000, K=512, seed=1004, n=64):
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(16, 65, size=N).astype(np.int64)
    loc, bits = _descriptors(rng, int(sizes.sum()), 128)
    w = _dirichlet_ragged(rng, sizes, 1.0, np.float32)
    objs = _pack(sizes, loc, w, "bf16", "f32", bits)
    cloc, cbits = _descriptors(rng, K * n, 128)
    cents = _pack(np.full(K, n, dtype=np.int64), cloc, np.full(K * n, 1.0 / n, np.float32),
                  "bf16", "f32", cbits)
    return objs, cents


def serving_centroids(K=1024, seed=1005, n=32):
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-5.0, 5.0, size=(32, 32))
    cents = _uniform_centroids(rng, K, n, 32, means, np.float32, np.float32)
    return cents, means


def serving_request(rng, means, size=None):
    """One assignment request: `size` bags (log-uniform on [1, 4096] when not
    given), 4-64 supports, d=32 mixture locations, Dirichlet(1) weights."""
    if size is None:
        size = int(np.floor(np.exp(rng.uniform(0.0, np.log(4097.0)))))
        size = max(1, min(4096, size))
    sizes = rng.integers(4, 65, size=size).astype(np.int64)
    loc, _ = _mixture_bags(rng, sizes, 32, 32, 5.0, np.float32, comp_means=means)
    w = _dirichlet_ragged(rng, sizes, 1.0, np.float32)
    return _pack(sizes, loc, w, "f32", "f32")


def image_two_bags(N=200_000, K=64, seed=1007, n=16, components=32):
    """Two bag types per image (the paper's colour and texture bags): each
    object draws one mixture component and, from it, a colour bag (d = 3)
    and a texture bag (d = 3) of 8-16 supports each, Dirichlet(0.5)
    weights, FP32.  Centroids: K of each type with n supports and uniform
    weights.  Returns ([colour objs, texture objs], [colour cents,
    texture cents])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out_o, out_c = [], []
    means = [rng.uniform(-5.0, 5.0, size=(components, 3)) for _ in range(2)]
    comp = rng.integers(0, components, size=N)
    for t in range(2):
        sizes = rng.integers(8, 17, size=N).astype(np.int64)
        loc = (means[t][np.repeat(comp, sizes)] + rng.normal(0, 1.0, size=(int(sizes.sum()), 3)))
        w = _dirichlet_ragged(rng, sizes, 0.5, np.float32)
        out_o.append(_pack(sizes, loc.astype(np.float32), w, "f32", "f32"))
        ccomp = rng.integers(0, components, size=K)
        cl = means[t][np.repeat(ccomp, n)] + rng.normal(0, 1.0, size=(K * n, 3))
        out_c.append(_pack(np.full(K, n, dtype=np.int64), cl.astype(np.float32),
                           np.full(K * n, 1.0 / n, np.float32), "f32", "f32"))
    return out_o, out_c


def sequence_like(N=100_000, K=64, A=20, seed=1006, classes=3):
    """Sequence-style bags (the protein experiment's shape): each bag is the
    histogram of a symbol sequence (length 100-600) drawn from one of
    `classes` class profiles over A symbols; its supports are the symbols
    present (ids stored as FP32, dim 1), weights their frequencies.
    Centroids: K such histograms.  Table: a substitution-style symbol
    distance D(s, t) = -(log P(s|t) + log P(t|s)) from a random symmetric
    similarity (softmax rows), nonnegative.  Returns (objs, cents, table)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    prof = rng.dirichlet(np.full(A, 0.6), size=classes)

    def hist_bags(count):
        cls = rng.integers(0, classes, size=count)
        lens = rng.integers(100, 601, size=count)
        syms, ws, sizes = [], [], []
        for c, L in zip(cls, lens):
            cnt = rng.multinomial(L, prof[c])
            nz = np.nonzero(cnt)[0]
            syms.append(nz.astype(np.float32))
            ws.append((cnt[nz] / L).astype(np.float32))
            sizes.append(len(nz))
        return _pack(np.asarray(sizes, dtype=np.int64), np.concatenate(syms).reshape(-1, 1),
                     np.concatenate(ws), "f32", "f32")

    objs = hist_bags(N)
    cents = hist_bags(K)
    e = rng.normal(size=(A, 6))
    sim = -((e[:, None, :] - e[None, :, :]) ** 2).sum(-1) / 4.0
    P = np.exp(sim)
    P /= P.sum(axis=1, keepdims=True)
    table = -(np.log(P) + np.log(P).T)
    return objs, cents, table


CONFIGS = {
    "plain_small": plain_small,
    "image_like": image_like,
    "uneven": uneven,
    "high_dim": high_dim,
}
