// d2_solver.cuh -- per-pair exact transportation LP (the Mallows distance of
// Eq. (D2opt) with the centroid fixed) solved by a lane group of G threads.
//
// Network simplex on the bipartite basis tree:
//   nodes 0..m-1 are object supports (rows, supply p_a), nodes m..m+n-1 are
//   centroid supports (columns, demand q_r); a basic cell (a,r) is a tree
//   edge.  The tree is rooted at row 0 and stored per node as
//     par  : parent node,
//     flow : flow on the edge (node, par) -- int64 fixed point, total mass
//            2^62, so feasibility, ratio tests and degeneracy are exact,
//     pot  : dual potential (u for rows, v for columns), u_a + v_r = c_ar
//            on every tree edge,
//     pos  : preorder index, sz : subtree size, so that
//            "x is an ancestor of y" is pos[x] <= pos[y] < pos[x]+sz[x].
// Each pivot: price all m*n cells in parallel (most negative reduced cost,
// ties to the smallest cell index; Bland's smallest-index rule after a run
// of degenerate pivots), walk the cycle from both ends of the entering cell
// to their meeting node, pick the leaving edge by an exact integer ratio
// test (ties to the smallest cell index), shift the flow, and re-hang the
// cut subtree under the entering edge.  The re-hang recomputes every node's
// preorder position, subtree size and potential independently in O(1) (plus
// a binary search over the re-rooted path), so all lanes share it.
// Potentials are refreshed from the tree by pointer jumping every 64 pivots
// and before optimality is accepted.
#pragma once
#include <cstdint>
#include <climits>

namespace d2k {

constexpr long long kMass = 1LL << 62;       // fixed-point unit of one bag's mass
constexpr double kInvMass = 1.0 / 4611686018427387904.0;  // 2^-62

enum : int { kStOk = 0, kStNotConverged = 1, kStInvalid = 2 };

template <int G>
struct Grp {
  unsigned mask;
  int lane;
  __device__ __forceinline__ Grp() {
    const int wl = threadIdx.x & 31;
    lane = wl & (G - 1);
    mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (wl & ~(G - 1)));
  }
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

template <int G, typename V>
__device__ __forceinline__ V gshfl_xor(const Grp<G>& g, V v, int o) {
  return __shfl_xor_sync(g.mask, v, o, G);
}

// minimum value, ties to the smallest index
template <int G, typename V>
__device__ __forceinline__ void gmin_idx(const Grp<G>& g, V& v, int& idx) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    V ov = gshfl_xor<G>(g, v, o);
    int oi = gshfl_xor<G>(g, idx, o);
    if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
}

template <int G>
__device__ __forceinline__ int gmin_int(const Grp<G>& g, int v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = min(v, gshfl_xor<G>(g, v, o));
  return v;
}

template <int G, typename V>
__device__ __forceinline__ V gsum(const Grp<G>& g, V v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += gshfl_xor<G>(g, v, o);
  return v;
}

template <int G, typename V>
__device__ __forceinline__ V gmax(const Grp<G>& g, V v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) { V w = gshfl_xor<G>(g, v, o); v = w > v ? w : v; }
  return v;
}

template <int G>
__device__ __forceinline__ bool gany(const Grp<G>& g, bool p) {
  return (__ballot_sync(g.mask, p) & g.mask) != 0u;
}

// Shared-memory slice of one lane group.  T is the cost/dual type.
template <typename T>
struct PairMem {
  T* cost;            // [m*n] row-major, stride n
  T* pot;             // [N]
  long long* flow;    // [N]
  int* par;           // [N]
  int* pos;           // [N]
  int* sz;            // [N]
  int* path;          // [2*N]: a-side at [0,..), b-side at [N,..)
  int* ppos;          // [N]
  int* psz;           // [N]
  long long* pflow;   // [N] flows staged for the re-rooted path
  long long* P;       // [mmax] inclusive prefix sums of object masses
  long long* Q;       // [nmax] inclusive prefix sums of centroid masses
  int* re;            // [mmax] last column of each row in the NW staircase
  int* pj0;           // [N] pointer-jumping scratch (ancestor | parity<<16)
  int* pj1;           // [N]
  T* acc0;            // [N]
  T* acc1;            // [N]
  int* sc;            // [16] group scalars
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes of one group's slice for supports up to (mmax, nmax).  The cost
// area is sized for doubles so one slice can host an FP32 or FP64 solve.
__host__ __device__ inline size_t pair_mem_bytes(int mmax, int nmax) {
  const size_t N = (size_t)(mmax + nmax);
  size_t b = 0;
  b += align_up((size_t)mmax * nmax * 8, 16);  // cost
  b += align_up(N * 8, 16);                    // pot
  b += align_up(N * 8, 16);                    // flow
  b += align_up(N * 4, 16) * 3;                // par pos sz
  b += align_up(2 * N * 4, 16);                // path
  b += align_up(N * 4, 16) * 2;                // ppos psz
  b += align_up(N * 8, 16);                    // pflow
  b += align_up((size_t)mmax * 8, 16);         // P
  b += align_up((size_t)nmax * 8, 16);         // Q
  b += align_up((size_t)mmax * 4, 16);         // re
  b += align_up(N * 4, 16) * 2;                // pj0 pj1
  b += align_up(N * 8, 16) * 2;                // acc0 acc1
  b += 64;                                     // sc
  return align_up(b, 128);
}

template <typename T>
__device__ inline PairMem<T> carve(unsigned char* base, int mmax, int nmax) {
  const size_t N = (size_t)(mmax + nmax);
  PairMem<T> s;
  unsigned char* p = base;
  s.cost = reinterpret_cast<T*>(p); p += align_up((size_t)mmax * nmax * 8, 16);
  s.pot = reinterpret_cast<T*>(p); p += align_up(N * 8, 16);
  s.flow = reinterpret_cast<long long*>(p); p += align_up(N * 8, 16);
  s.par = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.pos = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.sz = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.path = reinterpret_cast<int*>(p); p += align_up(2 * N * 4, 16);
  s.ppos = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.psz = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.pflow = reinterpret_cast<long long*>(p); p += align_up(N * 8, 16);
  s.P = reinterpret_cast<long long*>(p); p += align_up((size_t)mmax * 8, 16);
  s.Q = reinterpret_cast<long long*>(p); p += align_up((size_t)nmax * 8, 16);
  s.re = reinterpret_cast<int*>(p); p += align_up((size_t)mmax * 4, 16);
  s.pj0 = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.pj1 = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.acc0 = reinterpret_cast<T*>(p); p += align_up(N * 8, 16);
  s.acc1 = reinterpret_cast<T*>(p); p += align_up(N * 8, 16);
  s.sc = reinterpret_cast<int*>(p);
  return s;
}

// Reinterpret a slice for another cost type (same byte layout).
template <typename T2, typename T1>
__device__ inline PairMem<T2> recast(const PairMem<T1>& s) {
  PairMem<T2> o;
  o.cost = reinterpret_cast<T2*>(s.cost);
  o.pot = reinterpret_cast<T2*>(s.pot);
  o.flow = s.flow; o.par = s.par; o.pos = s.pos; o.sz = s.sz; o.path = s.path;
  o.ppos = s.ppos; o.psz = s.psz; o.pflow = s.pflow; o.P = s.P; o.Q = s.Q; o.re = s.re;
  o.pj0 = s.pj0; o.pj1 = s.pj1;
  o.acc0 = reinterpret_cast<T2*>(s.acc0);
  o.acc1 = reinterpret_cast<T2*>(s.acc1);
  o.sc = s.sc;
  return o;
}

// ----------------------------------------------------------------------
// Marginals: normalise a bag's weights in FP64 (divide by the sum, the
// total-mass-one constraint of Eq. (D2opt)), quantise to multiples of
// 2^-62, put the rounding residual on the largest weight so the total is
// exactly 2^62, and write inclusive prefix sums.  Returns false for a bag
// with a negative, NaN or infinite weight or a zero total.
// ----------------------------------------------------------------------
template <int G, typename W>
__device__ bool load_prefix(const Grp<G>& g, const W* w, int m, long long* pre) {
  double s = 0.0;
  bool bad = false;
  for (int a = g.lane; a < m; a += G) {
    double x = (double)w[a];
    bad |= !(x >= 0.0) || isinf(x);
    s += x;
  }
  s = gsum<G>(g, s);
  bad = gany<G>(g, bad) || !(s > 0.0) || isinf(s);
  if (bad) return false;
  const double inv = 1.0 / s;
  long long part = 0;
  long long bigv = -1;
  int bigi = INT_MAX;
  for (int a = g.lane; a < m; a += G) {
    long long q = __double2ll_rn((double)w[a] * inv * 4611686018427387904.0);
    if (q < 0) q = 0;
    pre[a] = q;
    part += q;
    if (q > bigv) { bigv = q; bigi = a; }
  }
  part = gsum<G>(g, part);
  // largest weight, ties to the smallest index
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    long long ov = gshfl_xor<G>(g, bigv, o);
    int oi = gshfl_xor<G>(g, bigi, o);
    if (ov > bigv || (ov == bigv && oi < bigi)) { bigv = ov; bigi = oi; }
  }
  g.sync();
  if (g.lane == 0) pre[bigi] += kMass - part;
  g.sync();
  // inclusive scan in chunks of G
  long long carry = 0;
  for (int base = 0; base < m; base += G) {
    const int a = base + g.lane;
    long long v = a < m ? pre[a] : 0;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      long long u = __shfl_up_sync(g.mask, v, o, G);
      if (g.lane >= o) v += u;
    }
    v += carry;
    if (a < m) pre[a] = v;
    carry = __shfl_sync(g.mask, v, G - 1, G);
  }
  g.sync();
  return true;
}

// ----------------------------------------------------------------------
// The solver proper.
// ----------------------------------------------------------------------
template <typename T, int G>
struct Simplex {
  PairMem<T> s;
  int m, n, N;
  Grp<G> g;
  bool bad = false;  // set if a walk leaves its bounds (corrupt tree): the
                     // solve stops with kStInvalid instead of looping

  __device__ __forceinline__ bool is_anc(int x, int y) const {
    const int px = s.pos[x];
    const int py = s.pos[y];
    return px <= py && py < px + s.sz[x];
  }
  // cell index a*n+r of the tree edge (y, par[y])
  __device__ __forceinline__ int edge_cell(int y, int py) const {
    return y < m ? y * n + (py - m) : py * n + (y - m);
  }

  // Northwest-corner basis: the staircase path from cell (0,0) to (m-1,n-1)
  // that moves down when the current row's cumulative mass is reached
  // (P_a <= Q_r), else right.  Row a spans columns [re(a-1), re(a)] with
  // re(a) = first r with Q_r >= P_a.  As a tree rooted at row 0, the
  // preorder of a node is the step at which the path first touches it.
  __device__ void init_northwest() {
    const long long* P = s.P;
    const long long* Q = s.Q;
    for (int a = g.lane; a < m; a += G) {
      int e = n - 1;
      if (a < m - 1) {
        int lo = 0, hi = n - 1;  // first r with Q[r] >= P[a]
        const long long key = P[a];
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (Q[mid] >= key) hi = mid; else lo = mid + 1;
        }
        e = lo;
      }
      s.re[a] = e;
    }
    g.sync();
    for (int a = g.lane; a < m; a += G) {
      if (a == 0) {
        s.par[0] = -1; s.pos[0] = 0; s.sz[0] = N; s.flow[0] = 0;
      } else {
        const int c = s.re[a - 1];
        const long long lo = max(P[a - 1], c > 0 ? Q[c - 1] : 0LL);
        const long long hi = min(P[a], Q[c]);
        s.par[a] = m + c;
        s.pos[a] = a + c + 1;
        s.flow[a] = hi > lo ? hi - lo : 0;
        s.sz[a] = (s.re[a] == c) ? 1 : N - (a + c + 1);
      }
    }
    for (int r = g.lane; r < n; r += G) {
      int af = 0;
      if (r > 0) {  // number of rows a < m-1 with P[a] <= Q[r-1]
        const long long key = Q[r - 1];
        int lo = 0, hi = m - 1;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (P[mid] <= key) lo = mid + 1; else hi = mid;
        }
        af = lo;
      }
      const long long lo = max(af > 0 ? P[af - 1] : 0LL, r > 0 ? Q[r - 1] : 0LL);
      const long long hi = min(P[af], Q[r]);
      const int y = m + r;
      s.par[y] = af;
      s.pos[y] = af + r + 1;
      s.flow[y] = hi > lo ? hi - lo : 0;
      const bool spine = (af < m - 1) && (s.re[af] == r);
      s.sz[y] = spine ? N - (af + r + 1) : 1;
    }
    g.sync();
  }

  // Potentials from the tree: pot(root) = 0, pot(y) = c(y,par y) - pot(par y),
  // by pointer jumping: pot(y) = acc(y) + (-1)^parity(y) * pot(anc(y)).
  __device__ void refresh_potentials() {
    int* pa = s.pj0; int* pb = s.pj1;
    T* aa = s.acc0; T* ab = s.acc1;
    bool lbad = false;
    for (int y = g.lane; y < N; y += G) {
      if (y == 0) { pa[y] = 0; aa[y] = T(0); }
      else {
        const int p = s.par[y];
        if (p < 0 || p >= N || (y < m) == (p < m)) {  // parent must be of the other side
          lbad = true;
          pa[y] = 0;
          aa[y] = T(0);
        } else {
          pa[y] = p | (1 << 16);
          aa[y] = s.cost[edge_cell(y, p)];
        }
      }
    }
    if (gany<G>(g, lbad)) bad = true;
    g.sync();
    for (int round = 0;; ++round) {
      if (round > 9) { bad = true; break; }  // depth < 128 needs <= 8 rounds
      bool moved = false;
      for (int y = g.lane; y < N; y += G) {
        const int code = pa[y];
        const int an = code & 0xffff;
        if (an != 0) {
          const int c2 = pa[an];
          const T v = aa[an];
          const int par1 = code >> 16;
          ab[y] = par1 ? aa[y] - v : aa[y] + v;
          pb[y] = (c2 & 0xffff) | ((par1 ^ (c2 >> 16)) << 16);
          moved = true;
        } else {
          ab[y] = aa[y];
          pb[y] = code;
        }
      }
      g.sync();
      int* tp = pa; pa = pb; pb = tp;
      T* ta = aa; aa = ab; ab = ta;
      if (!gany<G>(g, moved)) break;
    }
    for (int y = g.lane; y < N; y += G) s.pot[y] = aa[y];
    g.sync();
  }

  // Pricing.  Returns the entering cell (or -1) and its reduced cost.
  __device__ int price(bool bland, T tol, T& dbest) const {
    const int mn = m * n;
    const int q = G / n, rem = G - (G / n) * n;
    int a = g.lane / n, r = g.lane - (g.lane / n) * n;
    T best = -tol;
    int cell = INT_MAX;
    for (int t = g.lane; t < mn; t += G) {
      const T d = s.cost[t] - s.pot[a] - s.pot[m + r];
      if (bland) {
        if (d < -tol) { best = d; cell = t; break; }
      } else if (d < best) {
        best = d; cell = t;
      }
      r += rem; a += q;
      if (r >= n) { r -= n; ++a; }
    }
    if (bland) {
      const int c = gmin_int<G>(g, cell);
      const int src = __ffs(__ballot_sync(g.mask, cell == c && c != INT_MAX) & g.mask) - 1;
      T v = best;
      if (src >= 0) v = __shfl_sync(g.mask, best, src & (G - 1), G);
      dbest = v;
      return c == INT_MAX ? -1 : c;
    }
    gmin_idx<G>(g, best, cell);
    dbest = best;
    return cell == INT_MAX ? -1 : cell;
  }

  // One pivot on entering cell `cell` with reduced cost dE < 0.
  // Returns true when the pivot moved flow (theta > 0).
  __device__ bool pivot(int cell, T dE) {
    const int ea = cell / n;
    const int eB = m + (cell - ea * n);
    // 1. cycle: climb from the row until reaching an ancestor of the column,
    //    then from the column up to that apex.
    int la = 0, lb = 0;
    {
      int x = ea;
      while (!is_anc(x, eB)) {
        if (la >= N) { bad = true; break; }
        if (g.lane == 0) s.path[la] = x;
        ++la;
        x = s.par[x];
        if (x < 0 || x >= N) { bad = true; break; }
      }
      const int apex = x;
      int y = eB;
      while (!bad && y != apex) {
        if (lb >= N) { bad = true; break; }
        if (g.lane == 0) s.path[N + lb] = y;
        ++lb;
        y = s.par[y];
        if (y < 0 || y >= N) { bad = true; break; }
      }
    }
    g.sync();
    if (bad) return false;
    const int L = la + lb;
    // 2. ratio test over the "-" edges: on the row side the edges whose
    //    child is a row, on the column side those whose child is a column.
    long long th = LLONG_MAX;
    int lc = INT_MAX, le = -1;
    for (int e = g.lane; e < L; e += G) {
      const bool aside = e < la;
      const int y = aside ? s.path[e] : s.path[N + e - la];
      const bool minus = aside ? (y < m) : (y >= m);
      if (minus) {
        const long long f = s.flow[y];
        const int c = edge_cell(y, s.par[y]);
        if (f < th || (f == th && c < lc)) { th = f; lc = c; le = e; }
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const long long of = gshfl_xor<G>(g, th, o);
      const int oc = gshfl_xor<G>(g, lc, o);
      const int oe = gshfl_xor<G>(g, le, o);
      if (of < th || (of == th && oc < lc)) { th = of; lc = oc; le = oe; }
    }
    g.sync();
    // 3. shift theta around the cycle
    if (th > 0) {
      for (int e = g.lane; e < L; e += G) {
        const bool aside = e < la;
        const int y = aside ? s.path[e] : s.path[N + e - la];
        const bool minus = aside ? (y < m) : (y >= m);
        s.flow[y] += minus ? -th : th;
      }
    }
    // 4. re-hang.  The leaving edge (zL, par zL) lies on one side; the
    //    subtree S under it contains that side's end e of the entering edge
    //    and is re-rooted at e and hung under the other end o.
    const bool lside_a = le < la;
    const int k = lside_a ? le : le - la;
    const int* ph = lside_a ? s.path : s.path + N;
    const int enode = lside_a ? ea : eB;
    const int onode = lside_a ? eB : ea;
    const int zL = ph[k];
    const int P0 = s.pos[zL];
    const int Z = s.sz[zL];
    const int posO = s.pos[onode];
    for (int i = g.lane; i <= k; i += G) {
      const int y = ph[i];
      s.ppos[i] = s.pos[y];
      s.psz[i] = s.sz[y];
    }
    g.sync();
    const int remO = posO >= P0 + Z ? posO - Z : posO;
    const int Qi = remO + 1;
    const bool e_is_row = enode < m;
    for (int y = g.lane; y < N; y += G) {
      const int py = s.pos[y];
      const int sy = s.sz[y];
      int np, ns;
      if (py >= P0 && py < P0 + Z) {
        // ring index: smallest i with ppos[i] <= py < ppos[i]+psz[i]
        int lo = 0, hi = k;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          const int pp = s.ppos[mid];
          if (pp <= py && py < pp + s.psz[mid]) hi = mid; else lo = mid + 1;
        }
        const int i = lo;
        int off;
        if (i == 0) {
          off = py - s.ppos[0];
        } else {
          const int pp = s.ppos[i - 1], ps = s.psz[i - 1];
          off = ps + (py < pp ? py - s.ppos[i] : py - s.ppos[i] - ps);
        }
        np = Qi + off;
        ns = sy;
        if (py == s.ppos[i]) ns = (i == 0) ? Z : Z - s.psz[i - 1];
        s.pot[y] += ((y < m) == e_is_row) ? dE : -dE;
      } else {
        const int r0 = py >= P0 + Z ? py - Z : py;
        np = r0 + (r0 >= Qi ? Z : 0);
        ns = sy;
        if (py <= P0 && P0 < py + sy) ns -= Z;
        if (py <= posO && posO < py + sy) ns += Z;
      }
      s.pos[y] = np;
      s.sz[y] = ns;
    }
    // parent pointers and edge flows along the re-rooted path: the edge
    // (p_{i-1}, p_i) becomes p_i's parent edge, the entering edge e's.
    for (int i = g.lane + 1; i <= k; i += G) s.pflow[i] = s.flow[ph[i - 1]];
    g.sync();
    for (int i = g.lane; i <= k; i += G) {
      const int y = ph[i];
      if (i == 0) { s.par[y] = onode; s.flow[y] = th; }
      else { s.par[y] = ph[i - 1]; s.flow[y] = s.pflow[i]; }
    }
    g.sync();
    return th > 0;
  }

  // Pivot from the current basis until no reduced cost is below -tol
  // (with potentials freshly recomputed from the tree).  Returns kStOk or
  // kStNotConverged; *pivots accumulates the pivot count.
  __device__ int run(int max_pivots, T tol, int* pivots) {
    refresh_potentials();
    if (bad) return kStInvalid;
    int done = 0, degen = 0, since = 0;
    bool bland = false;
    int st = kStOk;
    for (;;) {
      T dE;
      const int cell = price(bland, tol, dE);
      if (cell < 0) {
        if (since == 0) break;
        refresh_potentials();
        if (bad) { st = kStInvalid; break; }
        since = 0;
        continue;
      }
      if (done >= max_pivots) { st = kStNotConverged; break; }
      const bool moved = pivot(cell, dE);
      if (bad) { st = kStInvalid; break; }
      ++done;
      ++since;
      if (moved) { degen = 0; bland = false; }
      else if (++degen >= 2 * N) bland = true;
      if (since >= 64) {
        refresh_potentials();
        if (bad) { st = kStInvalid; break; }
        since = 0;
      }
    }
    if (pivots) *pivots += done;
    return st;
  }

  // Full solve from the northwest corner.
  __device__ int solve(int max_pivots, T tol, int* pivots) {
    init_northwest();
    return run(max_pivots, tol, pivots);
  }
};

}  // namespace d2k
