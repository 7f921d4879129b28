// d2_solver.cuh -- per-pair exact transportation LP (the Mallows distance of
// Eq. (D2opt) with the centroid fixed) solved by a lane group of G threads.
//
// Network simplex on the bipartite basis tree:
//   nodes 0..m-1 are object supports (rows, supply p_a), nodes m..m+n-1 are
//   centroid supports (columns, demand q_r); a basic cell (a,r) is a tree
//   edge.  The tree is rooted at row 0.  Lane l of the group owns nodes
//   l, l+G, ... (NPL of them) and keeps for each owned node, in registers:
//     par  : parent node,
//     pos  : preorder index, sz : subtree size ("x is an ancestor of y" is
//            pos[x] <= pos[y] < pos[x]+sz[x]),
//     flow : flow on the edge (node, par) -- int64 fixed point, total mass
//            2^62, so feasibility, ratio tests and degeneracy are exact,
//     pot  : dual potential (u for rows, v for columns), u_a + v_r = c_ar
//            on every tree edge.
//   Shared memory holds the cost tile and mirrors of pos/sz (for the few
//   nodes every lane needs) and of the potentials (read by pricing).
// One pivot, all lanes busy:
//   1. price the lane's cells t = l, l+G, ... of the m*n tile; the group minimum of
//      (reduced cost, cell) enters (ties to the smallest cell; Bland's
//      smallest-index rule after a run of degenerate pivots);
//   2. a node is on the cycle's row side iff it is an ancestor of the
//      entering row but not of the entering column (and vice versa); the
//      "-" edges are the row-side edges hanging from rows and the
//      column-side edges hanging from columns; an exact integer group
//      minimum over them gives theta and the leaving edge;
//   3. the leaving side's path is ranked by preorder position (a bitmask of
//      positions), the cut subtree is re-rooted at the entering end and
//      hung under the other end: every node recomputes its own position,
//      size and potential in O(1) plus a binary search over the path.
// Potentials are recomputed from the tree by pointer jumping every 64
// pivots and before optimality is accepted.
#pragma once
#include <cstdint>
#include <climits>

namespace d2k {

constexpr long long kMass = 1LL << 62;       // fixed-point unit of one bag's mass
constexpr double kInvMass = 1.0 / 4611686018427387904.0;  // 2^-62

enum : int { kStOk = 0, kStNotConverged = 1, kStInvalid = 2 };
// Hand-over code of the two-launch exact solve: the FP32 launch restarted a
// pair from the basis the FP64 launch proved optimal in the previous joint
// round and needed no pivot, so that tree is still FP64-optimal.
enum : int { kStSameBasis = 3 };

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

// Shared-memory slice of one lane group.  The cost and potential areas hold
// eb bytes per entry: 8 (the default) gives the same byte layout for float
// and double, so that one slice can hold an FP32 solve and then its FP64
// continuation (recast); kernels that only ever solve in FP32 use eb = 4,
// half the cost tile, so more warps fit on an SM.
template <typename T>
struct PairMem {
  T* cost;            // [m*n] row-major, stride n
  T* pot;             // [N] potentials (mirror for pricing)
  int* pos;           // [N] mirror of preorder positions
  int* sz;            // [N] mirror of subtree sizes
  int* ppos;          // [N] leaving path, ranked: positions
  int* psz;           // [N]   sizes
  int* pnode;         // [N]   nodes
  long long* pflow;   // [N]   flows (after the shift)
  long long* P;       // [mmax] inclusive prefix sums of object masses
  long long* Q;       // [nmax] inclusive prefix sums of centroid masses
  int* re;            // [mmax] last column of each row in the NW staircase
  int* pj0;           // [N] pointer-jumping scratch (ancestor | parity<<16)
  int* pj1;           // [N]
  T* acc0;            // [N]
  T* acc1;            // [N]
  int* sc;            // [32] group scalars
  // projection order of the start basis (see order_rows / order_cols)
  int* rrank;         // [mmax] row -> rank
  int* rid;           // [mmax] rank -> row
  int* crank;         // [nmax] column -> rank
  int* cid;           // [nmax] rank -> column
  long long* Pr;      // [mmax] prefix masses in rank order
  long long* Qr;      // [nmax]
  float* dir;         // [dmax] principal direction of the object
  float* mu;          // [dmax] weighted mean of the object
  float* proj;        // [max(mmax,nmax)] projections
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// tile = false: no cost tile in shared memory (the solver reads a tile that
// already sits in global memory, see Simplex::set_cost).
__host__ __device__ inline size_t pair_mem_bytes(int mmax, int nmax, int dmax = 256, int eb = 8,
                                                 bool tile = true) {
  const size_t N = (size_t)(mmax + nmax);
  const size_t mx = (size_t)(mmax > nmax ? mmax : nmax);
  size_t b = 0;
  b += align_up((size_t)mmax * 4, 16) * 2 + align_up((size_t)nmax * 4, 16) * 2;  // ranks
  b += align_up((size_t)mmax * 8, 16) + align_up((size_t)nmax * 8, 16);          // Pr Qr
  b += align_up((size_t)dmax * 4, 16) * 2 + align_up(mx * 4, 16);               // dir mu proj
  if (tile) b += align_up((size_t)mmax * nmax * eb, 16);  // cost
  b += align_up(N * eb, 16);                    // pot
  b += align_up(N * 4, 16) * 2;                // pos sz
  b += align_up(N * 4, 16) * 3;                // ppos psz pnode
  b += align_up(N * 8, 16);                    // pflow
  b += align_up((size_t)mmax * 8, 16);         // P
  b += align_up((size_t)nmax * 8, 16);         // Q
  b += align_up((size_t)mmax * 4, 16);         // re
  b += align_up(N * 4, 16) * 2;                // pj0 pj1
  b += align_up(N * eb, 16) * 2;               // acc0 acc1
  b += 128;                                    // sc: 32 group scalars
  return align_up(b, 128);
}

template <typename T>
__device__ inline PairMem<T> carve(unsigned char* base, int mmax, int nmax, int dmax = 256,
                                   int eb = 8, bool tile = true) {
  const size_t N = (size_t)(mmax + nmax);
  const size_t mx = (size_t)(mmax > nmax ? mmax : nmax);
  PairMem<T> s;
  unsigned char* p = base;
  s.rrank = reinterpret_cast<int*>(p); p += align_up((size_t)mmax * 4, 16);
  s.rid = reinterpret_cast<int*>(p); p += align_up((size_t)mmax * 4, 16);
  s.crank = reinterpret_cast<int*>(p); p += align_up((size_t)nmax * 4, 16);
  s.cid = reinterpret_cast<int*>(p); p += align_up((size_t)nmax * 4, 16);
  s.Pr = reinterpret_cast<long long*>(p); p += align_up((size_t)mmax * 8, 16);
  s.Qr = reinterpret_cast<long long*>(p); p += align_up((size_t)nmax * 8, 16);
  s.dir = reinterpret_cast<float*>(p); p += align_up((size_t)dmax * 4, 16);
  s.mu = reinterpret_cast<float*>(p); p += align_up((size_t)dmax * 4, 16);
  s.proj = reinterpret_cast<float*>(p); p += align_up(mx * 4, 16);
  s.cost = nullptr;
  if (tile) { s.cost = reinterpret_cast<T*>(p); p += align_up((size_t)mmax * nmax * eb, 16); }
  s.pot = reinterpret_cast<T*>(p); p += align_up(N * eb, 16);
  s.pos = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.sz = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.ppos = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.psz = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.pnode = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.pflow = reinterpret_cast<long long*>(p); p += align_up(N * 8, 16);
  s.P = reinterpret_cast<long long*>(p); p += align_up((size_t)mmax * 8, 16);
  s.Q = reinterpret_cast<long long*>(p); p += align_up((size_t)nmax * 8, 16);
  s.re = reinterpret_cast<int*>(p); p += align_up((size_t)mmax * 4, 16);
  s.pj0 = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.pj1 = reinterpret_cast<int*>(p); p += align_up(N * 4, 16);
  s.acc0 = reinterpret_cast<T*>(p); p += align_up(N * eb, 16);
  s.acc1 = reinterpret_cast<T*>(p); p += align_up(N * eb, 16);
  s.sc = reinterpret_cast<int*>(p);
  return s;
}

template <typename T2, typename T1>
__device__ inline PairMem<T2> recast(const PairMem<T1>& s) {
  PairMem<T2> o;
  o.cost = reinterpret_cast<T2*>(s.cost);
  o.pot = reinterpret_cast<T2*>(s.pot);
  o.pos = s.pos; o.sz = s.sz; o.ppos = s.ppos; o.psz = s.psz; o.pnode = s.pnode;
  o.pflow = s.pflow; o.P = s.P; o.Q = s.Q; o.re = s.re; o.pj0 = s.pj0; o.pj1 = s.pj1;
  o.acc0 = reinterpret_cast<T2*>(s.acc0);
  o.acc1 = reinterpret_cast<T2*>(s.acc1);
  o.sc = s.sc;
  o.rrank = s.rrank; o.rid = s.rid; o.crank = s.crank; o.cid = s.cid; o.Pr = s.Pr; o.Qr = s.Qr;
  o.dir = s.dir; o.mu = s.mu; o.proj = s.proj;
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
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    long long ov = gshfl_xor<G>(g, bigv, o);
    int oi = gshfl_xor<G>(g, bigi, o);
    if (ov > bigv || (ov == bigv && oi < bigi)) { bigv = ov; bigi = oi; }
  }
  g.sync();
  if (g.lane == 0) pre[bigi] += kMass - part;
  g.sync();
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

// Tree registers of the nodes a lane owns (type independent: an FP32 solve
// hands its basis to an FP64 solve unchanged).
template <int NPL>
struct TreeRegs {
  int par[NPL], pos[NPL], sz[NPL];
  long long flow[NPL];
};

// ----------------------------------------------------------------------
// The solver proper.  m+n <= G*NPL <= 128, m, n <= 255.
// ----------------------------------------------------------------------
template <typename T, int G, int NPL>
struct Simplex {
  static constexpr int NW = (G * NPL + 31) / 32;  // position bitmask words
  PairMem<T> s;
  TreeRegs<NPL> t;  // hand over to another Simplex by copying
  int m, n, N;
  Grp<G> g;
  T pot[NPL];
  bool bad = false;  // a consistency check failed: the solve stops with kStInvalid
  // cell stepping of this lane: cells i = lane, lane+G, ... are (a, r) with
  // a += sq, r += sr per step (wrapping r at n)
  int a0, r0, sq, sr;
  // the cost tile: cell (a, r) at cost[a * cs + r] -- the shared-memory tile
  // (cs = n) or a tile row block in global memory (set_cost)
  T* cost;
  int cs;
  bool own_tile = true;
  int cand = -1;     // this lane's candidate cell (offset a * cs + r) from the last full pricing
  int cand_a = 0, cand_r = 0;
  int root = 0;      // the tree root: the node at preorder position 0

  __device__ __forceinline__ Simplex(const PairMem<T>& s_, int m_, int n_, const Grp<G>& g_)
      : s(s_), m(m_), n(n_), N(m_ + n_), g(g_), cost(s_.cost), cs(n_) {
    set_dims(m_, n_);
  }
  __device__ __forceinline__ void set_dims(int m_, int n_) {
    m = m_; n = n_; N = m_ + n_;
    a0 = g.lane / n; r0 = g.lane - a0 * n;
    sq = G / n; sr = G - sq * n;
    if (own_tile) cs = n;
    cand = -1;
  }
  // Price from a tile in global memory: cell (a, r) at c[a * stride + r].
  __device__ __forceinline__ void set_cost(T* c, int stride) {
    cost = c;
    cs = stride;
    own_tile = false;
    cand = -1;
  }
  __device__ __forceinline__ T cost_at(int a, int r) const { return cost[a * cs + r]; }

  __device__ __forceinline__ int node_of(int k) const { return g.lane + G * k; }
  // cell key of an edge: (row << 8) | col -- orders cells like row*n+col
  __device__ __forceinline__ static int key_rc(int a, int r) { return (a << 8) | r; }
  // tile offset of the edge (y, p)
  __device__ __forceinline__ int edge_idx(int y, int p) const {
    return y < m ? y * cs + (p - m) : p * cs + (y - m);
  }
  __device__ __forceinline__ int edge_key(int y, int p) const {
    return y < m ? key_rc(y, p - m) : key_rc(p, y - m);
  }

  // ---- Vogel start --------------------------------------------------
  // Smallest and second smallest alive cost of column r over the alive
  // rows `ra` (ties to the smaller row), by this lane alone.
  __device__ __forceinline__ void vogel_col_scan(int r, unsigned long long ra, T& v1, int& i1,
                                                 T& v2, int& i2) const {
    v1 = v2 = T(INFINITY);
    i1 = i2 = -1;
    for (unsigned long long b = ra; b; b &= b - 1) {
      const int a = __ffsll((long long)b) - 1;
      const T c = cost_at(a, r);
      if (c < v1) { v2 = v1; i2 = i1; v1 = c; i1 = a; }
      else if (c < v2) { v2 = c; i2 = a; }
    }
  }
  // The same for row a over the alive columns `ca`, by the whole warp; every
  // lane gets the result.
  __device__ __forceinline__ void vogel_row_scan(int a, unsigned long long ca, T& v1, int& i1,
                                                 T& v2, int& i2) const {
    T b1 = T(INFINITY), b2 = T(INFINITY);
    int j1 = INT_MAX, j2 = INT_MAX;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = g.lane + 32 * h;
      if (r < n && ((ca >> r) & 1ull)) {
        const T c = cost_at(a, r);
        if (c < b1) { b2 = b1; j2 = j1; b1 = c; j1 = r; }
        else if (c < b2) { b2 = c; j2 = r; }
      }
    }
    // smallest (value, column) over the warp
    T m1 = b1;
    int k1 = j1;
    gmin_val_key(m1, k1);
    // second: the best entry other than (m1, k1): the owner offers its own
    // second, everyone else their first
    T o = (j1 == k1) ? b2 : b1;
    int ko = (j1 == k1) ? j2 : j1;
    gmin_val_key(o, ko);
    v1 = m1; i1 = k1; v2 = o; i2 = (ko == INT_MAX) ? -1 : ko;
  }
  // Vogel's approximation: at every step the line (row or column) with the
  // largest penalty -- the gap between its two smallest alive costs; ties to
  // the smaller line, rows before columns -- gives its cheapest alive cell
  // as much flow as both ends still hold; the end that runs out (the row on
  // a tie) leaves.  Flows are the int64 masses, so the start is exactly
  // feasible.  Tree: every removed line hangs from the other end of the cell
  // that removed it, the last line standing is the root; sizes follow the
  // removal order and preorder positions its reverse.  m, n <= 64, G = 32.
  __device__ void init_vogel() {
    static_assert(G == 32, "Vogel start: one warp per pair");
    long long* mass = s.pflow;  // remaining mass of a line; its edge flow once removed
    int* par = s.pj0;
    int* ord = s.pj1;
    int* szs = s.ppos;
    int* poss = s.psz;
    int* offs = s.pnode;
    for (int y = g.lane; y < N; y += G) {
      long long v;
      if (y < m) v = s.P[y] - (y > 0 ? s.P[y - 1] : 0LL);
      else {
        const int r = y - m;
        v = s.Q[r] - (r > 0 ? s.Q[r - 1] : 0LL);
      }
      mass[y] = v;
      par[y] = -1;
      szs[y] = 1;
      offs[y] = 0;
    }
    unsigned long long ra = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
    unsigned long long ca = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
    // per-lane state of rows and columns lane, lane + 32
    T rv1[2], rv2[2], cv1[2], cv2[2];
    int ri1[2], ri2[2], ci1[2], ci2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      rv1[h] = rv2[h] = cv1[h] = cv2[h] = T(INFINITY);
      ri1[h] = ri2[h] = ci1[h] = ci2[h] = -1;
      const int r = g.lane + 32 * h;
      if (r < n) vogel_col_scan(r, ra, cv1[h], ci1[h], cv2[h], ci2[h]);
    }
    for (int a = 0; a < m; ++a) {
      T v1, v2;
      int i1, i2;
      vogel_row_scan(a, ca, v1, i1, v2, i2);
      if ((a & 31) == g.lane) {
        const int h = a >> 5;
        rv1[h] = v1; ri1[h] = i1; rv2[h] = v2; ri2[h] = i2;
      }
    }
    g.sync();
    int tcount = 0;
    int guard = 0;
    while (__popcll(ra) > 1 && __popcll(ca) > 1) {
      if (++guard > 2 * 128) { bad = true; break; }
      // the largest penalty (float keys: larger gap -> larger key)
      unsigned best = 0u;
      int bline = INT_MAX;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int a = g.lane + 32 * h;
        if (a < m && ((ra >> a) & 1ull)) {
          const unsigned k = __float_as_uint((float)(rv2[h] - rv1[h]));
          if (k > best || (k == best && a < bline)) { best = k; bline = a; }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = g.lane + 32 * h;
        if (r < n && ((ca >> r) & 1ull)) {
          const unsigned k = __float_as_uint((float)(cv2[h] - cv1[h]));
          if (k > best || (k == best && m + r < bline)) { best = k; bline = m + r; }
        }
      }
      const unsigned wbest = __reduce_max_sync(g.mask, best);
      const int L = (int)__reduce_min_sync(g.mask, best == wbest ? (unsigned)bline : 0xffffffffu);
      // its cheapest alive cell, from the owner lane
      int a, r;
      if (L < m) {
        a = L;
        const int h = a >> 5;
        r = __shfl_sync(g.mask, h ? ri1[1] : ri1[0], a & 31);
      } else {
        r = L - m;
        const int h = r >> 5;
        a = __shfl_sync(g.mask, h ? ci1[1] : ci1[0], r & 31);
      }
      if (a < 0 || r < 0) { bad = true; break; }
      const long long ma = mass[a], mr = mass[m + r];
      const bool row_leaves = ma <= mr;
      const long long f = row_leaves ? ma : mr;
      g.sync();
      if (g.lane == 0) {
        if (row_leaves) { mass[m + r] = mr - f; par[a] = m + r; ord[tcount] = a; }
        else { mass[a] = ma - f; par[m + r] = a; ord[tcount] = m + r; }
      }
      ++tcount;
      if (row_leaves) {
        ra &= ~(1ull << a);
        // columns whose two smallest included row a
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = g.lane + 32 * h;
          if (c < n && ((ca >> c) & 1ull) && (ci1[h] == a || ci2[h] == a))
            vogel_col_scan(c, ra, cv1[h], ci1[h], cv2[h], ci2[h]);
        }
      } else {
        ca &= ~(1ull << r);
        // rows whose two smallest included column r, one warp-wide rescan each
        unsigned long long hit = 0ull;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int b = g.lane + 32 * h;
          const bool p = b < m && ((ra >> b) & 1ull) && (ri1[h] == r || ri2[h] == r);
          hit |= (unsigned long long)__ballot_sync(g.mask, p) << (32 * h);
        }
        for (; hit; hit &= hit - 1) {
          const int b = __ffsll((long long)hit) - 1;
          T v1, v2;
          int i1, i2;
          vogel_row_scan(b, ca, v1, i1, v2, i2);
          if ((b & 31) == g.lane) {
            const int h = b >> 5;
            rv1[h] = v1; ri1[h] = i1; rv2[h] = v2; ri2[h] = i2;
          }
        }
      }
      g.sync();
    }
    // one line of one kind is left: it takes all remaining cells and is the root
    int rt;
    if (__popcll(ra) == 1) {
      rt = __ffsll((long long)ra) - 1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = g.lane + 32 * h;
        if (c < n && ((ca >> c) & 1ull)) {
          par[m + c] = rt;
          ord[tcount + __popcll(ca & ((1ull << c) - 1ull))] = m + c;
        }
      }
      tcount += __popcll(ca);
    } else {
      rt = m + __ffsll((long long)ca) - 1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int b = g.lane + 32 * h;
        if (b < m && ((ra >> b) & 1ull)) {
          par[b] = rt;
          ord[tcount + __popcll(ra & ((1ull << b) - 1ull))] = b;
        }
      }
      tcount += __popcll(ra);
    }
    if (tcount != N - 1 || __popcll(ra) < 1 || __popcll(ca) < 1) bad = true;
    g.sync();
    if (!bad && g.lane == 0) {
      // subtree sizes: children leave before their parents
      for (int q = 0; q < N - 1; ++q) {
        const int y = ord[q];
        szs[par[y]] += szs[y];
      }
      // preorder positions: parents are placed before their children
      poss[rt] = 0;
      for (int q = N - 2; q >= 0; --q) {
        const int y = ord[q];
        const int p = par[y];
        poss[y] = poss[p] + 1 + offs[p];
        offs[p] += szs[y];
      }
    }
    g.sync();
    root = rt;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) {
        t.par[k] = (y == rt) ? -1 : par[y];
        t.pos[k] = poss[y];
        t.sz[k] = szs[y];
        t.flow[k] = (y == rt) ? 0LL : mass[y];
        s.pos[y] = t.pos[k];
        s.sz[y] = t.sz[k];
      }
    }
    g.sync();
  }

  // Northwest-corner basis: the staircase path from cell (0,0) to (m-1,n-1)
  // that moves down when the current row's cumulative mass is reached
  // (P_a <= Q_r), else right.  Row a spans columns [re(a-1), re(a)] with
  // re(a) = first r with Q_r >= P_a.  As a tree rooted at row 0, a node's
  // preorder position is the step at which the path first touches it.
  __device__ __forceinline__ void init_northwest() {
    root = 0;
    const long long* P = s.P;
    const long long* Q = s.Q;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int a = node_of(k);
      if (a < m) {
        int e = n - 1;
        if (a < m - 1) {
          int lo = 0, hi = n - 1;
          const long long key = P[a];
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Q[mid] >= key) hi = mid; else lo = mid + 1;
          }
          e = lo;
        }
        s.re[a] = e;
      }
    }
    g.sync();
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < m) {
        const int a = y;
        if (a == 0) {
          t.par[k] = -1; t.pos[k] = 0; t.sz[k] = N; t.flow[k] = 0;
        } else {
          const int c = s.re[a - 1];
          const long long lo = max(P[a - 1], c > 0 ? Q[c - 1] : 0LL);
          const long long hi = min(P[a], Q[c]);
          t.par[k] = m + c;
          t.pos[k] = a + c + 1;
          t.flow[k] = hi > lo ? hi - lo : 0;
          t.sz[k] = (s.re[a] == c) ? 1 : N - (a + c + 1);
        }
      } else if (y < N) {
        const int r = y - m;
        int af = 0;
        if (r > 0) {  // rows a < m-1 with P[a] <= Q[r-1]
          const long long key = Q[r - 1];
          int lo = 0, hi = m - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (P[mid] <= key) lo = mid + 1; else hi = mid;
          }
          af = lo;
        }
        const long long lo = max(af > 0 ? P[af - 1] : 0LL, r > 0 ? Q[r - 1] : 0LL);
        const long long hi = min(P[af], Q[r]);
        t.par[k] = af;
        t.pos[k] = af + r + 1;
        t.flow[k] = hi > lo ? hi - lo : 0;
        const bool spine = (af < m - 1) && (s.re[af] == r);
        t.sz[k] = spine ? N - (af + r + 1) : 1;
      }
      if (y < N) { s.pos[y] = t.pos[k]; s.sz[y] = t.sz[k]; }
    }
    g.sync();
  }

  // The same northwest staircase taken in rank order: rows and columns are
  // visited in the order of their projections (rrank/crank, prefix masses
  // Pr/Qr in that order, see order_rows/order_cols).  Node ids stay the
  // real rows and columns; only the visiting order changes, so the result
  // is again a spanning-tree basis with its basic flows.
  __device__ __forceinline__ void init_northwest_ranked() {
    root = s.rid[0];
    const long long* P = s.Pr;
    const long long* Q = s.Qr;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int a = node_of(k);
      if (a < m) {
        const int ra = s.rrank[a];
        int e = n - 1;
        if (ra < m - 1) {
          int lo = 0, hi = n - 1;
          const long long key = P[ra];
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Q[mid] >= key) hi = mid; else lo = mid + 1;
          }
          e = lo;
        }
        s.re[ra] = e;
      }
    }
    g.sync();
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < m) {
        const int a = s.rrank[y];
        if (a == 0) {
          t.par[k] = -1; t.pos[k] = 0; t.sz[k] = N; t.flow[k] = 0;
        } else {
          const int c = s.re[a - 1];
          const long long lo = max(P[a - 1], c > 0 ? Q[c - 1] : 0LL);
          const long long hi = min(P[a], Q[c]);
          t.par[k] = m + s.cid[c];
          t.pos[k] = a + c + 1;
          t.flow[k] = hi > lo ? hi - lo : 0;
          t.sz[k] = (s.re[a] == c) ? 1 : N - (a + c + 1);
        }
      } else if (y < N) {
        const int r = s.crank[y - m];
        int af = 0;
        if (r > 0) {
          const long long key = Q[r - 1];
          int lo = 0, hi = m - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (P[mid] <= key) lo = mid + 1; else hi = mid;
          }
          af = lo;
        }
        const long long lo = max(af > 0 ? P[af - 1] : 0LL, r > 0 ? Q[r - 1] : 0LL);
        const long long hi = min(P[af], Q[r]);
        t.par[k] = s.rid[af];
        t.pos[k] = af + r + 1;
        t.flow[k] = hi > lo ? hi - lo : 0;
        const bool spine = (af < m - 1) && (s.re[af] == r);
        t.sz[k] = spine ? N - (af + r + 1) : 1;
      }
      if (y < N) { s.pos[y] = t.pos[k]; s.sz[y] = t.sz[k]; }
    }
    g.sync();
  }

  // Potentials from the tree: pot(root) = 0, pot(y) = c(y,par y) - pot(par y),
  // by pointer jumping: pot(y) = acc(y) + (-1)^parity(y) * pot(anc(y)).
  __device__ __forceinline__ void refresh_potentials() {
    if constexpr (NPL == 1 && G == 32) {
      // one node per lane: the same pointer jumping through shuffles
      const int y = g.lane;
      int code = y;
      T acc = T(0);
      bool lbad = false;
      if (y < N && y != root) {
        const int p = t.par[0];
        if (p < 0 || p >= N || (y < m) == (p < m)) { lbad = true; code = root; }
        else { code = p | (1 << 16); acc = cost[edge_idx(y, p)]; }
      }
      if (gany<G>(g, lbad)) bad = true;
      for (int round = 0;; ++round) {
        if (round > 9) { bad = true; break; }  // depth < 32 needs <= 6 rounds
        const int an = code & 0xffff;
        const int c2 = __shfl_sync(g.mask, code, an);
        const T v = __shfl_sync(g.mask, acc, an);
        const bool mv = y < N && an != root;
        if (mv) {
          const int par1 = code >> 16;
          acc = par1 ? acc - v : acc + v;
          code = (c2 & 0xffff) | ((par1 ^ (c2 >> 16)) << 16);
        }
        if (!gany<G>(g, mv)) break;
      }
      pot[0] = acc;
      if (y < N) s.pot[y] = acc;
      g.sync();
      return;
    }
    int* pa = s.pj0; int* pb = s.pj1;
    T* aa = s.acc0; T* ab = s.acc1;
    bool lbad = false;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y == root) { pa[y] = y; aa[y] = T(0); }   // the root points at itself
      else if (y < N) {
        const int p = t.par[k];
        if (p < 0 || p >= N || (y < m) == (p < m)) { lbad = true; pa[y] = root; aa[y] = T(0); }
        else { pa[y] = p | (1 << 16); aa[y] = cost[edge_idx(y, p)]; }
      }
    }
    if (gany<G>(g, lbad)) bad = true;
    g.sync();
    for (int round = 0;; ++round) {
      if (round > 9) { bad = true; break; }  // depth < 128 needs <= 8 rounds
      bool moved = false;
#pragma unroll
      for (int k = 0; k < NPL; ++k) {
        const int y = node_of(k);
        if (y < N) {
          const int code = pa[y];
          const int an = code & 0xffff;
          if (an != root) {
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
      }
      g.sync();
      int* tp = pa; pa = pb; pb = tp;
      T* ta = aa; aa = ab; ab = ta;
      if (!gany<G>(g, moved)) break;
    }
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) { pot[k] = aa[y]; s.pot[y] = aa[y]; }
    }
    g.sync();
  }

  // Pricing over the lane's cells t = lane, lane+G, ...  Returns the
  // entering cell key ((row << 8) | col) or -1, and its reduced cost.
  // order-preserving map of a value to an unsigned key (smaller value ->
  // smaller key), so group minima can use the integer reduction unit
  __device__ __forceinline__ static unsigned okey(float v) {
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  }

  // group minimum of (value, key): smallest value, ties to the smallest key
  __device__ __forceinline__ void gmin_val_key(T& v, int& key) const {
    if (sizeof(T) == 4) {
      const unsigned kv = okey((float)v);
      const unsigned mv = __reduce_min_sync(g.mask, kv);
      const unsigned mk = __reduce_min_sync(g.mask, kv == mv ? (unsigned)key : 0xffffffffu);
      const unsigned bal = __ballot_sync(g.mask, kv == mv && (unsigned)key == mk) & g.mask;
      v = __shfl_sync(g.mask, v, (__ffs(bal) - 1) & (G - 1), G);
      key = (int)mk;
    } else {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        const T ov = gshfl_xor<G>(g, v, o);
        const int ok = gshfl_xor<G>(g, key, o);
        if (ov < v || (ov == v && ok < key)) { v = ov; key = ok; }
      }
    }
  }

  // Full Dantzig scan of the lane's cells i = lane, lane+G, ...: the most
  // negative reduced cost (ties to the smallest cell).  Also records the
  // lane's best cell as its candidate for the following pivots.
  __device__ __forceinline__ void scan_full(T& best, int& cell) {
    if (NPL == 1 && sr == 0) {
      // n divides the group: this lane's cells share column r0 (rows a0,
      // a0 + sq, ...), so its column potential stays in a register (small
      // trees only: the larger instantiations keep their register budget)
      const T vr = s.pot[m + r0];
      best = T(0);
      int bi = -1, ba = 0;
      const int step = sq * cs;
      for (int a = a0, o = a0 * cs + r0; a < m; a += sq, o += step) {
        const T d = cost[o] - s.pot[a] - vr;
        const bool better = d < best;
        best = better ? d : best;
        bi = better ? o : bi;
        ba = better ? a : ba;
      }
      cell = bi >= 0 ? key_rc(ba, r0) : INT_MAX;
      cand = bi;
      cand_a = ba;
      cand_r = r0;
      return;
    }
    const int mn = m * n;
    int a = a0, r = r0;
    int o = a0 * cs + r0;  // offset of cell (a, r)
    const int ostep = sq * cs + sr, owrap = cs - n;
    best = T(0);
    cell = INT_MAX;
    int bi = -1, ba = 0, br = 0;
    const T* pv = s.pot + m;
    for (int i = g.lane; i < mn; i += G) {
      const T d = cost[o] - s.pot[a] - pv[r];
      const bool better = d < best;
      best = better ? d : best;
      cell = better ? key_rc(a, r) : cell;
      bi = better ? o : bi;
      ba = better ? a : ba;
      br = better ? r : br;
      r += sr; a += sq; o += ostep;
      const bool wrap = r >= n;
      r = wrap ? r - n : r;
      a = wrap ? a + 1 : a;
      o = wrap ? o + owrap : o;
    }
    cand = bi;
    cand_a = ba;
    cand_r = br;
  }

  // Bland's rule: the smallest cell with reduced cost below -tol.
  __device__ __forceinline__ int price_bland(T tol, T& dbest) const {
    const int mn = m * n;
    int a = a0, r = r0;
    T best = T(0);
    int cell = INT_MAX;
    const T* pv = s.pot + m;
    for (int i = g.lane; i < mn && cell == INT_MAX; i += G) {
      const T d = cost_at(a, r) - s.pot[a] - pv[r];
      if (d < -tol) { best = d; cell = key_rc(a, r); }
      r += sr; a += sq;
      if (r >= n) { r -= n; ++a; }
    }
    const int c = gmin_int<G>(g, cell);
    const unsigned bal = __ballot_sync(g.mask, cell == c && c != INT_MAX) & g.mask;
    T v = best;
    if (bal) v = __shfl_sync(g.mask, best, (__ffs(bal) - 1) & (G - 1), G);
    dbest = v;
    return c == INT_MAX ? -1 : c;
  }

  // Entering cell: on trees of one node per lane, the most negative reduced
  // cost of the whole tile; otherwise the lanes' candidates from the last
  // full scan are first re-priced with the current potentials (one cell per
  // lane), and only when none is below -tol is the whole tile scanned again.
  // Returns the cell key ((row << 8) | col) or -1 if no reduced cost is
  // below -tol.
  __device__ __forceinline__ int price(bool bland, T tol, T& dbest) {
    if (bland) return price_bland(tol, dbest);
    T best = T(0);
    int cell = INT_MAX;
    if constexpr (NPL == 1) {
      // small tiles (at most 8 cells per lane at 16 x 16): the full Dantzig
      // scan every pivot costs less than the pivots a candidate list adds
      scan_full(best, cell);
      gmin_val_key(best, cell);
      dbest = best;
      return (best < -tol && cell != INT_MAX) ? cell : -1;
    }
    if (cand >= 0) {
      best = cost[cand] - s.pot[cand_a] - s.pot[m + cand_r];
      cell = key_rc(cand_a, cand_r);
    }
    if (!(best < -tol)) { best = T(0); cell = INT_MAX; }
    gmin_val_key(best, cell);
    if (!(best < -tol)) {
      scan_full(best, cell);
      gmin_val_key(best, cell);
    }
    dbest = best;
    return (best < -tol && cell != INT_MAX) ? cell : -1;
  }

  // rank of a leaving-path position = number of path positions above it
  __device__ __forceinline__ static int rank_of(const unsigned (&wbits)[NW], int p) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const unsigned x = wbits[w];
      if (w > (p >> 5)) c += __popc(x);
      else if (w == (p >> 5)) c += ((p & 31) == 31) ? 0 : __popc(x >> ((p & 31) + 1));
    }
    return c;
  }

  // One pivot on entering cell key `cell` with reduced cost dE < 0.
  // Returns true when the pivot moved flow (theta > 0).
  __device__ __forceinline__ bool pivot(int cell, T dE) { return pivot_impl<false>(cell, dE, 0, 0); }

  // The pivot proper.  Primal (DUAL false): the leaving edge and theta come
  // from the ratio test over the cycle's decreasing edges.  Dual: the
  // leaving edge (the one above node zd, flow -thd < 0) was chosen first and
  // the entering cell crosses its cut so that the edge is an increasing one
  // of the cycle; theta = thd brings its flow to zero.  The cycle update,
  // the re-hanging of the leaving side and the potential shift by dE are
  // the same in both.
  template <bool DUAL>
  __device__ __forceinline__ bool pivot_impl(int cell, T dE, int zd, long long thd) {
    const int ea = cell >> 8;
    const int eB = m + (cell & 0xff);
    const int pa = s.pos[ea];
    const int pb = s.pos[eB];
    // 1. cycle membership of owned nodes and the ratio test candidates.
    //    side 1: row side (ancestor of ea only), 2: column side.
    int side[NPL];
    long long th = LLONG_MAX;
    int tkey = INT_MAX;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      side[k] = 0;
      if (y < N) {
        const int p0 = t.pos[k], p1 = p0 + t.sz[k];
        const bool isA = p0 <= pa && pa < p1;
        const bool isB = p0 <= pb && pb < p1;
        side[k] = (isA != isB) ? (isA ? 1 : 2) : 0;
        // "-" edges: row children on the row side, column children on the
        // column side
        if (!DUAL && side[k] == (y < m ? 1 : 2)) {
          const int key = (edge_key(y, t.par[k]) << 7) | y;
          if (t.flow[k] < th || (t.flow[k] == th && key < tkey)) { th = t.flow[k]; tkey = key; }
        }
      }
    }
    if constexpr (DUAL) {
      th = thd;
      tkey = zd;
    } else {  // group minimum of (flow, key) with the integer reduction unit
      if (th < 0) bad = true;  // flows are never negative
      const unsigned long long uf = (unsigned long long)th;
      const unsigned hi = (unsigned)(uf >> 32), lo = (unsigned)uf;
      const unsigned mh = __reduce_min_sync(g.mask, hi);
      const unsigned ml = __reduce_min_sync(g.mask, hi == mh ? lo : 0xffffffffu);
      const bool eq = hi == mh && lo == ml;
      tkey = (int)__reduce_min_sync(g.mask, eq ? (unsigned)tkey : 0xffffffffu);
      th = (long long)(((unsigned long long)mh << 32) | ml);
      if (gany<G>(g, bad)) bad = true;
    }
    if (bad || tkey == INT_MAX || th < 0) { bad = true; return false; }
    // 2. shift theta around the cycle
    if (th > 0) {
#pragma unroll
      for (int k = 0; k < NPL; ++k)
        if (side[k]) t.flow[k] += (side[k] == (node_of(k) < m ? 1 : 2)) ? -th : th;
    }
    // 3. the leaving edge hangs from zL; its side holds the entering end e
    const int zL = tkey & 0x7f;
    const int P0 = s.pos[zL];
    const int Z = s.sz[zL];
    const int lside = (P0 <= pa && pa < P0 + Z) ? 1 : 2;
    const int enode = lside == 1 ? ea : eB;
    const int onode = lside == 1 ? eB : ea;
    const int posO = s.pos[onode];
    // leaving path p_0 = e ... p_k = zL: the side's nodes inside zL's
    // subtree, ranked by decreasing preorder position
    unsigned wbits[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) wbits[w] = 0u;
    bool onpath[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      onpath[k] = side[k] == lside && t.pos[k] >= P0 && t.pos[k] < P0 + Z;
      if (onpath[k]) {
#pragma unroll
        for (int w = 0; w < NW; ++w)
          if ((t.pos[k] >> 5) == w) wbits[w] |= 1u << (t.pos[k] & 31);
      }
    }
    int tot = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      wbits[w] = __reduce_or_sync(g.mask, wbits[w]);
      tot += __popc(wbits[w]);
    }
    const int kk = tot - 1;  // index of zL on the path
    int rank[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      rank[k] = -1;
      if (onpath[k]) {
        const int i = rank_of(wbits, t.pos[k]);
        rank[k] = i;
        s.ppos[i] = t.pos[k]; s.psz[i] = t.sz[k]; s.pnode[i] = node_of(k); s.pflow[i] = t.flow[k];
      }
    }
    g.sync();
    if (kk < 0 || kk >= N || s.pnode[0] != enode || s.pnode[kk] != zL) {
      bad = true;
      return false;
    }
    // 4. every owned node: new preorder position, size, potential; the
    //    re-rooted path takes its new parent edges
    const int remO = posO >= P0 + Z ? posO - Z : posO;
    const int Qi = remO + 1;
    const bool e_is_row = enode < m;
    const int nsteps = 32 - __clz(kk);  // ceil(log2(kk+1)): group-uniform trip count
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) {
        const int py = t.pos[k], sy = t.sz[k];
        if (py >= P0 && py < P0 + Z) {
          int lo = 0, hi = kk;  // deepest path node that is an ancestor
          for (int it = 0; it < nsteps; ++it) {
            const int mid = (lo + hi) >> 1;
            const int pp = s.ppos[mid];
            const bool anc = pp <= py && py < pp + s.psz[mid];
            hi = anc ? mid : hi;
            lo = anc ? lo : mid + 1;
          }
          const int i = lo;
          int off;
          if (i == 0) {
            off = py - s.ppos[0];
          } else {
            const int pp = s.ppos[i - 1], ps = s.psz[i - 1];
            off = ps + (py < pp ? py - s.ppos[i] : py - s.ppos[i] - ps);
          }
          t.pos[k] = Qi + off;
          if (py == s.ppos[i]) t.sz[k] = (i == 0) ? Z : Z - s.psz[i - 1];
          pot[k] += ((y < m) == e_is_row) ? dE : -dE;
        } else {
          const int r0 = py >= P0 + Z ? py - Z : py;
          t.pos[k] = r0 + (r0 >= Qi ? Z : 0);
          int ns = sy;
          if (py <= P0 && P0 < py + sy) ns -= Z;
          if (py <= posO && posO < py + sy) ns += Z;
          t.sz[k] = ns;
        }
        const int i = rank[k];
        if (i == 0) { t.par[k] = onode; t.flow[k] = th; }
        else if (i > 0) { t.par[k] = s.pnode[i - 1]; t.flow[k] = s.pflow[i - 1]; }
      }
    }
    g.sync();
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) { s.pos[y] = t.pos[k]; s.sz[y] = t.sz[k]; s.pot[y] = pot[k]; }
    }
    g.sync();
    return th > 0;
  }

  // Pivot from the current basis until no reduced cost is below -tol.
  // With fresh_stop, optimality is only accepted on potentials freshly
  // recomputed from the tree (an FP32 screen whose error bound already
  // covers the drift of incrementally updated potentials passes false).
  // Returns kStOk, kStNotConverged or kStInvalid; *pivots accumulates the
  // pivot count.
  __device__ __forceinline__ int run(int max_pivots, T tol, int* pivots, bool fresh_stop = true) {
    refresh_potentials();
    if (bad) return kStInvalid;
    int done = 0, degen = 0, since = 0;
    bool bland = false;
    int st = kStOk;
    for (;;) {
      T dE;
      const int cell = price(bland, tol, dE);
      if (cell < 0) {
        if (since == 0 || !fresh_stop) break;
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

  __device__ __forceinline__ int solve(int max_pivots, T tol, int* pivots, bool fresh_stop = true) {
    init_northwest();
    return run(max_pivots, tol, pivots, fresh_stop);
  }

  // ---- restart from a basis saved for other marginals -----------------
  // A loaded tree (load_tree) is usable when every node's preorder range
  // lies inside [0, N) and the root spans all N nodes.
  __device__ __forceinline__ bool tree_sane() const {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) {
        ok &= t.sz[k] >= 1 && t.pos[k] + t.sz[k] <= N;
        if (y == root) ok &= t.pos[k] == 0 && t.sz[k] == N;
        else ok &= t.par[k] >= 0 && t.par[k] < N && (y < m) != (t.par[k] < m);
      }
    }
    return !gany<G>(g, !ok);
  }

  // Flows of the current tree for the current marginals (prefix masses
  // s.P, s.Q): the edge above node y carries the net supply of y's subtree
  // (rows supply their mass, columns demand theirs), read off a prefix sum
  // of the supplies laid out in preorder, where a subtree is a contiguous
  // range.  Returns true (group-uniform) when no flow is negative.
  __device__ __forceinline__ bool recompute_flows() {
    long long* B = s.pflow;  // [N]: supplies by preorder position, then prefix sums
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) {
        long long b;
        if (y < m) b = s.P[y] - (y > 0 ? s.P[y - 1] : 0LL);
        else {
          const int r = y - m;
          b = -(s.Q[r] - (r > 0 ? s.Q[r - 1] : 0LL));
        }
        B[t.pos[k]] = b;
      }
    }
    g.sync();
    // inclusive prefix: lane l sums positions [l*NPL, l*NPL + NPL), then an
    // exclusive scan of the lanes' totals
    long long loc[NPL];
    long long run = 0;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int p = g.lane * NPL + k;
      run += p < N ? B[p] : 0LL;
      loc[k] = run;
    }
    long long incl = run;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const long long v = __shfl_up_sync(g.mask, incl, o, G);
      if (g.lane >= o) incl += v;
    }
    const long long excl = incl - run;
    g.sync();
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int p = g.lane * NPL + k;
      if (p < N) B[p] = excl + loc[k];
    }
    g.sync();
    bool neg = false;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) {
        if (y == root) {
          t.flow[k] = 0;
        } else {
          const int p0 = t.pos[k], p1 = p0 + t.sz[k] - 1;
          const long long net = B[p1] - (p0 > 0 ? B[p0 - 1] : 0LL);
          t.flow[k] = y < m ? net : -net;
          neg |= t.flow[k] < 0;
        }
      }
    }
    g.sync();
    return !gany<G>(g, neg);
  }

  // Dual simplex from a tree whose reduced costs are (about) non-negative
  // but whose flows may not be: while an edge carries negative flow, the
  // most negative one leaves (ties to the smallest cell); the entering cell
  // is the cell of least reduced cost among those crossing the leaving
  // edge's cut in the direction that can carry its deficit (into the
  // subtree below a row node, out of the subtree below a column node), so
  // every other reduced cost stays non-negative.  The potentials are
  // recomputed first and then shifted incrementally; a primal run() after
  // this refreshes them.  Returns kStOk once every flow is non-negative,
  // kStNotConverged at max_pivots, kStInvalid on an inconsistent tree.
  __device__ int run_dual(int max_pivots, int* pivots) {
    refresh_potentials();
    if (bad) return kStInvalid;
    int done = 0;
    int st = kStOk;
    const int mn = m * n;
    for (;;) {
      // leaving edge: the most negative flow (signed order on the unsigned
      // reduction unit: flip the sign bit), ties to the smallest edge key
      long long fmin = 0;
      int lkey = INT_MAX;
#pragma unroll
      for (int k = 0; k < NPL; ++k) {
        const int y = node_of(k);
        if (y < N && y != root) {
          const int key = (edge_key(y, t.par[k]) << 7) | y;
          if (t.flow[k] < fmin || (t.flow[k] < 0 && t.flow[k] == fmin && key < lkey)) {
            fmin = t.flow[k];
            lkey = key;
          }
        }
      }
      const unsigned long long uf = (unsigned long long)fmin ^ 0x8000000000000000ull;
      const unsigned hi = (unsigned)(uf >> 32), lo = (unsigned)uf;
      const unsigned mh = __reduce_min_sync(g.mask, hi);
      const unsigned ml = __reduce_min_sync(g.mask, hi == mh ? lo : 0xffffffffu);
      lkey = (int)__reduce_min_sync(g.mask, (hi == mh && lo == ml) ? (unsigned)lkey : 0xffffffffu);
      fmin = (long long)((((unsigned long long)mh << 32) | ml) ^ 0x8000000000000000ull);
      if (fmin >= 0) break;  // feasible
      if (done >= max_pivots) { st = kStNotConverged; break; }
      if (lkey == INT_MAX) { bad = true; st = kStInvalid; break; }
      const int zL = lkey & 0x7f;
      const int P0 = s.pos[zL], P1 = P0 + s.sz[zL];
      const bool zrow = zL < m;
      // entering cell: least reduced cost over the eligible cells
      T best = T(INFINITY);
      int cell = INT_MAX;
      int a = a0, r = r0;
      int o = a0 * cs + r0;
      const int ostep = sq * cs + sr, owrap = cs - n;
      for (int i = g.lane; i < mn; i += G) {
        const int qa = s.pos[a], qb = s.pos[m + r];
        const bool inA = P0 <= qa && qa < P1, inB = P0 <= qb && qb < P1;
        if (zrow ? (!inA && inB) : (inA && !inB)) {
          const T d = cost[o] - s.pot[a] - s.pot[m + r];
          if (d < best) { best = d; cell = key_rc(a, r); }
        }
        r += sr; a += sq; o += ostep;
        if (r >= n) { r -= n; ++a; o += owrap; }
      }
      gmin_val_key(best, cell);
      if (cell == INT_MAX || !(best < T(INFINITY))) { bad = true; st = kStInvalid; break; }
      pivot_impl<true>(cell, best, zL, -fmin);
      if (bad) { st = kStInvalid; break; }
      ++done;
    }
    if (pivots) *pivots += done;
    return st;
  }

  // Saved basis of one pair: per node parent, preorder position, subtree
  // size (bytes) and edge flow (WITH_FLOW false: the tree only), at [y] of
  // arrays with room for N nodes.
  template <bool WITH_FLOW = true>
  __device__ __forceinline__ void store_tree(unsigned char* par8, unsigned char* pos8,
                                             unsigned char* sz8, long long* flow) const {
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) {
        par8[y] = (unsigned char)(t.par[k] & 0xff);  // root: 255, recognised by pos 0
        pos8[y] = (unsigned char)t.pos[k];
        sz8[y] = (unsigned char)t.sz[k];
        if constexpr (WITH_FLOW) flow[y] = t.flow[k];
      }
    }
  }
  // Restore a saved basis (the marginals must be those it was saved with,
  // so its flows are still the basic solution).  WITH_FLOW false: the tree
  // only; the caller recomputes the flows (recompute_flows).
  template <bool WITH_FLOW = true>
  __device__ __forceinline__ void load_tree(const unsigned char* par8, const unsigned char* pos8,
                                            const unsigned char* sz8, const long long* flow) {
    int r0 = INT_MAX;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N) {
        t.pos[k] = pos8[y];
        t.par[k] = t.pos[k] == 0 ? -1 : (int)par8[y];
        t.sz[k] = sz8[y];
        if constexpr (WITH_FLOW) t.flow[k] = flow[y];
        else t.flow[k] = 0LL;
        s.pos[y] = t.pos[k];
        s.sz[y] = t.sz[k];
        if (t.pos[k] == 0) r0 = y;
      }
    }
    root = (int)__reduce_min_sync(g.mask, (unsigned)r0);
    g.sync();
  }

  // sum over tree edges of flow * cost, in the accumulator type A
  template <typename A>
  __device__ __forceinline__ A objective() const {
    A acc = A(0);
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N && y != root)
        acc += ((A)t.flow[k] * (A)kInvMass) * (A)cost[edge_idx(y, t.par[k])];
    }
    return gsum<G>(g, acc);
  }

  // Basis flows as (cell, w) records: one entry per node but the root
  // (entry y, or y-1 past the root).
  __device__ __forceinline__ void write_flows(int* cell, double* w, long long stride) const {
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = node_of(k);
      if (y < N && y != root) {
        const int p = t.par[k];
        const int row = y < m ? y : p;
        const int col = y < m ? p - m : y - m;
        const int e = y < root ? y : y - 1;
        cell[e] = (row << 16) | col;
        w[e] = (double)t.flow[k] * kInvMass;
      }
    }
    for (long long e = N - 1 + g.lane; e < stride; e += G) {
      cell[e] = -1;
      w[e] = 0.0;
    }
  }
};

}  // namespace d2k
