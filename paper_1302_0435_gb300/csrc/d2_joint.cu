// d2_joint.cu -- Alg. 1 Step 1: new centroid weights p_z for every cluster
// from the joint LP of Eq. (WeightedD2) under the constraints of Eq. (D2opt),
// support locations fixed.
//
// With p fixed the joint LP separates into the members' own transportation
// LPs, so its value is F(p) = sum_i omega_i W_i(p): convex and piecewise
// linear over the simplex, and any minimiser p* with each member's optimal
// flows at p* is an optimum of the joint LP.  An exact member solve gives
// potentials (u, v), c - u - v >= 0, and by LP duality
// W_i(p') >= q_i.u + p'.v for every p' (with equality at the solved p).  So
// one round of member solves yields one supporting cut of F:
//   F(p') >= a.p' + b,  a = sum_i omega_i v_i,  b = sum_i omega_i (W_i - p.v_i).
// The members are dealt round-robin (in increasing object order) into G
// groups, and each group's sum gets its own cut, F_g(p') >= a_g.p' + b_g,
// so the model of F = sum_g F_g is far tighter than one aggregate cut per
// round (Kelley's cutting-plane method with disaggregated cuts).  The next
// p minimises sum_g max_k (a_gk.p + b_gk) over the simplex, a small LP
// solved per cluster by a revised primal simplex on its dual, where the
// new cuts enter as new columns and the previous optimal basis stays
// feasible.  The model minimum is a lower bound of min F, the best F seen
// an upper bound; a cluster stops when the two agree to the requested
// relative gap, and keeps the weights of the upper bound.  Cuts are stored
// per unit of the cluster's total omega.
#include <cuda_runtime.h>

#include <atomic>
#include <cfloat>
#include <climits>
#include <cmath>

#include "d2_internal.h"
#include "d2_joint.h"

namespace d2k {
namespace {

__host__ __device__ inline size_t al(size_t x) { return (x + 255) / 256 * 256; }

// Cluster status codes (also returned to the host).
constexpr int kJActive = 0, kJDone = 1, kJCap = 2, kJEmpty = 3, kJFail = 4;

__global__ void k_joint_init(JointView jv, const long long* start, const long long* coff,
                             const double* w64) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < jv.K;
       j += (long long)gridDim.x * blockDim.x) {
    jv.status[j] = start[j + 1] > start[j] ? kJActive : kJEmpty;
    jv.nk[j] = 0;
    jv.ub[j] = INFINITY;
    jv.lb[j] = -INFINITY;
    for (long long e = coff[j]; e < coff[j + 1]; ++e) {
      jv.wnext[e] = w64[e];
      jv.pbest[e] = w64[e];
    }
  }
}

// Exclusive prefix of the active clusters' member counts.  One block.
__global__ void k_joint_scan(const long long* start, const int* status, long long K,
                             long long* pstart) {
  __shared__ long long wsum[32];
  __shared__ long long carry_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (long long base = 0; base < K; base += blockDim.x) {
    const long long j = base + tid;
    const long long v = (j < K && status[j] == kJActive) ? start[j + 1] - start[j] : 0;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long s = lane < nw ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += u;
      }
      if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    const long long c = carry_s;
    if (j < K) pstart[j] = c + (warp > 0 ? wsum[warp - 1] : 0) + x - v;
    __syncthreads();
    if (tid == 0) carry_s = c + wsum[nw - 1];
    __syncthreads();
  }
  if (tid == 0) pstart[K] = carry_s;
}

// The pairs (i, C(i)) of the active clusters, one warp per cluster, members
// in increasing object order.
__global__ void k_joint_fill(const int* order, const long long* start, const int* status,
                             long long K, const long long* pstart, long long* pobj,
                             long long* pcen) {
  const int lane = threadIdx.x & 31;
  for (long long j = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; j < K;
       j += ((long long)gridDim.x * blockDim.x) >> 5) {
    if (status[j] != kJActive) continue;
    const long long s0 = start[j], cnt = start[j + 1] - s0, q0 = pstart[j];
    for (long long t = lane; t < cnt; t += 32) {
      pobj[q0 + t] = order[s0 + t];
      pcen[q0 + t] = j;
    }
  }
}

// One block per active cluster: this round's G group cuts and F at its p.
// Member t of the cluster (sorted order) belongs to group t % G, and G
// divides the block size, so every thread's members lie in one group.
// Each thread sums its members into its own shared row, then column c of
// group g is summed over that group's rows in thread order
// (deterministic).  Row layout: a_0..a_{n-1}, F, b, omega.
__global__ void k_joint_cut(JointView jv, const long long* pstart, const long long* pobj,
                            const double* omega, const double* W, const double* pot,
                            long long pstride, const int* pst, const long long* coff,
                            const double* w64) {
  extern __shared__ double rows[];
  const long long j = blockIdx.x;
  if (jv.status[j] != kJActive) return;
  const long long c0 = coff[j];
  const int n = (int)(coff[j + 1] - c0);
  const int cols = n + 3;
  const int G = jv.G;
  double* my = rows + (size_t)threadIdx.x * cols;
  for (int c = 0; c < cols; ++c) my[c] = 0.0;
  int bad = 0;
  for (long long t = pstart[j] + threadIdx.x; t < pstart[j + 1]; t += blockDim.x) {
    const long long i = pobj[t];
    const double om = omega ? omega[i] : 1.0;
    const double Wt = W[t];
    if (pst[t] != 0 || !isfinite(Wt)) { bad = 1; continue; }
    const double* v = pot + t * pstride;
    double pv = 0.0;
    for (int r = 0; r < n; ++r) {
      pv += w64[c0 + r] * v[r];
      my[r] += om * v[r];
    }
    my[n] += om * Wt;
    my[n + 1] += om * (Wt - pv);
    my[n + 2] += om;
  }
  bad = __syncthreads_or(bad);
  if (bad) {
    if (threadIdx.x == 0) jv.status[j] = kJFail;
    return;
  }
  // totals of the cluster (F, omega) first: every row in order
  __shared__ double tot_s[2];
  if (threadIdx.x < 2) {
    const int c = n + (threadIdx.x == 0 ? 0 : 2);
    double acc = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) acc += rows[(size_t)k * cols + c];
    tot_s[threadIdx.x] = acc;
  }
  __syncthreads();
  const double Om = tot_s[1];
  const int kk = jv.nk[j];
  const int per = (int)blockDim.x / G;  // rows of a group: threads g, g+G, ...
  for (int e = threadIdx.x; e < G * (n + 1); e += blockDim.x) {
    const int g = e / (n + 1), c = e - g * (n + 1);
    const int col = c < n ? c : n + 1;  // a_r, then b
    double acc = 0.0;
    for (int k = 0; k < per; ++k) acc += rows[(size_t)(g + k * G) * cols + col];
    if (c < n) jv.cutA[(((size_t)j * jv.itmax + kk) * G + g) * jv.nmax + c] = acc / Om;
    else jv.cutB[((size_t)j * jv.itmax + kk) * G + g] = acc / Om;
  }
  if (threadIdx.x == 0) {
    jv.F[j] = tot_s[0] / Om;
    jv.omsum[j] = Om;
  }
}

// ---- the master LP -----------------------------------------------------
// Model: min sum_g theta_g s.t. theta_g >= a_gk.p + b_gk (every round k < nk
// and group g), sum p = 1, p >= 0.  Solved through its dual, with
// R = G + n rows:
//   max sum_{k,g} b_gk mu_gk + nu
//   s.t. sum_k mu_gk = 1                              (row g < G)
//        nu - sum_{k,g} a_gk,r mu_gk + sigma_r = 0    (row G + r)
//        mu, sigma >= 0, nu free (always basic).
// The simplex multipliers of the optimal basis are (theta_g, p).  Variable
// ids: mu_gk = k*G + g, sigma_r = kSig + r, nu = kNu.  Cuts enter scaled by
// 1/S (S: the largest entry of the first round's cuts) so the matrix
// entries are O(1).  The basis and its inverse carry over from round to
// round (new cuts are new nonbasic columns); the inverse is updated by
// pivots and recomputed by Gauss-Jordan every kRefactor pivots.  FP64
// throughout: the lower bound certifies the relative gap.
constexpr int kSig = 1 << 24;
constexpr int kNu = -1;
constexpr int kRefactor = 64;
constexpr int kMT = 256;  // master block size
// Multipliers below this are rounding noise of a zero weight: they are set
// to 0 so that the support carries no mass (and keeps its location).
constexpr double kPTiny = 1e-13;

struct Master {
  const JointView& jv;
  long long j;
  int n, G, R, nk;
  double S, iS;  // the scale (a power of two) and its exact reciprocal
  double *Binv, *aug, *col, *y, *xB, *cB, *fac, *row;
  float* y32;
  int* bvar;
  unsigned* inB;  // basic flags as bits: [nk*G] mu, then [n] sigma

  __device__ Master(const JointView& jv_, long long j_, int n_, int nk_, unsigned char* sm)
      : jv(jv_), j(j_), n(n_), G(jv_.G), R(jv_.G + n_), nk(nk_) {
    double* d = reinterpret_cast<double*>(sm);
    Binv = d; d += R * R;
    aug = d; d += 2 * R * R;
    col = d; d += R;
    y = d; d += R;
    xB = d; d += R;
    cB = d; d += R;
    fac = d; d += R;
    row = d; d += R;
    y32 = reinterpret_cast<float*>(d);
    bvar = reinterpret_cast<int*>(y32 + ((R + 1) & ~1));
    inB = reinterpret_cast<unsigned*>(bvar + R);
  }
  __device__ const double* cut(int id) const {  // id = k*G + g
    return jv.cutA + ((size_t)j * jv.itmax * G + id) * jv.nmax;
  }
  __device__ double cutb(int id) const { return jv.cutB[(size_t)j * jv.itmax * G + id]; }
  __device__ const float* cut32(int id) const {
    return jv.cutA32 + ((size_t)j * jv.itmax * G + id) * jv.nmax;
  }
  __device__ float cutb32(int id) const { return jv.cutB32[(size_t)j * jv.itmax * G + id]; }
  // FP32 reduced cost of mu flag e (scaled units) and a bound on its
  // distance to the FP64 value: inputs rounded to FP32 (2^-24 each), n + 2
  // rounded terms summed in FP32; (n + 8) * 2^-23 of the sum of |terms|
  // covers both with a factor of two to spare.
  __device__ float reduced32(int e, float* bound) const {
    const float* a = cut32(e);
    const float b = cutb32(e), yg = y32[e % G];
    float s = b - yg, t = fabsf(b) + fabsf(yg);
    for (int r = 0; r < n; ++r) {
      const float pr = y32[G + r] * a[r];
      s += pr;
      t += fabsf(pr);
    }
    *bound = (float)(n + 8) * 0x1p-23f * t;
    return s;
  }
  __device__ double cost(int v) const {
    if (v == kNu) return 1.0;
    if (v >= kSig) return 0.0;
    return cutb(v) * iS;
  }
  __device__ int flag(int v) const { return v >= kSig ? nk * G + (v - kSig) : v; }
  __device__ bool basic(int f) const { return (inB[f >> 5] >> (f & 31)) & 1u; }
  __device__ void set_basic(int f, bool on) {  // one thread at a time
    if (on) inB[f >> 5] |= 1u << (f & 31);
    else inB[f >> 5] &= ~(1u << (f & 31));
  }
  // entry i of the column of variable v
  __device__ double entry(int v, int i) const {
    if (v == kNu) return i >= G ? 1.0 : 0.0;
    if (v >= kSig) return i == G + (v - kSig) ? 1.0 : 0.0;
    if (i < G) return i == v % G ? 1.0 : 0.0;
    return -cut(v)[i - G] * iS;
  }
  // reduced cost of nonbasic flag e (mu or sigma) and its variable id
  __device__ double reduced(int e, int* v) const {
    if (e < nk * G) {
      const double* a = cut(e);
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int r = 0;
      for (; r + 4 <= n; r += 4) {
        s0 += y[G + r] * a[r];
        s1 += y[G + r + 1] * a[r + 1];
        s2 += y[G + r + 2] * a[r + 2];
        s3 += y[G + r + 3] * a[r + 3];
      }
      for (; r < n; ++r) s0 += y[G + r] * a[r];
      *v = e;
      return (cutb(e) + ((s0 + s1) + (s2 + s3))) * iS - y[e % G];
    }
    *v = kSig + (e - nk * G);
    return -y[G + (e - nk * G)];
  }
  // xB = Binv * rhs (rhs: 1 on the G group rows), cB, and y = cB * Binv
  __device__ void basics() {
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
      double x = 0.0;
      for (int g = 0; g < G; ++g) x += Binv[i * R + g];
      xB[i] = x;
      cB[i] = cost(bvar[i]);
    }
    __syncthreads();
    matvec<true>(cB, y);
    for (int i = threadIdx.x; i < R; i += blockDim.x) y32[i] = (float)y[i];
    __syncthreads();
  }
  // out = Binv * v (TRANS false) or out = v * Binv (TRANS true), R x R in
  // FP64: P = blockDim/R threads per output entry each sum a slice of the
  // products (so every warp, on every SM sub-partition, shares the FP64
  // work), then one thread per entry adds the P partial sums in order.  The
  // partials use aug, which only refactor needs.  Ends synchronised.
  template <bool TRANS>
  __device__ void matvec(const double* v, double* out) {
    // >= 3 (R <= kMaxJointR); at most 2R, so the P*R partials fit in aug (2 R^2)
    const int P = min((int)blockDim.x / R, 2 * R);
    const int t = threadIdx.x;
    if (t < P * R) {
      const int i = t / P, pp = t - i * P;
      const int l0 = pp * R / P, l1 = (pp + 1) * R / P;
      double s0 = 0.0;
      for (int l = l0; l < l1; ++l) s0 += (TRANS ? Binv[l * R + i] : Binv[i * R + l]) * v[l];
      aug[t] = s0;
    }
    __syncthreads();
    for (int i = t; i < R; i += blockDim.x) {
      double s = 0.0;
      for (int pp = 0; pp < P; ++pp) s += aug[i * P + pp];
      out[i] = s;
    }
    __syncthreads();
  }
  // Binv = B^-1 by Gauss-Jordan with partial pivoting on [B | I] (rows with
  // a zero factor are skipped: B is mostly unit and 0/1 columns).
  __device__ bool refactor() {
    const int W2 = 2 * R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < R; i += nw)
      for (int l = lane; l < R; l += 32) {
        aug[i * W2 + l] = entry(bvar[l], i);
        aug[i * W2 + R + l] = i == l ? 1.0 : 0.0;
      }
    __syncthreads();
    __shared__ int piv_s;
    __shared__ int ok_s;
    __shared__ double inv_s;
    __shared__ double pv_s[kMT / 32];
    __shared__ int pi_s[kMT / 32];
    if (threadIdx.x == 0) ok_s = 1;
    for (int c = 0; c < R; ++c) {
      // pivot row: the largest |aug[i][c]|, i >= c (ties: smallest i)
      double bv = -1.0;
      int bi = INT_MAX;
      for (int i = c + threadIdx.x; i < R; i += blockDim.x) {
        const double x = fabs(aug[i * W2 + c]);
        if (x > bv) { bv = x; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double x2 = __shfl_down_sync(0xffffffffu, bv, o);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        if (x2 > bv || (x2 == bv && i2 < bi)) { bv = x2; bi = i2; }
      }
      if ((threadIdx.x & 31) == 0) { pv_s[threadIdx.x >> 5] = bv; pi_s[threadIdx.x >> 5] = bi; }
      __syncthreads();
      if (threadIdx.x == 0) {
        double b2 = pv_s[0];
        int i2 = pi_s[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
          if (pv_s[w] > b2 || (pv_s[w] == b2 && pi_s[w] < i2)) { b2 = pv_s[w]; i2 = pi_s[w]; }
        piv_s = i2;
        if (!(b2 > 1e-13) || i2 >= R) ok_s = 0;
      }
      __syncthreads();
      if (!ok_s) return false;
      const int pr = piv_s;
      if (pr != c)
        for (int e = threadIdx.x; e < W2; e += blockDim.x) {
          const double t = aug[c * W2 + e];
          aug[c * W2 + e] = aug[pr * W2 + e];
          aug[pr * W2 + e] = t;
        }
      __syncthreads();
      if (threadIdx.x == 0) inv_s = 1.0 / aug[c * W2 + c];  // one division, shared
      for (int i = threadIdx.x; i < R; i += blockDim.x) fac[i] = aug[i * W2 + c];
      __syncthreads();
      const double inv = inv_s;
      for (int e = threadIdx.x; e < W2; e += blockDim.x) aug[c * W2 + e] *= inv;
      __syncthreads();
      // a warp per row; rows with a zero factor (most: B is mostly unit
      // and 0/1 columns) are skipped whole
      for (int i = warp; i < R; i += nw) {
        const double f = fac[i];
        if (i == c || f == 0.0) continue;
        for (int k = lane; k < W2; k += 32) aug[i * W2 + k] -= f * aug[c * W2 + k];
      }
      __syncthreads();
    }
    for (int i = warp; i < R; i += nw)
      for (int k = lane; k < R; k += 32) Binv[i * R + k] = aug[i * W2 + R + k];
    __syncthreads();
    basics();
    return true;
  }
};

// Entering candidate of the block from each thread's (d, v): the largest d
// (Dantzig; ties to the smaller id), or with bland the smallest id.
// v == INT_MAX: no candidate.  Candidates have d > 0, whose IEEE patterns
// order like their values, so the warps reduce integer keys (the FP64
// compares of a shuffle tree would each take the FP64 pipe).
__device__ void block_pick(double d, int v, bool bland, double* sd, int* sv, int* out_v,
                           double* out_d) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool has = v != INT_MAX;
  const unsigned long long key = has ? (unsigned long long)__double_as_longlong(d) : 0ull;
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  int vw;
  unsigned long long kw;
  if (bland) {
    vw = __reduce_min_sync(0xffffffffu, has ? v : INT_MAX);
    const unsigned owner = __ballot_sync(0xffffffffu, has && v == vw);
    const long long k2 = __shfl_sync(0xffffffffu, (long long)key, owner ? __ffs(owner) - 1 : 0);
    kw = owner ? (unsigned long long)k2 : 0ull;
  } else {
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    vw = __reduce_min_sync(0xffffffffu, (has && hi == mh && lo == ml) ? v : INT_MAX);
    kw = ((unsigned long long)mh << 32) | ml;
  }
  if (lane == 0) { sd[warp] = __longlong_as_double((long long)kw); sv[warp] = vw; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long bk = (unsigned long long)__double_as_longlong(sd[0]);
    int bv = sv[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      const unsigned long long k2 = (unsigned long long)__double_as_longlong(sd[w]);
      const int v2 = sv[w];
      bool take;
      if (v2 == INT_MAX) take = false;
      else if (bv == INT_MAX) take = true;
      else if (bland) take = v2 < bv;
      else take = k2 > bk || (k2 == bk && v2 < bv);
      if (take) { bk = k2; bv = v2; }
    }
    *out_v = bv;
    *out_d = __longlong_as_double((long long)bk);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kMT) k_joint_master(JointView jv, const long long* coff,
                                                      const double* w64) {
  extern __shared__ __align__(16) unsigned char sm[];
  const long long j = blockIdx.x;
  if (jv.status[j] != kJActive) return;
  const long long c0 = coff[j];
  const int n = (int)(coff[j + 1] - c0);
  const int G = jv.G;
  const int kk = jv.nk[j];  // the round whose cuts were written
  const int nk = kk + 1;
  __shared__ double S_s, sd[kMT / 32], dq_s;
  __shared__ int sv[kMT / 32], enter_s, leave_s, state_s;
  __shared__ double inva_s;
  // incumbent
  const double F = jv.F[j];
  const bool better = F < jv.ub[j];
  __syncthreads();
  if (better)
    for (int r = threadIdx.x; r < n; r += blockDim.x) jv.pbest[c0 + r] = w64[c0 + r];
  if (threadIdx.x == 0) {
    if (better) jv.ub[j] = F;
    if (kk == 0) {
      double S = 0.0;
      for (int g = 0; g < G; ++g) {
        S = fmax(S, fabs(jv.cutB[(size_t)j * jv.itmax * G + g]));
        const double* a0 = jv.cutA + ((size_t)j * jv.itmax * G + g) * jv.nmax;
        for (int r = 0; r < n; ++r) S = fmax(S, fabs(a0[r]));
      }
      // a power of two >= the largest magnitude: scaling by it is exact
      int ex = 0;
      frexp(S, &ex);
      jv.scale[j] = S > 0.0 ? ldexp(1.0, ex) : 1.0;
    }
    S_s = jv.scale[j];
    jv.nk[j] = nk;
  }
  __syncthreads();
  Master M(jv, j, n, nk, sm);
  M.S = S_s;
  M.iS = 1.0 / S_s;  // exact: S is a power of two
  const int R = M.R;
  // FP32 copies of this round's cuts, scaled (the pricing filter reads them)
  for (int e = threadIdx.x; e < G * (n + 1); e += blockDim.x) {
    const int g = e / (n + 1), c = e - g * (n + 1);
    const int id = kk * G + g;
    if (c < n) jv.cutA32[((size_t)j * jv.itmax * G + id) * jv.nmax + c] = (float)(M.cut(id)[c] * M.iS);
    else jv.cutB32[(size_t)j * jv.itmax * G + id] = (float)(M.cutb(id) * M.iS);
  }
  int* bv_g = jv.bvar + (size_t)j * (jv.G + jv.nmax);
  double* bi_g = jv.binv + (size_t)j * (jv.G + jv.nmax) * (jv.G + jv.nmax);
  if (kk == 0) {
    // mu_g0 = 1 for every group, nu = min_r sum_g a_g0r, sigma_r basic for
    // every other r
    if (threadIdx.x == 0) {
      int rs = 0;
      double best = INFINITY;
      for (int r = 0; r < n; ++r) {
        double A = 0.0;
        for (int g = 0; g < G; ++g) A += M.cut(g)[r];
        if (A < best) { best = A; rs = r; }
      }
      int l = 0;
      for (int g = 0; g < G; ++g) M.bvar[l++] = g;
      M.bvar[l++] = kNu;
      for (int r = 0; r < n; ++r)
        if (r != rs) M.bvar[l++] = kSig + r;
    }
  } else {
    for (int l = threadIdx.x; l < R; l += blockDim.x) M.bvar[l] = bv_g[l];
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) M.Binv[e] = bi_g[e];
  }
  __syncthreads();
  const int nflag = nk * G + n;
  for (int e = threadIdx.x; e < (nflag + 31) / 32; e += blockDim.x) M.inB[e] = 0u;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int l = 0; l < R; ++l)
      if (M.bvar[l] != kNu) M.set_basic(M.flag(M.bvar[l]), true);
  __syncthreads();
  int status = kJActive;
  int since = kk == 0 ? 0 : jv.since[j];
  if (kk == 0 || since >= kRefactor) {
    if (!M.refactor()) status = kJFail;
    since = 0;
  } else {
    M.basics();
  }
  const double tol_d = 1e-12, tol_p = 1e-9;
  const int cap = 50 * R + 4 * nk * G;
  const int fresh0 = kk * G;  // this round's cuts: flags [fresh0, nk*G), then sigma
  int pivots = 0, degen = 0;
  bool bland = false;
  while (status == kJActive) {
    // partial pricing first (this round's cuts and the sigma columns), all
    // columns when that finds nothing or under Bland's rule
    int q = INT_MAX;
    for (int pass = bland ? 1 : 0; pass < 2 && q == INT_MAX; ++pass) {
      const int lo = pass == 0 ? fresh0 : 0, hi = nflag;  // (M.y32 follows M.y)
      double bd = -INFINITY;
      int bvv = INT_MAX;
      for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        if (M.basic(e)) continue;
        if (e < nk * G) {  // FP32 filter: only a cut that may enter is priced in FP64
          float eb;
          const float d32 = M.reduced32(e, &eb);
          if (!((double)d32 + (double)eb > tol_d)) continue;
        }
        int v;
        const double d = M.reduced(e, &v);
        if (d > tol_d) {
          const bool take =
              bvv == INT_MAX || (bland ? v < bvv : (d > bd || (d == bd && v < bvv)));
          if (take) { bd = d; bvv = v; }
        }
      }
      block_pick(bd, bvv, bland, sd, sv, &enter_s, &dq_s);
      q = enter_s;
    }
    if (q == INT_MAX) break;  // optimal
    if (pivots >= cap) { status = kJFail; break; }
    const double dq = dq_s;
    for (int i = threadIdx.x; i < R; i += blockDim.x) M.col[i] = M.entry(q, i);
    __syncthreads();
    M.matvec<false>(M.col, M.fac);  // alpha = Binv * col
    {  // ratio test over the basic rows (nu never leaves), in two passes
       // (Harris): the smallest ratio x_B / alpha over the rows with
       // alpha > tol_p, then among the rows within 1e-12 (1 + r*) of it the
       // largest alpha (Bland: the smallest variable).  The ratios go to
       // shared memory (aug is free here); one warp reduces integer keys
       // (non-negative doubles order like their bit patterns).
      for (int i = threadIdx.x; i < R; i += blockDim.x) {
        const double a = M.fac[i];
        const bool cand = M.bvar[i] != kNu && a > tol_p;
        M.aug[i] = cand ? (M.xB[i] > 0.0 ? M.xB[i] : 0.0) / a : -1.0;  // -1: no candidate
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long kmin = ~0ull;
        for (int i = lane; i < R; i += 32) {
          const double r = M.aug[i];
          if (r >= 0.0) {
            const unsigned long long k = (unsigned long long)__double_as_longlong(r);
            kmin = k < kmin ? k : kmin;
          }
        }
        const unsigned mh = __reduce_min_sync(0xffffffffu, (unsigned)(kmin >> 32));
        const unsigned ml = __reduce_min_sync(0xffffffffu, (unsigned)(kmin >> 32) == mh ? (unsigned)kmin : ~0u);
        const unsigned long long kbest = ((unsigned long long)mh << 32) | ml;
        int row = INT_MAX;
        if (kbest != ~0ull) {
          const double rs = __longlong_as_double((long long)kbest);
          const double thr = rs + 1e-12 * (1.0 + rs);
          // this lane's best row within the threshold
          unsigned long long ak = 0ull;
          int av = INT_MAX, ar = INT_MAX;
          for (int i = lane; i < R; i += 32) {
            const double r = M.aug[i];
            if (r >= 0.0 && r <= thr) {
              const unsigned long long k = (unsigned long long)__double_as_longlong(M.fac[i]);
              const int vid = M.bvar[i];
              const bool take = ar == INT_MAX ||
                                (bland ? vid < av : (k > ak || (k == ak && vid < av)));
              if (take) { ak = k; av = vid; ar = i; }
            }
          }
          int vw;
          if (bland) {
            vw = __reduce_min_sync(0xffffffffu, av);
          } else {
            const unsigned h2 = __reduce_max_sync(0xffffffffu, (unsigned)(ak >> 32));
            const unsigned l2 = __reduce_max_sync(0xffffffffu, (unsigned)(ak >> 32) == h2 ? (unsigned)ak : 0u);
            const unsigned long long kw = ((unsigned long long)h2 << 32) | l2;
            vw = __reduce_min_sync(0xffffffffu, (ar != INT_MAX && ak == kw) ? av : INT_MAX);
          }
          const unsigned own = __ballot_sync(0xffffffffu, ar != INT_MAX && av == vw);
          row = own ? __shfl_sync(0xffffffffu, ar, __ffs(own) - 1) : INT_MAX;
        }
        if (lane == 0) {
          leave_s = row;
          state_s = row == INT_MAX ? kJFail : kJActive;
          if (row != INT_MAX) inva_s = 1.0 / M.fac[row];  // one division, shared
        }
      }
      __syncthreads();
    }
    if (state_s != kJActive) { status = kJFail; break; }
    const int l = leave_s;
    const double inva = inva_s;
    const double theta = (M.xB[l] > 0.0 ? M.xB[l] : 0.0) * inva;
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
      if (i != l) M.xB[i] -= theta * M.fac[i];
      M.row[i] = M.Binv[l * R + i] * inva;  // new row l of Binv
    }
    __syncthreads();
    {  // a warp per row of Binv; a row with a zero factor keeps its values
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int i = warp; i < R; i += nw) {
        const double f = M.fac[i];
        if (i == l) {
          for (int k = lane; k < R; k += 32) M.Binv[i * R + k] = M.row[k];
        } else if (f != 0.0) {
          for (int k = lane; k < R; k += 32) M.Binv[i * R + k] -= f * M.row[k];
        }
      }
    }
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
      M.y[i] += dq * M.row[i];
      M.y32[i] = (float)M.y[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int old = M.bvar[l];
      if (old != kNu) M.set_basic(M.flag(old), false);
      M.set_basic(M.flag(q), true);
      M.bvar[l] = q;
      M.xB[l] = theta;
      M.cB[l] = M.cost(q);
    }
    __syncthreads();
    ++pivots;
    if (theta <= 1e-15) { if (++degen > 2 * R) bland = true; }
    else { degen = 0; bland = false; }
    if (++since >= kRefactor) {
      since = 0;
      if (!M.refactor()) { status = kJFail; break; }
    }
  }
  M.basics();  // multipliers recomputed from the inverse for the bound
  // lower bound sum_g theta_g and the next p
  __shared__ double psum_s, lb_s;
  if (threadIdx.x == 0) {
    double s = 0.0, t = 0.0;
    for (int r = 0; r < n; ++r) s += M.y[G + r] > kPTiny ? M.y[G + r] : 0.0;
    for (int g = 0; g < G; ++g) t += M.y[g];
    psum_s = s;
    lb_s = t * M.S;
  }
  __syncthreads();
  const double lb = lb_s;
  const double ub = jv.ub[j];
  if (status == kJActive) {
    if (ub <= 0.0 || ub - lb <= jv.tol * ub) status = kJDone;
    else if (nk >= jv.itmax) status = kJCap;
    else if (!(psum_s > 0.0)) status = kJFail;
  }
  for (int i = threadIdx.x; i < R; i += blockDim.x) bv_g[i] = M.bvar[i];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) bi_g[e] = M.Binv[e];
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double pr = M.y[G + r] > kPTiny ? M.y[G + r] : 0.0;
    jv.wnext[c0 + r] = status == kJActive ? pr / psum_s : jv.pbest[c0 + r];
  }
  if (threadIdx.x == 0) {
    jv.lb[j] = lb;
    jv.status[j] = status;
    jv.since[j] = since;
    atomicAdd(jv.pivots, (unsigned long long)pivots);
  }
}

// Clusters still active after the last round keep their best weights.
__global__ void k_joint_finish(JointView jv, const long long* coff) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < jv.K;
       j += (long long)gridDim.x * blockDim.x) {
    if (jv.status[j] == kJActive) {
      jv.status[j] = kJCap;
      for (long long e = coff[j]; e < coff[j + 1]; ++e) jv.wnext[e] = jv.pbest[e];
    }
  }
}

__global__ void k_joint_out(JointView jv, double* eps, int* iters, int* status) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < jv.K;
       j += (long long)gridDim.x * blockDim.x) {
    const bool has = jv.status[j] != kJEmpty && jv.nk[j] > 0;
    if (eps) eps[j] = has ? jv.ub[j] * jv.omsum[j] : 0.0;
    if (iters) iters[j] = jv.nk[j];
    if (status) status[j] = jv.status[j];
  }
}

unsigned blocks_for(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

size_t master_smem(int nmax, int itmax, int G) {
  const int R = G + nmax;
  return (size_t)(3 * R * R + 6 * R) * 8 + (size_t)(R + 1) * 4 + (size_t)R * 4 +
         ((size_t)itmax * G + nmax + 31) / 32 * 4 + 16;
}

std::atomic<long long> g_rounds{0}, g_mpiv{0};

}  // namespace

void joint_note(long long rounds, long long pivots) {
  g_rounds += rounds;
  g_mpiv += pivots;
}

void joint_counters(int64_t* rounds, int64_t* pivots) {
  *rounds = g_rounds.load();
  *pivots = g_mpiv.load();
}

size_t joint_state_bytes(long long K, long long Tc, int nmax, int itmax, int G) {
  return al((size_t)K * itmax * G * nmax * 8) + al((size_t)K * itmax * G * 8) +
         al((size_t)K * itmax * G * nmax * 4) + al((size_t)K * itmax * G * 4) +
         al((size_t)K * (G + nmax) * 4) + al((size_t)K * (G + nmax) * (G + nmax) * 8) +
         3 * al((size_t)K * 4) + 6 * al((size_t)K * 8) + 2 * al((size_t)Tc * 8) + al(8);
}

JointView joint_view(void* mem, long long K, long long Tc, int nmax, int itmax, int G,
                     double tol) {
  unsigned char* p = static_cast<unsigned char*>(mem);
  JointView v{};
  v.K = K;
  v.itmax = itmax;
  v.nmax = nmax;
  v.G = G;
  v.tol = tol;
  v.cutA = reinterpret_cast<double*>(p); p += al((size_t)K * itmax * G * nmax * 8);
  v.cutB = reinterpret_cast<double*>(p); p += al((size_t)K * itmax * G * 8);
  v.cutA32 = reinterpret_cast<float*>(p); p += al((size_t)K * itmax * G * nmax * 4);
  v.cutB32 = reinterpret_cast<float*>(p); p += al((size_t)K * itmax * G * 4);
  v.bvar = reinterpret_cast<int*>(p); p += al((size_t)K * (G + nmax) * 4);
  v.binv = reinterpret_cast<double*>(p); p += al((size_t)K * (G + nmax) * (G + nmax) * 8);
  v.since = reinterpret_cast<int*>(p); p += al((size_t)K * 4);
  v.nk = reinterpret_cast<int*>(p); p += al((size_t)K * 4);
  v.status = reinterpret_cast<int*>(p); p += al((size_t)K * 4);
  v.F = reinterpret_cast<double*>(p); p += al((size_t)K * 8);
  v.ub = reinterpret_cast<double*>(p); p += al((size_t)K * 8);
  v.lb = reinterpret_cast<double*>(p); p += al((size_t)K * 8);
  v.omsum = reinterpret_cast<double*>(p); p += al((size_t)K * 8);
  v.scale = reinterpret_cast<double*>(p); p += al((size_t)K * 8);
  p += al((size_t)K * 8);
  v.pbest = reinterpret_cast<double*>(p); p += al((size_t)Tc * 8);
  v.wnext = reinterpret_cast<double*>(p); p += al((size_t)Tc * 8);
  v.pivots = reinterpret_cast<unsigned long long*>(p);
  return v;
}

// The clusters [k0, k1) of a joint state as a state of their own: every
// per-cluster array shifted by k0 (the per-support arrays keep their global
// offsets, which the callers' coff + k0 supplies).
JointView joint_sub(const JointView& v, long long k0, long long k1) {
  JointView s = v;
  const size_t G = (size_t)v.G, nm = (size_t)v.nmax, it = (size_t)v.itmax, R = G + nm;
  const size_t k = (size_t)k0;
  s.cutA += k * it * G * nm;
  s.cutB += k * it * G;
  s.cutA32 += k * it * G * nm;
  s.cutB32 += k * it * G;
  s.bvar += k * R;
  s.binv += k * R * R;
  s.since += k;
  s.nk += k;
  s.status += k;
  s.F += k;
  s.ub += k;
  s.lb += k;
  s.omsum += k;
  s.scale += k;
  s.K = k1 - k0;
  return s;
}

cudaError_t joint_init(const JointView& jv, const long long* start, const long long* coff,
                       const double* w64, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(jv.pivots, 0, 8, st);
  if (e != cudaSuccess) return e;
  k_joint_init<<<blocks_for(jv.K), 256, 0, st>>>(jv, start, coff, w64);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t joint_list(const JointView& jv, const int* order, const long long* start,
                       long long* pstart, long long* pobj, long long* pcen, cudaStream_t st) {
  k_joint_scan<<<1, 1024, 0, st>>>(start, jv.status, jv.K, pstart);
  const long long warps = jv.K;
  const unsigned gb = (unsigned)((warps * 32 + 255) / 256 < 8192 ? (warps * 32 + 255) / 256 : 8192);
  k_joint_fill<<<gb > 0 ? gb : 1, 256, 0, st>>>(order, start, jv.status, jv.K, pstart, pobj, pcen);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t joint_round(const JointView& jv, const long long* pstart, const long long* pobj,
                        const double* omega, const double* W, const double* pot,
                        long long pstride, const int* pst, const long long* coff,
                        const double* w64, cudaStream_t st) {
  if (jv.nmax > kMaxJointN || jv.G < 1 || 128 % jv.G != 0 || jv.G + jv.nmax > kMaxJointR)
    return cudaErrorInvalidValue;
  const size_t cs = (size_t)128 * (jv.nmax + 3) * 8;
  cudaError_t e = cudaFuncSetAttribute(k_joint_cut, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cs);
  if (e != cudaSuccess) return e;
  k_joint_cut<<<(unsigned)jv.K, 128, cs, st>>>(jv, pstart, pobj, omega, W, pot, pstride, pst, coff,
                                               w64);
  const size_t ms = master_smem(jv.nmax, jv.itmax, jv.G);
  e = cudaFuncSetAttribute(k_joint_master, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms);
  if (e != cudaSuccess) return e;
  k_joint_master<<<(unsigned)jv.K, kMT, ms, st>>>(jv, coff, w64);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t joint_finish(const JointView& jv, const long long* coff, double* eps, int* iters,
                         int* status, cudaStream_t st) {
  k_joint_finish<<<blocks_for(jv.K), 256, 0, st>>>(jv, coff);
  k_joint_out<<<blocks_for(jv.K), 256, 0, st>>>(jv, eps, iters, status);
  note_launches(2);
  return cudaGetLastError();
}

}  // namespace d2k
