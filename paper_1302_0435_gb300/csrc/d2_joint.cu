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
// The rounds follow Kelley's cutting-plane method: the next p minimises the
// largest cut over the simplex, a small LP solved here per cluster by a
// revised primal simplex on its dual, where each new cut enters as a new
// column and the previous optimal basis stays feasible.  The model minimum
// is a lower bound of min F, the best F seen an upper bound; a cluster stops
// when the two agree to the requested relative gap, and keeps the weights of
// the upper bound.  Cuts are stored per unit of the cluster's total omega.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "d2_internal.h"

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

// One block per active cluster: the cut of this round and F at its p.  Each
// thread sums a fixed stride of the members into its own shared row, then
// column c is summed over the rows in order (deterministic).  Row layout:
// a_0..a_{n-1}, F, b, omega.
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
  __shared__ double tot[kMaxJointN + 3];
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) s += rows[(size_t)k * cols + c];
    tot[c] = s;
  }
  __syncthreads();
  const double Om = tot[n + 2];
  const int kk = jv.nk[j];
  double* a = jv.cutA + ((size_t)j * jv.itmax + kk) * jv.nmax;
  for (int r = threadIdx.x; r < n; r += blockDim.x) a[r] = tot[r] / Om;
  if (threadIdx.x == 0) {
    jv.cutB[(size_t)j * jv.itmax + kk] = tot[n + 1] / Om;
    jv.F[j] = tot[n] / Om;
    jv.omsum[j] = Om;
  }
}

// ---- the master LP -----------------------------------------------------
// Model: min theta s.t. theta >= a_k.p + b_k (k < nk), sum p = 1, p >= 0.
// Solved through its dual, with R = n + 1 rows:
//   max sum_k b_k mu_k + nu
//   s.t. sum_k mu_k = 1                              (row 0)
//        nu - sum_k a_kr mu_k + sigma_r = 0          (row 1 + r)
//        mu, sigma >= 0, nu free (always basic).
// The simplex multipliers of the optimal basis are (theta, p).  Variable ids:
// mu_k = k, sigma_r = kSig + r, nu = kNu.  Cuts enter scaled by 1/S (S: the
// largest entry of the first cut) so the matrix entries are O(1).
constexpr int kSig = 1 << 20;
constexpr int kNu = -1;

struct Master {
  const JointView& jv;
  long long j;
  int n, R, nk;
  double S;
  double *Binv, *aug, *col, *y, *xB, *cB, *fac;
  int* bvar;
  unsigned char* inB;

  __device__ Master(const JointView& jv_, long long j_, int n_, int nk_, unsigned char* sm)
      : jv(jv_), j(j_), n(n_), R(n_ + 1), nk(nk_) {
    double* d = reinterpret_cast<double*>(sm);
    Binv = d; d += R * R;
    aug = d; d += 2 * R * R;
    col = d; d += R;
    y = d; d += R;
    xB = d; d += R;
    cB = d; d += R;
    fac = d; d += R;
    bvar = reinterpret_cast<int*>(d);
    inB = reinterpret_cast<unsigned char*>(bvar + R);
  }
  __device__ const double* cut(int k) const {
    return jv.cutA + ((size_t)j * jv.itmax + k) * jv.nmax;
  }
  __device__ double cutb(int k) const { return jv.cutB[(size_t)j * jv.itmax + k]; }
  __device__ double cost(int v) const {
    if (v == kNu) return 1.0;
    if (v >= kSig) return 0.0;
    return cutb(v) / S;
  }
  // column of variable v into col[] (all threads call; ends synchronised)
  __device__ void load_col(int v) {
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
      double x;
      if (v == kNu) x = i == 0 ? 0.0 : 1.0;
      else if (v >= kSig) x = (i == 1 + (v - kSig)) ? 1.0 : 0.0;
      else x = i == 0 ? 1.0 : -cut(v)[i - 1] / S;
      col[i] = x;
    }
    __syncthreads();
  }
  // Binv = B^-1 by Gauss-Jordan with partial pivoting on [B | I]; xB = Binv e0.
  __device__ bool refactor() {
    const int W2 = 2 * R;
    for (int l = 0; l < R; ++l) {
      const int v = bvar[l];
      for (int i = threadIdx.x; i < R; i += blockDim.x) {
        double x;
        if (v == kNu) x = i == 0 ? 0.0 : 1.0;
        else if (v >= kSig) x = (i == 1 + (v - kSig)) ? 1.0 : 0.0;
        else x = i == 0 ? 1.0 : -cut(v)[i - 1] / S;
        aug[i * W2 + l] = x;
        aug[i * W2 + R + l] = i == l ? 1.0 : 0.0;
      }
    }
    __syncthreads();
    __shared__ int piv_s;
    __shared__ int ok_s;
    if (threadIdx.x == 0) ok_s = 1;
    for (int c = 0; c < R; ++c) {
      if (threadIdx.x == 0) {  // R <= 65: a serial pivot search is cheap
        int best = c;
        double bv = fabs(aug[c * W2 + c]);
        for (int i = c + 1; i < R; ++i) {
          const double x = fabs(aug[i * W2 + c]);
          if (x > bv) { bv = x; best = i; }
        }
        piv_s = best;
        if (!(bv > 1e-13)) ok_s = 0;
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
      const double inv = 1.0 / aug[c * W2 + c];
      for (int i = threadIdx.x; i < R; i += blockDim.x) fac[i] = aug[i * W2 + c];
      __syncthreads();
      for (int e = threadIdx.x; e < W2; e += blockDim.x) aug[c * W2 + e] *= inv;
      __syncthreads();
      for (int e = threadIdx.x; e < R * W2; e += blockDim.x) {
        const int i = e / W2, k = e - i * W2;
        if (i != c) aug[e] -= fac[i] * aug[c * W2 + k];
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      const int i = e / R, k = e - i * R;
      Binv[e] = aug[i * W2 + R + k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
      xB[i] = Binv[i * R + 0];
      cB[i] = cost(bvar[i]);
    }
    __syncthreads();
    return true;
  }
  __device__ void duals() {
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
      double s = 0.0;
      for (int l = 0; l < R; ++l) s += cB[l] * Binv[l * R + i];
      y[i] = s;
    }
    __syncthreads();
  }
};

// Best entering candidate of the block: the largest reduced cost above tol
// (Dantzig), or with bland the smallest variable id above tol.
__device__ void block_pick(double d, int v, bool bland, double* sd, int* sv, double* out_d,
                           int* out_v) {
  // order key: Dantzig -> larger d first, then smaller id; Bland -> smaller id
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double d2 = __shfl_down_sync(0xffffffffu, d, o);
    const int v2 = __shfl_down_sync(0xffffffffu, v, o);
    bool take;
    if (v2 == INT_MAX) take = false;
    else if (v == INT_MAX) take = true;
    else if (bland) take = v2 < v;
    else take = d2 > d || (d2 == d && v2 < v);
    if (take) { d = d2; v = v2; }
  }
  if (lane == 0) { sd[warp] = d; sv[warp] = v; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bd = sd[0];
    int bv = sv[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      const double d2 = sd[w];
      const int v2 = sv[w];
      bool take;
      if (v2 == INT_MAX) take = false;
      else if (bv == INT_MAX) take = true;
      else if (bland) take = v2 < bv;
      else take = d2 > bd || (d2 == bd && v2 < bv);
      if (take) { bd = d2; bv = v2; }
    }
    *out_d = bd;
    *out_v = bv;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(128) k_joint_master(JointView jv, const long long* coff,
                                                      const double* w64) {
  extern __shared__ __align__(16) unsigned char sm[];
  const long long j = blockIdx.x;
  if (jv.status[j] != kJActive) return;
  const long long c0 = coff[j];
  const int n = (int)(coff[j + 1] - c0);
  const int kk = jv.nk[j];  // the cut written this round
  const int nk = kk + 1;
  __shared__ double S_s, sd[4];
  __shared__ int sv[4], enter_s, leave_s, state_s;
  __shared__ double dbest_s;
  // incumbent
  const double F = jv.F[j];
  const bool better = F < jv.ub[j];
  __syncthreads();
  if (better) {
    for (int r = threadIdx.x; r < n; r += blockDim.x) jv.pbest[c0 + r] = w64[c0 + r];
  }
  if (threadIdx.x == 0) {
    if (better) jv.ub[j] = F;
    if (kk == 0) {
      double S = fabs(jv.cutB[(size_t)j * jv.itmax]);
      const double* a0 = jv.cutA + (size_t)j * jv.itmax * jv.nmax;
      for (int r = 0; r < n; ++r) S = fmax(S, fabs(a0[r]));
      jv.scale[j] = S > 0.0 ? S : 1.0;
    }
    S_s = jv.scale[j];
    jv.nk[j] = nk;
  }
  __syncthreads();
  Master M(jv, j, n, nk, sm);
  M.S = S_s;
  int* bv_g = jv.bvar + (size_t)j * (jv.nmax + 1);
  if (kk == 0) {
    // mu_0 = 1, nu = min_r a_0r, sigma_r basic for every other r
    if (threadIdx.x == 0) {
      const double* a0 = M.cut(0);
      int rs = 0;
      for (int r = 1; r < n; ++r)
        if (a0[r] < a0[rs]) rs = r;
      int l = 0;
      M.bvar[l++] = 0;
      M.bvar[l++] = kNu;
      for (int r = 0; r < n; ++r)
        if (r != rs) M.bvar[l++] = kSig + r;
    }
  } else {
    for (int l = threadIdx.x; l < M.R; l += blockDim.x) M.bvar[l] = bv_g[l];
  }
  __syncthreads();
  const int nflag = nk + n;
  for (int e = threadIdx.x; e < nflag; e += blockDim.x) M.inB[e] = 0;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int l = 0; l < M.R; ++l) {
      const int v = M.bvar[l];
      if (v >= kSig) M.inB[nk + (v - kSig)] = 1;
      else if (v >= 0) M.inB[v] = 1;
    }
  int status = kJActive;
  if (!M.refactor()) status = kJFail;
  const double tol_d = 1e-12, tol_p = 1e-9;
  const int cap = 50 * M.R + 4 * nk;
  int pivots = 0, degen = 0, since = 0;
  bool bland = false;
  while (status == kJActive) {
    M.duals();
    // price every nonbasic mu_k and sigma_r
    double bd = -INFINITY;
    int bvv = INT_MAX;
    for (int k = threadIdx.x; k < nk + n; k += blockDim.x) {
      if (M.inB[k]) continue;
      double d;
      int v;
      if (k < nk) {
        const double* a = M.cut(k);
        double s = M.cutb(k) / M.S - M.y[0];
        for (int r = 0; r < n; ++r) s += M.y[1 + r] * (a[r] / M.S);
        d = s;
        v = k;
      } else {
        d = -M.y[1 + (k - nk)];
        v = kSig + (k - nk);
      }
      if (d > tol_d) {
        const bool take = bvv == INT_MAX || (bland ? v < bvv : (d > bd || (d == bd && v < bvv)));
        if (take) { bd = d; bvv = v; }
      }
    }
    block_pick(bd, bvv, bland, sd, sv, &dbest_s, &enter_s);
    const int q = enter_s;
    if (q == INT_MAX) break;  // optimal
    if (pivots >= cap) { status = kJFail; break; }
    M.load_col(q);
    // alpha = Binv * col (into fac)
    for (int i = threadIdx.x; i < M.R; i += blockDim.x) {
      double s = 0.0;
      for (int l = 0; l < M.R; ++l) s += M.Binv[i * M.R + l] * M.col[l];
      M.fac[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int lv = -1;
      double br = INFINITY, ba = 0.0;
      for (int l = 0; l < M.R; ++l) {
        if (M.bvar[l] == kNu) continue;
        const double al_ = M.fac[l];
        if (!(al_ > tol_p)) continue;
        const double xl = M.xB[l] > 0.0 ? M.xB[l] : 0.0;
        const double rt = xl / al_;
        bool take;
        if (lv < 0) take = true;
        else if (rt < br - 1e-12 * (1.0 + br)) take = true;
        else if (rt > br + 1e-12 * (1.0 + br)) take = false;
        else if (bland) take = M.bvar[l] < M.bvar[lv];
        else take = al_ > ba;
        if (take) { lv = l; br = rt; ba = al_; }
      }
      leave_s = lv;
      state_s = lv < 0 ? kJFail : kJActive;  // unbounded cannot happen for a valid model
    }
    __syncthreads();
    if (state_s != kJActive) { status = kJFail; break; }
    const int l = leave_s;
    const double apiv = M.fac[l];
    const double theta = (M.xB[l] > 0.0 ? M.xB[l] : 0.0) / apiv;
    // x_B and B^-1 update
    for (int i = threadIdx.x; i < M.R; i += blockDim.x)
      if (i != l) M.xB[i] -= theta * M.fac[i];
    __syncthreads();
    for (int e = threadIdx.x; e < M.R; e += blockDim.x) M.Binv[l * M.R + e] /= apiv;
    __syncthreads();
    for (int e = threadIdx.x; e < M.R * M.R; e += blockDim.x) {
      const int i = e / M.R, k = e - i * M.R;
      if (i != l) M.Binv[e] -= M.fac[i] * M.Binv[l * M.R + k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int old = M.bvar[l];
      if (old >= kSig) M.inB[nk + (old - kSig)] = 0;
      else if (old >= 0) M.inB[old] = 0;
      if (q >= kSig) M.inB[nk + (q - kSig)] = 1;
      else M.inB[q] = 1;
      M.bvar[l] = q;
      M.xB[l] = theta;
      M.cB[l] = M.cost(q);
    }
    __syncthreads();
    ++pivots;
    if (theta <= 1e-15) { if (++degen > 2 * M.R) bland = true; }
    else { degen = 0; bland = false; }
    if (++since >= 32) {
      since = 0;
      if (!M.refactor()) { status = kJFail; break; }
    }
  }
  if (status == kJActive && since > 0 && !M.refactor()) status = kJFail;
  M.duals();
  // lower bound and the next p
  __shared__ double psum_s;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += M.y[1 + r] > 0.0 ? M.y[1 + r] : 0.0;
    psum_s = s;
  }
  __syncthreads();
  const double lb = M.y[0] * M.S;
  const double ub = jv.ub[j];
  if (status == kJActive) {
    if (ub <= 0.0 || ub - lb <= jv.tol * ub) status = kJDone;
    else if (nk >= jv.itmax) status = kJCap;
    else if (!(psum_s > 0.0)) status = kJFail;
  }
  for (int l = threadIdx.x; l < M.R; l += blockDim.x) bv_g[l] = M.bvar[l];
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double pr = M.y[1 + r] > 0.0 ? M.y[1 + r] : 0.0;
    jv.wnext[c0 + r] = status == kJActive ? pr / psum_s : jv.pbest[c0 + r];
  }
  if (threadIdx.x == 0) {
    jv.lb[j] = lb;
    jv.status[j] = status;
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

size_t master_smem(int nmax, int itmax) {
  const int R = nmax + 1;
  return (size_t)(3 * R * R + 5 * R) * 8 + (size_t)R * 4 + (size_t)(itmax + nmax) + 16;
}

}  // namespace

size_t joint_state_bytes(long long K, long long Tc, int nmax, int itmax) {
  return al((size_t)K * itmax * nmax * 8) + al((size_t)K * itmax * 8) +
         al((size_t)K * (nmax + 1) * 4) + 2 * al((size_t)K * 4) + 6 * al((size_t)K * 8) +
         2 * al((size_t)Tc * 8) + al(8);
}

JointView joint_view(void* mem, long long K, long long Tc, int nmax, int itmax, double tol) {
  unsigned char* p = static_cast<unsigned char*>(mem);
  JointView v{};
  v.K = K;
  v.itmax = itmax;
  v.nmax = nmax;
  v.tol = tol;
  v.cutA = reinterpret_cast<double*>(p); p += al((size_t)K * itmax * nmax * 8);
  v.cutB = reinterpret_cast<double*>(p); p += al((size_t)K * itmax * 8);
  v.bvar = reinterpret_cast<int*>(p); p += al((size_t)K * (nmax + 1) * 4);
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
  if (jv.nmax > kMaxJointN) return cudaErrorInvalidValue;
  const size_t cs = (size_t)128 * (jv.nmax + 3) * 8;
  cudaError_t e = cudaFuncSetAttribute(k_joint_cut, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cs);
  if (e != cudaSuccess) return e;
  k_joint_cut<<<(unsigned)jv.K, 128, cs, st>>>(jv, pstart, pobj, omega, W, pot, pstride, pst, coff,
                                               w64);
  const size_t ms = master_smem(jv.nmax, jv.itmax);
  e = cudaFuncSetAttribute(k_joint_master, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms);
  if (e != cudaSuccess) return e;
  k_joint_master<<<(unsigned)jv.K, 128, ms, st>>>(jv, coff, w64);
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
