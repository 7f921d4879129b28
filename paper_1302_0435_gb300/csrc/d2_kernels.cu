// d2_kernels.cu -- the small kernels of the assignment step for sm_103a
// (bag validation, centroid preparation, node bins, single-pair cost
// matrices, fixed-order sums) and the dispatch of the solver launches
// (per-pair Mallows distance, Eq. (D2opt) with z fixed; nearest-centroid
// assignment, Alg. 2 Step 2) to the units d2_npl1..4.cu that instantiate
// them for 1..4 tree nodes per lane.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include "d2_internal.h"
#include "d2_solver.cuh"

#include "d2_solve.cuh"

namespace d2k {

__global__ void k_scan_bags(const long long* off, long long count, int* info) {
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < count;
       b += (long long)gridDim.x * blockDim.x) {
    const long long m = off[b + 1] - off[b];
    if (m < 1 || (b == 0 && off[0] != 0)) atomicOr(&info[1], 1);
    atomicMax(&info[0], (int)(m > INT_MAX ? INT_MAX : (m < 0 ? 0 : m)));
  }
}

__global__ void k_check_bags(const long long* off, long long count, int maxm, int* err) {
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < count;
       b += (long long)gridDim.x * blockDim.x) {
    const long long m = off[b + 1] - off[b];
    if (m < 1 || m > maxm || (b == 0 && off[0] != 0)) atomicOr(err, kErrInvalid);
  }
}

template <int G>
__global__ void k_prep_centroids(const void* loc, int ldt, const void* w, int wdt,
                                 const long long* off, long long K, int d, float* loc32,
                                 double* loc64, long long* Qpre, double* w64, int* err) {
  Grp<G> g;
  const int gpb = blockDim.x / G;
  for (long long j = (long long)blockIdx.x * gpb + threadIdx.x / G; j < K;
       j += (long long)gridDim.x * gpb) {
    const long long c0 = off[j];
    const long long n = off[j + 1] - c0;
    if (n < 1 || n > 64) {
      if (g.lane == 0) atomicOr(err, kErrInvalid);
      continue;
    }
    bool ok = wdt == 0 ? load_prefix<G>(g, static_cast<const double*>(w) + c0, (int)n, Qpre + c0)
                       : load_prefix<G>(g, static_cast<const float*>(w) + c0, (int)n, Qpre + c0);
    if (!ok && g.lane == 0) atomicOr(err, kErrInvalid);
    // normalised FP64 weights as seen by the solver
    for (int r = g.lane; r < n; r += G) {
      const long long prev = r > 0 ? Qpre[c0 + r - 1] : 0LL;
      w64[c0 + r] = ok ? (double)(Qpre[c0 + r] - prev) * kInvMass : 0.0;
    }
    for (long long e = g.lane; e < n * d; e += G) {
      const double v = ldx<double>(loc, ldt, c0 * d + e);
      loc64[c0 * d + e] = v;
      loc32[c0 * d + e] = (float)v;
    }
  }
}

__global__ void k_bin_of(const long long* off, long long count, int nmax, int* bins) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const long long m = off[i + 1] - off[i];
    const long long nn = m + nmax;
    bins[i] = (m < 1 || nn > 128) ? -1 : (int)((nn + 31) / 32 - 1);
  }
}

__global__ void k_cost_matrix(ObjView ob, CentView cv, long long i, long long j, int mode,
                              double* C) {
  const long long o0 = ob.off[i];
  const int m = (int)(ob.off[i + 1] - o0);
  const long long c0 = cv.off[j];
  const int n = (int)(cv.off[j + 1] - c0);
  for (int t = threadIdx.x; t < m * n; t += blockDim.x) {
    const int a = t / n, r = t % n;
    if (cv.A) {  // symbol table (ids checked before the launch; clamped reads)
      int xs = (int)ldx<double>(ob.loc, ob.ldt, o0 + a), ys = (int)cv.loc64[c0 + r];
      xs = xs < 0 ? 0 : (xs >= cv.A ? cv.A - 1 : xs);
      ys = ys < 0 ? 0 : (ys >= cv.A ? cv.A - 1 : ys);
      C[t] = mode == 0 ? cv.tab64[xs * cv.A + ys] : (double)cv.tab32[xs * cv.A + ys];
    } else if (mode == 0) {
      double acc = 0.0;
      for (int k = 0; k < cv.d; ++k) {
        const double df = ldx<double>(ob.loc, ob.ldt, (o0 + a) * cv.d + k) - cv.loc64[(c0 + r) * cv.d + k];
        acc = fma(df, df, acc);
      }
      C[t] = acc;
    } else {
      float acc = 0.f;
      for (int k = 0; k < cv.d; ++k) {
        const float df = ldx<float>(ob.loc, ob.ldt, (o0 + a) * cv.d + k) - cv.loc32[(c0 + r) * cv.d + k];
        acc = fmaf(df, df, acc);
      }
      C[t] = (double)acc;
    }
  }
}

__global__ void k_check_symbols(const void* loc, int ldt, long long T, int A, int* err) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = ldx<double>(loc, ldt, t);
    if (!(v >= 0.0 && v < (double)A && v == floor(v))) atomicOr(err, kErrInvalid);
  }
}

__global__ void k_check_bag_symbols(const void* loc, int ldt, const long long* off, long long count,
                                    int A, int* err) {
  const long long T = off[count];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = ldx<double>(loc, ldt, t);
    if (!(v >= 0.0 && v < (double)A && v == floor(v))) atomicOr(err, kErrInvalid);
  }
}

// Mean and spread of one bag from its masses (inclusive int64 prefix, units
// of 2^-62) in FP64: lanes over coordinates for the mean, over supports for
// the spread.
template <typename GetX>
__device__ __forceinline__ void bag_mean_var(const Grp<32>& g, const long long* pre, int m, int d,
                                             GetX x, double* mu, double* var) {
  for (int k = g.lane; k < d; k += 32) {
    double acc = 0.0;
    for (int a = 0; a < m; ++a) {
      const double w = (double)(pre[a] - (a > 0 ? pre[a - 1] : 0LL)) * kInvMass;
      acc = fma(w, x(a, k), acc);
    }
    mu[k] = acc;
  }
  __syncwarp();
  double v = 0.0;
  for (int a = g.lane; a < m; a += 32) {
    const double w = (double)(pre[a] - (a > 0 ? pre[a - 1] : 0LL)) * kInvMass;
    double s2 = 0.0;
    for (int k = 0; k < d; ++k) {
      const double df = x(a, k) - mu[k];
      s2 = fma(df, df, s2);
    }
    v = fma(w, s2, v);
  }
  v = gsum<32>(g, v);
  if (g.lane == 0) *var = v;
}

// One warp per object: the masses the solver will use (load_prefix), then
// the mean and spread.
__global__ void k_bag_moments(ObjView ob, double* mu, double* var) {
  __shared__ long long pre[4][64];
  Grp<32> g;
  const int wb = threadIdx.x >> 5;
  for (long long i = (long long)blockIdx.x * 4 + wb; i < ob.count; i += (long long)gridDim.x * 4) {
    const long long o0 = ob.off[i];
    const int m = (int)(ob.off[i + 1] - o0);
    const int d = ob.d;
    bool ok = m >= 1 && m <= 64;
    if (ok) ok = ob.wdt == 0 ? load_prefix<32>(g, static_cast<const double*>(ob.w) + o0, m, pre[wb])
                             : load_prefix<32>(g, static_cast<const float*>(ob.w) + o0, m, pre[wb]);
    if (!ok) {
      if (g.lane == 0) var[i] = NAN;
      continue;
    }
    const void* loc = ob.loc;
    const int ldt = ob.ldt;
    bag_mean_var(g, pre[wb], m, d,
                 [&](int a, int k) { return ldx<double>(loc, ldt, (o0 + a) * d + k); },
                 mu + i * d, var + i);
    __syncwarp();
  }
}

__global__ void k_cent_moments(CentView cv, double* mu, double* var) {
  Grp<32> g;
  const int wb = threadIdx.x >> 5;
  for (long long j = (long long)blockIdx.x * 4 + wb; j < cv.K; j += (long long)gridDim.x * 4) {
    const long long c0 = cv.off[j];
    const int n = (int)(cv.off[j + 1] - c0);
    const int d = cv.d;
    const double* y = cv.loc64 + c0 * d;
    bag_mean_var(g, cv.Qpre + c0, n, d, [&](int r, int k) { return y[r * d + k]; }, mu + j * d,
                 var + j);
    __syncwarp();
  }
}

// One warp per object: UB over its segment's K centroids, then the keep bits.
__global__ void k_prune_keep(ObjView ob, long long seg_size, int K, long long KT, int d,
                             const double* mu_o, const double* var_o, const double* mu_c,
                             const double* var_c, unsigned* keep, int kw) {
  Grp<32> g;
  const int wb = threadIdx.x >> 5;
  for (long long i = (long long)blockIdx.x * 4 + wb; i < ob.count; i += (long long)gridDim.x * 4) {
    const long long cb = seg_of(ob, i, seg_size) * (long long)K;
    const double vi = var_o[i];
    const double* xi = mu_o + i * d;
    const bool valid = !isnan(vi) && cb + K <= KT;
    auto lb = [&](int j) {
      const double* yj = mu_c + (cb + j) * d;
      double s2 = 0.0;
      for (int k = 0; k < d; ++k) {
        const double df = xi[k] - yj[k];
        s2 = fma(df, df, s2);
      }
      return s2;
    };
    double best = INFINITY;
    if (valid)
      for (int j = g.lane; j < K; j += 32) best = fmin(best, lb(j) + var_c[cb + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    const double ub = (vi + best) * (1.0 + 0x1p-40);
    for (int w = 0; w < kw; ++w) {
      const int j = w * 32 + g.lane;
      // keep unless the lower bound is above the upper bound (NaN keeps)
      const bool k = j < K && (!valid || !(lb(j) * (1.0 - 0x1p-40) > ub));
      const unsigned bits = __ballot_sync(0xffffffffu, k);
      if (g.lane == 0) keep[i * kw + w] = bits;
    }
  }
}

// Fixed-order sum (one block, strided partials then a tree): deterministic.
__global__ void k_sum_fixed(const double* v, long long n, double* out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) acc += v[t];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// ------------------------------------------------------------ launchers --

static unsigned long long g_launches = 0;
void note_launches(long long k) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }
long long launches() { return (long long)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

// Sum of the solver counters of the units that hold the solver kernels.
cudaError_t solver_stats(long long out[6]) {
  cudaError_t (*const units[4])(long long*) = {stats_npl1, stats_npl2, stats_npl3, stats_npl4};
  for (int i = 0; i < 6; ++i) out[i] = 0;
  for (auto f : units) {
    long long v[6];
    const cudaError_t e = f(v);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < 6; ++i) out[i] += v[i];
  }
  return cudaSuccess;
}

int device_sms(int dev) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

cudaError_t scan_bags(const long long* off, long long count, int* d_info, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_info, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (count <= 0) return cudaSuccess;
  const long long blocks = (count + 255) / 256;
  k_scan_bags<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(off, count, d_info);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t check_bags(const long long* off, long long count, int maxm, int* d_err,
                       cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const long long blocks = (count + 255) / 256;
  k_check_bags<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(off, count, maxm, d_err);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t prep_centroids(const void* loc, int ldt, const void* w, int wdt, const long long* off,
                           long long K, int d, float* loc32, double* loc64, long long* Qpre,
                           double* w64, int* d_err, cudaStream_t st) {
  const long long blocks = (K + 3) / 4;
  k_prep_centroids<32><<<(unsigned)(blocks < 65535 ? blocks : 65535), 128, 0, st>>>(
      loc, ldt, w, wdt, off, K, d, loc32, loc64, Qpre, w64, d_err);
  note_launches(1);
  return cudaGetLastError();
}

// Tree shape for supports up to (mmax, nmax): one warp (G = 32 lanes) per
// pair, each lane owning NPL tree nodes (m+n <= 32*NPL).
#define D2_BINS(X) \
  X(32, 1)         \
  X(32, 2)         \
  X(32, 3)         \
  X(32, 4)

static bool pick_shape(int mmax, int nmax, int* G, int* npl) {
  const int N = mmax + nmax;
  if (N > 128) return false;
  *G = 32;
  *npl = (N + 31) / 32;
  return true;
}

cudaError_t mallows_pairs(const ObjView& ob, const CentView& cv, const long long* pobj,
                          const long long* pcen, long long npairs, const SolveCfg& cfg,
                          double* dist2, FlowOut fo, int* status, int* d_err, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  int G, NP;
  if (!pick_shape(cfg.mmax, cfg.nmax, &G, &NP)) return cudaErrorInvalidValue;
#define X(g_, n_)                                                                          \
  if (G == g_ && NP == n_)                                                                \
    return mallows_pairs_npl##n_(ob, cv, pobj, pcen, npairs, cfg, dist2, fo, status, d_err, st);
  D2_BINS(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t assign(const ObjView& ob, const CentView& cv, long long seg_size, int K,
                   const SolveCfg& cfg, const double* omega, int* labels, double* dist2,
                   double* eps_terms, FlowOut fo, int* cand, int* d_err, cudaStream_t st,
                   const WarmStore* ws, const TcWork* tw) {
  if (ob.count <= 0) return cudaSuccess;
  int G, NP;
  if (!pick_shape(cfg.mmax, cfg.nmax, &G, &NP)) return cudaErrorInvalidValue;
#define X(g_, n_)                                                                            \
  if (G == g_ && NP == n_)                                                                  \
    return assign_npl##n_(ob, cv, seg_size, K, cfg, omega, labels, dist2, eps_terms, fo, cand, d_err, st, ws, tw);
  D2_BINS(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t bin_objects(const ObjView& ob, int nmax, int* bins_out, cudaStream_t st) {
  if (ob.count <= 0) return cudaSuccess;
  const unsigned b = (unsigned)std::min<long long>((ob.count + 255) / 256, 4096);
  k_bin_of<<<b, 256, 0, st>>>(ob.off, ob.count, nmax, bins_out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t cost_matrix(const ObjView& ob, const CentView& cv, long long i, long long j, int mode,
                        double* C, cudaStream_t st) {
  k_cost_matrix<<<1, 256, 0, st>>>(ob, cv, i, j, mode, C);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t check_symbols(const void* loc, int ldt, long long T, int A, int* d_err,
                          cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  const unsigned b = (unsigned)std::min<long long>((T + 255) / 256, 4096);
  k_check_symbols<<<b, 256, 0, st>>>(loc, ldt, T, A, d_err);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t check_bag_symbols(const void* loc, int ldt, const long long* off, long long count,
                              int A, int* d_err, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_check_bag_symbols<<<(unsigned)(152 * 4), 256, 0, st>>>(loc, ldt, off, count, A, d_err);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t bag_moments(const ObjView& ob, double* mu, double* var, cudaStream_t st) {
  if (ob.count <= 0) return cudaSuccess;
  const long long blocks = (ob.count + 3) / 4;
  k_bag_moments<<<(unsigned)(blocks < 8192 ? blocks : 8192), 128, 0, st>>>(ob, mu, var);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t cent_moments(const CentView& cv, double* mu, double* var, cudaStream_t st) {
  if (cv.K <= 0) return cudaSuccess;
  const long long blocks = (cv.K + 3) / 4;
  k_cent_moments<<<(unsigned)(blocks < 8192 ? blocks : 8192), 128, 0, st>>>(cv, mu, var);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t prune_keep(const ObjView& ob, long long seg_size, int K, long long KT, int d,
                       const double* mu_o, const double* var_o, const double* mu_c,
                       const double* var_c, unsigned* keep, int kw, cudaStream_t st) {
  if (ob.count <= 0) return cudaSuccess;
  if (kw < (K + 31) / 32) return cudaErrorInvalidValue;
  const long long blocks = (ob.count + 3) / 4;
  k_prune_keep<<<(unsigned)(blocks < 8192 ? blocks : 8192), 128, 0, st>>>(
      ob, seg_size, K, KT, d, mu_o, var_o, mu_c, var_c, keep, kw);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t sum_fixed_order(const double* v, long long n, double* out, cudaStream_t st) {
  k_sum_fixed<<<1, 256, 0, st>>>(v, n, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace d2k
