// d2_solve.cuh -- device side of the solver kernels and their launch
// templates, shared by the translation units that instantiate them (one per
// nodes-per-lane shape, compiled in parallel).  Everything here has internal
// linkage: each unit carries its own copy, so no relocatable device code is
// needed; each unit also counts its own solver activity.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include "d2_internal.h"
#include "d2_solver.cuh"

namespace d2k {
namespace {


// Solver activity counters: pairs screened, their pivots, pairs solved
// exactly, their pivots, screened pairs certified in FP64, cells the
// certificate checked in FP64.  Accumulated once per lane group per launch.
constexpr int kStatWords = 6;
__device__ unsigned long long g_solver_stats[kStatWords];

__device__ __forceinline__ void add_stats(unsigned long long a, unsigned long long b,
                                          unsigned long long c, unsigned long long d,
                                          unsigned long long e = 0, unsigned long long f = 0) {
  if (a) atomicAdd(&g_solver_stats[0], a);
  if (b) atomicAdd(&g_solver_stats[1], b);
  if (c) atomicAdd(&g_solver_stats[2], c);
  if (d) atomicAdd(&g_solver_stats[3], d);
  if (e) atomicAdd(&g_solver_stats[4], e);
  if (f) atomicAdd(&g_solver_stats[5], f);
}

// ---------------------------------------------------------------- loads --

template <typename T>
__device__ __forceinline__ T ldx(const void* p, int dt, long long idx) {
  if (dt == 0) return (T)(static_cast<const double*>(p)[idx]);
  if (dt == 1) return (T)(static_cast<const float*>(p)[idx]);
  return (T)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[idx]);
}

template <typename T> __device__ __forceinline__ T cvt(float v) { return (T)v; }
template <typename T> __device__ __forceinline__ T cvt(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T cvt(__nv_bfloat16 v) { return (T)__bfloat162float(v); }

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// Ground-cost tile of Eq. (D2opt): C[a*n+r] = sum_k (x_ak - y_rk)^2, by
// explicit differences accumulated with FMA in coordinate order.  Returns
// the tile maximum (group-uniform).
template <typename T, typename X, int G>
__device__ __forceinline__ T cost_cells(const Grp<G>& g, T* C, int m, int n, const X* x, const T* yl,
                                        int d) {
  const int mn = m * n;
  const int q = G / n, rem = G - (G / n) * n;
  int a = g.lane / n, r = g.lane - (g.lane / n) * n;
  T cmax = T(0);
  for (int t = g.lane; t < mn; t += G) {
    const T* yr = yl + (long long)r * d;
    const X* xr = x + (long long)a * d;
    T acc = T(0);
    for (int k = 0; k < d; ++k) {
      const T df = cvt<T>(xr[k]) - yr[k];
      acc = fmaT(df, df, acc);
    }
    C[t] = acc;
    cmax = acc > cmax ? acc : cmax;
    r += rem; a += q;
    if (r >= n) { r -= n; ++a; }
  }
  return cmax;
}

// The same tile for FP32 bags when n divides the group and d is a small
// compile-time constant: lane l keeps centroid support r = l mod n in
// registers and takes rows a = l/n, l/n + G/n, ...; the object row is read
// with vector loads where its alignment allows.  Same operations in the same
// order as cost_cells, so the tile is bitwise the same.
template <int D, int G>
__device__ __forceinline__ float cost_cells_fixed(const Grp<G>& g, float* C, int m, int n,
                                                  const float* __restrict__ x,
                                                  const float* __restrict__ yl) {
  const int step = G / n;
  const int r = g.lane - (g.lane / n) * n;
  float y[D];
#pragma unroll
  for (int k = 0; k < D; ++k) y[k] = yl[r * D + k];
  float cmax = 0.f;
  for (int a = g.lane / n; a < m; a += step) {
    const float* xr = x + (long long)a * D;
    float acc = 0.f;
    if constexpr (D % 4 == 0) {
#pragma unroll
      for (int k = 0; k < D; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(xr + k);
        float df = v.x - y[k];
        acc = fmaf(df, df, acc);
        df = v.y - y[k + 1];
        acc = fmaf(df, df, acc);
        df = v.z - y[k + 2];
        acc = fmaf(df, df, acc);
        df = v.w - y[k + 3];
        acc = fmaf(df, df, acc);
      }
    } else if constexpr (D % 2 == 0) {
#pragma unroll
      for (int k = 0; k < D; k += 2) {
        const float2 v = *reinterpret_cast<const float2*>(xr + k);
        float df = v.x - y[k];
        acc = fmaf(df, df, acc);
        df = v.y - y[k + 1];
        acc = fmaf(df, df, acc);
      }
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float df = xr[k] - y[k];
        acc = fmaf(df, df, acc);
      }
    }
    C[a * n + r] = acc;
    cmax = acc > cmax ? acc : cmax;
  }
  return cmax;
}

// Ground-cost tile of Eq. (D2opt): C[a*n+r] = sum_k (x_ak - y_rk)^2, by
// explicit differences accumulated with FMA in coordinate order.  Returns
// the tile maximum (group-uniform).
template <typename T, int G, int DMAX = 32>
__device__ T build_cost(const Grp<G>& g, T* C, int m, int n, const void* xl, int xdt,
                        long long xrow0, const T* yl, int d) {
  T cmax;
  const long long o = xrow0 * (long long)d;
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    // FP32 bags, n dividing the group, common small d: register-resident
    // centroid supports (vector loads need 8- or 16-byte aligned rows)
    const float* xf = static_cast<const float*>(xl) + o;
    const uintptr_t al = reinterpret_cast<uintptr_t>(xf);
    if (xdt == 1 && n <= G && G % n == 0) {
      done = true;
      if (d == 6 && (al & 7) == 0) cmax = cost_cells_fixed<6, G>(g, C, m, n, xf, yl);
      else if (d == 3) cmax = cost_cells_fixed<3, G>(g, C, m, n, xf, yl);
      else if constexpr (DMAX >= 32) {
        if (d == 16 && (al & 15) == 0) cmax = cost_cells_fixed<16, G>(g, C, m, n, xf, yl);
        else if (d == 32 && (al & 15) == 0) cmax = cost_cells_fixed<32, G>(g, C, m, n, xf, yl);
        else done = false;
      } else {
        done = false;
      }
    }
  }
  if (done) {
  } else if (xdt == 1) cmax = cost_cells<T, float, G>(g, C, m, n, static_cast<const float*>(xl) + o, yl, d);
  else if (xdt == 0) cmax = cost_cells<T, double, G>(g, C, m, n, static_cast<const double*>(xl) + o, yl, d);
  else cmax = cost_cells<T, __nv_bfloat16, G>(g, C, m, n, static_cast<const __nv_bfloat16*>(xl) + o, yl, d);
  cmax = gmax<G>(g, cmax);
  g.sync();
  return cmax;
}

// Ground-cost tile from a symbol table (the sequence variant of Eq. (D2opt)):
// C[a*n+r] = tab[x_a*A + y_r] with x, y symbol ids (d = 1).  Ids are checked
// before the launch; the clamp only keeps reads inside the table.  Returns
// the tile maximum (group-uniform).
template <typename T, int G>
__device__ T build_cost_tab(const Grp<G>& g, T* C, int m, int n, const void* xl, int xdt,
                            long long xrow0, const T* ysym, const T* tab, int A) {
  const int mn = m * n;
  const int q = G / n, rem = G - (G / n) * n;
  int a = g.lane / n, r = g.lane - (g.lane / n) * n;
  T cmax = T(0);
  for (int t = g.lane; t < mn; t += G) {
    int xs = (int)ldx<T>(xl, xdt, xrow0 + a);
    int ys = (int)ysym[r];
    xs = xs < 0 ? 0 : (xs >= A ? A - 1 : xs);
    ys = ys < 0 ? 0 : (ys >= A ? A - 1 : ys);
    const T c = tab[xs * A + ys];
    C[t] = c;
    cmax = c > cmax ? c : cmax;
    r += rem; a += q;
    if (r >= n) { r -= n; ++a; }
  }
  cmax = gmax<G>(g, cmax);
  g.sync();
  return cmax;
}

// ---------------------------------------------------------- start order --
// The cold-start basis is the northwest staircase taken in the order of
// the supports' projections onto the object's principal direction (in 1-D
// that staircase is the optimal monotone coupling; in d dimensions it is a
// start close to it along the dominant axis).

// inclusive prefix of per-id masses (from the by-id inclusive prefix `pre`)
// in the order id_of[0..cnt)
template <int G>
__device__ void prefix_in_order(const Grp<G>& g, const long long* pre, const int* id_of, int cnt,
                                long long* out) {
  long long carry = 0;
  for (int base = 0; base < cnt; base += G) {
    const int r = base + g.lane;
    long long v = 0;
    if (r < cnt) {
      const int id = id_of[r];
      v = pre[id] - (id > 0 ? pre[id - 1] : 0LL);
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const long long u = __shfl_up_sync(g.mask, v, o, G);
      if (g.lane >= o) v += u;
    }
    v += carry;
    if (r < cnt) out[r] = v;
    carry = __shfl_sync(g.mask, v, G - 1, G);
  }
  g.sync();
}

// stable ranks of proj[0..cnt) (ties to the smaller index)
template <int G>
__device__ void rank_by_proj(const Grp<G>& g, const float* proj, int cnt, int* rank, int* id) {
  for (int a = g.lane; a < cnt; a += G) {
    const float v = proj[a];
    int r = 0;
    for (int b = 0; b < cnt; ++b) {
      const float u = proj[b];
      r += (u < v || (u == v && b < a)) ? 1 : 0;
    }
    rank[a] = r;
    id[r] = a;
  }
  g.sync();
}

// Object side: weighted mean, principal direction by power iteration from
// the farthest support, row ranks and rank-order prefix masses.
template <int G>
__device__ void order_rows(const Grp<G>& g, const PairMem<float>& s, const ObjView& ob, long long o0,
                           int m, int d) {
  const float wscale = (float)kInvMass;
  for (int k = g.lane; k < d; k += G) {
    float acc = 0.f;
    for (int a = 0; a < m; ++a) {
      const float pa = (float)(s.P[a] - (a > 0 ? s.P[a - 1] : 0LL)) * wscale;
      acc = fmaf(pa, ldx<float>(ob.loc, ob.ldt, (o0 + a) * d + k), acc);
    }
    s.mu[k] = acc;
  }
  g.sync();
  // start: the support farthest from the mean (largest weighted deviation)
  float best = -1.f;
  int bi = 0;
  for (int a = g.lane; a < m; a += G) {
    float dev = 0.f;
    for (int k = 0; k < d; ++k) {
      const float x = ldx<float>(ob.loc, ob.ldt, (o0 + a) * d + k) - s.mu[k];
      dev = fmaf(x, x, dev);
    }
    dev *= (float)(s.P[a] - (a > 0 ? s.P[a - 1] : 0LL)) * wscale;
    if (dev > best) { best = dev; bi = a; }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float ob2 = gshfl_xor<G>(g, best, o);
    const int oi = gshfl_xor<G>(g, bi, o);
    if (ob2 > best || (ob2 == best && oi < bi)) { best = ob2; bi = oi; }
  }
  for (int k = g.lane; k < d; k += G) s.dir[k] = ldx<float>(ob.loc, ob.ldt, (o0 + bi) * d + k) - s.mu[k];
  g.sync();
  for (int it = 0; it < 6; ++it) {
    for (int a = g.lane; a < m; a += G) {
      float dot = 0.f;
      for (int k = 0; k < d; ++k) dot = fmaf(ldx<float>(ob.loc, ob.ldt, (o0 + a) * d + k) - s.mu[k], s.dir[k], dot);
      s.proj[a] = dot * (float)(s.P[a] - (a > 0 ? s.P[a - 1] : 0LL)) * wscale;
    }
    g.sync();
    float nrm = 0.f;
    float vk[8];
    int nk = 0;
    for (int k = g.lane; k < d; k += G) {
      float acc = 0.f;
      for (int a = 0; a < m; ++a) acc = fmaf(s.proj[a], ldx<float>(ob.loc, ob.ldt, (o0 + a) * d + k) - s.mu[k], acc);
      if (nk < 8) vk[nk++] = acc;
      nrm = fmaf(acc, acc, nrm);
    }
    nrm = gsum<G>(g, nrm);
    g.sync();
    const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
    nk = 0;
    for (int k = g.lane; k < d; k += G) {
      if (nk < 8) s.dir[k] = inv > 0.f ? vk[nk] * inv : s.dir[k];
      ++nk;
    }
    g.sync();
  }
  for (int a = g.lane; a < m; a += G) {
    float dot = 0.f;
    for (int k = 0; k < d; ++k) dot = fmaf(ldx<float>(ob.loc, ob.ldt, (o0 + a) * d + k) - s.mu[k], s.dir[k], dot);
    s.proj[a] = dot;
  }
  g.sync();
  rank_by_proj<G>(g, s.proj, m, s.rrank, s.rid);
  prefix_in_order<G>(g, s.P, s.rid, m, s.Pr);
}

// Centroid side: column ranks along the object's direction and their
// rank-order prefix masses (s.Q holds the centroid's by-id prefix).
template <int G>
__device__ void order_cols(const Grp<G>& g, const PairMem<float>& s, const float* y32, int n, int d) {
  for (int r = g.lane; r < n; r += G) {
    float dot = 0.f;
    for (int k = 0; k < d; ++k) dot = fmaf(y32[(long long)r * d + k] - s.mu[k], s.dir[k], dot);
    s.proj[r] = dot;
  }
  g.sync();
  rank_by_proj<G>(g, s.proj, n, s.crank, s.cid);
  prefix_in_order<G>(g, s.Q, s.cid, n, s.Qr);
}

template <int G>
__device__ bool load_obj_prefix(const Grp<G>& g, const ObjView& ob, long long o0, int m,
                                long long* P) {
  if (ob.wdt == 0) return load_prefix<G>(g, static_cast<const double*>(ob.w) + o0, m, P);
  return load_prefix<G>(g, static_cast<const float*>(ob.w) + o0, m, P);
}

template <int G>
__device__ void load_cent_prefix(const Grp<G>& g, const CentView& cv, long long c0, int n,
                                 long long* Q) {
  for (int r = g.lane; r < n; r += G) Q[r] = cv.Qpre[c0 + r];
  g.sync();
}

// Tolerances on the most negative reduced cost accepted as optimal.
__device__ __forceinline__ double tol64(double cmax) { return cmax * 0x1p-43; }
__device__ __forceinline__ float tol32(float cmax) { return cmax * 0x1p-20f; }

// Exact solve of pair (object at o0/m, centroid at c0/n) into the tree
// registers `tr`.  With fp32_start the basis is first driven to FP32
// optimality on the FP32 tile (cheap pivots); the same tree and integer
// flows then continue on the FP64 tile with FP64 potentials until no FP64
// reduced cost is below -tol64, so the result is FP64-optimal either way.
// *obj: FP64 objective.
template <int G, int NPL, int ST>
__device__ __forceinline__ int solve_exact(const Grp<G>& g, const PairMem<double>& s,
                                           Simplex<double, G, NPL>& S, const ObjView& ob,
                                           long long o0, int m, const CentView& cv, long long c0,
                                           int n, int budget, bool fp32_start, double* obj,
                                           int* piv_out) {
  load_cent_prefix<G>(g, cv, c0, n, s.Q);
  const int cap = budget * (m + n);
  int piv = 0;
  if (fp32_start) {
    const PairMem<float> s32 = recast<float>(s);
    const float c32 =
        cv.A ? build_cost_tab<float, G>(g, s32.cost, m, n, ob.loc, ob.ldt, o0, cv.loc32 + c0,
                                        cv.tab32, cv.A)
             : build_cost<float, G, 8>(g, s32.cost, m, n, ob.loc, ob.ldt, o0,
                                       cv.loc32 + c0 * cv.d, cv.d);
    Simplex<float, G, NPL> S32(s32, m, n, g);
    if constexpr (ST == 1) {
      S32.init_vogel();
    } else {
      order_rows<G>(g, s32, ob, o0, m, cv.d);
      order_cols<G>(g, s32, cv.loc32 + c0 * cv.d, n, cv.d);
      S32.init_northwest_ranked();
    }
    if (S32.run(cap, tol32(c32), &piv) == kStInvalid) { *piv_out += piv; return kStInvalid; }
    S.t = S32.t;
    S.root = S32.root;
    g.sync();
  }
  const double cmax =
      cv.A ? build_cost_tab<double, G>(g, s.cost, m, n, ob.loc, ob.ldt, o0, cv.loc64 + c0,
                                       cv.tab64, cv.A)
           : build_cost<double, G>(g, s.cost, m, n, ob.loc, ob.ldt, o0, cv.loc64 + c0 * cv.d,
                                   cv.d);
  S.set_dims(m, n);
  S.bad = false;
  if (!fp32_start) S.init_northwest();
  const int st = S.run(cap, tol64(cmax), &piv);
  *obj = S.template objective<double>();
  *piv_out += piv;
  return st;
}

// FP64 ground cost of cell (a, r) of a pair, by explicit differences in
// coordinate order (the arithmetic of build_cost<double>, so the same value
// as the FP64 tile's cell); the table entry with symbol ground costs.
__device__ __forceinline__ double cost64_cell(const ObjView& ob, long long o0, const CentView& cv,
                                              long long c0, int a, int r) {
  if (cv.A) {  // ids checked before the launch; the clamp only keeps reads in the table
    int xs = (int)ldx<double>(ob.loc, ob.ldt, o0 + a);
    int ys = (int)cv.loc64[c0 + r];
    xs = xs < 0 ? 0 : (xs >= cv.A ? cv.A - 1 : xs);
    ys = ys < 0 ? 0 : (ys >= cv.A ? cv.A - 1 : ys);
    return cv.tab64[xs * cv.A + ys];
  }
  const int d = cv.d;
  const double* y = cv.loc64 + (c0 + r) * d;
  const long long x0 = (o0 + a) * d;
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    const double df = ldx<double>(ob.loc, ob.ldt, x0 + k) - y[k];
    acc = fma(df, df, acc);
  }
  return acc;
}

// -------------------------------------------------------------- kernels --

template <int G, int NPL, int ST>
__global__ void __launch_bounds__(128) k_mallows_pairs(ObjView ob, CentView cv,
                                                       const long long* pobj, const long long* pcen,
                                                       long long npairs, SolveCfg cfg, size_t slice,
                                                       double* dist2, FlowOut fo, int* status, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  Grp<G> g;
  const int gpb = blockDim.x / G;
  unsigned char* base = smem + (threadIdx.x / G) * slice;
  int n_pairs = 0, n_piv = 0;
  for (long long t = (long long)blockIdx.x * gpb + threadIdx.x / G; t < npairs;
       t += (long long)gridDim.x * gpb) {
    const long long i = pobj[t], j = pcen[t];
    int st = kStInvalid;
    double res = nan("");
    if (i >= 0 && i < ob.count && j >= 0 && j < cv.K) {
      const long long o0 = ob.off[i];
      const int m = (int)(ob.off[i + 1] - o0);
      const long long c0 = cv.off[j];
      const int n = (int)(cv.off[j + 1] - c0);
      if (m >= 1 && m <= cfg.mmax && n >= 1 && n <= cfg.nmax && m + n <= G * NPL) {
        PairMem<double> s64 = carve<double>(base, cfg.mmax, cfg.nmax, cv.d);
        if (load_obj_prefix<G>(g, ob, o0, m, s64.P)) {
          Simplex<double, G, NPL> S(s64, m, n, g);
          st = solve_exact<G, NPL, ST>(g, s64, S, ob, o0, m, cv, c0, n, cfg.budget, cfg.mode == 1,
                                       &res, &n_piv);
          ++n_pairs;
          if (fo.cell && st != kStInvalid)
            S.write_flows(fo.cell + t * fo.stride, fo.w + t * fo.stride, fo.stride);
          if (fo.pot && st == kStOk)  // potentials of the final, freshly priced basis
            for (int r = g.lane; r < n; r += G) fo.pot[t * fo.pstride + r] = s64.pot[m + r];
        }
      }
    }
    if (g.lane == 0) {
      dist2[t] = res;
      if (status) status[t] = st == kStOk ? 0 : (st == kStNotConverged ? -3 : -1);
      if (st == kStInvalid) atomicOr(err, kErrInvalid);
      if (st == kStNotConverged) atomicOr(err, kErrNotConverged);
    }
    g.sync();
  }
  if (g.lane == 0) add_stats(0, 0, n_pairs, n_piv);
}

// The same exact solve in two launches: the FP32 start and pivots here,
// the FP64 continuation in k_pairs64 from the basis handed over in global
// memory (the same tree and integer flows solve_exact hands over in
// registers, so the results are identical).  Each kernel then carries only
// one Simplex instantiation, which keeps its code within the instruction
// cache.
template <int G, int NPL, int ST>
__global__ void __launch_bounds__(128, (NPL <= 1 ? 8 : 5))
    k_pairs32(ObjView ob, CentView cv, const long long* pobj, const long long* pcen,
              long long npairs, SolveCfg cfg, size_t slice, WarmStore tr, int* st32) {
  extern __shared__ __align__(16) unsigned char smem[];
  Grp<G> g;
  const int gpb = blockDim.x / G;
  unsigned char* base = smem + (threadIdx.x / G) * slice;
  int n_piv = 0;
  for (long long t = (long long)blockIdx.x * gpb + threadIdx.x / G; t < npairs;
       t += (long long)gridDim.x * gpb) {
    const long long i = pobj[t], j = pcen[t];
    int st = kStInvalid;
    if (i >= 0 && i < ob.count && j >= 0 && j < cv.K) {
      const long long o0 = ob.off[i];
      const int m = (int)(ob.off[i + 1] - o0);
      const long long c0 = cv.off[j];
      const int n = (int)(cv.off[j + 1] - c0);
      if (m >= 1 && m <= cfg.mmax && n >= 1 && n <= cfg.nmax && m + n <= G * NPL) {
        const PairMem<float> s32 = carve<float>(base, cfg.mmax, cfg.nmax, cv.d, 4);  // FP32 only
        if (load_obj_prefix<G>(g, ob, o0, m, s32.P)) {
          load_cent_prefix<G>(g, cv, c0, n, s32.Q);
          const float c32 =
              cv.A ? build_cost_tab<float, G>(g, s32.cost, m, n, ob.loc, ob.ldt, o0, cv.loc32 + c0,
                                              cv.tab32, cv.A)
                   : build_cost<float, G, 8>(g, s32.cost, m, n, ob.loc, ob.ldt, o0,
                                             cv.loc32 + c0 * cv.d, cv.d);
          Simplex<float, G, NPL> S32(s32, m, n, g);
          // restart from the object's basis of the previous joint round:
          // same tree, flows for the new centroid weights, dual pivots to
          // feasibility, then the primal run
          const long long wi = i * (long long)cfg.jw.ns;
          bool same = false;  // restarted, and no pivot moved the saved tree
          if (cfg.jw.par8 && m + n <= cfg.jw.ns && cfg.jw.sz8[wi] != 0) {
            S32.load_tree(cfg.jw.par8 + wi, cfg.jw.pos8 + wi, cfg.jw.sz8 + wi, cfg.jw.flow + wi);
            if (S32.tree_sane()) {
              S32.recompute_flows();
              int pw = 0;
              st = S32.run_dual(cfg.budget * (m + n), &pw);
              if (st == kStOk) st = S32.run(cfg.budget * (m + n), tol32(c32), &pw);
              n_piv += pw;
              same = st == kStOk && pw == 0;
            }
            if (st != kStOk) {  // start over cold
              S32.bad = false;
              S32.set_dims(m, n);
            }
          }
          if (st != kStOk) {
            if constexpr (ST == 1) {
              S32.init_vogel();
            } else {
              order_rows<G>(g, s32, ob, o0, m, cv.d);
              order_cols<G>(g, s32, cv.loc32 + c0 * cv.d, n, cv.d);
              S32.init_northwest_ranked();
            }
            st = S32.run(cfg.budget * (m + n), tol32(c32), &n_piv);
          }
          if (st != kStInvalid) {
            const long long wt = t * tr.ns;
            S32.store_tree(tr.par8 + wt, tr.pos8 + wt, tr.sz8 + wt, tr.flow + wt);
          }
          if (same) st = kStSameBasis;
        }
      }
    }
    if (g.lane == 0) st32[t] = st;
    g.sync();
  }
  if (g.lane == 0) add_stats(0, 0, 0, n_piv);
}

template <int G, int NPL>
__global__ void __launch_bounds__(128) k_pairs64(ObjView ob, CentView cv, const long long* pobj,
                                                 const long long* pcen, long long npairs,
                                                 SolveCfg cfg, size_t slice, WarmStore tr,
                                                 const int* st32, double* dist2, FlowOut fo,
                                                 int* status, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  Grp<G> g;
  const int gpb = blockDim.x / G;
  unsigned char* base = smem + (threadIdx.x / G) * slice;
  int n_pairs = 0, n_piv = 0;
  for (long long t = (long long)blockIdx.x * gpb + threadIdx.x / G; t < npairs;
       t += (long long)gridDim.x * gpb) {
    const long long i = pobj[t], j = pcen[t];
    int st = kStInvalid;
    double res = nan("");
    if (st32[t] != kStInvalid && i >= 0 && i < ob.count && j >= 0 && j < cv.K) {
      const long long o0 = ob.off[i];
      const int m = (int)(ob.off[i + 1] - o0);
      const long long c0 = cv.off[j];
      const int n = (int)(cv.off[j + 1] - c0);
      const PairMem<double> s64 = carve<double>(base, cfg.mmax, cfg.nmax, cv.d);
      if (load_obj_prefix<G>(g, ob, o0, m, s64.P)) {
        load_cent_prefix<G>(g, cv, c0, n, s64.Q);
        Simplex<double, G, NPL> S(s64, m, n, g);
        const long long wt = t * tr.ns;
        if (st32[t] == kStSameBasis) {
          // the tree the previous round proved FP64-optimal, unchanged (same
          // costs, so the same reduced costs): only its basic cells' costs
          // are needed, for the potentials and the objective
          S.load_tree(tr.par8 + wt, tr.pos8 + wt, tr.sz8 + wt, tr.flow + wt);
#pragma unroll
          for (int k = 0; k < NPL; ++k) {
            const int y = S.node_of(k);
            if (y < S.N && y != S.root) {
              const int p = S.t.par[k];
              if (p >= 0 && p < S.N && (y < m) != (p < m)) {
                const int a = y < m ? y : p, r = y < m ? p - m : y - m;
                s64.cost[S.edge_idx(y, p)] = cost64_cell(ob, o0, cv, c0, a, r);
              }
            }
          }
          g.sync();
          S.refresh_potentials();
          st = S.bad ? kStInvalid : kStOk;
        } else {
          const double cmax =
              cv.A ? build_cost_tab<double, G>(g, s64.cost, m, n, ob.loc, ob.ldt, o0,
                                               cv.loc64 + c0, cv.tab64, cv.A)
                   : build_cost<double, G>(g, s64.cost, m, n, ob.loc, ob.ldt, o0,
                                           cv.loc64 + c0 * cv.d, cv.d);
          S.load_tree(tr.par8 + wt, tr.pos8 + wt, tr.sz8 + wt, tr.flow + wt);
          S.bad = false;
          st = S.run(cfg.budget * (m + n), tol64(cmax), &n_piv);
        }
        res = S.template objective<double>();
        ++n_pairs;
        if (fo.cell && st != kStInvalid)
          S.write_flows(fo.cell + t * fo.stride, fo.w + t * fo.stride, fo.stride);
        if (fo.pot && st == kStOk)  // potentials of the final, freshly priced basis
          for (int r = g.lane; r < n; r += G) fo.pot[t * fo.pstride + r] = s64.pot[m + r];
        if (cfg.jw.par8 && st == kStOk && m + n <= cfg.jw.ns) {  // the next joint round's start
          const long long wi = i * (long long)cfg.jw.ns;
          S.store_tree(cfg.jw.par8 + wi, cfg.jw.pos8 + wi, cfg.jw.sz8 + wi, cfg.jw.flow + wi);
        }
      }
    }
    if (g.lane == 0) {
      dist2[t] = res;
      if (status) status[t] = st == kStOk ? 0 : (st == kStNotConverged ? -3 : -1);
      if (st == kStInvalid) atomicOr(err, kErrInvalid);
      if (st == kStNotConverged) atomicOr(err, kErrNotConverged);
    }
    g.sync();
  }
  if (g.lane == 0) add_stats(0, 0, n_pairs, n_piv);
}

// Nearest centroid, Alg. 2 Step 2, in two kernels.  Object i uses the
// centroids [seg(i)*K, seg(i)*K + K) of the set (seg(i) = i/seg_size, or
// the object's entry of ob.segof).
//
// k_screen: every centroid is solved with an FP32 tile and FP32 pivots.
// The FP32 objective D32_j has a bound err_j on its distance to the FP64
// optimum (cost rounding (d+3)*2^-24 relative, summation 2^-17 relative,
// basis optimality 2^-14 * max cost absolute, which covers the stopping
// tolerance 2^-20 * max cost and the drift of the incrementally updated
// FP32 potentials, refreshed every 64 pivots); every centroid whose interval
// [D32_j - err_j, D32_j + err_j] reaches below the smallest upper end is a
// candidate.  With tensor-core tiles (cfg.tile) the bound adds the tile's
// own error, see tc_bound.
// Work items are (object i, centroid block jb) with blocks of KB centroids,
// so small batches still fill the GPU; lane groups take items from an
// atomic counter (persistent kernel).  Output per item (kItemInts ints at
// item*kItemInts): count (-1: more than kCandCap, -2: invalid object),
// kCandCap candidate indices in increasing order, their lower ends (float
// bits), and the block's smallest upper end (float bits).

// Objects of a launch: their count and list (oidx, or obase.. when null);
// with a device-side range the count is read here (SolveCfg::dev_range).
__device__ __forceinline__ long long launch_objects(const SolveCfg& cfg, long long count,
                                                    const int** oidx) {
  if (cfg.dev_range) {
    const long long lo = cfg.dev_range[0];
    *oidx = cfg.oidx + lo;
    return cfg.dev_range[1] - lo;
  }
  *oidx = cfg.oidx;
  return cfg.nobj >= 0 ? cfg.nobj : count;
}

// Centroid blocks of the screen: enough (object, block) items to fill the
// GPU (sms x items per SM), blocks of at least 8 centroids.
__host__ __device__ inline void centroid_blocks(const SolveCfg& cfg, long long cnt, int K, int* NB,
                                                int* KB) {
  const int ip = cfg.ipsm < 8 ? 8 : (cfg.ipsm > 256 ? 256 : cfg.ipsm);
  const long long want = (long long)cfg.sms * ip;
  long long nb = cnt > 0 ? (want + cnt - 1) / cnt : 1;
  const long long cap = K / 8 > 1 ? K / 8 : 1;
  nb = nb < 1 ? 1 : (nb > cap ? cap : nb);
  const int kb = (int)((K + nb - 1) / nb);
  *KB = kb;
  *NB = (K + kb - 1) / kb;
}

// Largest cost of a pair's block of a chunk's tile (read in place).
template <int G>
__device__ __forceinline__ float tile_max(const Grp<G>& g, const float* __restrict__ src, int m,
                                          int n, long long ldc) {
  const int mn = m * n;
  const int q = G / n, rem = G - (G / n) * n;
  int a = g.lane / n, r = g.lane - (g.lane / n) * n;
  float cmax = 0.f;
#pragma unroll 4
  for (int t = g.lane; t < mn; t += G) {
    cmax = fmaxf(cmax, __ldg(src + (long long)a * ldc + r));
    r += rem; a += q;
    if (r >= n) { r -= n; ++a; }
  }
  return gmax<G>(g, cmax);
}

// Bound on |C^ - C| for every cell of a tensor-core tile (C^ = the FP32
// tile of ||x||^2 + ||y^||^2 - 2 x.y^ over BF16 x and y^ = BF16(y)), from the
// largest FP32 squared norms nxm (object rows) and cn (centroid rows) and
// the largest rounding distance cd = max ||y - y^||:
//   accumulation of d exact products in FP32 by the tensor cores, modelled
//   as at most one unit in the last place of sum|x_k y^_k| <= ||x|| ||y^||
//   lost by every aligned addend (d products plus one accumulator per
//   block of at least 4 products: <= 1.25 d units of 2^-23), taken twice:
//   d * 2^-22; the two FP32 norm sums and the final FMA ((d+3) * 2^-24);
//   both relative to ||x||^2 + ||y^||^2 >= 2 ||x|| ||y^||; then the move from
//   y^ back to y: | ||x-y^||^2 - ||x-y||^2 | <= (2(||x|| + ||y^||) + cd) cd.
// Since a pair's flows sum to 1, the same bound holds for the objective of
// any basis, hence for the optimum.
__device__ __forceinline__ float tc_bound(int d, float nxm, float cn, float cd) {
  const float rel = (float)d * 0x1p-22f + (float)(d + 3) * 0x1p-24f;
  const float e1 = rel * (nxm + cn);
  const float e2 = (2.f * (sqrtf(nxm) + sqrtf(cn)) + 2.f * cd) * cd;
  return (e1 + e2) * (1.f + 0x1p-10f);
}

// ---- double-float arithmetic (an unevaluated sum hi + lo of two floats,
// about 48 significant bits) on the FP32 pipes, which run 64 times the FP64
// rate on this GPU.  The intrinsics keep every product and sum rounded on
// its own (no contraction into FMA), which the error-free steps rely on.

// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) + (bh, bl) -> normalised (hi, lo): relative error <= 4 u^2 of the
// magnitudes involved (u = 2^-24).
__device__ __forceinline__ void dd_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// Ground cost of cell (a, r) as hi + lo, for FP32 or BF16 object data (X)
// and a centroid set whose FP32 copy is exact (loc32 == loc64: the screen's
// precondition).  Per coordinate: x - y exactly by two-sum (s + e), s^2
// exactly as p + q (q = fma(s, s, -p)), the cross term 2se + q rounded once
// (e^2 <= u^2 s^2 dropped), and the running sum kept as hi + lo.  Error:
// |hi + lo - c| <= (6d + 4) u^2 c.
// One coordinate's term added to the running sum H + L.
__device__ __forceinline__ void dd_sq_acc(float xv, float yv, float& H, float& L) {
  float s, e;
  two_sum(xv, -yv, s, e);
  const float p = __fmul_rn(s, s);
  const float q = fmaf(s, s, -p);
  const float rr = fmaf(__fadd_rn(s, s), e, q);
  float t, z;
  two_sum(H, p, t, z);
  L = __fadd_rn(L, __fadd_rn(z, rr));
  H = t;
}

// Two independent running sums (even and odd coordinates) shorten the
// dependent chain; they are added exactly at the end (two-sum).
template <typename X>
__device__ __forceinline__ void cost_dd_x(const X* __restrict__ x, const float* __restrict__ y,
                                          int d, float& hi, float& lo) {
  float H0 = 0.f, L0 = 0.f, H1 = 0.f, L1 = 0.f;
  int k = 0;
  for (; k + 1 < d; k += 2) {
    dd_sq_acc(cvt<float>(x[k]), y[k], H0, L0);
    dd_sq_acc(cvt<float>(x[k + 1]), y[k + 1], H1, L1);
  }
  if (k < d) dd_sq_acc(cvt<float>(x[k]), y[k], H0, L0);
  float t, z;
  two_sum(H0, H1, t, z);
  const float L = __fadd_rn(__fadd_rn(L0, L1), z);
  hi = __fadd_rn(t, L);
  lo = __fsub_rn(L, __fsub_rn(hi, t));
}

// The cell cost of FP64 data or of a symbol table: the FP64 cost (the
// arithmetic of cost64_cell) split into hi + lo.  Out of line, with scalar
// arguments: only those rare inputs take it.
__device__ __noinline__ float2 cost_dd_slow(const void* xloc, int ldt, long long xrow, int d,
                                            const double* y64, const double* tab64, int A) {
  double c;
  if (A) {
    int xs = (int)ldx<double>(xloc, ldt, xrow);
    int ys = (int)y64[0];
    xs = xs < 0 ? 0 : (xs >= A ? A - 1 : xs);
    ys = ys < 0 ? 0 : (ys >= A ? A - 1 : ys);
    c = tab64[xs * A + ys];
  } else {
    c = 0.0;
    for (int k = 0; k < d; ++k) {
      const double df = ldx<double>(xloc, ldt, xrow * d + k) - y64[k];
      c = fma(df, df, c);
    }
  }
  const float hi = __double2float_rn(c);
  return make_float2(hi, __double2float_rn(c - (double)hi));
}

// Cost of cell (a, r) as hi + lo: cost_dd_x for FP32 (xt == 1) or BF16
// (xt == 2) object data, cost_dd_slow otherwise (xt == 0).  Only the load
// loop depends on the type, so the certificate around it exists once.
__device__ __forceinline__ void cost_dd(int xt, const ObjView& ob, long long o0,
                                        const CentView& cv, long long c0, int a, int r,
                                        float& hi, float& lo) {
  if (xt == 1) {
    cost_dd_x(static_cast<const float*>(ob.loc) + (o0 + a) * cv.d, cv.loc32 + (c0 + r) * cv.d,
              cv.d, hi, lo);
  } else if (xt == 2) {
    cost_dd_x(static_cast<const __nv_bfloat16*>(ob.loc) + (o0 + a) * cv.d,
              cv.loc32 + (c0 + r) * cv.d, cv.d, hi, lo);
  } else {
    const float2 c = cost_dd_slow(ob.loc, ob.ldt, o0 + a, cv.d,
                                  cv.A ? cv.loc64 + c0 + r : cv.loc64 + (c0 + r) * cv.d, cv.tab64,
                                  cv.A);
    hi = c.x;
    lo = c.y;
  }
}

// Group maximum of non-negative floats (or NaN) by the integer reduction
// unit: their bit patterns order like the values, and a NaN (above +inf as
// an unsigned pattern) survives, where fmaxf would drop it.
template <int G>
__device__ __forceinline__ float gmax_nonneg(const Grp<G>& g, float v) {
  return __uint_as_float(__reduce_max_sync(g.mask, __float_as_uint(v)));
}

// Optimality certificate of the basis an FP32 solve stopped at (precision
// pattern: FP32 pivots, then a check and objective of FP64 accuracy).
//   1. Costs of the m+n-1 basic cells (tree edges) in double-float; the
//      objective D = sum w c of the basic flows (exact integer masses) in
//      FP64 -- an upper bound of the optimum, the basis being feasible.
//   2. Potentials u_a + v_r = c_ar on every tree edge: the FP32 solve's own
//      potentials plus a correction delta, from the residuals
//      c_ar - pot_a - pot_r of the tree edges (double-float costs, so the
//      small residuals are exact to about 2^-48 c) propagated down the tree
//      by pointer jumping in FP32 (delta is small, its own rounding
//      negligible).
//   3. LP duality: for an optimal plan w*, D* = sum w* (u + v + d) =
//      D + sum w* d >= D + min d, because sum w* = 1 and the marginals are
//      the basis's.  So D - D* <= max(0, -min d) over all cells.
//   4. min d is checked in FP32 against a rounding bound: with the FP32
//      tile c32, the potentials rounded to FP32 and two FP32 subtractions,
//      |d32 - d~| <= E = ecost + 2^-24 (2 c_max + 5 p_max) (ecost bounds
//      |c32 - c| per cell, p_max the largest |potential|, d~ the reduced
//      cost of the computed potentials), and |d~ - d| <= err = (N + 1)
//      ((6d + 32) 2^-48 c_max + 2^-24 delta_max) covers the double-float
//      costs and the corrections; so d32 >= E + err - tau implies
//      d >= -tau.  The few cells below that are re-priced in double-float
//      and must reach err - tau.
// Returns true when every reduced cost is >= -tau, tau = max(2^-24 D,
// 2^-43 c_max) (*tau_out, FP32 rounded down): the pair's D^2 is then
// certified, D - tau <= D* <= D (up to (6d + 4) 2^-48 relative for the
// double-float costs in D).  *D64: the FP64 objective of the basis (NaN if
// the tree was inconsistent); *nchk: cells re-priced.  Overwrites the
// basic cells of the FP32 tile and the solver's pivot scratch; the tree
// and the solver's potentials are kept.
template <int G, int NPL>
__device__ bool certify_fp64(Simplex<float, G, NPL>& S, const ObjView& ob, long long o0,
                             const CentView& cv, long long c0, float cmax, float ecost,
                             double* D64, float* tau_out, int* nchk) {
  const Grp<G>& g = S.g;
  const int m = S.m, n = S.n, N = S.N;
  const PairMem<float>& s = S.s;
  const int xt = (cv.A == 0 && ob.ldt != 0) ? ob.ldt : 0;  // cost_dd's path
  float rres[NPL];
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < NPL; ++k) {
    const int y = S.node_of(k);
    rres[k] = 0.f;
    if (y < N && y != S.root) {
      const int p = S.t.par[k];
      const int a = y < m ? y : p;
      const int r = y < m ? p - m : y - m;
      float ch, cl;
      cost_dd(xt, ob, o0, cv, c0, a, r, ch, cl);
      const double w = (double)S.t.flow[k] * kInvMass;
      acc = fma(w, (double)ch, acc);
      acc = fma(w, (double)cl, acc);
      // residual of the FP32 potentials on this edge: c - pot_y - pot_p
      float s1, e1;
      two_sum(ch, -S.pot[k], s1, e1);
      e1 = __fadd_rn(e1, cl);
      float s2, e2;
      two_sum(s1, -s.pot[p], s2, e2);
      rres[k] = __fadd_rn(s2, __fadd_rn(e2, e1));
    }
  }
  const double D = gsum<G>(g, acc);
  *D64 = D;
  // corrections: delta(root) = 0, delta(y) = residual(y) - delta(par y)
  float2* PD = reinterpret_cast<float2*>(s.pflow);  // [N] (solver potential, correction)
  float dl[NPL];
  bool bad = false;
  if constexpr (NPL == 1 && G == 32) {
    const int y = g.lane;
    int code = y;
    float a = 0.f;
    if (y < N && y != S.root) {
      const int p = S.t.par[0];
      if (p < 0 || p >= N || (y < m) == (p < m)) { bad = true; code = S.root; }
      else { code = p | (1 << 16); a = rres[0]; }
    }
    for (int round = 0;; ++round) {
      if (round > 9) { bad = true; break; }
      const int an = code & 0xffff;
      const int c2 = __shfl_sync(g.mask, code, an);
      const float v = __shfl_sync(g.mask, a, an);
      const bool mv = y < N && an != S.root;
      if (mv) {
        const int par1 = code >> 16;
        a = par1 ? a - v : a + v;
        code = (c2 & 0xffff) | ((par1 ^ (c2 >> 16)) << 16);
      }
      if (!gany<G>(g, mv)) break;
    }
    dl[0] = a;
  } else {
    int* pa = s.pj0;
    int* pb = s.pj1;
    float* aa = s.acc0;
    float* ab = s.acc1;
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = S.node_of(k);
      if (y == S.root) { pa[y] = y; aa[y] = 0.f; }
      else if (y < N) {
        const int p = S.t.par[k];
        if (p < 0 || p >= N || (y < m) == (p < m)) { bad = true; pa[y] = S.root; aa[y] = 0.f; }
        else { pa[y] = p | (1 << 16); aa[y] = rres[k]; }
      }
    }
    g.sync();
    for (int round = 0;; ++round) {
      if (round > 9) { bad = true; break; }
      bool moved = false;
#pragma unroll
      for (int k = 0; k < NPL; ++k) {
        const int y = S.node_of(k);
        if (y < N) {
          const int code = pa[y];
          const int an = code & 0xffff;
          if (an != S.root) {
            const int c2 = pa[an];
            const float v = aa[an];
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
      float* ta = aa; aa = ab; ab = ta;
      if (!gany<G>(g, moved)) break;
    }
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
      const int y = S.node_of(k);
      dl[k] = y < N ? aa[y] : 0.f;
    }
    g.sync();
  }
  // potentials to shared memory ((base, correction) for re-pricing, their
  // FP32 sum for the scan); the basic cells leave the scan (+inf in the tile)
  // (|u| and |delta| maxima as unsigned patterns: a NaN potential wins the
  // maximum and fails the finiteness test below)
  unsigned pm = 0u, dm = 0u;
#pragma unroll
  for (int k = 0; k < NPL; ++k) {
    const int y = S.node_of(k);
    if (y < N) {
      PD[y] = make_float2(S.pot[k], dl[k]);
      const float u = S.pot[k] + dl[k];
      s.pot[y] = u;
      pm = max(pm, __float_as_uint(fabsf(u)));
      dm = max(dm, __float_as_uint(fabsf(dl[k])));
      if (y != S.root) S.cost[S.edge_idx(y, S.t.par[k])] = INFINITY;
    }
  }
  const float pmax = gmax_nonneg<G>(g, __uint_as_float(pm));
  const float dmax = gmax_nonneg<G>(g, __uint_as_float(dm));
  g.sync();
  if (gany<G>(g, bad)) { *D64 = NAN; return false; }
  if (!isfinite(D) || !isfinite(pmax) || !isfinite(dmax) || !(cmax < FLT_MAX)) return false;
  // tau and the bounds in FP32, rounded toward the safe side
  const float tau = fmaxf(__fmul_rd(__double2float_rd(D), 0x1p-24f), __fmul_rd(cmax, 0x1p-43f));
  *tau_out = tau;
  const float err = __fmul_ru((float)(N + 1),
                              __fmaf_ru((float)(6 * cv.d + 32) * 0x1p-48f, cmax,
                                        __fmul_ru(dmax, 0x1p-24f)));
  const float E = __fmul_ru(__fadd_ru(ecost, __fmul_ru(__fmaf_ru(5.f, pmax, 2.f * cmax), 0x1p-24f)),
                            1.f + 0x1p-10f);
  const float thr = __fsub_ru(__fadd_ru(E, err), tau);  // d32 >= thr    =>  d >= -tau
  const float thr_dd = __fsub_ru(err, tau);              // d~ >= thr_dd  =>  d >= -tau
  const int mn = m * n;
  // pass 1: the FP32 test of every cell (a NaN reduced cost is flagged)
  bool flagged = false;
  if (S.sr == 0) {
    // n divides the group: the lane's cells share column r0, whose
    // potential stays in a register
    const float vr = s.pot[m + S.r0];
    const int step = S.sq * S.cs;
    for (int a = S.a0, o = S.a0 * S.cs + S.r0; a < m; a += S.sq, o += step)
      flagged |= !(S.cost[o] - s.pot[a] - vr >= thr);
  } else {
    int a = S.a0, r = S.r0;
    int o = S.a0 * S.cs + S.r0;  // offset of cell (a, r) in the tile
    const int ostep = S.sq * S.cs + S.sr, owrap = S.cs - n;
    for (int i = g.lane; i < mn; i += G) {
      flagged |= !(S.cost[o] - s.pot[a] - s.pot[m + r] >= thr);
      r += S.sr; a += S.sq; o += ostep;
      if (r >= n) { r -= n; ++a; o += owrap; }
    }
  }
  if (!gany<G>(g, flagged)) return true;
  // pass 2 (few pairs): the flagged cells re-priced in double-float, where
  // they must reach thr_dd
  bool fail = false;
  int cnt = 0;
  if (flagged) {
    int a = S.a0, r = S.r0;
    int o = S.a0 * S.cs + S.r0;
    const int ostep = S.sq * S.cs + S.sr, owrap = S.cs - n;
    for (int i = g.lane; i < mn; i += G) {
      if (!(S.cost[o] - s.pot[a] - s.pot[m + r] >= thr)) {
        ++cnt;
        float ch, cl;
        cost_dd(xt, ob, o0, cv, c0, a, r, ch, cl);
        const float2 u = PD[a], v = PD[m + r];
        dd_add(ch, cl, -u.x, -u.y);
        dd_add(ch, cl, -v.x, -v.y);
        fail |= !((double)ch + (double)cl >= (double)thr_dd);
      }
      r += S.sr; a += S.sq; o += ostep;
      if (r >= n) { r -= n; ++a; o += owrap; }
    }
  }
  *nchk += cnt;
  return !gany<G>(g, fail);
}

template <int G, int NPL, bool TC, int ST, bool CERT>
__global__ void __launch_bounds__(128, (NPL <= 1 ? 8 : 5)) k_screen(ObjView ob, CentView cv, long long seg_size, int K,
                                                SolveCfg cfg, size_t slice,
                                                int* items_out, unsigned long long* queue,
                                                WarmStore ws, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  Grp<G> g;
  unsigned char* base = smem + (threadIdx.x / G) * slice;
  // FP32 only; with tensor-core tiles the solver reads them in place
  const PairMem<float> s32 = carve<float>(base, cfg.mmax, cfg.nmax, cv.d, 4, !TC);
  int* cand = s32.sc;                                          // [kCandCap]
  float* clo = reinterpret_cast<float*>(s32.sc + kCandCap);    // [kCandCap]
  int n_scr = 0, p_scr = 0, n_cert = 0, n_chk = 0;
  const float rel = (float)(cv.d + 3) * 0x1p-24f + 0x1p-17f;
  const int* oidx;
  const long long nobj = launch_objects(cfg, ob.count, &oidx);
  int NB, KB;
  centroid_blocks(cfg, nobj, K, &NB, &KB);
  const unsigned long long total = nobj > 0 ? (unsigned long long)nobj * NB : 0ull;
  for (;;) {
    unsigned long long item = 0;
    if (g.lane == 0) item = atomicAdd(queue, 1ull);
    item = __shfl_sync(g.mask, item, 0, G);
    if (item >= total) break;
    const long long tt = (long long)(item / NB);
    const long long i = oidx ? (long long)oidx[tt] : cfg.obase + tt;
    const int jb = (int)(item - (unsigned long long)tt * NB);
    const int j0 = jb * KB, j1 = min(K, j0 + KB);
    const long long o0 = ob.off[i];
    const int m = (int)(ob.off[i + 1] - o0);
    const long long cb = seg_of(ob, i, seg_size) * (long long)K;
    bool ok = m >= 1 && m <= cfg.mmax && cb + K <= cv.K && load_obj_prefix<G>(g, ob, o0, m, s32.P);
    const bool cold = !(ws.par8 && ws.warm);
    // the cold-start rule is a compile-time choice (ST: 0 ranked staircase,
    // 1 Vogel), so each instantiation carries only its own start code
    constexpr bool vogel = ST == 1;
    if (ok && cold && !vogel) order_rows<G>(g, s32, ob, o0, m, cv.d);
    constexpr bool tcp = TC;  // FP32 tiles precomputed by the tensor cores (cfg.tile)
    long long trow0 = 0;
    float nxm = 0.f;
    if (ok && tcp) {
      trow0 = cfg.tile.trow[tt];
      for (int a = g.lane; a < m; a += G) nxm = fmaxf(nxm, cfg.tile.nx[trow0 + a]);
      nxm = gmax<G>(g, nxm);
    }
    int ncand = 0;
    bool all = false;
    float best_hi = FLT_MAX;
    double best_d64 = NAN;  // certified FP64 value of the smallest upper end's centroid
    for (int j = j0; ok && j < j1; ++j) {
      const long long c0 = cv.off[cb + j];
      const int n = (int)(cv.off[cb + j + 1] - c0);
      if (n < 1 || n > cfg.nmax || m + n > G * NPL) { ok = false; break; }
      const long long wt = (i * (long long)K + j) * ws.ns;
      if constexpr (!CERT) {
        // a centroid whose lower bound is above the object's upper bound
        // cannot be its argmin: no solve (and no saved basis: a later warm
        // round starts that pair cold)
        if (cfg.keep && !((cfg.keep[i * cfg.keep_words + (j >> 5)] >> (j & 31)) & 1u)) {
          if (ws.par8 && g.lane == 0) ws.sz8[wt] = 0;
          continue;
        }
      }
      // a warm round restarts the pairs whose basis was not saved (a
      // certify-all level never skips a pair, so its warm rounds always
      // find one)
      const bool fresh = cold || (!CERT && ws.sz8[wt] == 0);
      // warm bases saved with their flows need no Q (the larger
      // instantiations load it regardless: fewer live values across the
      // solve); bases saved as trees only (never in certify-all levels,
      // whose kernel carries no code for them) recompute their flows from it
      constexpr bool kTreeOnly = !CERT;
      const bool tree_only = kTreeOnly && !ws.flow;
      if (fresh || NPL > 1 || tree_only) load_cent_prefix<G>(g, cv, c0, n, s32.Q);
      float cmax;
      float* tile_g = nullptr;  // the pair's block of the chunk's tile (TC)
      if constexpr (TC) {
        tile_g = const_cast<float*>(cfg.tile.C) + trow0 * cfg.tile.ldc + (c0 - cfg.tile.col0);
        cmax = tile_max<G>(g, tile_g, m, n, cfg.tile.ldc);
      } else if (cv.A)
        cmax = build_cost_tab<float, G>(g, s32.cost, m, n, ob.loc, ob.ldt, o0, cv.loc32 + c0,
                                        cv.tab32, cv.A);
      else
        cmax = build_cost<float, G, (NPL <= 1 ? 8 : 32)>(g, s32.cost, m, n, ob.loc, ob.ldt, o0,
                                                         cv.loc32 + c0 * cv.d, cv.d);
      Simplex<float, G, NPL> S(s32, m, n, g);
      if constexpr (TC) S.set_cost(tile_g, (int)cfg.tile.ldc);
      int st;
      if (!fresh) {
        if (kTreeOnly && tree_only) {
          S.template load_tree<false>(ws.par8 + wt, ws.pos8 + wt, ws.sz8 + wt, nullptr);
          S.recompute_flows();  // the same marginals: the saved flows, exactly
        } else {
          S.load_tree(ws.par8 + wt, ws.pos8 + wt, ws.sz8 + wt, ws.flow + wt);
        }
      } else if (!CERT && !cold) {
        S.init_northwest();  // warm round, no saved basis (the object's order was not built)
      } else if constexpr (vogel) {
        S.init_vogel();
      } else {
        order_cols<G>(g, s32, cv.loc32 + c0 * cv.d, n, cv.d);
        S.init_northwest_ranked();
      }
      st = S.run(cfg.budget * (m + n), tol32(cmax), &p_scr, false);
      if (ws.par8) {
        // always leave a valid basis for the next round
        if (st == kStInvalid) {
          if (!fresh && NPL == 1 && !tree_only) load_cent_prefix<G>(g, cv, c0, n, s32.Q);
          S.init_northwest();
        }
        if (kTreeOnly && tree_only) S.template store_tree<false>(ws.par8 + wt, ws.pos8 + wt, ws.sz8 + wt, nullptr);
        else S.store_tree(ws.par8 + wt, ws.pos8 + wt, ws.sz8 + wt, ws.flow + wt);
      }
      ++n_scr;
      float lo, hi;
      double pair_d64 = NAN;
      if constexpr (CERT) {
        // every pair certified in FP64 (certify_fp64); one that fails is
        // always a candidate, so the exact pass solves it
        double D64 = NAN;
        float tau = 0.f;
        bool cert = false;
        if (st == kStOk) {
          float ecost;
          if constexpr (TC) ecost = tc_bound(cv.d, nxm, cfg.tile.cn[cb + j], cfg.tile.cd[cb + j]);
          else ecost = (cv.A ? 0x1p-23f : (float)(cv.d + 3) * 0x1p-24f) * cmax;
          cert = certify_fp64<G, NPL>(S, ob, o0, cv, c0, cmax, ecost, &D64, &tau, &n_chk);
        }
        // D64 is within (6d + 4) 2^-48 relative of the basis's objective
        // (double-float costs, FP64 sum); the FP32 interval ends, widened by
        // 2^-22 relative, cover it
        const float dhi = __double2float_ru(D64);
        if (cert) {
          ++n_cert;
          lo = __fsub_rd(__fmul_rd(__double2float_rd(D64), 1.f - 0x1p-22f), tau);
          hi = __fmul_ru(dhi, 1.f + 0x1p-22f);
          pair_d64 = D64;
        } else {
          lo = -FLT_MAX;
          hi = isfinite(D64) ? __fmul_ru(dhi, 1.f + 0x1p-22f) : FLT_MAX;
        }
        if (cfg.pair64 && g.lane == 0) cfg.pair64[i * (long long)K + j] = pair_d64;
      } else {
        if (st != kStOk) all = true;  // no bound: let the exact pass decide
        const float D = S.template objective<float>();
        float e = D * rel + cmax * 0x1p-14f;
        if constexpr (TC) e += tc_bound(cv.d, nxm, cfg.tile.cn[cb + j], cfg.tile.cd[cb + j]);
        if (cfg.pair_out && g.lane == 0) {
          float* po = cfg.pair_out + 2 * (i * (long long)K + j);
          po[0] = D;
          po[1] = st != kStOk ? INFINITY : e;
        }
        lo = D - e;
        hi = D + e;
      }
      if (lo <= best_hi) {
        if (ncand < kCandCap) {
          if (g.lane == 0) { cand[ncand] = j; clo[ncand] = lo; }
          ++ncand;
        } else {
          all = true;
        }
      }
      g.sync();
      if (hi < best_hi) {
        best_hi = hi;
        best_d64 = pair_d64;
        int k2 = 0;
        for (int c = 0; c < ncand; ++c) {
          const int cj = cand[c];
          const float cl = clo[c];
          g.sync();
          if (cl <= best_hi) {
            if (g.lane == 0) { cand[k2] = cj; clo[k2] = cl; }
            ++k2;
          }
          g.sync();
        }
        ncand = k2;
      }
    }
    if (!ok && cfg.pair_out && g.lane == 0)
      for (int j = j0; j < j1; ++j) cfg.pair_out[2 * (i * (long long)K + j)] = NAN;
    if (!ok && cfg.pair64 && g.lane == 0)
      for (int j = j0; j < j1; ++j) cfg.pair64[i * (long long)K + j] = NAN;
    int* out = items_out + item * kItemInts;
    if (g.lane == 0) {
      out[0] = !ok ? -2 : (all ? -1 : ncand);
      out[2 * kCandCap + 1] = __float_as_int(best_hi);
      const long long bits = __double_as_longlong(best_d64);
      out[2 * kCandCap + 2] = (int)(unsigned)(bits & 0xffffffffLL);
      out[2 * kCandCap + 3] = (int)(bits >> 32);
    }
    if (g.lane >= 1 && g.lane <= kCandCap) {
      out[g.lane] = (g.lane <= ncand) ? cand[g.lane - 1] : -1;
      out[kCandCap + g.lane] = __float_as_int((g.lane <= ncand) ? clo[g.lane - 1] : FLT_MAX);
    }
    g.sync();
  }
  n_chk = gsum<G>(g, n_chk);
  if (g.lane == 0) add_stats(n_scr, p_scr, 0, 0, n_cert, n_chk);
}

// Per object: merge its NB block lists into one candidate list (count,
// kCandCap indices increasing) at cand[i*kMergedInts]: keep the block
// candidates whose lower end reaches the smallest upper end over all blocks.
__global__ void k_merge(const int* items, long long count, int K, SolveCfg cfg, int* cand) {
  const int* oidx;
  const long long N = launch_objects(cfg, count, &oidx);
  int NB, KB;
  centroid_blocks(cfg, N, K, &NB, &KB);
  for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt < N;
       tt += (long long)gridDim.x * blockDim.x) {
    const long long i = oidx ? (long long)oidx[tt] : cfg.obase + tt;
    const int* it = items + tt * NB * kItemInts;
    float best_hi = FLT_MAX;
    int state = 0;  // 0 ok, -1 all, -2 invalid
    int bbest = 0;  // first block holding the smallest upper end
    for (int b = 0; b < NB; ++b) {
      const int c = it[b * kItemInts];
      if (c == -2) state = -2;
      else if (c == -1 && state == 0) state = -1;
      const float h = __int_as_float(it[b * kItemInts + 2 * kCandCap + 1]);
      if (h < best_hi) { best_hi = h; bbest = b; }
    }
    int cnt = 0;
    int* out = cand + i * kMergedInts;
    if (state == 0) {
      for (int b = 0; b < NB && state == 0; ++b) {
        const int* blk = it + b * kItemInts;
        for (int c = 0; c < blk[0]; ++c) {
          if (__int_as_float(blk[kCandCap + 1 + c]) <= best_hi) {
            if (cnt < kCandCap) out[1 + cnt] = blk[1 + c];
            ++cnt;
          }
        }
      }
      if (cnt > kCandCap) state = -1;
    }
    out[0] = state == 0 ? cnt : state;
    // the certified FP64 value of the smallest upper end's centroid (the
    // only candidate when cnt == 1)
    out[1 + kCandCap] = it[bbest * kItemInts + 2 * kCandCap + 2];
    out[2 + kCandCap] = it[bbest * kItemInts + 2 * kCandCap + 3];
  }
}

// k_exact: the candidates of each object (all K for mode 0, for
// count -1, or where the FP32 screen could not run) are solved to FP64
// optimality; the label is the smallest-index minimum of those FP64
// values, so it agrees with an all-FP64 argmin.
template <int G, int NPL, int ST>
__global__ void __launch_bounds__(128) k_exact(ObjView ob, CentView cv, long long seg_size, int K,
                                               SolveCfg cfg, size_t slice, const int* cand_in,
                                               const double* omega, int* labels, double* dist2,
                                               double* eps_terms, FlowOut fo, WarmStore ws,
                                               int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  Grp<G> g;
  const int gpb = blockDim.x / G;
  unsigned char* base = smem + (threadIdx.x / G) * slice;
  const PairMem<double> s64 = carve<double>(base, cfg.mmax, cfg.nmax, cv.d);
  int n_ex = 0, p_ex = 0;
  const int* oidx;
  const long long nobj = launch_objects(cfg, ob.count, &oidx);
  for (long long tt = (long long)blockIdx.x * gpb + threadIdx.x / G; tt < nobj;
       tt += (long long)gridDim.x * gpb) {
    const long long i = oidx ? (long long)oidx[tt] : cfg.obase + tt;
    const long long o0 = ob.off[i];
    const int m = (int)(ob.off[i + 1] - o0);
    const long long cb = seg_of(ob, i, seg_size) * (long long)K;
    int best_j = -1;
    double best = nan("");
    int st = kStOk;
    const int cnt = cand_in ? cand_in[i * kMergedInts] : -1;
    const bool okm = m >= 1 && m <= cfg.mmax && cb + K <= cv.K && cnt != -2;
    double d64c = NAN;  // certified FP64 value of the single candidate, if any
    if (cfg.certify && cnt == 1) {
      const int* mr = cand_in + i * kMergedInts;
      d64c = __longlong_as_double(((long long)mr[2 + kCandCap] << 32) |
                                  (long long)(unsigned)mr[1 + kCandCap]);
    }
    if (!okm || !load_obj_prefix<G>(g, ob, o0, m, s64.P)) {
      st = kStInvalid;
    } else if (!isnan(d64c)) {
      // one candidate, certified by the screen: its FP64 value stands; its
      // flows come from the basis the screen saved (or a re-solve)
      const int j = cand_in[i * kMergedInts + 1];
      const long long c0 = cv.off[cb + j];
      const int n = (int)(cv.off[cb + j + 1] - c0);
      if (j < 0 || j >= K || n < 1 || n > cfg.nmax || m + n > G * NPL) {
        st = kStInvalid;
      } else {
        best_j = j;
        best = d64c;
        if (fo.cell) {
          Simplex<double, G, NPL> S(s64, m, n, g);
          if (ws.par8) {
            const long long wt = (i * (long long)K + j) * ws.ns;
            if (ws.flow) {
              S.load_tree(ws.par8 + wt, ws.pos8 + wt, ws.sz8 + wt, ws.flow + wt);
            } else {
              load_cent_prefix<G>(g, cv, c0, n, s64.Q);
              S.template load_tree<false>(ws.par8 + wt, ws.pos8 + wt, ws.sz8 + wt, nullptr);
              S.recompute_flows();
            }
          } else {
            double D;
            const int s2 = solve_exact<G, NPL, ST>(g, s64, S, ob, o0, m, cv, c0, n, cfg.budget,
                                                   true, &D, &p_ex);
            ++n_ex;
            if (s2 != kStOk) st = s2;
          }
          if (st != kStInvalid) S.write_flows(fo.cell + i * fo.stride, fo.w + i * fo.stride, fo.stride);
        }
      }
    } else {
      const bool all = cnt < 0;
      const int count = all ? K : cnt;
      for (int c = 0; c < count; ++c) {
        const int j = all ? c : cand_in[i * kMergedInts + 1 + c];
        const long long c0 = cv.off[cb + j];
        const int n = (int)(cv.off[cb + j + 1] - c0);
        if (j < 0 || j >= K || n < 1 || n > cfg.nmax || m + n > G * NPL) { st = kStInvalid; break; }
        double D;
        Simplex<double, G, NPL> S(s64, m, n, g);
        int s2;
        if (ws.par8 && cand_in && !all) {
          // the screen just saved this pair's FP32-optimal basis: continue in FP64
          const long long wt = (i * (long long)K + j) * ws.ns;
          load_cent_prefix<G>(g, cv, c0, n, s64.Q);
          const double cmax =
              cv.A ? build_cost_tab<double, G>(g, s64.cost, m, n, ob.loc, ob.ldt, o0,
                                               cv.loc64 + c0, cv.tab64, cv.A)
                   : build_cost<double, G>(g, s64.cost, m, n, ob.loc, ob.ldt, o0,
                                           cv.loc64 + c0 * cv.d, cv.d);
          if (ws.flow) {
            S.load_tree(ws.par8 + wt, ws.pos8 + wt, ws.sz8 + wt, ws.flow + wt);
          } else {
            S.template load_tree<false>(ws.par8 + wt, ws.pos8 + wt, ws.sz8 + wt, nullptr);
            S.recompute_flows();
          }
          s2 = S.run(cfg.budget * (m + n), tol64(cmax), &p_ex);
          D = S.template objective<double>();
        } else {
          s2 = solve_exact<G, NPL, ST>(g, s64, S, ob, o0, m, cv, c0, n, cfg.budget, cfg.mode == 1,
                                       &D, &p_ex);
        }
        ++n_ex;
        if (cfg.pair64 && g.lane == 0) cfg.pair64[i * (long long)K + j] = s2 == kStInvalid ? NAN : D;
        if (s2 != kStOk) st = s2;
        if (s2 == kStInvalid) break;
        if (best_j < 0 || D < best) {
          best = D;
          best_j = j;
          if (fo.cell) S.write_flows(fo.cell + i * fo.stride, fo.w + i * fo.stride, fo.stride);
        }
        g.sync();
      }
    }
    if (g.lane == 0) {
      labels[i] = st == kStInvalid ? -1 : best_j;
      dist2[i] = st == kStInvalid ? nan("") : best;
      if (eps_terms) eps_terms[i] = (omega ? omega[i] : 1.0) * dist2[i];
      if (st == kStInvalid) atomicOr(err, kErrInvalid);
      if (st == kStNotConverged) atomicOr(err, kErrNotConverged);
    }
    g.sync();
  }
  if (g.lane == 0) add_stats(0, 0, n_ex, p_ex);
}

// Groups per block: up to 128 threads, whole warps only, within the
// 227 KB shared-memory limit of a block.  0 if one warp does not fit.
static int groups_per_block(int G, size_t slice, int tpb = 128) {
  const size_t limit = 227 * 1024;
  const int per_warp = 32 / G;
  int gpb = (tpb >= 32 && tpb <= 128 ? tpb : 128) / G;
  while (gpb >= per_warp && (size_t)gpb * slice > limit) gpb -= per_warp;
  return gpb >= per_warp ? gpb : 0;
}

template <typename KernelT>
static cudaError_t launch_cfg(KernelT kern, size_t smem, int threads, int sms, long long work,
                              int gpb, unsigned* grid) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (work + gpb - 1) / gpb;
  long long cap = (long long)per_sm * sms;
  long long gsz = need < cap ? need : cap;
  *grid = (unsigned)(gsz > 0 ? gsz : 1);
  return cudaSuccess;
}

template <int G, int NPL, int ST>
static cudaError_t mallows_pairs_g(const ObjView& ob, const CentView& cv, const long long* pobj,
                                   const long long* pcen, long long npairs, const SolveCfg& cfg,
                                   double* dist2, FlowOut fo, int* status, int* d_err,
                                   cudaStream_t st) {
  const size_t slice = pair_mem_bytes(cfg.mmax, cfg.nmax, cv.d);
  const int gpb = groups_per_block(G, slice);
  if (gpb == 0) return cudaErrorInvalidConfiguration;
  const size_t smem = slice * gpb;
  unsigned grid = 1;
  if (cfg.mode == 1 && cfg.tree &&
      cfg.tree_bytes >= pair_tree_bytes(npairs, cfg.mmax, cfg.nmax)) {
    const int ns = cfg.mmax + cfg.nmax;
    const size_t nodes = (size_t)npairs * ns;
    WarmStore tr{cfg.tree, cfg.tree + nodes, cfg.tree + 2 * nodes,
                 reinterpret_cast<long long*>(cfg.tree + (nodes * 3 + 15) / 16 * 16), ns, 0};
    int* st32 = reinterpret_cast<int*>(tr.flow + nodes);
    const size_t slice32 = pair_mem_bytes(cfg.mmax, cfg.nmax, cv.d, 4);  // FP32-only kernel
    const int gpb32 = groups_per_block(G, slice32);
    if (gpb32 == 0) return cudaErrorInvalidConfiguration;
    const size_t smem32 = slice32 * gpb32;
    unsigned g1 = 1, g2 = 1;
    cudaError_t e = launch_cfg(k_pairs32<G, NPL, ST>, smem32, gpb32 * G, cfg.sms, npairs, gpb32, &g1);
    if (e != cudaSuccess) return e;
    e = launch_cfg(k_pairs64<G, NPL>, smem, gpb * G, cfg.sms, npairs, gpb, &g2);
    if (e != cudaSuccess) return e;
    k_pairs32<G, NPL, ST><<<g1, gpb32 * G, smem32, st>>>(ob, cv, pobj, pcen, npairs, cfg, slice32,
                                                          tr, st32);
    k_pairs64<G, NPL><<<g2, gpb * G, smem, st>>>(ob, cv, pobj, pcen, npairs, cfg, slice, tr, st32,
                                                 dist2, fo, status, d_err);
    note_launches(2);
    return cudaGetLastError();
  }
  cudaError_t e = launch_cfg(k_mallows_pairs<G, NPL, ST>, smem, gpb * G, cfg.sms, npairs, gpb, &grid);
  if (e != cudaSuccess) return e;
  k_mallows_pairs<G, NPL, ST><<<grid, gpb * G, smem, st>>>(ob, cv, pobj, pcen, npairs, cfg, slice,
                                                            dist2, fo, status, d_err);
  note_launches(1);
  return cudaGetLastError();
}

template <int G, int NPL, int ST>
static cudaError_t assign_g(const ObjView& ob, const CentView& cv, long long seg_size, int K,
                            const SolveCfg& cfg, const double* omega, int* labels, double* dist2,
                            double* eps_terms, FlowOut fo, int* cand, int* d_err, cudaStream_t st,
                            const WarmStore* wsp, const TcWork* tw) {
  WarmStore ws{nullptr, nullptr, nullptr, nullptr, 0, 0};
  if (wsp) ws = *wsp;
  const size_t slice = pair_mem_bytes(cfg.mmax, cfg.nmax, cv.d);
  const int gpb = groups_per_block(G, slice, cfg.tpb);
  if (gpb == 0) return cudaErrorInvalidConfiguration;
  const size_t smem = slice * gpb;
  // the screen solves in FP32 only: the tighter slice of 4-byte costs
  const size_t slice32 = pair_mem_bytes(cfg.mmax, cfg.nmax, cv.d, 4);
  const int gpb32 = groups_per_block(G, slice32, cfg.tpb);
  if (gpb32 == 0) return cudaErrorInvalidConfiguration;
  const size_t smem32 = slice32 * gpb32;
  unsigned grid = 1;
  cudaError_t e;
  const bool screen = cfg.mode == 1 && cand != nullptr;
  // with a device-side range the count is not known here: persistent
  // grids, sized by the batch
  const long long nobj = cfg.dev_range ? ob.count : (cfg.nobj >= 0 ? cfg.nobj : ob.count);
  if (nobj <= 0) return cudaSuccess;
  if (screen) {
    // scratch layout: [queue counter: 4 ints][merged lists: count*kMergedInts][items]
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(cand);
    int* merged = cand + 4;
    int* items = merged + ((ob.count * kMergedInts + 3) & ~3LL);  // merged is indexed by object
    // one screening launch over objects [t0, t0+cnt) of this launch
    // with tensor-core tiles the screen reads them in place: no tile slice
    const size_t slice_tc = pair_mem_bytes(cfg.mmax, cfg.nmax, cv.d, 4, false);
    const int gpb_tc = groups_per_block(G, slice_tc, cfg.tpb);
    auto screen_part = [&](const SolveCfg& sc, long long cnt) -> cudaError_t {
      // items: (object, centroid block), the blocks chosen on the device
      // (centroid_blocks) from the launch's object count
      int NB, KB;
      centroid_blocks(sc, cnt, K, &NB, &KB);
      const long long work = sc.dev_range ? (1LL << 40) : cnt * (long long)NB;
      cudaError_t e2 = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st);
      if (e2 != cudaSuccess) return e2;
      const size_t sl = sc.tile.C ? slice_tc : slice32;
      const int gp = sc.tile.C ? gpb_tc : gpb32;
      auto launch = [&](auto kern) -> cudaError_t {
        unsigned g2 = 1;
        cudaError_t e3 = launch_cfg(kern, sl * gp, gp * G, sc.sms, work, gp, &g2);
        if (e3 != cudaSuccess) return e3;
        kern<<<g2, gp * G, sl * gp, st>>>(ob, cv, seg_size, K, sc, sl, items, queue, ws, d_err);
        return cudaSuccess;
      };
      if (sc.tile.C)
        e2 = sc.certify ? launch(k_screen<G, NPL, true, ST, true>)
                        : launch(k_screen<G, NPL, true, ST, false>);
      else
        e2 = sc.certify ? launch(k_screen<G, NPL, false, ST, true>)
                        : launch(k_screen<G, NPL, false, ST, false>);
      if (e2 != cudaSuccess) return e2;
      const unsigned mb = (unsigned)std::max<long long>(1, std::min<long long>((cnt + 255) / 256, 4096));
      k_merge<<<mb, 256, 0, st>>>(items, ob.count, K, sc, merged);
      note_launches(2);
      return cudaGetLastError();
    };
    if (tw && tw->C && cfg.mmax <= 64) {
      if (cfg.dev_range) return cudaErrorInvalidValue;  // chunks are cut on the host
      // tensor-core tiles, chunk by chunk within the tile buffer
      const long long per = std::max<long long>(1, tw->rows_cap / cfg.mmax);
      for (long long t0 = 0; t0 < nobj; t0 += per) {
        const long long cnt = std::min(per, nobj - t0);
        SolveCfg sc = cfg;
        sc.oidx = cfg.oidx ? cfg.oidx + t0 : nullptr;
        sc.obase = cfg.oidx ? 0 : cfg.obase + t0;
        sc.nobj = cnt;
        e = tc_chunk(ob, *tw, sc.oidx, sc.obase, cnt, cfg.mmax, 0, -1, d_err, st);
        if (e != cudaSuccess) return e;
        sc.tile.C = tw->C;
        sc.tile.trow = tw->trow;
        sc.tile.nx = tw->nx;
        sc.tile.cn = tw->cents.cn;
        sc.tile.cd = tw->cents.cd;
        sc.tile.ldc = tw->cents.ncols;
        sc.tile.col0 = 0;
        e = screen_part(sc, cnt);
        if (e != cudaSuccess) return e;
      }
    } else {
      e = screen_part(cfg, nobj);
      if (e != cudaSuccess) return e;
    }
  }
  if (screen && cfg.screen_only) return cudaGetLastError();
  e = launch_cfg(k_exact<G, NPL, ST>, smem, gpb * G, cfg.sms,
                 cfg.dev_range ? (1LL << 40) : nobj, gpb, &grid);
  if (e != cudaSuccess) return e;
  WarmStore wx = ws;
  if (!screen) wx.par8 = nullptr;
  k_exact<G, NPL, ST><<<grid, gpb * G, smem, st>>>(ob, cv, seg_size, K, cfg, slice,
                                               screen ? cand + 4 : nullptr, omega, labels, dist2,
                                               eps_terms, fo, wx, d_err);
  note_launches(1);
  return cudaGetLastError();
}

// Cold-start rule dispatch: Vogel's start (ST = 1) exists for trees of
// more than one node per lane only.
template <int G, int NPL>
static cudaError_t assign_st(const ObjView& ob, const CentView& cv, long long seg_size, int K,
                             const SolveCfg& cfg, const double* omega, int* labels, double* dist2,
                             double* eps_terms, FlowOut fo, int* cand, int* d_err, cudaStream_t st,
                             const WarmStore* ws, const TcWork* tw) {
  if constexpr (NPL > 1) {
    if (cfg.start == 1)
      return assign_g<G, NPL, 1>(ob, cv, seg_size, K, cfg, omega, labels, dist2, eps_terms, fo,
                                 cand, d_err, st, ws, tw);
  }
  return assign_g<G, NPL, 0>(ob, cv, seg_size, K, cfg, omega, labels, dist2, eps_terms, fo, cand,
                             d_err, st, ws, tw);
}

template <int G, int NPL>
static cudaError_t mallows_pairs_st(const ObjView& ob, const CentView& cv, const long long* pobj,
                                    const long long* pcen, long long npairs, const SolveCfg& cfg,
                                    double* dist2, FlowOut fo, int* status, int* d_err,
                                    cudaStream_t st) {
  if constexpr (NPL > 1) {
    if (cfg.start == 1)
      return mallows_pairs_g<G, NPL, 1>(ob, cv, pobj, pcen, npairs, cfg, dist2, fo, status, d_err,
                                        st);
  }
  return mallows_pairs_g<G, NPL, 0>(ob, cv, pobj, pcen, npairs, cfg, dist2, fo, status, d_err, st);
}

// This unit's solver counters (see g_solver_stats).
cudaError_t read_unit_stats(long long out[kStatWords]) {
  unsigned long long v[kStatWords] = {};
  cudaError_t e = cudaMemcpyFromSymbol(v, g_solver_stats, sizeof(v));
  for (int i = 0; i < kStatWords; ++i) out[i] = (long long)v[i];
  return e;
}

}  // namespace
}  // namespace d2k
