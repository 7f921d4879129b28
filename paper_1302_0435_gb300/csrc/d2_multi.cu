// d2_multi.cu -- nearest centroid under the combined distance of several
// bag types (Eq. (imgdist)): D^2(I_i, Z_j) = sum_b D^2(U_i^b, Z_j^b).
// Each type's FP32 screen leaves, per (object, centroid) pair, its value
// and error bound; here the bounds are summed over the types, the
// candidates of each object are listed (every centroid whose summed
// interval reaches the smallest summed upper end), and after each type has
// solved the listed pairs exactly the summed FP64 values give the label
// (ties to the smallest centroid index).
#include <cuda_runtime.h>

#include <cmath>

#include "d2_internal.h"

namespace d2k {
namespace {

// Candidates of object i: count (or -1: a type could not screen the bag).
__device__ int cand_of(const MultiScreen& ms, long long i, int K, long long* out) {
  float best_hi = INFINITY;
  for (int j = 0; j < K; ++j) {
    float v = 0.f, e = 0.f;
    for (int b = 0; b < ms.B; ++b) {
      const float* p = ms.pair[b] + 2 * (i * (long long)K + j);
      v += p[0];
      e += p[1] + fabsf(p[0]) * 0x1p-23f;  // the type's bound, plus the FP32 sum's rounding
    }
    if (isnan(v)) return -1;
    best_hi = fminf(best_hi, v + e);
  }
  int cnt = 0;
  for (int j = 0; j < K; ++j) {
    float v = 0.f, e = 0.f;
    for (int b = 0; b < ms.B; ++b) {
      const float* p = ms.pair[b] + 2 * (i * (long long)K + j);
      v += p[0];
      e += p[1] + fabsf(p[0]) * 0x1p-23f;
    }
    if (v - e <= best_hi) {
      if (out) out[cnt] = j;
      ++cnt;
    }
  }
  return cnt;
}

__global__ void k_multi_count(MultiScreen ms, long long N, int K, long long* cnt, int* err) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = cand_of(ms, i, K, nullptr);
    if (c < 0) atomicOr(err, kErrInvalid);
    cnt[i] = c < 0 ? 0 : c;
  }
}

// Exclusive prefix over N counts, start[N] = total.  One block.
__global__ void k_multi_scan(const long long* cnt, long long N, long long* start) {
  __shared__ long long wsum[32];
  __shared__ long long carry_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (long long base = 0; base < N; base += blockDim.x) {
    const long long t = base + tid;
    const long long v = t < N ? cnt[t] : 0;
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
    if (t < N) start[t] = c + (warp > 0 ? wsum[warp - 1] : 0) + x - v;
    __syncthreads();
    if (tid == 0) carry_s = c + wsum[nw - 1];
    __syncthreads();
  }
  if (tid == 0) start[N] = carry_s;
}

__global__ void k_multi_fill(MultiScreen ms, long long N, int K, const long long* start,
                             long long* pobj, long long* pcen) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s0 = start[i];
    const int c = cand_of(ms, i, K, pcen + s0);
    for (int t = 0; t < c; ++t) pobj[s0 + t] = i;
  }
}

__global__ void k_multi_argmin(long long N, const long long* start, const long long* pcen,
                               MultiExact mx, int* labels, double* dist2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    int best_j = -1;
    double best = NAN;
    for (long long t = start[i]; t < start[i + 1]; ++t) {
      double s = 0.0;
      for (int b = 0; b < mx.B; ++b) s += mx.d2[b][t];
      if (best_j < 0 || s < best) {  // candidates run in increasing j
        best = s;
        best_j = (int)pcen[t];
      }
    }
    labels[i] = best_j;
    dist2[i] = best;
  }
}

unsigned blocks_for(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t multi_candidates(const MultiScreen& ms, long long N, int K, long long* cnt,
                             long long* start, int* d_err, cudaStream_t st) {
  k_multi_count<<<blocks_for(N), 256, 0, st>>>(ms, N, K, cnt, d_err);
  k_multi_scan<<<1, 1024, 0, st>>>(cnt, N, start);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t multi_fill(const MultiScreen& ms, long long N, int K, const long long* start,
                       long long* pobj, long long* pcen, cudaStream_t st) {
  k_multi_fill<<<blocks_for(N), 256, 0, st>>>(ms, N, K, start, pobj, pcen);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t multi_argmin(long long N, const long long* start, const long long* pcen,
                         const MultiExact& mx, int* labels, double* dist2, cudaStream_t st) {
  k_multi_argmin<<<blocks_for(N), 256, 0, st>>>(N, start, pcen, mx, labels, dist2);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace d2k
