// d2_segment.cu -- device helpers of the initial data segmentation
// (Alg. 3 Step 1): gather one segment's bags into a compact view, and build
// the uniform-weight start centroids of a binary constrained split
// (Alg. 2 Step 3*) from member bags.  The split loop itself (assign,
// location update, partition, largest-first order) runs on the host in
// d2_api.cu with the assignment and update kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "d2_internal.h"
#include "d2_segment.h"

namespace d2k {
namespace {

// Row offsets of the gathered bags: off_out[t] = sum of sizes of
// members[0..t), t = 0..cnt.  One block.
__global__ void k_seg_offsets(const long long* __restrict__ off, const int* __restrict__ members,
                              long long cnt, long long* __restrict__ off_out) {
  __shared__ long long wsum[32];
  __shared__ long long carry_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (long long base = 0; base < cnt; base += blockDim.x) {
    const long long t = base + tid;
    long long v = 0;
    if (t < cnt) {
      const long long i = members[t];
      v = off[i + 1] - off[i];
    }
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
    if (t < cnt) off_out[t] = c + (warp > 0 ? wsum[warp - 1] : 0) + x - v;
    __syncthreads();
    if (tid == 0) carry_s = c + wsum[nw - 1];
    __syncthreads();
  }
  if (tid == 0) off_out[cnt] = carry_s;
}

// One warp per member: its location rows and weights (bytes, any element
// type) and its omega.
__global__ void k_seg_gather(ObjView v, const int* __restrict__ members, long long cnt,
                             const long long* __restrict__ off_out, int lsz, int wsz,
                             unsigned char* __restrict__ loc_out, unsigned char* __restrict__ w_out,
                             const double* __restrict__ om_in, double* __restrict__ om_out) {
  const int lane = threadIdx.x & 31;
  for (long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; t < cnt;
       t += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long i = members[t];
    const long long r0 = v.off[i], r1 = v.off[i + 1], q0 = off_out[t];
    const long long lb = (r1 - r0) * v.d * lsz, wb = (r1 - r0) * wsz;
    const unsigned char* ls = static_cast<const unsigned char*>(v.loc) + r0 * v.d * lsz;
    const unsigned char* ws = static_cast<const unsigned char*>(v.w) + r0 * wsz;
    for (long long b = lane; b < lb; b += 32) loc_out[q0 * v.d * lsz + b] = ls[b];
    for (long long b = lane; b < wb; b += 32) w_out[q0 * wsz + b] = ws[b];
    if (lane == 0) om_out[t] = om_in ? om_in[i] : 1.0;
  }
}

__device__ __forceinline__ double ld_any(const void* p, int dt, long long idx) {
  if (dt == 0) return static_cast<const double*>(p)[idx];
  if (dt == 1) return (double)static_cast<const float*>(p)[idx];
  return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[idx]);
}

// Start centroids of a split: the supports of compact bags idx[0..K) with
// uniform weights 1/s, FP64 locations.  One block.
__global__ void k_seg_cents(const void* loc, int ldt, const long long* __restrict__ off, int d,
                            int i0, int i1, int K, double* __restrict__ cloc,
                            double* __restrict__ cw, long long* __restrict__ coff) {
  const int idx[2] = {i0, i1};
  long long base = 0;
  for (int j = 0; j < K; ++j) {
    const long long r0 = off[idx[j]], n = off[idx[j] + 1] - r0;
    for (long long e = threadIdx.x; e < n * d; e += blockDim.x)
      cloc[base * d + e] = ld_any(loc, ldt, r0 * d + e);
    for (long long r = threadIdx.x; r < n; r += blockDim.x) cw[base + r] = 1.0 / (double)n;
    if (threadIdx.x == 0) coff[j] = base;
    base += n;
  }
  if (threadIdx.x == 0) coff[K] = base;
}

// Start centroids of several splits at once: centroid t is compact bag
// idx[t] with uniform weights 1/s, FP64 locations, at row coff[t] (the
// prefix of the bags' sizes, k_seg_offsets).  One warp per centroid.
__global__ void k_seg_cents_list(const void* loc, int ldt, const long long* __restrict__ off,
                                 int d, const int* __restrict__ idx, long long KT,
                                 const long long* __restrict__ coff, double* __restrict__ cloc,
                                 double* __restrict__ cw) {
  const int lane = threadIdx.x & 31;
  for (long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; t < KT;
       t += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long i = idx[t];
    const long long r0 = off[i], n = off[i + 1] - r0, base = coff[t];
    for (long long e = lane; e < n * d; e += 32) cloc[base * d + e] = ld_any(loc, ldt, r0 * d + e);
    for (long long r = lane; r < n; r += 32) cw[base + r] = 1.0 / (double)n;
  }
}

}  // namespace

cudaError_t seg_cents_list(const ObjView& v, const int* idx, long long KT, double* cloc,
                           double* cw, long long* coff, cudaStream_t st) {
  if (KT <= 0) return cudaSuccess;
  k_seg_offsets<<<1, 1024, 0, st>>>(v.off, idx, KT, coff);
  const unsigned gb = (unsigned)((KT * 32 + 255) / 256 < 8192 ? (KT * 32 + 255) / 256 : 8192);
  k_seg_cents_list<<<gb, 256, 0, st>>>(v.loc, v.ldt, v.off, v.d, idx, KT, coff, cloc, cw);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t seg_gather(const ObjView& v, const int* members, long long cnt, const double* om_in,
                       long long* off_out, void* loc_out, void* w_out, double* om_out,
                       cudaStream_t st) {
  if (cnt <= 0) return cudaSuccess;
  const int lsz = v.ldt == 0 ? 8 : (v.ldt == 1 ? 4 : 2);
  const int wsz = v.wdt == 0 ? 8 : 4;
  k_seg_offsets<<<1, 1024, 0, st>>>(v.off, members, cnt, off_out);
  const unsigned gb = (unsigned)((cnt * 32 + 255) / 256 < 8192 ? (cnt * 32 + 255) / 256 : 8192);
  k_seg_gather<<<gb, 256, 0, st>>>(v, members, cnt, off_out, lsz, wsz,
                                   static_cast<unsigned char*>(loc_out),
                                   static_cast<unsigned char*>(w_out), om_in, om_out);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t seg_cents(const ObjView& v, int i0, int i1, int K, double* cloc, double* cw,
                      long long* coff, cudaStream_t st) {
  if (K < 1 || K > 2) return cudaErrorInvalidValue;
  k_seg_cents<<<1, 256, 0, st>>>(v.loc, v.ldt, v.off, v.d, i0, i1, K, cloc, cw, coff);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace d2k
