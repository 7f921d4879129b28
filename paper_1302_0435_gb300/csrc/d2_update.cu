// d2_update.cu -- centroid location update of Eq. (WeightedUpdate)
// (Eq. (UpdateZ) with unit weights), centroid weights held fixed:
//   z_j^(r) = sum_{i:C(i)=j} omega_i sum_a w_{r,a}^(i) v_i^(a)
//             / sum_{i:C(i)=j} omega_i sum_a w_{r,a}^(i).
// Deterministic: objects are grouped by centroid with a stable counting
// sort (chunk histograms, per-label prefix, in-order warp scatter), then one
// block per centroid accumulates its members in increasing object index, and
// each member's flow entries in stored order, in FP64.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "d2_internal.h"

namespace d2k {

namespace {
constexpr int kChunk = 1024;

__host__ __device__ inline size_t al(size_t x) { return (x + 255) / 256 * 256; }

__global__ void k_global_label(const int* labels, long long N, long long seg_size, const int* segof,
                               int K, long long KT, int* gl) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int l = labels[i];
    const long long g = (segof ? (long long)segof[i] : i / seg_size) * (long long)K + l;
    gl[i] = (l < 0 || l >= K || g >= KT) ? -1 : (int)g;
  }
}

__global__ void k_chunk_hist(const int* gl, long long N, long long KT, int* counts) {
  const long long c = blockIdx.x;
  const long long lo = c * kChunk;
  const long long hi = lo + kChunk < N ? lo + kChunk : N;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int g = gl[i];
    if (g >= 0) atomicAdd(&counts[c * KT + g], 1);
  }
}

// per label: exclusive prefix over chunks (in place), totals out
__global__ void k_label_prefix(int* counts, long long nchunks, long long KT, long long* tot) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < KT;
       g += (long long)gridDim.x * blockDim.x) {
    long long run = 0;
    for (long long c = 0; c < nchunks; ++c) {
      const int v = counts[c * KT + g];
      counts[c * KT + g] = (int)run;
      run += v;
    }
    tot[g] = run;
  }
}

// exclusive scan over labels, one block
__global__ void k_exclusive_scan(const long long* tot, long long KT, long long* start) {
  __shared__ long long sh[1024];
  long long carry = 0;
  for (long long base = 0; base < KT; base += blockDim.x) {
    const long long g = base + threadIdx.x;
    long long v = g < KT ? tot[g] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
      long long u = (int)threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += u;
      __syncthreads();
    }
    if (g < KT) start[g] = carry + sh[threadIdx.x] - v;
    const long long last = sh[blockDim.x - 1];
    __syncthreads();
    carry += last;
  }
  if (threadIdx.x == 0) start[KT] = carry;
}

// one warp per chunk, objects in order: stable positions
__global__ void k_scatter(const int* gl, long long N, long long KT, int* counts,
                          const long long* start, int* order) {
  const long long c = blockIdx.x;
  const long long lo = c * kChunk;
  const long long hi = lo + kChunk < N ? lo + kChunk : N;
  const int lane = threadIdx.x;
  for (long long b = lo; b < hi; b += 32) {
    const long long i = b + lane;
    const int g = i < hi ? gl[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, g);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int basev = 0;
    if (g >= 0) basev = counts[c * KT + g];
    __syncwarp();
    if (g >= 0) {
      order[start[g] + basev + rank] = (int)i;
      if (rank == 0) counts[c * KT + g] = basev + __popc(peers);
    }
    __syncwarp();
  }
}

__device__ __forceinline__ double ldloc(const void* p, int dt, long long idx) {
  if (dt == 0) return static_cast<const double*>(p)[idx];
  if (dt == 1) return (double)static_cast<const float*>(p)[idx];
  return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[idx]);
}

__device__ __forceinline__ double round_to(double v, int dt) {
  if (dt == 1) return (double)(float)v;
  if (dt == 2) return (double)__bfloat162float(__float2bfloat16_rn((float)v));
  return v;
}

constexpr int kStageEntries = 1024;  // flow entries staged per step
constexpr int kMaxStride = 127;

// One block per centroid.  Members (objects assigned to it, increasing
// index) are staged as many whole members at a time as fit kStageEntries
// flow entries: each entry's centroid support r, object row and coefficient
// omega_i * w go to shared memory, and one warp lists the entries of every
// column r in entry order (a stable counting sort by r).  Then every (r, k)
// slot of the numerator sums, in entry order, the entries of its column
// (coef * v^(a)_k) in FP64; the k == 0 slot also sums the denominator.  The
// order of every sum is fixed, so results are deterministic.  Dynamic smem:
// num [n*d] + den [n] doubles, then the staged entries and column lists.
//
// Large clusters are split over U blocks (blockIdx.y = part p takes the p-th
// of U equal runs of the members); with U > 1 each part writes its sums to
// `part` and k_accumulate_sum adds the parts in part order, so the result is
// still deterministic.
__global__ void k_accumulate(ObjView ob, const double* omega, FlowOut fo, const int* order,
                             const long long* start, const long long* coff, int d, int cent_ldt,
                             float* loc32, double* loc64, int U, double* part) {
  extern __shared__ __align__(16) double acc[];
  const long long g = blockIdx.x;
  const long long c0 = coff[g];
  const int n = (int)(coff[g + 1] - c0);
  double* num = acc;
  double* den = acc + (size_t)n * d;
  double* e_coef = den + n;
  long long* e_row = reinterpret_cast<long long*>(e_coef + kStageEntries);
  int* e_r = reinterpret_cast<int*>(e_row + kStageEntries);
  int* blist = e_r + kStageEntries;
  int* bend = blist + kStageEntries;  // [n+1]
  const int stride = (int)(fo.stride < kMaxStride ? fo.stride : kMaxStride);
  const int per = kStageEntries / stride;
  const int slots = n * d;
  const int lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < slots; t += blockDim.x) num[t] = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) den[t] = 0.0;
  const long long gb = start[g], ge = start[g + 1];
  const long long len = (ge - gb + U - 1) / U;
  const long long b = gb + (long long)blockIdx.y * len;
  const long long e = b + len < ge ? b + len : ge;
  for (long long c = b; c < e; c += per) {
    const int cm = (int)(e - c < per ? e - c : per);
    __syncthreads();
    for (int q = threadIdx.x; q < cm * stride; q += blockDim.x) {
      const int mi = q / stride, qq = q - mi * stride;
      const long long i = order[c + mi];
      const long long o0 = ob.off[i];
      const int m = (int)(ob.off[i + 1] - o0);
      const int cl = fo.cell[i * fo.stride + qq];
      const int a = cl >> 16, r = cl & 0xffff;
      const bool ok = cl >= 0 && a < m && r < n;  // other entries are ignored
      e_r[q] = ok ? r : -1;
      e_row[q] = o0 + a;
      e_coef[q] = ok ? (omega ? omega[i] : 1.0) * fo.w[i * fo.stride + qq] : 0.0;
    }
    __syncthreads();
    const int ne = cm * stride;
    if (threadIdx.x < 32) {
      // counts per column, then starts, then a stable scatter in entry order
      for (int r = lane; r <= n; r += 32) bend[r] = 0;
      __syncwarp();
      for (int base = 0; base < ne; base += 32) {
        const int q = base + lane;
        const int rr = q < ne ? e_r[q] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, rr);
        if (rr >= 0 && lane == __ffs(peers) - 1) bend[rr + 1] += __popc(peers);
        __syncwarp();
      }
      if (lane == 0)
        for (int r = 0; r < n; ++r) bend[r + 1] += bend[r];
      __syncwarp();
      for (int base = 0; base < ne; base += 32) {
        const int q = base + lane;
        const int rr = q < ne ? e_r[q] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, rr);
        if (rr >= 0) blist[bend[rr] + __popc(peers & ((1u << lane) - 1u))] = q;
        __syncwarp();
        if (rr >= 0 && lane == __ffs(peers) - 1) bend[rr] += __popc(peers);
        __syncwarp();
      }
      // column r now spans blist[(r ? bend[r-1] : 0) .. bend[r])
    }
    __syncthreads();
    for (int t = threadIdx.x; t < slots; t += blockDim.x) {
      const int r = t / d, k = t - r * d;
      double sn = num[t], sd = (k == 0) ? den[r] : 0.0;
      const int lo = r > 0 ? bend[r - 1] : 0, hi = bend[r];
      for (int x = lo; x < hi; ++x) {
        const int q = blist[x];
        const double cf = e_coef[q];
        sn = fma(cf, ldloc(ob.loc, ob.ldt, e_row[q] * d + k), sn);
        if (k == 0) sd += cf;
      }
      num[t] = sn;
      if (k == 0) den[r] = sd;
    }
  }
  __syncthreads();
  if (U > 1) {
    double* out = part + ((size_t)g * U + blockIdx.y) * ((size_t)64 * d + 64);
    for (int t = threadIdx.x; t < n * d; t += blockDim.x) out[t] = num[t];
    for (int t = threadIdx.x; t < n; t += blockDim.x) out[(size_t)64 * d + t] = den[t];
    return;
  }
  for (int t = threadIdx.x; t < n * d; t += blockDim.x) {
    const int r = t / d;
    if (den[r] > 0.0) {
      const double v = round_to(num[t] / den[r], cent_ldt);
      loc64[c0 * d + t] = v;
      loc32[c0 * d + t] = (float)v;
    }
  }
}

// The parts of each centroid added in part order, then the new locations.
__global__ void k_accumulate_sum(const long long* coff, int d, int cent_ldt, int U,
                                 const double* part, float* loc32, double* loc64) {
  const long long g = blockIdx.x;
  const long long c0 = coff[g];
  const int n = (int)(coff[g + 1] - c0);
  const size_t ps = (size_t)64 * d + 64;
  const double* in = part + (size_t)g * U * ps;
  for (int t = threadIdx.x; t < n * d; t += blockDim.x) {
    const int r = t / d;
    double sn = 0.0, sd = 0.0;
    for (int q = 0; q < U; ++q) {
      sn += in[q * ps + t];
      sd += in[q * ps + (size_t)64 * d + r];
    }
    if (sd > 0.0) {
      const double v = round_to(sn / sd, cent_ldt);
      loc64[c0 * d + t] = v;
      loc32[c0 * d + t] = (float)v;
    }
  }
}
}  // namespace

// group sums of per-object values in the sorted order: out[g] = sum of
// v[i] over members i of g, i increasing (deterministic)
__global__ void k_group_sum(const double* v, const int* order, const long long* start, long long KT,
                            double* out) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < KT;
       g += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (long long t = start[g]; t < start[g + 1]; ++t) acc += v ? v[order[t]] : 1.0;
    out[g] = acc;
  }
}

size_t update_scratch_bytes(long long N, long long KT) {
  const long long nchunks = (N + kChunk - 1) / kChunk;
  return al((size_t)(nchunks > 0 ? nchunks : 1) * KT * 4) + al((size_t)(KT + 1) * 8) * 2 +
         al((size_t)N * 4) * 2;
}

size_t update_part_bytes(long long N, long long KT, int d) {
  const long long U = update_parts(N, KT);
  return U > 1 ? (size_t)(KT * U) * ((size_t)64 * d + 64) * sizeof(double) : 0;
}

cudaError_t update_locations(const ObjView& ob, const double* omega, const int* labels,
                             long long seg_size, int K, const FlowOut& fo, long long KT,
                             const long long* coff, int d, int cent_ldt, float* loc32,
                             double* loc64, void* scratch, cudaStream_t st, double* part,
                             size_t part_bytes) {
  const long long N = ob.count;
  if (N <= 0 || KT <= 0) return cudaSuccess;
  const long long nchunks = (N + kChunk - 1) / kChunk;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  int* counts = reinterpret_cast<int*>(p); p += al((size_t)nchunks * KT * 4);
  long long* tot = reinterpret_cast<long long*>(p); p += al((size_t)(KT + 1) * 8);
  long long* start = reinterpret_cast<long long*>(p); p += al((size_t)(KT + 1) * 8);
  int* order = reinterpret_cast<int*>(p); p += al((size_t)N * 4);
  int* gl = reinterpret_cast<int*>(p);
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)nchunks * KT * 4, st);
  if (e != cudaSuccess) return e;
  const unsigned gb = (unsigned)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
  k_global_label<<<gb, 256, 0, st>>>(labels, N, seg_size, ob.segof, K, KT, gl);
  k_chunk_hist<<<(unsigned)nchunks, 256, 0, st>>>(gl, N, KT, counts);
  const unsigned kb = (unsigned)((KT + 255) / 256);
  k_label_prefix<<<kb, 256, 0, st>>>(counts, nchunks, KT, tot);
  k_exclusive_scan<<<1, 1024, 0, st>>>(tot, KT, start);
  k_scatter<<<(unsigned)nchunks, 32, 0, st>>>(gl, N, KT, counts, start, order);
  note_launches(5);
  if (!fo.cell) return cudaGetLastError();  // sort only
  // largest centroid support bounds the accumulator size
  const size_t smem = ((size_t)64 * d + 64) * sizeof(double) +
                      (size_t)kStageEntries * (8 + 8 + 4 + 4) + 65 * 4;
  e = cudaFuncSetAttribute(k_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // several blocks per centroid when the clusters are large (few centroids,
  // many members) and the caller gave room for the parts
  int U = (int)update_parts(N, KT);
  if (!part || part_bytes < update_part_bytes(N, KT, d)) U = 1;
  k_accumulate<<<dim3((unsigned)KT, (unsigned)U), 128, smem, st>>>(
      ob, omega, fo, order, start, coff, d, cent_ldt, loc32, loc64, U, part);
  note_launches(1);
  if (U > 1) {
    k_accumulate_sum<<<(unsigned)KT, 128, 0, st>>>(coff, d, cent_ldt, U, part, loc32, loc64);
    note_launches(1);
  }
  return cudaGetLastError();
}

void sorted_groups(void* scratch, long long N, long long KT, const long long** start,
                   const int** order) {
  const long long nchunks = (N + kChunk - 1) / kChunk;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  p += al((size_t)nchunks * KT * 4);
  p += al((size_t)(KT + 1) * 8);
  *start = reinterpret_cast<const long long*>(p); p += al((size_t)(KT + 1) * 8);
  *order = reinterpret_cast<const int*>(p);
}

cudaError_t group_weight_sum(const double* omega, long long N, long long KT, void* scratch,
                             double* out, cudaStream_t st) {
  const long long nchunks = (N + kChunk - 1) / kChunk;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  p += al((size_t)nchunks * KT * 4);
  p += al((size_t)(KT + 1) * 8);
  const long long* start = reinterpret_cast<const long long*>(p); p += al((size_t)(KT + 1) * 8);
  const int* order = reinterpret_cast<const int*>(p);
  const unsigned kb = (unsigned)((KT + 255) / 256);
  k_group_sum<<<kb, 256, 0, st>>>(omega, order, start, KT, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace d2k
