// d2_tc.cu -- ground-cost tiles of Eq. (D2opt) on the tensor cores for the
// FP32 screen at high support dimension.
//
// The squared Euclidean cost expands as ||x||^2 + ||y||^2 - 2 x.y, so the
// cost of every object support against every centroid support of a chunk is
// one contraction over the d coordinates: rows = the chunk's object supports
// (gathered in the order the screen visits the objects), columns = all
// centroid supports.  Operands are BF16 (the objects are stored as BF16;
// the centroids are rounded to BF16 with a measured per-centroid bound),
// products are exact in FP32 and accumulate in FP32 in tensor memory; the
// epilogue adds the FP32 squared norms and stores an FP32 tile to HBM that
// the screen reads instead of building its cost tile with SIMT arithmetic.
//
// k_cost_tc: one CTA of 4 warps per (256-column tile, run of 128-row tiles).
// The centroid tile (256 x d) is staged once in shared memory in the
// no-swizzle K-major core-matrix layout; each row tile (128 x d) is gathered
// with cp.async, one thread issues d/16 tcgen05.mma (M=128, N=256, K=16,
// kind::f16 with BF16 inputs) into a 128 x 256 FP32 accumulator in TMEM,
// and the four warps read their 32 TMEM lanes back with tcgen05.ld for the
// epilogue.  Every wait on the MMA completion barrier is bounded: on expiry
// the kernel raises kErrTimeout, waits (bounded) once more, frees its TMEM
// and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "d2_internal.h"

namespace d2k {
namespace {

constexpr int kTcBM = 128;       // rows per tile (TMEM lanes)
constexpr int kTcBN = 256;       // columns per tile (TMEM columns, FP32)
constexpr int kTcThreads = 128;  // 4 warps: warp w owns TMEM lanes 32w..32w+31
constexpr int kTcRowTiles = 8;   // row tiles per CTA (the centroid tile is reused)
constexpr long long kWaitIters = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of row r, 8-element chunk k8 in a no-swizzle K-major tile of
// d columns: 8x8 core matrices of 128 contiguous bytes (8 rows x 16 bytes),
// the core matrices of one 8-row group adjacent along K (128 bytes apart),
// 8-row groups (d/8)*128 bytes apart.
__device__ __forceinline__ uint32_t cm_off(int r, int k8, int d) {
  return (uint32_t)((((r >> 3) * (d >> 3) + k8) << 7) + ((r & 7) << 4));
}

// Shared-memory matrix descriptor of tcgen05: start address, leading byte
// offset (K-adjacent core matrices), stride byte offset (8-row groups), all
// in 16-byte units; bits 46-48 hold the fixed value 0b001; no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t v = (uint64_t)((addr >> 4) & 0x3FFFu);
  v |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  v |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  v |= (uint64_t)1 << 46;
  return v;
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kWaitIters && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// Non-blocking polls of a barrier, at most `polls` of them.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity, long long polls) {
  uint32_t done = 0;
  for (long long it = 0; it < polls && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_cost_tc(const __nv_bfloat16* __restrict__ X, const long long* __restrict__ rowsrc,
              const float* __restrict__ nx, const long long* __restrict__ total_p,
              const __nv_bfloat16* __restrict__ Y, const float* __restrict__ yn, int d,
              long long ldc, int ct0, float* __restrict__ C, int* err, long long probe_polls) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) unsigned long long mbar;
  // diagnostic (probe_polls > 0): the first completion wait polls this
  // barrier instead, which nothing ever arrives on, so it runs out and the
  // kernel takes its timeout path with MMAs really in flight
  __shared__ __align__(8) unsigned long long mbar_probe;
  __shared__ uint32_t tmem_slot;
  unsigned char* sA = sm;                                                   // 128 x d BF16
  unsigned char* sB = sm + (size_t)kTcBM * d * 2;                          // 256 x d BF16
  float* sYn = reinterpret_cast<float*>(sB + (size_t)kTcBN * d * 2);       // 256 FP32
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long total = *total_p;
  const long long col0 = (long long)(ct0 + blockIdx.x) * kTcBN;
  const long long rt0 = (long long)blockIdx.y * kTcRowTiles;
  if (rt0 * kTcBM >= total) return;  // CTA-uniform, before any allocation
  const int kc = d >> 3;             // 16-byte chunks per row
  // centroid tile and its norms, once per CTA (consecutive threads take
  // consecutive rows of a core matrix: conflict-free shared stores)
  for (int c = tid; c < kTcBN * kc; c += kTcThreads) {
    const int r = (c & 7) + ((c / (8 * kc)) << 3);
    const int k8 = (c >> 3) % kc;
    cp16(smem_u32(sB) + cm_off(r, k8, d), Y + (col0 + r) * d + k8 * 8, true);
  }
  for (int c = tid; c < kTcBN; c += kTcThreads) sYn[c] = yn[col0 + c];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTcBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_probe)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t bar = smem_u32(&mbar);
  const uint32_t lbo = 128, sbo = (uint32_t)kc * 128;
  // kind::f16 instruction descriptor: D FP32 (bits 4-5 = 1), A and B BF16
  // (bits 7-9, 10-12 = 1), both K-major, N/8 at bit 17, M/16 at bit 24
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcBN >> 3) << 17) |
                         ((uint32_t)(kTcBM >> 4) << 24);
  uint32_t phase = 0;
  bool alive = true, issued = false;
  for (int q = 0; q < kTcRowTiles; ++q) {
    const long long row0 = (rt0 + q) * kTcBM;
    if (row0 >= total) break;  // CTA-uniform
    for (int c = tid; c < kTcBM * kc; c += kTcThreads) {
      const int r = (c & 7) + ((c / (8 * kc)) << 3);
      const int k8 = (c >> 3) % kc;
      const long long R = row0 + r;
      const bool v = R < total;
      const long long src = v ? rowsrc[R] : 0;
      cp16(smem_u32(sA) + cm_off(r, k8, d), X + src * d + k8 * 8, v);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      for (int s = 0; s < (d >> 4); ++s) {
        const uint64_t ad = sdesc(smem_u32(sA) + (uint32_t)s * 256u, lbo, sbo);
        const uint64_t bd = sdesc(smem_u32(sB) + (uint32_t)s * 256u, lbo, sbo);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
          : "memory");
    }
    issued = true;
    const bool got = probe_polls > 0 ? mbar_test(smem_u32(&mbar_probe), 0u, probe_polls)
                                     : mbar_wait(bar, phase);
    const bool ok = __syncthreads_and(got ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) atomicOr(err, kErrTimeout);
      alive = false;
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: thread owns tile row 32*warp + lane
    const long long R = row0 + warp * 32 + lane;
    const bool live = R < total;
    const float nr = live ? nx[R] : 0.f;
    float* crow = C + (live ? R : 0) * ldc + col0;
#pragma unroll 1
    for (int cb = 0; cb < kTcBN; cb += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      if (live) {
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          float4 o;
          o.x = fmaxf(0.f, fmaf(-2.f, __uint_as_float(v[j + 0]), nr + sYn[cb + j + 0]));
          o.y = fmaxf(0.f, fmaf(-2.f, __uint_as_float(v[j + 1]), nr + sYn[cb + j + 1]));
          o.z = fmaxf(0.f, fmaf(-2.f, __uint_as_float(v[j + 2]), nr + sYn[cb + j + 2]));
          o.w = fmaxf(0.f, fmaf(-2.f, __uint_as_float(v[j + 3]), nr + sYn[cb + j + 3]));
          *reinterpret_cast<float4*>(crow + cb + j) = o;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // TMEM and the row tile are free for the next step
  }
  if (!alive && issued) {
    // the MMAs of the abandoned step may still be in flight: give them one
    // more bounded wait before the accumulator is released
    mbar_wait(bar, phase);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcBN));
}

// Per centroid support row: BF16 rounding, FP32 squared norm of the rounded
// vector (FMA in coordinate order), FP64 distance to the FP64 original.
__global__ void k_tc_prep_rows(const double* __restrict__ loc64, long long Tc, long long ncols,
                               int d, __nv_bfloat16* __restrict__ yb, float* __restrict__ yn,
                               double* __restrict__ ydel) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < ncols;
       r += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    double del = 0.0;
    for (int k = 0; k < d; ++k) {
      const double y = r < Tc ? loc64[r * d + k] : 0.0;
      const __nv_bfloat16 b = __float2bfloat16_rn(__double2float_rn(y));
      const float bf = __bfloat162float(b);
      yb[r * d + k] = b;
      acc = fmaf(bf, bf, acc);
      const double e = y - (double)bf;
      del = fma(e, e, del);
    }
    yn[r] = acc;
    ydel[r] = sqrt(del);
  }
}

__global__ void k_tc_prep_cent(const long long* __restrict__ off, long long K,
                               const float* __restrict__ yn, const double* __restrict__ ydel,
                               float* __restrict__ cn, float* __restrict__ cd) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < K;
       j += (long long)gridDim.x * blockDim.x) {
    float mx = 0.f;
    double dl = 0.0;
    for (long long r = off[j]; r < off[j + 1]; ++r) {
      mx = fmaxf(mx, yn[r]);
      dl = fmax(dl, ydel[r]);
    }
    cn[j] = mx;
    cd[j] = dl > 0.0 ? __double2float_ru(dl * (1.0 + 0x1p-40)) : 0.f;
  }
}

// Exclusive prefix of the chunk objects' row counts (objects with m outside
// 1..mmax get no rows): trow[t], t = 0..cnt.  One block.
__global__ void k_tc_scan(const long long* __restrict__ off, const int* __restrict__ oidx,
                          long long obase, long long cnt, int mmax, long long* __restrict__ trow) {
  __shared__ long long wsum[32];
  __shared__ long long carry_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (long long base = 0; base < cnt; base += blockDim.x) {
    const long long t = base + tid;
    long long v = 0;
    if (t < cnt) {
      const long long i = oidx ? (long long)oidx[t] : obase + t;
      const long long m = off[i + 1] - off[i];
      v = (m >= 1 && m <= mmax) ? m : 0;
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
      if (lane < nw) wsum[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const long long c = carry_s;
    const long long excl = c + (warp > 0 ? wsum[warp - 1] : 0) + x - v;
    if (t < cnt) trow[t] = excl;
    __syncthreads();
    if (tid == 0) carry_s = c + wsum[nw - 1];
    __syncthreads();
  }
  if (tid == 0) trow[cnt] = carry_s;
}

// One warp per chunk object: source row and FP32 squared norm of each of
// its tile rows (lane a takes support a).
__global__ void k_tc_gather(const long long* __restrict__ off, const __nv_bfloat16* __restrict__ X,
                            const int* __restrict__ oidx, long long obase, long long cnt, int d,
                            const long long* __restrict__ trow, long long* __restrict__ rowsrc,
                            float* __restrict__ nx) {
  const int lane = threadIdx.x & 31;
  for (long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; t < cnt;
       t += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long i = oidx ? (long long)oidx[t] : obase + t;
    const long long r0 = trow[t];
    const int rows = (int)(trow[t + 1] - r0);
    for (int a = lane; a < rows; a += 32) {
      const long long src = off[i] + a;
      const __nv_bfloat16* x = X + src * d;
      float acc = 0.f;
      for (int k = 0; k < d; ++k) {
        const float v = __bfloat162float(x[k]);
        acc = fmaf(v, v, acc);
      }
      rowsrc[r0 + a] = src;
      nx[r0 + a] = acc;
    }
  }
}

__global__ void k_tc_extract(const float* __restrict__ C, long long ldc, int m, long long c0,
                             int n, double* __restrict__ out) {
  for (int t = threadIdx.x; t < m * n; t += blockDim.x) {
    const int a = t / n, r = t - (t / n) * n;
    out[t] = (double)C[a * ldc + c0 + r];
  }
}

size_t tc_smem(int d) {
  const size_t need = (size_t)(kTcBM + kTcBN) * d * 2 + kTcBN * 4;
  // at least 100 KB so that no more than two CTAs (2 x 256 TMEM columns)
  // share an SM
  return need < 102400 ? 102400 : need;
}

}  // namespace

cudaError_t tc_prep_centroids(const double* loc64, const long long* off, long long K, long long Tc,
                              int d, void* yb, float* yn, double* ydel, float* cn, float* cd,
                              cudaStream_t st) {
  if (!tc_dim_ok(d)) return cudaErrorInvalidValue;
  const long long ncols = tc_cols(Tc);
  const unsigned b1 = (unsigned)std::min<long long>((ncols + 255) / 256, 4096);
  k_tc_prep_rows<<<b1, 256, 0, st>>>(loc64, Tc, ncols, d, static_cast<__nv_bfloat16*>(yb), yn,
                                     ydel);
  const unsigned b2 = (unsigned)std::min<long long>((K + 255) / 256, 4096);
  k_tc_prep_cent<<<b2, 256, 0, st>>>(off, K, yn, ydel, cn, cd);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t tc_chunk(const ObjView& ob, const TcWork& w, const int* oidx, long long obase,
                     long long cnt, int mmax, int ct0, int nct, int* d_err, cudaStream_t st) {
  if (w.probe_polls < 0) return cudaErrorInvalidValue;
  if (cnt <= 0) return cudaSuccess;
  if (ob.ldt != 2 || !tc_dim_ok(ob.d) || mmax < 1 || mmax > 64) return cudaErrorInvalidValue;
  const int d = ob.d;
  const __nv_bfloat16* X = static_cast<const __nv_bfloat16*>(ob.loc);
  k_tc_scan<<<1, 1024, 0, st>>>(ob.off, oidx, obase, cnt, mmax, w.trow);
  const unsigned gb = (unsigned)std::min<long long>((cnt * 32 + 255) / 256, 8192);
  k_tc_gather<<<gb, 256, 0, st>>>(ob.off, X, oidx, obase, cnt, d, w.trow, w.rowsrc, w.nx);
  const long long ncols = w.cents.ncols;
  const int ctiles = (int)(ncols / kTcBN);
  if (nct < 0) nct = ctiles - ct0;
  if (ct0 < 0 || nct < 1 || ct0 + nct > ctiles) return cudaErrorInvalidValue;
  const long long row_tiles = (cnt * mmax + kTcBM - 1) / kTcBM;
  const long long gy = (row_tiles + kTcRowTiles - 1) / kTcRowTiles;
  if (gy > 65535) return cudaErrorInvalidValue;
  const size_t smem = tc_smem(d);
  cudaError_t e =
      cudaFuncSetAttribute(k_cost_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)nct, (unsigned)gy);
  k_cost_tc<<<grid, kTcThreads, smem, st>>>(X, w.rowsrc, w.nx, w.trow + cnt,
                                            static_cast<const __nv_bfloat16*>(w.cents.yb),
                                            w.cents.yn, d, ncols, ct0, w.C, d_err, w.probe_polls);
  note_launches(3);
  return cudaGetLastError();
}

cudaError_t tc_extract(const float* C, long long ldc, int m, long long c0, int n, double* out,
                       cudaStream_t st) {
  k_tc_extract<<<1, 256, 0, st>>>(C, ldc, m, c0, n, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace d2k
