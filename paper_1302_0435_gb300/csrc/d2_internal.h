// d2_internal.h -- host-side launchers shared by the C-ABI implementation.
// Device views are plain structs of pointers (all device memory).
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace d2k {

struct ObjView {
  const void* loc;       // [T][d] element type ldt
  const void* w;         // [T] element type wdt
  const long long* off;  // [count+1]
  long long count;
  int d;
  int ldt;  // 0 f64, 1 f32, 2 bf16
  int wdt;  // 0 f64, 1 f32
};

struct CentView {
  const float* loc32;    // [T][d] FP32 copy (exact for FP32/BF16 centroids)
  const double* loc64;   // [T][d] FP64 copy
  const long long* Qpre; // [T] inclusive prefix of quantised masses, per centroid
  const long long* off;  // [K+1]
  long long K;           // number of centroids in the set
  int d;
};

struct FlowOut {
  int* cell;
  double* w;
  long long stride;
};

// Saved optimal bases of every (object, centroid) pair of an assign call,
// pair t = i*K + j, node y at [t*ns + y]: parent / position / size bytes and
// int64 flow.  `warm`: the arrays hold bases saved by a previous call on the
// same pairs (same marginals), so solves start from them.
struct WarmStore {
  unsigned char* par8;
  unsigned char* pos8;
  unsigned char* sz8;
  long long* flow;
  int ns;
  int warm;
};

// Launch-wide solver settings.
struct SolveCfg {
  int mode;        // 0: FP64 throughout; 1: FP32 screen/pivots + FP64 certify
  int group;       // lanes per pair (1,2,4,8,16,32)
  int mmax, nmax;  // support bounds of the launch
  int budget;      // pivots per pair = budget*(m+n)
  int sms;         // SM count
  int tpb = 128;   // threads per block of the solver kernels (64 or 128)
  int ipsm = 96;   // screening work items per SM the centroid blocks aim for
  const int* oidx = nullptr;  // objects of this launch (nullptr: 0..count-1)
  long long nobj = -1;        // entries of oidx (-1: all ob.count objects)
};

// Error bits raised by kernels into a device int.
enum : int { kErrInvalid = 1, kErrNotConverged = 2 };

cudaError_t scan_bags(const long long* off, long long count, int* d_info, cudaStream_t st);
cudaError_t prep_centroids(const void* loc, int ldt, const void* w, int wdt, const long long* off,
                           long long K, int d, float* loc32, double* loc64, long long* Qpre,
                           double* w64, int* d_err, cudaStream_t st);
cudaError_t mallows_pairs(const ObjView& ob, const CentView& cv, const long long* pobj,
                          const long long* pcen, long long npairs, const SolveCfg& cfg,
                          double* dist2, FlowOut fo, int* status, int* d_err, cudaStream_t st);
// cand: int scratch of assign_scratch_ints(count, K) for the FP32 screen's
// candidate lists (required when cfg.mode == 1; nullptr solves every
// centroid exactly).
// ws (may be null): saved bases, see WarmStore.
cudaError_t assign(const ObjView& ob, const CentView& cv, long long seg_size, int K,
                   const SolveCfg& cfg, const double* omega, int* labels, double* dist2,
                   double* eps_terms, FlowOut fo, int* cand, int* d_err, cudaStream_t st,
                   const WarmStore* ws = nullptr);
// ints of assign scratch for `count` objects and K centroids per object:
// queue counter, merged lists [count*9], and per-(object, centroid block)
// items; a launch over nobj <= count objects makes at most
// nobj*ceil(want/nobj) <= want + count items, want <= sms*256.
inline long long assign_scratch_ints(long long count, long long K, int sms = 160) {
  (void)K;
  return 4 + ((count * 9 + 3) & ~3LL) + (count + (long long)sms * 256) * 18 + 4;
}
cudaError_t cost_matrix(const ObjView& ob, const CentView& cv, long long i, long long j, int mode,
                        double* C, cudaStream_t st);
cudaError_t sum_fixed_order(const double* v, long long n, double* out, cudaStream_t st);

// Location update (Eq. (WeightedUpdate)): objects grouped by label with a
// stable counting sort, then one block per centroid sums its members in
// object-index order.  labels index the centroid set `cv` (seg_size/K map
// an object's local label to a global centroid: g = (i/seg_size)*K + label).
struct UpdateScratch {
  int* chunk_counts;   // [nchunks * KT]
  long long* start;    // [KT+1]
  int* order;          // [N]
  int* seg_label;      // [N] global centroid per object
};
size_t update_scratch_bytes(long long N, long long KT);
cudaError_t update_locations(const ObjView& ob, const double* omega, const int* labels,
                             long long seg_size, int K, const FlowOut& fo, long long KT,
                             const long long* coff, int d, int cent_ldt, float* loc32,
                             double* loc64, void* scratch, cudaStream_t st);

// After update_locations (or update_locations with fo.cell == nullptr, which
// only sorts): per centroid sum of omega over its members, object order.
cudaError_t group_weight_sum(const double* omega, long long N, long long KT, void* scratch,
                             double* out, cudaStream_t st);

// Bin of each object by the lanes' node count its tree needs with centroid
// supports up to nmax: bin b holds m + nmax <= 32*(b+1); -1 if m is out of
// range.  labels_out: [count] ints.
cudaError_t bin_objects(const ObjView& ob, int nmax, int* bins_out, cudaStream_t st);

int device_sms(int dev);

// kernel launches issued by this library (all contexts)
void note_launches(long long k);
long long launches();
// pairs screened, their pivots, pairs solved exactly, their pivots
cudaError_t solver_stats(long long out[4]);

}  // namespace d2k
