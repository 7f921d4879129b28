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
  // segment of each object (nullptr: object i is in segment i / seg_size)
  const int* segof = nullptr;
};

__host__ __device__ inline long long seg_of(const ObjView& ob, long long i, long long seg_size) {
  return ob.segof ? (long long)ob.segof[i] : i / seg_size;
}

struct CentView {
  const float* loc32;    // [T][d] FP32 copy (exact for FP32/BF16 centroids)
  const double* loc64;   // [T][d] FP64 copy
  const long long* Qpre; // [T] inclusive prefix of quantised masses, per centroid
  const long long* off;  // [K+1]
  long long K;           // number of centroids in the set
  int d;
  // symbol ground costs (A > 0): supports are symbol ids (d = 1) and the
  // cost of symbols (s, t) is tab[s*A + t] instead of the squared distance
  const float* tab32 = nullptr;
  const double* tab64 = nullptr;
  int A = 0;
};

struct FlowOut {
  int* cell;
  double* w;
  long long stride;
  // optional (mallows_pairs only): the FP64 potentials of the centroid
  // supports of each solved pair, pot[t*pstride + r], from the final basis
  // (c(a, r) - u_a - v_r >= 0 on every cell, = 0 on the basis)
  double* pot = nullptr;
  long long pstride = 0;
};

// Saved optimal bases of every (object, centroid) pair of an assign call,
// pair t = i*K + j, node y at [t*ns + y]: parent / position / size bytes and
// int64 flow (flow == nullptr: trees only, the flows recomputed from the
// marginals on reload).  `warm`: the arrays hold bases saved by a previous
// call on the same pairs (same marginals), so solves start from them.
struct WarmStore {
  unsigned char* par8;
  unsigned char* pos8;
  unsigned char* sz8;
  long long* flow;
  int ns;
  int warm;
};

// FP32 ground-cost tiles made ahead of the screen by the tensor-core
// contraction (d2_tc.cu) for the objects of one chunk: row R of C holds
// ||x||^2 + ||y||^2 - 2 x.y of tile row R (an object support) against every
// centroid support column.  Launch object tt owns rows trow[tt] ..
// trow[tt+1]; the cost of its support a against centroid support row c0+r
// is C[(trow[tt]+a)*ldc + (c0 - col0) + r].  C == nullptr: the screen builds
// its tiles itself.
struct TileView {
  const float* C = nullptr;
  const long long* trow = nullptr;  // [nobj+1]
  const float* nx = nullptr;        // [rows] ||x||^2 of each tile row (FP32)
  const float* cn = nullptr;        // [K] max ||y^||^2 over each centroid's BF16 supports
  const float* cd = nullptr;        // [K] max ||y - y^|| over each centroid's supports
  long long ldc = 0;
  long long col0 = 0;
};

// Resident centroids rounded to BF16 for the contraction, with the data of
// its error bound (see TileView).
struct TcCents {
  const void* yb = nullptr;  // [ncols][d] BF16 (rows >= Tc are zero)
  const float* yn = nullptr;  // [ncols] ||y^||^2 in FP32
  const float* cn = nullptr;  // [K]
  const float* cd = nullptr;  // [K]
  long long ncols = 0;        // centroid support rows rounded up to the tile width
};

// Per-call buffers of the tensor-core screen: the tile buffer and the row
// maps of one chunk (a chunk of c objects of at most mmax supports has
// c*mmax <= rows_cap; trow holds rows_cap+1 entries).
struct TcWork {
  TcCents cents;
  float* C = nullptr;
  long long* trow = nullptr;    // [rows_cap+1]
  long long* rowsrc = nullptr;  // [rows_cap]
  float* nx = nullptr;          // [rows_cap]
  long long rows_cap = 0;       // tile rows the buffers hold (C: rows_cap*ncols floats)
  // diagnostic: > 0 makes the contraction's first completion wait poll a
  // barrier nothing arrives on, at most this many times (timeout path tests)
  long long probe_polls = 0;
};

// Launch-wide solver settings.
struct SolveCfg {
  int mode;        // 0: FP64 throughout; 1: FP32 screen/pivots + FP64 certify
  int group;       // lanes per pair (32: one warp)
  int mmax, nmax;  // support bounds of the launch
  int budget;      // pivots per pair = budget*(m+n)
  int sms;         // SM count
  int tpb = 128;   // threads per block of the solver kernels (64 or 128)
  int ipsm = 96;   // screening work items per SM the centroid blocks aim for
  const int* oidx = nullptr;  // objects of this launch (nullptr: obase..obase+nobj-1)
  long long nobj = -1;        // entries of oidx (-1: all ob.count objects)
  long long obase = 0;        // first object when oidx is nullptr
  // device-side object range (bins whose counts stay on the device): the
  // launch takes oidx[dev_range[0] .. dev_range[1]); overrides nobj
  const long long* dev_range = nullptr;
  int start = 0;              // cold start basis: 0 ranked northwest staircase, 1 Vogel
  // per-pair screen output (optional): pair_out[2*(i*K + j)] = FP32 value,
  // [..+1] = its error bound (+inf when the screen could not bound it, NaN
  // for an invalid bag); screen_only: no FP64 certification launch
  float* pair_out = nullptr;
  bool screen_only = false;
  // certify every screened pair in FP64 (see certify_fp64 in d2_solve.cuh):
  // a pair whose FP32-optimal basis passes the FP64 reduced-cost check keeps
  // its FP64 objective; one that fails is sent to the exact pass with its
  // object's candidates.  pair64 (optional, certify only): [count][K] FP64
  // D^2 of every pair, pair64[i*K + j] (j local to the object's segment).
  bool certify = false;
  double* pair64 = nullptr;
  // pairs that cannot be the argmin are skipped (see prune_keep): bit j of
  // keep[i*keep_words + j/32] set = centroid j (local to the object's
  // segment) kept for object i.  Null: every pair is solved.  Only for
  // screens that pick argmin candidates (not certify, not pair_out).
  const unsigned* keep = nullptr;
  int keep_words = 0;
  TileView tile;              // precomputed FP32 tiles of the screen (optional)
  // mallows_pairs with mode 1: room (pair_tree_bytes) for the FP32 bases
  // handed from the FP32 launch to the FP64 launch; null: one fused launch
  unsigned char* tree = nullptr;
  size_t tree_bytes = 0;
  // joint-weights rounds (mallows_pairs with the hand-over above): the
  // optimal basis of each object's pair from the previous round, indexed by
  // OBJECT (node y of object i at [i*jw.ns + y]; sz8 of node 0 == 0: none
  // saved).  Only the centroid weights change between rounds, so that basis
  // stays dual feasible: the FP32 launch restarts from it (flows recomputed
  // for the new weights, dual pivots until they are feasible, then primal
  // pivots), and the FP64 launch saves its final basis there.
  WarmStore jw{};
};

// Bases of npairs pairs of up to mmax + nmax nodes (par/pos/size bytes and
// int64 flows per node) plus a status int per pair.
inline size_t pair_tree_bytes(long long npairs, int mmax, int nmax) {
  const size_t nodes = (size_t)npairs * (size_t)(mmax + nmax);
  return (nodes * 3 + 15) / 16 * 16 + nodes * 8 + (size_t)npairs * 4;
}

// Error bits raised by kernels into a device int.
enum : int { kErrInvalid = 1, kErrNotConverged = 2, kErrTimeout = 4 };

cudaError_t scan_bags(const long long* off, long long count, int* d_info, cudaStream_t st);
// Raise kErrInvalid into d_err unless off[0] = 0 and every bag has 1..maxm
// supports (no host wait: callers that declare their largest bag).
cudaError_t check_bags(const long long* off, long long count, int maxm, int* d_err,
                       cudaStream_t st);
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
                   const WarmStore* ws = nullptr, const TcWork* tw = nullptr);

// ---- solver launches, one translation unit per nodes-per-lane shape ----
#define D2_NPL_DECL(N)                                                                         \
  cudaError_t assign_npl##N(const ObjView& ob, const CentView& cv, long long seg_size, int K,  \
                            const SolveCfg& cfg, const double* omega, int* labels,           \
                            double* dist2, double* eps_terms, FlowOut fo, int* cand,           \
                            int* d_err, cudaStream_t st, const WarmStore* ws,                 \
                            const TcWork* tw);                                                 \
  cudaError_t mallows_pairs_npl##N(const ObjView& ob, const CentView& cv,                     \
                                   const long long* pobj, const long long* pcen,              \
                                   long long npairs, const SolveCfg& cfg, double* dist2,       \
                                   FlowOut fo, int* status, int* d_err, cudaStream_t st);     \
  cudaError_t stats_npl##N(long long out[6]);
D2_NPL_DECL(1)
D2_NPL_DECL(2)
D2_NPL_DECL(3)
D2_NPL_DECL(4)
#undef D2_NPL_DECL

// ---- pairs that cannot be the argmin (Alg. 2 Step 2 needs only it) ----
// Under a pair's own marginals (the quantised masses the solver uses), for
// every transport plan: D^2(P, Q) >= ||mu_P - mu_Q||^2 (Jensen, the plan's
// masses summing to one), and the product plan p_a q_r costs
// ||mu_P - mu_Q||^2 + var_P + var_Q (var: the mass-weighted squared spread
// about the mean), an upper bound of D^2.  So centroid j cannot be object
// i's argmin when ||mu_i - mu_j||^2 > UB_i = var_i + min_j' (||mu_i -
// mu_j'||^2 + var_j').  All in FP64, compared with 2^-40 relative margins.
// Means [count][d] and spreads [count] of a batch (FP64; NaN for a bag the
// solver rejects, which keeps all its pairs).
cudaError_t bag_moments(const ObjView& ob, double* mu, double* var, cudaStream_t st);
// The same for the centroids of a set (masses from Qpre, locations loc64).
cudaError_t cent_moments(const CentView& cv, double* mu, double* var, cudaStream_t st);
// Keep bits of every object: kw = ceil(K / 32) words per object.
cudaError_t prune_keep(const ObjView& ob, long long seg_size, int K, long long KT, int d,
                       const double* mu_o, const double* var_o, const double* mu_c,
                       const double* var_c, unsigned* keep, int kw, cudaStream_t st);

// Raise kErrInvalid into d_err unless every location of the T supports is
// an integer symbol id in [0, A) (d = 1).
// The same for the supports of a bag batch (their count read on the device).
cudaError_t check_bag_symbols(const void* loc, int ldt, const long long* off, long long count,
                              int A, int* d_err, cudaStream_t st);
cudaError_t check_symbols(const void* loc, int ldt, long long T, int A, int* d_err,
                          cudaStream_t st);

// ---- combined distance of several bag types (d2_multi.cu) ----
constexpr int kMaxBagTypes = 8;
struct MultiScreen {  // per type: the screen's pair values and bounds [N*K*2]
  const float* pair[kMaxBagTypes];
  int B;
};
struct MultiExact {  // per type: exact D^2 of the listed pairs
  const double* d2[kMaxBagTypes];
  int B;
};
// Candidate counts per object (cnt [N]) and their offsets (start [N+1]).
cudaError_t multi_candidates(const MultiScreen& ms, long long N, int K, long long* cnt,
                             long long* start, int* d_err, cudaStream_t st);
// The listed pairs (object, centroid), objects in order, centroids increasing.
cudaError_t multi_fill(const MultiScreen& ms, long long N, int K, const long long* start,
                       long long* pobj, long long* pcen, cudaStream_t st);
// Label and summed D^2 of every object from its listed pairs' exact values.
cudaError_t multi_argmin(long long N, const long long* start, const long long* pcen,
                         const MultiExact& mx, int* labels, double* dist2, cudaStream_t st);

// ---- initial data segmentation helpers (d2_segment.cu) ----
// Gather bags members[0..cnt) of v into a compact view: off_out [cnt+1],
// loc_out / w_out in v's element types (room for all their rows), om_out
// [cnt] (1 where om_in is nullptr).
cudaError_t seg_gather(const ObjView& v, const int* members, long long cnt, const double* om_in,
                       long long* off_out, void* loc_out, void* w_out, double* om_out,
                       cudaStream_t st);
// K (1 or 2) start centroids from bags i0 (, i1) of v: FP64 locations,
// uniform FP64 weights, offsets [K+1].
cudaError_t seg_cents(const ObjView& v, int i0, int i1, int K, double* cloc, double* cw,
                      long long* coff, cudaStream_t st);

// ---- tensor-core ground cost (d2_tc.cu) ----
// Whether the contraction supports dimension d (a multiple of 16 in 16..256).
inline bool tc_dim_ok(int d) { return d >= 16 && d <= 256 && d % 16 == 0; }
inline long long tc_cols(long long Tc) { return (Tc + 255) / 256 * 256; }
// BF16 copies, FP32 squared norms and rounding bounds of the resident
// centroids (loc64: [Tc][d]); yb [ncols][d], yn [ncols], ydel [ncols] FP64
// scratch, cn/cd [K].
cudaError_t tc_prep_centroids(const double* loc64, const long long* off, long long K, long long Tc,
                              int d, void* yb, float* yn, double* ydel, float* cn, float* cd,
                              cudaStream_t st);
// Tiles of one chunk: objects oidx[0..cnt) (or obase..obase+cnt-1) with
// supports of at most mmax rows (others get no rows); fills w.trow,
// w.rowsrc, w.nx and C rows [0, trow[cnt]) x columns of col tiles
// [ct0, ct0+nct) (nct = -1: all).  Objects' loc must be BF16.
cudaError_t tc_chunk(const ObjView& ob, const TcWork& w, const int* oidx, long long obase,
                     long long cnt, int mmax, int ct0, int nct, int* d_err, cudaStream_t st);
// Copy rows [0,m) x columns [c0, c0+n) of a chunk's tile to FP64.
cudaError_t tc_extract(const float* C, long long ldc, int m, long long c0, int n, double* out,
                       cudaStream_t st);
// ints of assign scratch for `count` objects and K centroids per object:
// queue counter, merged lists [count*9], and per-(object, centroid block)
// items; a launch over nobj <= count objects makes at most
// nobj*ceil(want/nobj) <= want + count items, want <= sms*256.
// The screen keeps up to kCandCap candidates per (object, centroid block)
// item and per object; more means the object is certified against all K.
// An item record also carries the FP64 value of its smallest upper end's
// centroid when that pair was certified (two ints of double bits, NaN
// otherwise); a merged record carries the object's.
constexpr int kCandCap = 16;
// count, centroids, lower ends, best upper end, certified FP64 value of that centroid
constexpr int kItemInts = 2 + 2 * kCandCap + 2;
constexpr int kMergedInts = 1 + kCandCap + 2;  // count, centroids, certified FP64 value
inline long long assign_scratch_ints(long long count, long long K, int sms = 160) {
  (void)K;
  return 4 + ((count * kMergedInts + 3) & ~3LL) + (count + (long long)sms * 256) * kItemInts + 4;
}
cudaError_t cost_matrix(const ObjView& ob, const CentView& cv, long long i, long long j, int mode,
                        double* C, cudaStream_t st);
cudaError_t sum_fixed_order(const double* v, long long n, double* out, cudaStream_t st);

// Location update (Eq. (WeightedUpdate)): objects grouped by label with a
// stable counting sort, then one block per centroid sums its members in
// object-index order.  labels index the centroid set `cv` (seg_size/K map
// an object's local label to a global centroid: g = seg_of(i)*K + label).
struct UpdateScratch {
  int* chunk_counts;   // [nchunks * KT]
  long long* start;    // [KT+1]
  int* order;          // [N]
  int* seg_label;      // [N] global centroid per object
};
size_t update_scratch_bytes(long long N, long long KT);
// Blocks per centroid of the accumulation: about 512 members each, at most 64.
inline long long update_parts(long long N, long long KT) {
  const long long u = (N + KT * 512 - 1) / (KT * 512);
  return u < 1 ? 1 : (u > 64 ? 64 : u);
}
// Room for the per-part sums (0: one block per centroid suffices).
size_t update_part_bytes(long long N, long long KT, int d);
// part / part_bytes (optional): room for the per-part sums of large
// clusters (update_part_bytes); without it one block sums each centroid.
cudaError_t update_locations(const ObjView& ob, const double* omega, const int* labels,
                             long long seg_size, int K, const FlowOut& fo, long long KT,
                             const long long* coff, int d, int cent_ldt, float* loc32,
                             double* loc64, void* scratch, cudaStream_t st,
                             double* part = nullptr, size_t part_bytes = 0);

// After update_locations with fo.cell == nullptr (the sort only): the
// members of group g are order[start[g] .. start[g+1]), increasing index.
void sorted_groups(void* scratch, long long N, long long KT, const long long** start,
                   const int** order);



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
// pairs screened, their pivots, pairs solved exactly, their pivots,
// screened pairs certified in FP64, cells the certificate checked in FP64
cudaError_t solver_stats(long long out[6]);

}  // namespace d2k
