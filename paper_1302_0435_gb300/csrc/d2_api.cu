// d2_api.cu -- implementation of the C-ABI declared in include/d2.h:
// context, host/device pointer staging, and the five calls of the
// assignment step (cost matrix, Mallows batch, assign, location update,
// hierarchical level driver).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "d2.h"
#include "d2_internal.h"
#include "d2_segment.h"
#include "d2_joint.h"
#include "d2_trace.h"

using d2k::CentView;
using d2k::FlowOut;
using d2k::ObjView;
using d2k::SolveCfg;

namespace {

enum Slot {
  kObjOff, kObjLoc, kObjW, kOmega, kPairObj, kPairCen, kOutD2, kOutLab, kOutStatus, kFlowCell,
  kFlowW, kEpsTerms, kEpsOut, kUpd, kLabelsIn, kCentIn0, kCentIn1, kCentIn2,
  // level driver
  kLvDataLoc, kLvDataW, kLvDataOff, kLvOmega, kLvOmegaNew, kLvC, kLvCT, kLvLab, kLvD2,
  kLvCLoc32, kLvCLoc64, kLvCQ, kLvCW, kLvCOff, kLvTmp, kCand, kWarmMeta, kWarmFlow, kBins,
  kBinSort, kTuneLab, kTuneD2, kTcTile, kTcRow, kTcSrc, kTcNx, kTcDel,
  // initial data segmentation
  kSgMem, kSgOff, kSgLoc, kSgW, kSgOm, kSgCLoc, kSgCW, kSgCOff, kSgC32, kSgC64, kSgCQ, kSgCW64,
  kSgLab, kSgD2, kSgCell, kSgFw, kSgUpd, kSgCand, kSgOut, kLvSegof, kSgPart, kUpdPart, kLvPart,
  kSgSid, kSgIdx, kSgAct, kSgULab,
  kLvTerms, kLvEps,
  // combined distance of several bag types
  kMbPair, kMbTmpLab, kMbTmpD2, kMbCnt, kMbStart, kMbPObj, kMbPCen, kMbD2, kMbSt,
  // joint weights (Alg. 1 Step 1)
  kJState, kJPot, kJPStart, kJEps, kJIters, kJSort, kJPObj, kJPCen, kJW, kJSt, kJTree,
  kPairTree, kPairTree2,
  // d2_mallows_all
  kAllLab, kAllD2, kAllPair,
  // pruning of pairs that cannot be the argmin
  kPrMuO, kPrVarO, kPrMuC, kPrVarC, kPrKeep,
  kSlots
};

struct Buf {
  void* p = nullptr;
  size_t n = 0;
};

}  // namespace

struct d2_ctx {
  int device = 0;
  int sms = 1;
  cudaStream_t own = nullptr;
  cudaStream_t stream = nullptr;
  d2_config cfg{};
  // resident centroids
  long long K = 0, Tc = 0;
  int d = 0, nmax = 0, cent_ldt = D2_F32;
  float* c_loc32 = nullptr;
  double* c_loc64 = nullptr;
  long long* c_Q = nullptr;
  double* c_w64 = nullptr;
  long long* c_off = nullptr;
  std::vector<long long> h_coff;
  // BF16 copy of the resident centroids for the tensor-core contraction
  // (dimension a multiple of 16 in 16..256), rebuilt when the set changes
  void* c_yb = nullptr;
  float* c_yn = nullptr;
  float* c_cn = nullptr;
  float* c_cd = nullptr;
  bool tc_stale = true;
  // symbol ground-cost table (A > 0): FP64 and FP32 copies of [A][A]
  double* tab64 = nullptr;
  float* tab32 = nullptr;
  int A = 0;
  // scratch
  Buf slot[kSlots];
  int* d_err = nullptr;
  int* d_info = nullptr;
  int* h_pin = nullptr;  // pinned host ints
  // autotuned launch per (nodes-per-lane bin, K, m bound, n bound, d, mode):
  // threads per block, screening items per SM, cold-start rule
  std::map<std::tuple<int, long long, int, int, int, int>, std::tuple<int, int, int>> tuned;
  int tuning_runs = 0;
};

namespace {

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      return e_ == cudaErrorMemoryAllocation ? D2_ENOMEM : D2_ECUDA; \
    }                                           \
  } while (0)

void* grow(d2_ctx* c, int s, size_t bytes, int* rc) {
  Buf& b = c->slot[s];
  if (bytes == 0) bytes = 16;
  if (b.n >= bytes) return b.p;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.n = 0;
  size_t want = bytes + bytes / 4;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    *rc = D2_ENOMEM;
    return nullptr;
  }
  b.n = want;
  return b.p;
}

// As grow, without the slack (for buffers sized to a memory budget).
void* grow_exact(d2_ctx* c, int s, size_t bytes, int* rc) {
  Buf& b = c->slot[s];
  if (bytes == 0) bytes = 16;
  if (b.n >= bytes) return b.p;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.n = 0;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *rc = D2_ENOMEM;
    return nullptr;
  }
  b.n = bytes;
  return b.p;
}

// 1 = device-accessible allocation, 0 = host memory, -1 = null
int where(const void* p) {
  if (!p) return -1;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
}

size_t esize(int dt) { return dt == D2_F64 ? 8 : (dt == D2_F32 ? 4 : 2); }

bool bags_ok(const d2_bags* b) {
  if (!b || !b->loc || !b->w || !b->off || b->count < 0 || b->dim < 1 || b->dim > D2_MAX_DIM)
    return false;
  if (b->loc_dtype < D2_F64 || b->loc_dtype > D2_BF16) return false;
  if (b->w_dtype != D2_F64 && b->w_dtype != D2_F32) return false;
  const int w0 = where(b->off), w1 = where(b->loc), w2 = where(b->w);
  return w0 == w1 && w1 == w2;
}

// Stage a bag batch on the device.  Host batches are copied into slots.
int stage_bags(d2_ctx* c, const d2_bags* b, int s_off, int s_loc, int s_w, ObjView* v) {
  v->count = b->count;
  v->d = b->dim;
  v->ldt = b->loc_dtype;
  v->wdt = b->w_dtype;
  if (where(b->off) == 1) {
    v->loc = b->loc;
    v->w = b->w;
    v->off = reinterpret_cast<const long long*>(b->off);
    return D2_OK;
  }
  const long long T = b->count > 0 ? b->off[b->count] : 0;
  if (b->off[0] != 0 || T < 0) return D2_EINVAL;
  int rc = D2_OK;
  void* doff = grow(c, s_off, (size_t)(b->count + 1) * 8, &rc);
  void* dloc = grow(c, s_loc, (size_t)T * b->dim * esize(b->loc_dtype), &rc);
  void* dw = grow(c, s_w, (size_t)T * esize(b->w_dtype), &rc);
  if (rc != D2_OK) return rc;
  CK(cudaMemcpyAsync(doff, b->off, (size_t)(b->count + 1) * 8, cudaMemcpyHostToDevice, c->stream));
  if (T > 0) {
    CK(cudaMemcpyAsync(dloc, b->loc, (size_t)T * b->dim * esize(b->loc_dtype),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(dw, b->w, (size_t)T * esize(b->w_dtype), cudaMemcpyHostToDevice, c->stream));
  }
  v->loc = dloc;
  v->w = dw;
  v->off = static_cast<const long long*>(doff);
  return D2_OK;
}

// Device copy of a caller array (host arrays are staged into slot s).
template <typename T>
int stage_in(d2_ctx* c, const T* p, size_t n, int s, const T** out) {
  if (!p) { *out = nullptr; return D2_OK; }
  if (where(p) == 1) { *out = p; return D2_OK; }
  int rc = D2_OK;
  void* d = grow(c, s, n * sizeof(T), &rc);
  if (rc != D2_OK) return rc;
  if (n) CK(cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  *out = static_cast<const T*>(d);
  return D2_OK;
}

// Device destination for a caller output (host outputs get a slot).
template <typename T>
int stage_out(d2_ctx* c, T* p, size_t n, int s, T** out, bool* host) {
  *host = false;
  if (!p) { *out = nullptr; return D2_OK; }
  if (where(p) == 1) { *out = p; return D2_OK; }
  int rc = D2_OK;
  void* d = grow(c, s, n * sizeof(T), &rc);
  if (rc != D2_OK) return rc;
  *out = static_cast<T*>(d);
  *host = true;
  return D2_OK;
}

// Largest bag of a batch: declared by the caller (d2_bags.max_support,
// checked on the device with the other bag errors, no wait), else read back
// from a scan of the offsets (a wait).
int scan(d2_ctx* c, const ObjView& v, int* mmax);
int bag_bound(d2_ctx* c, const d2_bags* b, const ObjView& v, int* mmax) {
  if (b->max_support > 0) {
    if (b->max_support > D2_MAX_SUPPORT) return D2_EUNSUPPORTED;
    *mmax = b->max_support;
    CK(d2k::check_bags(v.off, v.count, *mmax, c->d_err, c->stream));
    return D2_OK;
  }
  return scan(c, v, mmax);
}

// max support and offset validity of a bag batch (device offsets)
int scan(d2_ctx* c, const ObjView& v, int* mmax) {
  CK(d2k::scan_bags(v.off, v.count, c->d_info, c->stream));
  CK(cudaMemcpyAsync(c->h_pin, c->d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->h_pin[1]) return D2_EINVAL;
  *mmax = c->h_pin[0];
  if (v.count > 0 && (*mmax < 1 || *mmax > D2_MAX_SUPPORT)) return D2_EUNSUPPORTED;
  return D2_OK;
}

int mode_for(const d2_ctx* c, int obj_ldt) {
  if (c->cfg.precision == D2_PREC_FP64) return 0;
  if (obj_ldt == D2_F64 || c->cent_ldt == D2_F64) return 0;
  return 1;
}

// Cold-start rule when nothing was timed: Vogel's approximation pays for
// its bookkeeping on wide centroids (64 supports), the ranked staircase
// elsewhere.
int start_default(const d2_ctx* c) {
  if (c->cfg.start_rule == D2_START_VOGEL) return 1;
  if (c->cfg.start_rule == D2_START_RANKED) return 0;
  return c->nmax >= 64 ? 1 : 0;
}

SolveCfg solve_cfg(const d2_ctx* c, int mode, int mmax) {
  SolveCfg s;
  s.mode = mode;
  s.group = 32;  // one warp per pair
  s.mmax = std::max(mmax, 1);
  s.nmax = std::max(c->nmax, 1);
  s.budget = c->cfg.pivot_budget > 0 ? c->cfg.pivot_budget : 64;
  s.sms = c->sms;
  s.start = start_default(c);
  s.certify = mode == 1 && c->cfg.certify == D2_CERTIFY_ALL;
  return s;
}

// Room for the FP32 bases of a two-launch exact solve (SolveCfg::tree);
// past 2 GiB the solve stays one fused launch.
int attach_tree(d2_ctx* c, SolveCfg* cfg, long long npairs, int slot = kPairTree) {
  if (cfg->mode != 1 || npairs <= 0) return D2_OK;
  const size_t b = d2k::pair_tree_bytes(npairs, cfg->mmax, cfg->nmax);
  if (b > ((size_t)2 << 30)) return D2_OK;
  int rc = D2_OK;
  void* p = grow(c, slot, b, &rc);
  if (rc != D2_OK) return rc;
  cfg->tree = static_cast<unsigned char*>(p);
  cfg->tree_bytes = b;
  return D2_OK;
}

CentView resident_view(const d2_ctx* c) {
  CentView v;
  v.loc32 = c->c_loc32;
  v.loc64 = c->c_loc64;
  v.Qpre = c->c_Q;
  v.off = c->c_off;
  v.K = c->K;
  v.d = c->d;
  v.tab32 = c->tab32;
  v.tab64 = c->tab64;
  v.A = c->A;
  return v;
}

// With a symbol table set: the bags must be one-dimensional symbol ids in
// [0, A); raises kErrInvalid otherwise (reported with the call's errors).
int check_bag_symbols(d2_ctx* c, const ObjView& v) {
  if (c->A <= 0) return D2_OK;
  if (v.d != 1) return D2_EINVAL;
  CK(d2k::check_bag_symbols(v.loc, v.ldt, v.off, v.count, c->A, c->d_err, c->stream));
  return D2_OK;
}

// Read and clear the context's error word (waits for the stream).
int read_err(d2_ctx* c, int* bits) {
  CK(cudaMemcpyAsync(c->h_pin + 2, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *bits = c->h_pin[2];
  return D2_OK;
}

int bits_code(int bits) {
  if (bits & d2k::kErrTimeout) return D2_ETIMEOUT;
  if (bits & d2k::kErrInvalid) return D2_EINVAL;
  if (bits & d2k::kErrNotConverged) return D2_ENOTCONVERGED;
  return D2_OK;
}

// Wait for the stream and report (and clear) the errors its kernels raised,
// those of earlier calls that returned without waiting included.
int take_errors(d2_ctx* c) {
  int bits = 0;
  const int rc = read_err(c, &bits);
  return rc != D2_OK ? rc : bits_code(bits);
}

// The end of a call that may return without waiting: with a host output it
// waits and reports the stream's errors; otherwise they wait for d2_sync.
int finish(d2_ctx* c, bool host_output) { return host_output ? take_errors(c) : D2_OK; }

void free_centroids(d2_ctx* c) {
  cudaFree(c->c_loc32); cudaFree(c->c_loc64); cudaFree(c->c_Q); cudaFree(c->c_w64); cudaFree(c->c_off);
  c->c_loc32 = nullptr; c->c_loc64 = nullptr; c->c_Q = nullptr; c->c_w64 = nullptr; c->c_off = nullptr;
  cudaFree(c->c_yb); cudaFree(c->c_yn); cudaFree(c->c_cn); cudaFree(c->c_cd);
  c->c_yb = nullptr; c->c_yn = nullptr; c->c_cn = nullptr; c->c_cd = nullptr;
  c->tc_stale = true;
  c->K = c->Tc = 0;
  c->h_coff.clear();
}

__global__ void k_pairs_from_labels(const int* labels, long long N, long long* pobj, long long* pcen) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    pobj[i] = i;
    pcen[i] = labels[i];
  }
}

// pairs (i, global centroid of i) of a level: g = seg(i) * K + labels[i]
__global__ void k_pairs_global(const int* labels, long long N, long long seg_size, const int* segof,
                               int K, long long* pobj, long long* pcen) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    pobj[i] = i;
    pcen[i] = (segof ? (long long)segof[i] : i / seg_size) * K + labels[i];
  }
}

// replicate the resident set M times (level centroid sets)
__global__ void k_replicate(const float* l32, const double* l64, const long long* Q, const double* w,
                            const long long* off, long long K, long long Tc, int d, long long M,
                            float* o32, double* o64, long long* oQ, double* ow, long long* ooff) {
  const long long tot = M * Tc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long src = t % Tc;
    oQ[t] = Q[src];
    ow[t] = w[src];
    for (int k = 0; k < d; ++k) {
      o32[t * d + k] = l32[src * d + k];
      o64[t * d + k] = l64[src * d + k];
    }
  }
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j <= M * K;
       j += (long long)gridDim.x * blockDim.x) {
    const long long mu = j / K, jj = j % K;
    ooff[j] = (j == M * K) ? M * Tc : mu * Tc + off[jj];
  }
}

// C~ = label + segment*K (Eq. (UpdateLabel)); C = C~[C] (Eq. (UpdateGlobalLabel))
__global__ void k_merge_labels(const int* lab, long long n_l, long long seg, const int* segof,
                               int K, int* ct) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_l;
       i += (long long)gridDim.x * blockDim.x)
    ct[i] = lab[i] < 0 ? -1 : (int)((segof ? (long long)segof[i] : i / seg) * K + lab[i]);
}
__global__ void k_compose(int* C, long long N, const int* ct) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    C[i] = C[i] < 0 ? -1 : ct[C[i]];
}

// Device memory the level driver may use for saved bases (warm starts):
// d2_config.warm_budget_mib, else 40 % of what is free when the level starts.
size_t warm_budget_bytes(const d2_ctx* c) {
  if (c->cfg.warm_budget_mib > 0) return (size_t)c->cfg.warm_budget_mib << 20;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return fr / 5 * 2;
}

unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)std::max<long long>(1, std::min<long long>(b, 8192));
}

}  // namespace

namespace {

// Object bins by the nodes per lane their trees need (see d2k::bin_objects),
// as a stable partition: order[start[b] .. start[b+1]) are bin b's objects
// in increasing index.  start stays on the device (the solver launches read
// their bin's range there); the host copy hstart is read only when needed
// (autotuning, tensor-core chunks), which waits.
struct Bins {
  int* order = nullptr;
  const long long* start = nullptr;
  long long hstart[5] = {0, 0, 0, 0, 0};
  bool binned = false;
  bool host = false;
};

int make_bins(d2_ctx* c, const ObjView& v, int nmax, Bins* b) {
  int rc = D2_OK;
  const long long N = v.count;
  int* bins = static_cast<int*>(grow(c, kBins, (size_t)N * 4, &rc));
  void* scr = grow(c, kBinSort, d2k::update_scratch_bytes(N, 4), &rc);
  if (rc != D2_OK) return rc;
  CK(d2k::bin_objects(v, nmax, bins, c->stream));
  d2k::FlowOut none{nullptr, nullptr, 0};
  ObjView flat = v;  // the bin sort is one group of 4 labels, whatever the segments
  flat.segof = nullptr;
  CK(d2k::update_locations(flat, nullptr, bins, N, 4, none, 4, nullptr, v.d, 0, nullptr, nullptr, scr,
                           c->stream));
  const long long* start;
  const int* order;
  d2k::sorted_groups(scr, N, 4, &start, &order);
  b->start = start;
  b->order = const_cast<int*>(order);
  b->binned = true;
  b->host = false;
  return D2_OK;
}

int bins_to_host(d2_ctx* c, Bins* b) {
  if (b->host) return D2_OK;
  CK(cudaMemcpyAsync(b->hstart, b->start, 5 * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  b->host = true;
  return D2_OK;
}

// One assign over a batch, bin by bin (largest trees first), each bin with
// its autotuned launch shape.  ws may be null.
// Whether run_assign screens with pruning bits for these arguments.
bool prunes(const d2_ctx* c, const SolveCfg& base, const CentView& cv) {
  return base.mode == 1 && !base.certify && !base.pair64 && cv.A == 0 && !c->cfg.no_prune;
}

// The bags' means and spreads into the slots run_assign reads (the rounds
// of a level reuse them: the bags do not change).
int prune_moments(d2_ctx* c, const ObjView& v) {
  int rc = D2_OK;
  double* mu_o = static_cast<double*>(grow(c, kPrMuO, (size_t)v.count * v.d * 8, &rc));
  double* var_o = static_cast<double*>(grow(c, kPrVarO, (size_t)v.count * 8, &rc));
  if (rc != D2_OK) return rc;
  CK(d2k::bag_moments(v, mu_o, var_o, c->stream));
  return D2_OK;
}

int run_assign(d2_ctx* c, const ObjView& v, const CentView& cv, long long seg, int K, int mode,
               int mmax, const double* om, int* lab, double* d2o, double* terms, FlowOut fo,
               int* cand, const d2k::WarmStore* ws, Bins& bins,
               const d2k::TcWork* tw = nullptr, bool certify_all = false,
               double* pair64 = nullptr, bool obj_moments_ready = false) {
  const int nmax = std::max(c->nmax, 1);
  SolveCfg base = solve_cfg(c, mode, mmax);
  if (certify_all && mode == 1) base.certify = true;
  base.pair64 = pair64;
  if (prunes(c, base, cv)) {
    // pairs whose lower bound is above their object's upper bound cannot be
    // the argmin: bounds from the bags' means and spreads, keep bits per object
    int rc = D2_OK;
    const int kw = (K + 31) / 32;
    double* mu_o = static_cast<double*>(grow(c, kPrMuO, (size_t)v.count * v.d * 8, &rc));
    double* var_o = static_cast<double*>(grow(c, kPrVarO, (size_t)v.count * 8, &rc));
    double* mu_c = static_cast<double*>(grow(c, kPrMuC, (size_t)cv.K * cv.d * 8, &rc));
    double* var_c = static_cast<double*>(grow(c, kPrVarC, (size_t)cv.K * 8, &rc));
    unsigned* keep = static_cast<unsigned*>(grow(c, kPrKeep, (size_t)v.count * kw * 4, &rc));
    if (rc != D2_OK) return rc;
    // (a level computes its bags' moments once: prune_moments)
    if (!obj_moments_ready) CK(d2k::bag_moments(v, mu_o, var_o, c->stream));
    CK(d2k::cent_moments(cv, mu_c, var_c, c->stream));
    CK(d2k::prune_keep(v, seg, K, cv.K, v.d, mu_o, var_o, mu_c, var_c, keep, kw, c->stream));
    base.keep = keep;
    base.keep_words = kw;
  }
  if (!bins.binned) {
    CK(d2k::assign(v, cv, seg, K, base, om, lab, d2o, terms, fo, cand, c->d_err, c->stream, ws, tw));
    return D2_OK;
  }
  const bool tuning = c->cfg.group_lanes == 0 && mode == 1 && v.count >= 8192;
  const int lo_bin = (1 + nmax + 31) / 32 - 1;
  const int hi_bin = std::min(3, (mmax + nmax + 31) / 32 - 1);
  for (int b = hi_bin; b >= lo_bin; --b) {
    SolveCfg cfg = base;
    cfg.mmax = std::max(1, std::min(mmax, 32 * (b + 1) - nmax));
    const auto key = std::make_tuple(b, (long long)K, cfg.mmax, nmax, v.d,
                                     mode + (cfg.certify ? 2 : 0));
    auto it = c->tuned.find(key);
    // the host needs the bin's count for tensor-core chunks and to tune a
    // new launch shape (a wait); otherwise the launches read it on the device
    const bool host = tw != nullptr || (it == c->tuned.end() && tuning);
    long long cnt = -1;
    if (host) {
      int rc0 = bins_to_host(c, &bins);
      if (rc0 != D2_OK) return rc0;
      cnt = bins.hstart[b + 1] - bins.hstart[b];
      if (cnt <= 0) continue;
      cfg.oidx = bins.order + bins.hstart[b];
      cfg.nobj = cnt;
    } else {
      cfg.oidx = bins.order;
      cfg.dev_range = bins.start + b;
    }
    if (it == c->tuned.end() && tuning && cnt < 8192) {
      // too few objects to time: the default shape, kept for this key
      it = c->tuned.emplace(key, std::make_tuple(cfg.tpb, cfg.ipsm, cfg.start)).first;
    }
    if (it == c->tuned.end() && tuning) {
      // autotune on a sample of this bin: threads per block x screening items per SM
      SolveCfg t = cfg;
      t.pair64 = nullptr;
      // a sample of about 2^20 pairs, at least 256 objects: several waves of
      // warps, so the timing ranks throughput (a one-wave sample ranks the
      // per-pair latency and favoured Vogel's start where the staircase is
      // faster at scale)
      t.nobj = std::min<long long>(cnt, std::max<long long>(256, (1LL << 20) / std::max(K, 1)));
      int rc = D2_OK;
      int* tl = static_cast<int*>(grow(c, kTuneLab, (size_t)v.count * 4, &rc));
      double* td = static_cast<double*>(grow(c, kTuneD2, (size_t)v.count * 8, &rc));
      if (rc != D2_OK) return rc;
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      auto time_one = [&](const SolveCfg& tc, float* ms) -> int {
        CK(cudaEventRecord(e0, c->stream));
        CK(d2k::assign(v, cv, seg, K, tc, om, tl, td, nullptr, FlowOut{nullptr, nullptr, 0}, cand,
                       c->d_err, c->stream, nullptr, tw));
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        *ms = 0.f;
        cudaEventElapsedTime(ms, e0, e1);
        return D2_OK;
      };
      // cold-start rule first (default shape), unless the caller fixed it
      if (c->cfg.start_rule == D2_START_AUTO) {
        float best_s = 1e30f;
        for (int sr = 0; sr < 2; ++sr) {
          t.start = sr;
          float ms = 0.f;
          if ((rc = time_one(t, &ms))) return rc;
          if (ms < best_s) { best_s = ms; cfg.start = sr; }
        }
      }
      t.start = cfg.start;
      float best = 1e30f;
      std::tuple<int, int, int> pick(128, 96, cfg.start);
      const int tpbs[2] = {64, 128};
      const int ipsms[3] = {48, 96, 192};
      for (int tp : tpbs)
        for (int ip : ipsms) {
          t.tpb = tp;
          t.ipsm = ip;
          float ms = 0.f;
          if ((rc = time_one(t, &ms))) return rc;
          if (ms < best) { best = ms; pick = std::make_tuple(tp, ip, cfg.start); }
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      ++c->tuning_runs;
      it = c->tuned.emplace(key, pick).first;
    }
    if (it != c->tuned.end()) {
      cfg.tpb = std::get<0>(it->second);
      cfg.ipsm = std::get<1>(it->second);
      cfg.start = std::get<2>(it->second);
    }
    CK(d2k::assign(v, cv, seg, K, cfg, om, lab, d2o, terms, fo, cand, c->d_err, c->stream, ws, tw));
  }
  return D2_OK;
}

// The tensor-core copy of the resident centroids, built on first use after
// the set changed.
int tc_cents(d2_ctx* c, d2k::TcCents* out) {
  const long long ncols = d2k::tc_cols(c->Tc);
  if (c->tc_stale) {
    cudaFree(c->c_yb); cudaFree(c->c_yn); cudaFree(c->c_cn); cudaFree(c->c_cd);
    c->c_yb = nullptr; c->c_yn = nullptr; c->c_cn = nullptr; c->c_cd = nullptr;
    if (cudaMalloc(&c->c_yb, (size_t)ncols * c->d * 2) != cudaSuccess ||
        cudaMalloc(&c->c_yn, (size_t)ncols * 4) != cudaSuccess ||
        cudaMalloc(&c->c_cn, (size_t)c->K * 4) != cudaSuccess ||
        cudaMalloc(&c->c_cd, (size_t)c->K * 4) != cudaSuccess) {
      cudaGetLastError();
      return D2_ENOMEM;
    }
    int rc = D2_OK;
    double* del = static_cast<double*>(grow(c, kTcDel, (size_t)ncols * 8, &rc));
    if (rc != D2_OK) return rc;
    CK(d2k::tc_prep_centroids(c->c_loc64, c->c_off, c->K, c->Tc, c->d, c->c_yb, c->c_yn, del,
                              c->c_cn, c->c_cd, c->stream));
    c->tc_stale = false;
  }
  out->yb = c->c_yb;
  out->yn = c->c_yn;
  out->cn = c->c_cn;
  out->cd = c->c_cd;
  out->ncols = ncols;
  return D2_OK;
}

// Whether d2_assign screens with tensor-core tiles for these objects.
bool tc_wanted(const d2_ctx* c, const d2_bags* objs, const ObjView& v, int mode) {
  if (c->cfg.cost_tc == D2_TC_OFF || mode != 1) return false;
  if (objs->loc_dtype != D2_BF16 || !d2k::tc_dim_ok(c->d)) return false;
  if (c->cfg.cost_tc != D2_TC_ON && c->d < 64) return false;
  return (reinterpret_cast<uintptr_t>(v.loc) & 15) == 0;
}

// Tile buffers for `rows` tile rows at most (capped by the budget).
int tc_work(d2_ctx* c, long long rows, int mmax, d2k::TcWork* w) {
  int rc = tc_cents(c, &w->cents);
  if (rc != D2_OK) return rc;
  size_t budget = (size_t)c->cfg.tile_budget_mib << 20;
  if (c->cfg.tile_budget_mib <= 0) {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    budget = std::min<size_t>((size_t)32 << 30, fr / 5 * 2);
  }
  const size_t row_bytes = (size_t)w->cents.ncols * 4;
  long long cap = (long long)(budget / row_bytes);
  cap = std::min(cap, rows);
  if (cap < mmax) return D2_ENOMEM;  // not even one object of mmax rows fits
  w->C = static_cast<float*>(grow_exact(c, kTcTile, (size_t)cap * row_bytes, &rc));
  if (rc != D2_OK) return rc;
  w->trow = static_cast<long long*>(grow(c, kTcRow, (size_t)(cap + 1) * 8, &rc));
  w->rowsrc = static_cast<long long*>(grow(c, kTcSrc, (size_t)cap * 8, &rc));
  w->nx = static_cast<float*>(grow(c, kTcNx, (size_t)cap * 4, &rc));
  if (rc != D2_OK) return rc;
  w->rows_cap = cap;
  w->probe_polls = c->cfg.tc_wait_probe;
  return D2_OK;
}

// Initial data segmentation of Alg. 3 Step 1 on the device view v (see
// d2_segment in d2.h): largest-first binary splits, each a constrained
// D2-clustering with k = 2 (farthest-bag start, uniform centroid weights held
// fixed, at most `iters` update rounds, early stop when the labels repeat).
// Writes the segment of every object to segof (device, [v.count]); segments
// are numbered by their smallest member.
int segment_impl(d2_ctx* c, const ObjView& v, int mmax, const double* om, long long tau, int iters,
                 int* segof, long long* M_out) {
  // Every segment above tau splits in two; a split depends only on its own
  // members (in increasing object order), so all the splits of one
  // generation run together: one gathered view, one centroid set of two
  // per segment, one assignment and one update per round.  The result is
  // the partition of largest-first splitting, one split at a time.
  const long long N = v.count;
  int rc = D2_OK;
  const long long rows_cap = N * (long long)mmax;
  const long long stride = 2LL * mmax - 1;
  int* dmem = static_cast<int*>(grow(c, kSgMem, (size_t)N * 4, &rc));
  int* dsid = static_cast<int*>(grow(c, kSgSid, (size_t)N * 4, &rc));
  long long* soff = static_cast<long long*>(grow(c, kSgOff, (size_t)(N + 1) * 8, &rc));
  void* sloc = grow(c, kSgLoc, (size_t)rows_cap * v.d * esize(v.ldt), &rc);
  void* sw = grow(c, kSgW, (size_t)rows_cap * esize(v.wdt), &rc);
  double* som = static_cast<double*>(grow(c, kSgOm, (size_t)N * 8, &rc));
  int* lab = static_cast<int*>(grow(c, kSgLab, (size_t)N * 4, &rc));
  double* dd = static_cast<double*>(grow(c, kSgD2, (size_t)N * 8, &rc));
  int* fcell = static_cast<int*>(grow(c, kSgCell, (size_t)(N * stride) * 4, &rc));
  double* fw = static_cast<double*>(grow(c, kSgFw, (size_t)(N * stride) * 8, &rc));
  int* cand = static_cast<int*>(grow(c, kSgCand, (size_t)d2k::assign_scratch_ints(N, 2, c->sms) * 4, &rc));
  if (rc != D2_OK) return rc;
  SolveCfg cfg = solve_cfg(c, mode_for(c, v.ldt), mmax);
  cfg.nmax = mmax;  // the split centroids are bags of the data
  // the splits' centroids are FP64 (their FP32 copies are not exact), and
  // only their labels are used: no per-pair certificate
  cfg.certify = false;
  cfg.start = c->cfg.start_rule == D2_START_VOGEL ? 1
            : c->cfg.start_rule == D2_START_RANKED ? 0 : (mmax >= 64 ? 1 : 0);
  const FlowOut fo{fcell, fw, stride};
  std::vector<std::vector<int>> segs(1, std::vector<int>((size_t)N));
  for (long long i = 0; i < N; ++i) segs[0][(size_t)i] = (int)i;
  auto check = [&]() -> int {
    int bits = 0;
    int r = read_err(c, &bits);
    if (r != D2_OK) return r;
    if (bits & d2k::kErrTimeout) return D2_ETIMEOUT;
    if (bits & d2k::kErrInvalid) return D2_EINVAL;
    if (bits & d2k::kErrNotConverged) return D2_ENOTCONVERGED;
    return D2_OK;
  };
  std::vector<double> hd;
  std::vector<int> hl, hl2, list, sid, idx;
  for (;;) {
    std::vector<size_t> B;  // the segments split in this generation
    for (size_t k = 0; k < segs.size(); ++k)
      if ((long long)segs[k].size() > tau) B.push_back(k);
    if (B.empty()) break;
    if ((long long)(segs.size() + B.size()) > N) return D2_EINVAL;  // every split makes progress
    const long long nB = (long long)B.size();
    std::vector<long long> s0((size_t)nB + 1, 0);
    list.clear();
    sid.clear();
    for (long long b = 0; b < nB; ++b) {
      s0[(size_t)b] = (long long)list.size();
      const std::vector<int>& S = segs[B[(size_t)b]];
      list.insert(list.end(), S.begin(), S.end());
      sid.insert(sid.end(), S.size(), (int)b);
    }
    s0[(size_t)nB] = (long long)list.size();
    const long long cnt = (long long)list.size();
    // room for two centroids of at most mmax supports per segment
    const long long KT = 2 * nB;
    double* zloc = static_cast<double*>(grow(c, kSgCLoc, (size_t)KT * mmax * v.d * 8, &rc));
    double* zw = static_cast<double*>(grow(c, kSgCW, (size_t)KT * mmax * 8, &rc));
    long long* zoff = static_cast<long long*>(grow(c, kSgCOff, (size_t)(KT + 1) * 8, &rc));
    float* z32 = static_cast<float*>(grow(c, kSgC32, (size_t)KT * mmax * v.d * 4, &rc));
    double* z64 = static_cast<double*>(grow(c, kSgC64, (size_t)KT * mmax * v.d * 8, &rc));
    long long* zQ = static_cast<long long*>(grow(c, kSgCQ, (size_t)KT * mmax * 8, &rc));
    double* zw64 = static_cast<double*>(grow(c, kSgCW64, (size_t)KT * mmax * 8, &rc));
    int* didx = static_cast<int*>(grow(c, kSgIdx, (size_t)KT * 4, &rc));
    void* uscr = grow(c, kSgUpd, d2k::update_scratch_bytes(cnt, KT), &rc);
    const size_t spart_n = d2k::update_part_bytes(cnt, KT, v.d);
    double* spart = static_cast<double*>(grow(c, kSgPart, spart_n, &rc));
    if (rc != D2_OK) return rc;
    CK(cudaMemcpyAsync(dmem, list.data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(dsid, sid.data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, c->stream));
    CK(d2k::seg_gather(v, dmem, cnt, om, soff, sloc, sw, som, c->stream));
    ObjView sub;
    sub.loc = sloc;
    sub.w = sw;
    sub.off = soff;
    sub.count = cnt;
    sub.d = v.d;
    sub.ldt = v.ldt;
    sub.wdt = v.wdt;
    sub.segof = dsid;  // segment b of the generation uses centroids [b*K, b*K + K)
    auto set_cents = [&](int K) -> int {  // centroids from compact bags idx[0 .. K*nB)
      CK(cudaMemcpyAsync(didx, idx.data(), (size_t)(K * nB) * 4, cudaMemcpyHostToDevice,
                         c->stream));
      CK(d2k::seg_cents_list(sub, didx, K * nB, zloc, zw, zoff, c->stream));
      CK(d2k::prep_centroids(zloc, D2_F64, zw, D2_F64, zoff, K * nB, v.d, z32, z64, zQ, zw64,
                             c->d_err, c->stream));
      return D2_OK;
    };
    // objects of the segments still open (nullptr: all of them)
    const int* act_d = nullptr;
    long long act_n = cnt;
    auto solve = [&](int K) -> int {
      const CentView zc{z32, z64, zQ, zoff, K * nB, v.d};
      SolveCfg sc = cfg;
      sc.oidx = act_d;
      sc.nobj = act_d ? act_n : -1;
      CK(d2k::assign(sub, zc, cnt, K, sc, nullptr, lab, dd, nullptr, fo, cand, c->d_err,
                     c->stream));
      return check();
    };
    auto labels_to = [&](std::vector<int>& h) -> int {
      h.resize((size_t)cnt);
      CK(cudaMemcpyAsync(h.data(), lab, (size_t)cnt * 4, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      return D2_OK;
    };
    // start: each segment's first member, then the member farthest from it
    idx.assign((size_t)nB, 0);
    for (long long b = 0; b < nB; ++b) idx[(size_t)b] = (int)s0[(size_t)b];
    if ((rc = set_cents(1)) || (rc = solve(1))) return rc;
    hd.resize((size_t)cnt);
    CK(cudaMemcpyAsync(hd.data(), dd, (size_t)cnt * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    idx.assign((size_t)KT, 0);
    for (long long b = 0; b < nB; ++b) {
      long long i2 = s0[(size_t)b];
      for (long long t = s0[(size_t)b] + 1; t < s0[(size_t)b + 1]; ++t)
        if (hd[(size_t)t] > hd[(size_t)i2]) i2 = t;
      idx[(size_t)(2 * b)] = (int)s0[(size_t)b];
      idx[(size_t)(2 * b + 1)] = (int)i2;
    }
    if ((rc = set_cents(2)) || (rc = solve(2)) || (rc = labels_to(hl))) return rc;
    // rounds: a segment whose labels repeat is done; its labels are frozen
    // there (the serial loop stops at that round) while the others go on
    std::vector<char> done((size_t)nB, 0);
    long long open = nB;
    int* dact = static_cast<int*>(grow(c, kSgAct, (size_t)cnt * 4, &rc));
    int* ulab = static_cast<int*>(grow(c, kSgULab, (size_t)cnt * 4, &rc));
    if (rc != D2_OK) return rc;
    std::vector<int> act, hul;
    for (int r = 0; r < iters && open > 0; ++r) {
      // finished segments drop out: their objects are not re-solved and
      // carry label -1 into the update, which leaves their centroids alone
      const int* ul = lab;
      if (open < nB) {
        act.clear();
        hul = hl;
        for (long long b = 0; b < nB; ++b) {
          if (done[(size_t)b]) {
            std::fill(hul.begin() + s0[(size_t)b], hul.begin() + s0[(size_t)b + 1], -1);
          } else {
            for (long long t = s0[(size_t)b]; t < s0[(size_t)b + 1]; ++t) act.push_back((int)t);
          }
        }
        CK(cudaMemcpyAsync(dact, act.data(), act.size() * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(ulab, hul.data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, c->stream));
        act_d = dact;
        act_n = (long long)act.size();
        ul = ulab;
      }
      CK(d2k::update_locations(sub, som, ul, cnt, 2, fo, KT, zoff, v.d, D2_F64, z32, z64, uscr,
                               c->stream, spart, spart_n));
      if ((rc = solve(2)) || (rc = labels_to(hl2))) return rc;
      for (long long b = 0; b < nB; ++b) {
        if (done[(size_t)b]) continue;
        const auto lo = hl.begin() + s0[(size_t)b], hi = hl.begin() + s0[(size_t)b + 1];
        if (std::equal(lo, hi, hl2.begin() + s0[(size_t)b])) {
          done[(size_t)b] = 1;
          --open;
        } else {
          std::copy(hl2.begin() + s0[(size_t)b], hl2.begin() + s0[(size_t)b + 1], lo);
        }
      }
    }
    for (long long b = 0; b < nB; ++b) {
      const std::vector<int>& S = segs[B[(size_t)b]];
      std::vector<int> pa, pb;
      for (size_t t = 0; t < S.size(); ++t)
        (hl[(size_t)s0[(size_t)b] + t] == 0 ? pa : pb).push_back(S[t]);
      if (pa.empty() || pb.empty()) {
        const size_t h = S.size() / 2;
        pa.assign(S.begin(), S.begin() + h);
        pb.assign(S.begin() + h, S.end());
      }
      segs[B[(size_t)b]] = std::move(pa);
      segs.push_back(std::move(pb));
    }
  }
  std::vector<size_t> order(segs.size());
  for (size_t k = 0; k < segs.size(); ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return segs[x][0] < segs[y][0]; });
  std::vector<int> hs((size_t)N);
  for (size_t id = 0; id < order.size(); ++id)
    for (int i : segs[order[id]]) hs[(size_t)i] = (int)id;
  CK(cudaMemcpyAsync(segof, hs.data(), (size_t)N * 4, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *M_out = (long long)segs.size();
  return D2_OK;
}

// Bin only when the batch is large and its trees span more than one bin.
bool want_bins(const d2_ctx* c, long long count, int mmax) {
  const int nmax = std::max(c->nmax, 1);
  const int lo_bin = (1 + nmax + 31) / 32 - 1;
  const int hi_bin = (mmax + nmax + 31) / 32 - 1;
  return count >= 4096 && hi_bin > lo_bin;
}

}  // namespace

namespace d2k {
bool ctx_prune(const d2_ctx* c) { return c->cfg.no_prune == 0; }
CentView ctx_centroids(const d2_ctx* c, int* nmax, int* d, int* device, int* mode, int* budget,
                       int* sms, long long* K, int* start) {
  *nmax = c->nmax;
  *d = c->d;
  *device = c->device;
  *mode = (c->cfg.precision == D2_PREC_FP64 || c->cent_ldt == D2_F64) ? 0 : 1;
  *budget = c->cfg.pivot_budget > 0 ? c->cfg.pivot_budget : 64;
  *sms = c->sms;
  *K = c->K;
  *start = start_default(c);
  return resident_view(c);
}
}  // namespace d2k

extern "C" {

const char* d2_strerror(int32_t s) {
  switch (s) {
    case D2_OK: return "ok";
    case D2_EINVAL: return "invalid argument, offsets, sizes or weights";
    case D2_ENOMEM: return "out of memory";
    case D2_ENOTCONVERGED: return "a pair hit its pivot budget";
    case D2_ETIMEOUT: return "device wait timed out";
    case D2_ECUDA: return "CUDA runtime error";
    case D2_EUNSUPPORTED: return "size or type not supported by the kernels";
    case D2_ENOCENTROIDS: return "no resident centroid set";
    default: return "unknown status";
  }
}

const char* d2_version(void) { return "d2-gb300 0.1 (sm_103a)"; }

// Every field of the configuration within its documented values.
static bool config_ok(const d2_config& f) {
  auto in = [](int32_t v, int32_t lo, int32_t hi) { return v >= lo && v <= hi; };
  return in(f.precision, D2_PREC_AUTO, D2_PREC_FP32) && f.pivot_budget >= 0 &&
         (f.group_lanes == 0 || f.group_lanes == 32) && in(f.cost_tc, D2_TC_AUTO, D2_TC_ON) &&
         f.tile_budget_mib >= 0 && in(f.start_rule, D2_START_AUTO, D2_START_VOGEL) &&
         in(f.segmentation, D2_SEG_SLICES, D2_SEG_CONSTRAINED) && f.split_iters >= 0 &&
         f.eps_tol >= 0.0 && in(f.centroid_update, D2_UPDATE_CONSTRAINED, D2_UPDATE_ALG1) &&
         f.joint_max_iter >= 0 && f.joint_tol >= 0.0 &&
         in(f.certify, D2_CERTIFY_CANDIDATES, D2_CERTIFY_ALL) && f.tc_wait_probe >= 0 &&
         in(f.no_prune, 0, 1) && in(f.joint_cold_start, 0, 1) && f.warm_budget_mib >= 0;
}

int d2_ctx_create(d2_ctx** out, int32_t device, const d2_config* cfg) {
  if (!out) return D2_EINVAL;
  *out = nullptr;
  if (cfg && !config_ok(*cfg)) return D2_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return D2_ECUDA;
  }
  d2_ctx* c = new (std::nothrow) d2_ctx();
  if (!c) return D2_ENOMEM;
  c->device = device;
  if (cfg) c->cfg = *cfg;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->own, cudaStreamDefault) != cudaSuccess ||
      cudaMalloc(&c->d_err, 4 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_info, 4 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->h_pin, 16 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    d2_ctx_destroy(c);
    return D2_ECUDA;
  }
  c->stream = c->own;
  c->sms = d2k::device_sms(device);
  *out = c;
  return D2_OK;
}

int d2_ctx_destroy(d2_ctx* c) {
  if (!c) return D2_EINVAL;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_centroids(c);
  cudaFree(c->tab64); cudaFree(c->tab32);
  for (auto& b : c->slot) if (b.p) cudaFree(b.p);
  if (c->d_err) cudaFree(c->d_err);
  if (c->d_info) cudaFree(c->d_info);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
  return D2_OK;
}

int d2_set_stream(d2_ctx* c, void* s) {
  if (!c) return D2_EINVAL;
  c->stream = s ? static_cast<cudaStream_t>(s) : c->own;
  return D2_OK;
}

int d2_sync(d2_ctx* c) {
  if (!c) return D2_EINVAL;
  cudaSetDevice(c->device);
  return take_errors(c);
}

int d2_set_centroids(d2_ctx* c, const d2_bags* b) {
  d2k::TraceRange trace_("d2_set_centroids");
  if (!c || !bags_ok(b) || b->count < 1) return D2_EINVAL;
  cudaSetDevice(c->device);
  int rc = take_errors(c);  // errors left by earlier calls that did not wait
  if (rc != D2_OK) return rc;
  ObjView v;
  rc = stage_bags(c, b, kCentIn0, kCentIn1, kCentIn2, &v);
  if (rc != D2_OK) return rc;
  std::vector<long long> h(b->count + 1);
  CK(cudaMemcpyAsync(h.data(), v.off, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (h[0] != 0) return D2_EINVAL;
  int nmax = 0;
  for (long long j = 0; j < b->count; ++j) {
    const long long n = h[j + 1] - h[j];
    if (n < 1) return D2_EINVAL;
    if (n > D2_MAX_SUPPORT) return D2_EUNSUPPORTED;
    nmax = std::max<int>(nmax, (int)n);
  }
  free_centroids(c);
  const long long Tc = h[b->count];
  const int d = b->dim;
  if (cudaMalloc(&c->c_loc32, (size_t)Tc * d * 4) != cudaSuccess ||
      cudaMalloc(&c->c_loc64, (size_t)Tc * d * 8) != cudaSuccess ||
      cudaMalloc(&c->c_Q, (size_t)Tc * 8) != cudaSuccess ||
      cudaMalloc(&c->c_w64, (size_t)Tc * 8) != cudaSuccess ||
      cudaMalloc(&c->c_off, (size_t)(b->count + 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    free_centroids(c);
    return D2_ENOMEM;
  }
  CK(cudaMemcpyAsync(c->c_off, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->stream));
  CK(d2k::prep_centroids(v.loc, v.ldt, v.w, v.wdt, c->c_off, b->count, d, c->c_loc32, c->c_loc64,
                         c->c_Q, c->c_w64, c->d_err, c->stream));
  int bits = 0;
  rc = read_err(c, &bits);
  if (rc != D2_OK) return rc;
  if (bits) {
    free_centroids(c);
    return D2_EINVAL;
  }
  if (c->A > 0) {  // a symbol table is set: the centroids must be symbol ids
    if (d != 1) { free_centroids(c); return D2_EINVAL; }
    CK(d2k::check_symbols(c->c_loc64, D2_F64, Tc, c->A, c->d_err, c->stream));
    if ((rc = read_err(c, &bits))) return rc;
    if (bits) { free_centroids(c); return D2_EINVAL; }
  }
  c->K = b->count;
  c->Tc = Tc;
  c->d = d;
  c->nmax = nmax;
  c->cent_ldt = b->loc_dtype;
  c->h_coff = h;
  return D2_OK;
}

int d2_set_cost_table(d2_ctx* c, const double* table, int32_t A) {
  if (!c || A < 0 || (A > 0 && !table)) return D2_EINVAL;
  cudaSetDevice(c->device);
  if (A == 0 || !table) {
    cudaFree(c->tab64); cudaFree(c->tab32);
    c->tab64 = nullptr; c->tab32 = nullptr; c->A = 0;
    return D2_OK;
  }
  if ((long long)A * A > (1LL << 26)) return D2_EUNSUPPORTED;
  std::vector<double> h((size_t)A * A);
  CK(cudaMemcpy(h.data(), table, h.size() * 8, cudaMemcpyDefault));
  std::vector<float> h32(h.size());
  for (size_t t = 0; t < h.size(); ++t) {
    if (!(h[t] >= 0.0) || std::isinf(h[t])) return D2_EINVAL;  // nonnegative, finite
    h32[t] = (float)h[t];
  }
  if (c->K > 0) {  // the resident centroids must already be symbol ids
    if (c->d != 1) return D2_EINVAL;
    std::vector<double> loc((size_t)c->Tc);
    CK(cudaMemcpy(loc.data(), c->c_loc64, loc.size() * 8, cudaMemcpyDeviceToHost));
    for (double x : loc)
      if (!(x >= 0.0 && x < (double)A && x == std::floor(x))) return D2_EINVAL;
  }
  cudaFree(c->tab64); cudaFree(c->tab32);
  c->tab64 = nullptr; c->tab32 = nullptr; c->A = 0;
  if (cudaMalloc(&c->tab64, h.size() * 8) != cudaSuccess ||
      cudaMalloc(&c->tab32, h.size() * 4) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->tab64); cudaFree(c->tab32);
    c->tab64 = nullptr; c->tab32 = nullptr;
    return D2_ENOMEM;
  }
  CK(cudaMemcpy(c->tab64, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->tab32, h32.data(), h32.size() * 4, cudaMemcpyHostToDevice));
  c->A = A;
  return D2_OK;
}

int d2_get_centroids(d2_ctx* c, double* loc_out, double* w_out, int64_t* off_out, int64_t* k_out,
                     int64_t* t_out) {
  if (!c) return D2_EINVAL;
  if (c->K == 0) return D2_ENOCENTROIDS;
  cudaSetDevice(c->device);
  if (k_out) *k_out = c->K;
  if (t_out) *t_out = c->Tc;
  if (loc_out) CK(cudaMemcpyAsync(loc_out, c->c_loc64, (size_t)c->Tc * c->d * 8, cudaMemcpyDefault, c->stream));
  if (w_out) CK(cudaMemcpyAsync(w_out, c->c_w64, (size_t)c->Tc * 8, cudaMemcpyDefault, c->stream));
  if (off_out) CK(cudaMemcpyAsync(off_out, c->c_off, (size_t)(c->K + 1) * 8, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return D2_OK;
}

int d2_cost_matrix(d2_ctx* c, const d2_bags* objs, int64_t i, int64_t j, int32_t precision,
                   double* C) {
  d2k::TraceRange trace_("d2_cost_matrix");
  if (!c || !C || !bags_ok(objs)) return D2_EINVAL;
  if (c->K == 0) return D2_ENOCENTROIDS;
  if (i < 0 || i >= objs->count || j < 0 || j >= c->K || objs->dim != c->d) return D2_EINVAL;
  cudaSetDevice(c->device);
  int rc = take_errors(c);  // errors left by earlier calls that did not wait
  if (rc != D2_OK) return rc;
  ObjView v;
  rc = stage_bags(c, objs, kObjOff, kObjLoc, kObjW, &v);
  if (rc != D2_OK) return rc;
  long long oo[2];
  CK(cudaMemcpyAsync(oo, v.off + i, 16, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const long long m = oo[1] - oo[0];
  const long long n = c->h_coff[j + 1] - c->h_coff[j];
  if (m < 1) return D2_EINVAL;
  if (m > D2_MAX_SUPPORT) return D2_EUNSUPPORTED;
  double* dC;
  bool host;
  rc = stage_out(c, C, (size_t)(m * n), kOutD2, &dC, &host);
  if (rc != D2_OK) return rc;
  if (precision == D2_PREC_TC) {
    if (objs->loc_dtype != D2_BF16 || !d2k::tc_dim_ok(c->d) ||
        (reinterpret_cast<uintptr_t>(v.loc) & 15) != 0)
      return D2_EUNSUPPORTED;
    d2k::TcWork tw;
    if ((rc = tc_work(c, m, (int)m, &tw))) return rc;
    const long long c0 = c->h_coff[j];
    const int ct0 = (int)(c0 / 256), ct1 = (int)((c0 + n - 1) / 256);
    CK(d2k::tc_chunk(v, tw, nullptr, i, 1, (int)m, ct0, ct1 - ct0 + 1, c->d_err, c->stream));
    CK(d2k::tc_extract(tw.C, tw.cents.ncols, (int)m, c0, (int)n, dC, c->stream));
    int bits = 0;
    if ((rc = read_err(c, &bits))) return rc;
    if (bits & d2k::kErrTimeout) return D2_ETIMEOUT;
  } else {
    const int mode = precision == D2_PREC_FP32 ? 1 : 0;
    if ((rc = check_bag_symbols(c, v))) return rc;
    CK(d2k::cost_matrix(v, resident_view(c), i, j, mode, dC, c->stream));
    int bits = 0;
    if ((rc = read_err(c, &bits))) return rc;
    if (bits & d2k::kErrInvalid) return D2_EINVAL;
  }
  if (host) CK(cudaMemcpyAsync(C, dC, (size_t)(m * n) * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return D2_OK;
}

int d2_mallows_batch(d2_ctx* c, const d2_bags* objs, const int64_t* pair_obj, const int64_t* pair_cen,
                     int64_t npairs, double* dist2, d2_flows* flows, int32_t* status) {
  d2k::TraceRange trace_("d2_mallows_batch");
  if (!c || !bags_ok(objs) || npairs < 0 || (npairs > 0 && (!pair_obj || !pair_cen || !dist2)))
    return D2_EINVAL;
  if (c->K == 0) return D2_ENOCENTROIDS;
  if (objs->dim != c->d) return D2_EINVAL;
  if (npairs == 0) return D2_OK;
  cudaSetDevice(c->device);
  ObjView v;
  int rc = stage_bags(c, objs, kObjOff, kObjLoc, kObjW, &v);
  if (rc != D2_OK) return rc;
  int mmax = 0;
  rc = bag_bound(c, objs, v, &mmax);
  if (rc != D2_OK) return rc;
  if (flows && flows->stride < (long long)mmax + c->nmax - 1) return D2_EINVAL;
  const long long* po;
  const long long* pc;
  if ((rc = stage_in(c, reinterpret_cast<const long long*>(pair_obj), (size_t)npairs, kPairObj, &po)) ||
      (rc = stage_in(c, reinterpret_cast<const long long*>(pair_cen), (size_t)npairs, kPairCen, &pc)))
    return rc;
  double* dd;
  int* ds = nullptr;
  bool h1 = false, h2 = false, h3 = false, h4 = false;
  if ((rc = stage_out(c, dist2, (size_t)npairs, kOutD2, &dd, &h1))) return rc;
  if ((rc = stage_out(c, status, (size_t)npairs, kOutStatus, &ds, &h2))) return rc;
  FlowOut fo{nullptr, nullptr, 0};
  if (flows) {
    fo.stride = flows->stride;
    if ((rc = stage_out(c, flows->cell, (size_t)(npairs * flows->stride), kFlowCell, &fo.cell, &h3)) ||
        (rc = stage_out(c, flows->w, (size_t)(npairs * flows->stride), kFlowW, &fo.w, &h4)))
      return rc;
  }
  if ((rc = check_bag_symbols(c, v))) return rc;
  SolveCfg cfg = solve_cfg(c, mode_for(c, objs->loc_dtype), mmax);
  if ((rc = attach_tree(c, &cfg, npairs))) return rc;
  CK(d2k::mallows_pairs(v, resident_view(c), po, pc, npairs, cfg, dd, fo, ds, c->d_err, c->stream));
  if (h1) CK(cudaMemcpyAsync(dist2, dd, (size_t)npairs * 8, cudaMemcpyDeviceToHost, c->stream));
  if (h2) CK(cudaMemcpyAsync(status, ds, (size_t)npairs * 4, cudaMemcpyDeviceToHost, c->stream));
  if (h3) CK(cudaMemcpyAsync(flows->cell, fo.cell, (size_t)(npairs * fo.stride) * 4, cudaMemcpyDeviceToHost, c->stream));
  if (h4) CK(cudaMemcpyAsync(flows->w, fo.w, (size_t)(npairs * fo.stride) * 8, cudaMemcpyDeviceToHost, c->stream));
  return finish(c, h1 || h2 || h3 || h4);
}

namespace {

// d2_assign, and with dist2_all (or certify_all) d2_mallows_all: every pair
// certified in FP64, the pair values into dist2_all [N][K].
int assign_impl(d2_ctx* c, const d2_bags* objs, const double* omega, int32_t* labels,
                double* dist2, double* eps_total, d2_flows* flows, double* dist2_all,
                bool certify_all) {
  if (!c || !bags_ok(objs)) return D2_EINVAL;
  if (c->K == 0) return D2_ENOCENTROIDS;
  if (objs->dim != c->d) return D2_EINVAL;
  if (objs->count == 0) {
    if (eps_total) {
      const double z = 0.0;
      CK(cudaMemcpy(eps_total, &z, 8, cudaMemcpyDefault));
    }
    return D2_OK;
  }
  cudaSetDevice(c->device);
  const long long N = objs->count;
  ObjView v;
  int rc = stage_bags(c, objs, kObjOff, kObjLoc, kObjW, &v);
  if (rc != D2_OK) return rc;
  int mmax = 0;
  if ((rc = bag_bound(c, objs, v, &mmax))) return rc;
  if (flows && flows->stride < (long long)mmax + c->nmax - 1) return D2_EINVAL;
  const double* om;
  if ((rc = stage_in(c, omega, (size_t)N, kOmega, &om))) return rc;
  int* dl;
  double* dd;
  double* dall = nullptr;
  bool h1 = false, h2 = false, h3 = false, h4 = false, h5 = false;
  if (labels) {
    if ((rc = stage_out(c, labels, (size_t)N, kOutLab, &dl, &h1))) return rc;
  } else {
    dl = static_cast<int*>(grow(c, kAllLab, (size_t)N * 4, &rc));
  }
  if (dist2) {
    if ((rc = stage_out(c, dist2, (size_t)N, kOutD2, &dd, &h2))) return rc;
  } else {
    dd = static_cast<double*>(grow(c, kAllD2, (size_t)N * 8, &rc));
  }
  if (rc != D2_OK) return rc;
  if (dist2_all && (rc = stage_out(c, dist2_all, (size_t)(N * c->K), kAllPair, &dall, &h5)))
    return rc;
  FlowOut fo{nullptr, nullptr, 0};
  if (flows) {
    fo.stride = flows->stride;
    if ((rc = stage_out(c, flows->cell, (size_t)(N * flows->stride), kFlowCell, &fo.cell, &h3)) ||
        (rc = stage_out(c, flows->w, (size_t)(N * flows->stride), kFlowW, &fo.w, &h4)))
      return rc;
  }
  double* terms = nullptr;
  if (eps_total) {
    terms = static_cast<double*>(grow(c, kEpsTerms, (size_t)N * 8, &rc));
    if (rc != D2_OK) return rc;
  }
  int* cand = static_cast<int*>(grow(c, kCand, (size_t)d2k::assign_scratch_ints(N, c->K, c->sms) * 4, &rc));
  if (rc != D2_OK) return rc;
  if ((rc = check_bag_symbols(c, v))) return rc;
  Bins bins;
  if (want_bins(c, N, mmax) && (rc = make_bins(c, v, c->nmax, &bins))) return rc;
  const int mode = mode_for(c, objs->loc_dtype);
  d2k::TcWork tw;
  const bool tc = tc_wanted(c, objs, v, mode);
  if (tc && (rc = tc_work(c, N * (long long)mmax, mmax, &tw))) return rc;
  if ((rc = run_assign(c, v, resident_view(c), N, (int)c->K, mode, mmax, om, dl, dd, terms, fo,
                       cand, nullptr, bins, tc ? &tw : nullptr, certify_all, dall)))
    return rc;
  if (eps_total) {
    double* de = static_cast<double*>(grow(c, kEpsOut, 8, &rc));
    if (rc != D2_OK) return rc;
    CK(d2k::sum_fixed_order(terms, N, de, c->stream));
    CK(cudaMemcpyAsync(eps_total, de, 8, cudaMemcpyDefault, c->stream));
  }
  if (h1) CK(cudaMemcpyAsync(labels, dl, (size_t)N * 4, cudaMemcpyDeviceToHost, c->stream));
  if (h2) CK(cudaMemcpyAsync(dist2, dd, (size_t)N * 8, cudaMemcpyDeviceToHost, c->stream));
  if (h3) CK(cudaMemcpyAsync(flows->cell, fo.cell, (size_t)(N * fo.stride) * 4, cudaMemcpyDeviceToHost, c->stream));
  if (h4) CK(cudaMemcpyAsync(flows->w, fo.w, (size_t)(N * fo.stride) * 8, cudaMemcpyDeviceToHost, c->stream));
  if (h5) CK(cudaMemcpyAsync(dist2_all, dall, (size_t)(N * c->K) * 8, cudaMemcpyDeviceToHost, c->stream));
  const bool eps_host = eps_total && where(eps_total) != 1;
  return finish(c, h1 || h2 || h3 || h4 || h5 || eps_host);
}

}  // namespace

int d2_assign(d2_ctx* c, const d2_bags* objs, const double* omega, int32_t* labels, double* dist2,
              double* eps_total, d2_flows* flows) {
  d2k::TraceRange trace_("d2_assign");
  if (!labels || !dist2) return D2_EINVAL;
  return assign_impl(c, objs, omega, labels, dist2, eps_total, flows, nullptr, false);
}

int d2_mallows_all(d2_ctx* c, const d2_bags* objs, double* dist2_all, int32_t* labels,
                   double* dist2) {
  d2k::TraceRange trace_("d2_mallows_all");
  if (!dist2_all) return D2_EINVAL;
  return assign_impl(c, objs, nullptr, labels, dist2, nullptr, nullptr, dist2_all, true);
}

namespace {

// A centroid set the joint-weights core works on: the resident set, or a
// level's replicated sets (K = all centroids of the set).
struct CentSet {
  float* loc32;
  double* loc64;
  long long* Q;
  double* w64;
  const long long* off;
  long long K;
  long long Tc;
};

// Alg. 1 Step 1 for every centroid of `cs` (cluster g = seg(i)*K + label):
// cutting-plane rounds of exact member solves and per-cluster master LPs
// (d2_joint.cu); the set's weights (w64, Q) end as the best weights found.
// eps_d / it_d: [cs.K] device outputs (may be null).  *certified: every
// non-empty cluster closed its gap within max_iter rounds.
int joint_core(d2_ctx* c, const ObjView& v, const double* om, const int* dl, long long seg, int K,
               const CentSet& cs, int mmax, int max_iter, double tol, double* eps_d, int* it_d,
               bool* certified) {
  const long long N = v.count, KT = cs.K;
  int rc = D2_OK;
  const int nmax = std::max(c->nmax, 1);
  const int itmax = max_iter;
  const int G = d2k::joint_groups(nmax);
  // the clusters in two halves, each with its own pair lists and stream: a
  // half's member solves run while the other half's masters (one block per
  // cluster) hold only some of the SMs
  const int H = KT >= 2 ? 2 : 1;
  const long long NB = std::max(N, 1LL);  // pair room per half
  void* scr = grow(c, kJSort, d2k::update_scratch_bytes(std::max(N, 1LL), KT), &rc);
  void* jmem = grow(c, kJState, d2k::joint_state_bytes(KT, cs.Tc, nmax, itmax, G), &rc);
  long long* pobj = static_cast<long long*>(grow(c, kJPObj, (size_t)(H * NB) * 8, &rc));
  long long* pcen = static_cast<long long*>(grow(c, kJPCen, (size_t)(H * NB) * 8, &rc));
  double* W = static_cast<double*>(grow(c, kJW, (size_t)(H * NB) * 8, &rc));
  int* pst = static_cast<int*>(grow(c, kJSt, (size_t)std::max(H * NB, KT) * 4, &rc));
  double* pot = static_cast<double*>(grow(c, kJPot, (size_t)(H * NB) * nmax * 8, &rc));
  long long* pstart = static_cast<long long*>(grow(c, kJPStart, (size_t)(KT + H) * 8, &rc));
  if (rc != D2_OK) return rc;
  const long long* start;
  const int* order;
  if (N > 0) {  // members of every cluster, increasing object index
    FlowOut none{nullptr, nullptr, 0};
    CK(d2k::update_locations(v, nullptr, dl, seg, K, none, KT, cs.off, c->d, c->cent_ldt,
                             cs.loc32, cs.loc64, scr, c->stream));
    d2k::sorted_groups(scr, N, KT, &start, &order);
  } else {
    long long* z = static_cast<long long*>(scr);  // no members: start = 0
    CK(cudaMemsetAsync(z, 0, (size_t)(KT + 1) * 8, c->stream));
    start = z;
    order = nullptr;
  }
  d2k::JointView jv = d2k::joint_view(jmem, KT, cs.Tc, nmax, itmax, G, tol);
  CK(d2k::joint_init(jv, start, cs.off, cs.w64, c->stream));
  SolveCfg cfg = solve_cfg(c, mode_for(c, v.ldt), mmax);
  FlowOut fo{nullptr, nullptr, 0};
  fo.pot = pot;
  fo.pstride = nmax;
  CentView cv{cs.loc32, cs.loc64, cs.Q, cs.off, KT, c->d};
  cv.tab32 = c->tab32;
  cv.tab64 = c->tab64;
  cv.A = c->A;
  // each object's optimal basis from the previous round (the solves of a
  // round restart from it); none saved yet
  if (N > 0 && c->cfg.joint_cold_start == 0 && cfg.mode == 1) {
    const int ns = cfg.mmax + cfg.nmax;
    const size_t nodes = (size_t)N * ns;
    const size_t b3 = (nodes * 3 + 15) / 16 * 16;
    unsigned char* jt = static_cast<unsigned char*>(grow(c, kJTree, b3 + nodes * 8, &rc));
    if (rc != D2_OK) return rc;
    cfg.jw = d2k::WarmStore{jt, jt + nodes, jt + 2 * nodes, reinterpret_cast<long long*>(jt + b3),
                            ns, 1};
    CK(cudaMemsetAsync(cfg.jw.sz8, 0, nodes, c->stream));
  }
  struct Half {
    long long k0, k1;
    d2k::JointView jv;
    long long *pobj, *pcen, *pstart, *hP;
    double *W, *pot;
    int* pst;
    SolveCfg cfg;
    CentView cv;
    FlowOut fo;
    cudaStream_t s;
    cudaEvent_t ev;
    bool done;
  };
  // the second stream and the events live for this call only
  struct Owned {
    cudaStream_t s = nullptr;
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~Owned() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
      if (s) cudaStreamDestroy(s);
    }
  } own;
  for (int h = 0; h < 3; ++h) CK(cudaEventCreateWithFlags(&own.e[h], cudaEventDisableTiming));
  if (H > 1) {
    CK(cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking));
    CK(cudaEventRecord(own.e[2], c->stream));  // the set-up above, then both halves
    CK(cudaStreamWaitEvent(own.s, own.e[2], 0));
  }
  Half hf[2];
  const long long kmid = H > 1 ? KT / 2 : KT;
  for (int h = 0; h < H; ++h) {
    Half& x = hf[h];
    x.k0 = h == 0 ? 0 : kmid;
    x.k1 = h == 0 ? kmid : KT;
    x.jv = d2k::joint_sub(jv, x.k0, x.k1);
    x.pobj = pobj + h * NB;
    x.pcen = pcen + h * NB;
    x.W = W + h * NB;
    x.pot = pot + (size_t)(h * NB) * nmax;
    x.pst = pst + h * NB;
    x.pstart = pstart + (h == 0 ? 0 : kmid + 1);
    x.hP = reinterpret_cast<long long*>(c->h_pin + 4 + 4 * h);
    x.cfg = cfg;
    x.cv = cv;
    x.cv.off = cs.off + x.k0;  // the half's clusters as centroids 0 .. k1-k0-1
    x.cv.K = x.k1 - x.k0;
    x.fo = fo;
    x.fo.pot = x.pot;
    x.s = h == 0 ? c->stream : own.s;
    x.ev = own.e[h];
    x.done = false;
  }
  for (int it = 0; it < itmax; ++it) {
    d2k::TraceRange round_("joint round");
    for (int h = 0; h < H; ++h) {
      Half& x = hf[h];
      if (x.done) continue;
      if (it > 0)  // the weights chosen by the half's last master solves
        CK(d2k::prep_centroids(cs.loc64, D2_F64, jv.wnext, D2_F64, cs.off + x.k0, x.k1 - x.k0, c->d,
                               cs.loc32, cs.loc64, cs.Q, cs.w64, c->d_err, x.s));
      CK(d2k::joint_list(x.jv, order, start + x.k0, x.pstart, x.pobj, x.pcen, x.s));
      CK(cudaMemcpyAsync(x.hP, x.pstart + (x.k1 - x.k0), 8, cudaMemcpyDeviceToHost, x.s));
      CK(cudaEventRecord(x.ev, x.s));
    }
    bool any = false;
    for (int h = 0; h < H; ++h) {
      Half& x = hf[h];
      if (x.done) continue;
      CK(cudaEventSynchronize(x.ev));  // the other half keeps running meanwhile
      const long long P = *x.hP;
      if (P == 0) {
        x.done = true;
        continue;
      }
      any = true;
      if ((rc = attach_tree(c, &x.cfg, P, h == 0 ? kPairTree : kPairTree2))) return rc;
      CK(d2k::mallows_pairs(v, x.cv, x.pobj, x.pcen, P, x.cfg, x.W, x.fo, x.pst, c->d_err, x.s));
      CK(d2k::joint_round(x.jv, x.pstart, x.pobj, om, x.W, x.pot, nmax, x.pst, cs.off + x.k0,
                          cs.w64, x.s));
    }
    if (!any) break;
    d2k::joint_note(1, 0);
  }
  if (H > 1) {  // both halves done before the results are read
    CK(cudaEventRecord(own.e[2], own.s));
    CK(cudaStreamWaitEvent(c->stream, own.e[2], 0));
  }
  int* jst = pst;  // per-cluster status, reusing the pair status room
  CK(d2k::joint_finish(jv, cs.off, eps_d, it_d, jst, c->stream));
  CK(d2k::prep_centroids(cs.loc64, D2_F64, jv.wnext, D2_F64, cs.off, KT, c->d, cs.loc32, cs.loc64,
                         cs.Q, cs.w64, c->d_err, c->stream));
  unsigned long long* hpiv = reinterpret_cast<unsigned long long*>(c->h_pin + 4);
  CK(cudaMemcpyAsync(hpiv, jv.pivots, 8, cudaMemcpyDeviceToHost, c->stream));
  std::vector<int> hs((size_t)KT);
  CK(cudaMemcpyAsync(hs.data(), jst, (size_t)KT * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  d2k::joint_note(0, (long long)*hpiv);
  *certified = true;
  for (int s2 : hs)
    if (s2 == 2 || s2 == 4) *certified = false;
  return D2_OK;
}

// flows for pairs (i, labels[i]) re-solved in FP64 into slots
int resolve_assigned(d2_ctx* c, const ObjView& v, const int* dl, int mmax, const CentView& cv,
                     FlowOut* fo) {
  const long long N = v.count;
  int rc = D2_OK;
  long long* po = static_cast<long long*>(grow(c, kPairObj, (size_t)N * 8, &rc));
  long long* pc = static_cast<long long*>(grow(c, kPairCen, (size_t)N * 8, &rc));
  double* dd = static_cast<double*>(grow(c, kOutD2, (size_t)N * 8, &rc));
  fo->stride = (long long)mmax + c->nmax - 1;
  fo->cell = static_cast<int*>(grow(c, kFlowCell, (size_t)(N * fo->stride) * 4, &rc));
  fo->w = static_cast<double*>(grow(c, kFlowW, (size_t)(N * fo->stride) * 8, &rc));
  if (rc != D2_OK) return rc;
  k_pairs_from_labels<<<blocks_for(N), 256, 0, c->stream>>>(dl, N, po, pc);
  d2k::note_launches(1);
  SolveCfg cfg = solve_cfg(c, 0, mmax);
  CK(d2k::mallows_pairs(v, cv, po, pc, N, cfg, dd, *fo, nullptr, c->d_err, c->stream));
  return D2_OK;
}

}  // namespace

int d2_update_locations(d2_ctx* c, const d2_bags* objs, const double* omega, const int32_t* labels,
                        const d2_flows* flows) {
  d2k::TraceRange trace_("d2_update_locations");
  if (!c || !bags_ok(objs) || !labels) return D2_EINVAL;
  if (c->K == 0) return D2_ENOCENTROIDS;
  if (c->A > 0) return D2_EUNSUPPORTED;  // symbolic supports are not moved
  if (objs->dim != c->d) return D2_EINVAL;
  const long long N = objs->count;
  if (N == 0) return D2_OK;
  cudaSetDevice(c->device);
  ObjView v;
  int rc = stage_bags(c, objs, kObjOff, kObjLoc, kObjW, &v);
  if (rc != D2_OK) return rc;
  int mmax = 0;
  if ((rc = bag_bound(c, objs, v, &mmax))) return rc;
  const double* om;
  const int* dl;
  if ((rc = stage_in(c, omega, (size_t)N, kOmega, &om))) return rc;
  if ((rc = stage_in(c, labels, (size_t)N, kLabelsIn, &dl))) return rc;
  FlowOut fo{nullptr, nullptr, 0};
  if (flows) {
    if (!flows->cell || !flows->w || flows->stride < 1) return D2_EINVAL;
    fo.stride = flows->stride;
    const int* fc;
    const double* fw;
    if ((rc = stage_in(c, flows->cell, (size_t)(N * flows->stride), kFlowCell, &fc)) ||
        (rc = stage_in(c, flows->w, (size_t)(N * flows->stride), kFlowW, &fw)))
      return rc;
    fo.cell = const_cast<int*>(fc);
    fo.w = const_cast<double*>(fw);
  } else {
    if ((rc = resolve_assigned(c, v, dl, mmax, resident_view(c), &fo))) return rc;
  }
  void* scr = grow(c, kUpd, d2k::update_scratch_bytes(N, c->K), &rc);
  const size_t upart_n = d2k::update_part_bytes(N, c->K, c->d);
  double* upart = static_cast<double*>(grow(c, kUpdPart, upart_n, &rc));
  if (rc != D2_OK) return rc;
  c->tc_stale = true;
  CK(d2k::update_locations(v, om, dl, N, (int)c->K, fo, c->K, c->c_off, c->d, c->cent_ldt,
                           c->c_loc32, c->c_loc64, scr, c->stream, upart, upart_n));
  return D2_OK;  // device work only: errors are reported by d2_sync
}

int d2_update_weights(d2_ctx* c, const d2_bags* objs, const double* omega, const int32_t* labels,
                      int32_t max_iter, double tol, double* eps_out, int32_t* iters_out) {
  d2k::TraceRange trace_("d2_update_weights");
  if (!c || !bags_ok(objs) || !labels || max_iter < 1 || max_iter > D2_JOINT_MAX_ITER ||
      !(tol >= 0.0 && tol < 1.0))
    return D2_EINVAL;
  if (c->K == 0) return D2_ENOCENTROIDS;
  if (objs->dim != c->d) return D2_EINVAL;
  if (c->nmax > d2k::kMaxJointN) return D2_EUNSUPPORTED;
  cudaSetDevice(c->device);
  const long long N = objs->count, K = c->K;
  int rc = take_errors(c);  // errors left by earlier calls that did not wait
  if (rc != D2_OK) return rc;
  ObjView v;
  if ((rc = stage_bags(c, objs, kObjOff, kObjLoc, kObjW, &v))) return rc;
  int mmax = 0;
  if ((rc = bag_bound(c, objs, v, &mmax))) return rc;
  if ((rc = check_bag_symbols(c, v))) return rc;
  const double* om;
  const int* dl;
  if ((rc = stage_in(c, omega, (size_t)N, kOmega, &om))) return rc;
  if ((rc = stage_in(c, labels, (size_t)N, kLabelsIn, &dl))) return rc;
  double* eps_d;
  int* it_d;
  bool eps_h, it_h;
  if ((rc = stage_out(c, eps_out, (size_t)K, kJEps, &eps_d, &eps_h)) ||
      (rc = stage_out(c, reinterpret_cast<int*>(iters_out), (size_t)K, kJIters, &it_d, &it_h)))
    return rc;
  CentSet cs{c->c_loc32, c->c_loc64, c->c_Q, c->c_w64, c->c_off, K, c->Tc};
  bool certified = true;
  if ((rc = joint_core(c, v, om, dl, std::max(N, 1LL), (int)K, cs, mmax, max_iter, tol, eps_d,
                       it_d, &certified)))
    return rc;
  if (eps_h) CK(cudaMemcpyAsync(eps_out, eps_d, (size_t)K * 8, cudaMemcpyDeviceToHost, c->stream));
  if (it_h) CK(cudaMemcpyAsync(iters_out, it_d, (size_t)K * 4, cudaMemcpyDeviceToHost, c->stream));
  int bits = 0;
  if ((rc = read_err(c, &bits))) return rc;
  if (bits & d2k::kErrTimeout) return D2_ETIMEOUT;
  if (bits & d2k::kErrInvalid) return D2_EINVAL;
  return certified ? D2_OK : D2_ENOTCONVERGED;
}

int d2_assign_multi(d2_ctx* const* ctxs, int32_t B, const d2_bags* objs, int32_t* labels,
                    double* dist2) {
  d2k::TraceRange trace_("d2_assign_multi");
  if (!ctxs || B < 1 || B > d2k::kMaxBagTypes || !objs || !labels || !dist2) return D2_EINVAL;
  d2_ctx* c = ctxs[0];
  if (!c) return D2_EINVAL;
  const long long N = objs[0].count;
  for (int b = 0; b < B; ++b) {
    d2_ctx* cb = ctxs[b];
    if (!cb || !bags_ok(&objs[b])) return D2_EINVAL;
    if (cb->K == 0) return D2_ENOCENTROIDS;
    if (cb->device != c->device || cb->K != c->K || objs[b].count != N || objs[b].dim != cb->d)
      return D2_EINVAL;
    for (int a = 0; a < b; ++a)
      if (ctxs[a] == cb) return D2_EINVAL;  // one context per bag type
  }
  if (N == 0) return D2_OK;
  cudaSetDevice(c->device);
  const int K = (int)c->K;
  int rc = D2_OK;
  for (int b = 0; b < B; ++b)  // errors left by earlier calls that did not wait
    if ((rc = take_errors(ctxs[b]))) return rc;
  ObjView v[d2k::kMaxBagTypes];
  int mmax[d2k::kMaxBagTypes];
  d2k::MultiScreen ms{};
  ms.B = B;
  auto check = [](d2_ctx* cx) -> int {
    int bits = 0;
    int r = read_err(cx, &bits);
    if (r != D2_OK) return r;
    if (bits & d2k::kErrTimeout) return D2_ETIMEOUT;
    if (bits & d2k::kErrInvalid) return D2_EINVAL;
    if (bits & d2k::kErrNotConverged) return D2_ENOTCONVERGED;
    return D2_OK;
  };
  // 1. every type screens every pair: FP32 value and its bound
  for (int b = 0; b < B; ++b) {
    d2_ctx* cb = ctxs[b];
    if ((rc = stage_bags(cb, &objs[b], kObjOff, kObjLoc, kObjW, &v[b]))) return rc;
    if ((rc = bag_bound(cb, &objs[b], v[b], &mmax[b]))) return rc;
    float* pair = static_cast<float*>(grow(cb, kMbPair, (size_t)N * K * 2 * 4, &rc));
    int* cand = static_cast<int*>(grow(cb, kCand, (size_t)d2k::assign_scratch_ints(N, K, cb->sms) * 4, &rc));
    int* tl = static_cast<int*>(grow(cb, kMbTmpLab, (size_t)N * 4, &rc));
    double* td = static_cast<double*>(grow(cb, kMbTmpD2, (size_t)N * 8, &rc));
    if (rc != D2_OK) return rc;
    if ((rc = check_bag_symbols(cb, v[b]))) return rc;
    SolveCfg cfg = solve_cfg(cb, 1, mmax[b]);  // the FP32 screen, whatever the data type
    cfg.certify = false;  // the summed bounds decide; candidates are solved exactly below
    cfg.pair_out = pair;
    cfg.screen_only = true;
    CK(d2k::assign(v[b], resident_view(cb), N, K, cfg, nullptr, tl, td, nullptr,
                   FlowOut{nullptr, nullptr, 0}, cand, cb->d_err, cb->stream));
    if ((rc = check(cb))) return rc;
    ms.pair[b] = pair;
  }
  // 2. candidates from the summed intervals, listed as pairs
  long long* cnt = static_cast<long long*>(grow(c, kMbCnt, (size_t)N * 8, &rc));
  long long* start = static_cast<long long*>(grow(c, kMbStart, (size_t)(N + 1) * 8, &rc));
  if (rc != D2_OK) return rc;
  CK(d2k::multi_candidates(ms, N, K, cnt, start, c->d_err, c->stream));
  long long P = 0;
  CK(cudaMemcpyAsync(&P, start + N, 8, cudaMemcpyDeviceToHost, c->stream));
  if ((rc = check(c))) return rc;
  long long* pobj = static_cast<long long*>(grow(c, kMbPObj, (size_t)std::max(P, 1LL) * 8, &rc));
  long long* pcen = static_cast<long long*>(grow(c, kMbPCen, (size_t)std::max(P, 1LL) * 8, &rc));
  double* dd = static_cast<double*>(grow(c, kMbD2, (size_t)std::max(P, 1LL) * B * 8, &rc));
  int* pst = static_cast<int*>(grow(c, kMbSt, (size_t)std::max(P, 1LL) * 4, &rc));
  if (rc != D2_OK) return rc;
  CK(d2k::multi_fill(ms, N, K, start, pobj, pcen, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // 3. every type solves the listed pairs exactly
  d2k::MultiExact mx{};
  mx.B = B;
  for (int b = 0; b < B; ++b) {
    d2_ctx* cb = ctxs[b];
    SolveCfg cfg = solve_cfg(cb, mode_for(cb, objs[b].loc_dtype), mmax[b]);
    if ((rc = attach_tree(cb, &cfg, P))) return rc;
    if (P > 0)
      CK(d2k::mallows_pairs(v[b], resident_view(cb), pobj, pcen, P, cfg, dd + (size_t)b * P,
                            FlowOut{nullptr, nullptr, 0}, pst, cb->d_err, cb->stream));
    if ((rc = check(cb))) return rc;
    mx.d2[b] = dd + (size_t)b * P;
  }
  // 4. labels from the summed exact values
  int* dl;
  double* dD;
  bool h1 = false, h2 = false;
  if ((rc = stage_out(c, labels, (size_t)N, kOutLab, &dl, &h1))) return rc;
  if ((rc = stage_out(c, dist2, (size_t)N, kOutD2, &dD, &h2))) return rc;
  CK(d2k::multi_argmin(N, start, pcen, mx, dl, dD, c->stream));
  if (h1) CK(cudaMemcpyAsync(labels, dl, (size_t)N * 4, cudaMemcpyDeviceToHost, c->stream));
  if (h2) CK(cudaMemcpyAsync(dist2, dD, (size_t)N * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return D2_OK;
}

int d2_segment(d2_ctx* c, const d2_bags* objs, const double* omega, int64_t tau, int32_t iters,
               int32_t* seg_id, int64_t* n_segments) {
  d2k::TraceRange trace_("d2_segment");
  if (!c || !bags_ok(objs) || tau < 1 || iters < 0 || !seg_id || !n_segments) return D2_EINVAL;
  const long long N = objs->count;
  if (N < 1) return D2_EINVAL;
  cudaSetDevice(c->device);
  int rc = take_errors(c);  // errors left by earlier calls that did not wait
  if (rc != D2_OK) return rc;
  ObjView v;
  if ((rc = stage_bags(c, objs, kObjOff, kObjLoc, kObjW, &v))) return rc;
  int mmax = 0;
  if ((rc = bag_bound(c, objs, v, &mmax))) return rc;
  const double* om;
  if ((rc = stage_in(c, omega, (size_t)N, kOmega, &om))) return rc;
  int* ds;
  bool host = false;
  if ((rc = stage_out(c, seg_id, (size_t)N, kSgOut, &ds, &host))) return rc;
  long long M = 0;
  if ((rc = segment_impl(c, v, mmax, om, tau, iters, ds, &M))) return rc;
  if (host) CK(cudaMemcpyAsync(seg_id, ds, (size_t)N * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *n_segments = M;
  return D2_OK;
}

int d2_cluster_level(d2_ctx* c, const d2_bags* objs, const double* omega, int32_t K, int64_t seg_size,
                     int32_t iters, double* out_loc, double* out_cent_weight, int32_t* labels) {
  return d2_cluster_level_ex(c, objs, omega, K, seg_size, iters, out_loc, nullptr, out_cent_weight,
                             labels);
}

int d2_cluster_level_ex(d2_ctx* c, const d2_bags* objs, const double* omega, int32_t K,
                        int64_t seg_size, int32_t iters, double* out_loc, double* out_support_w,
                        double* out_cent_weight, int32_t* labels) {
  d2k::TraceRange trace_("d2_cluster_level");
  if (!c || !bags_ok(objs) || K < 1 || iters < 0 || !out_loc || !out_cent_weight || !labels)
    return D2_EINVAL;
  const bool alg1 = c->cfg.centroid_update == D2_UPDATE_ALG1;
  if (c->cfg.centroid_update != D2_UPDATE_CONSTRAINED && !alg1) return D2_EINVAL;
  if (alg1 && c->nmax > d2k::kMaxJointN) return D2_EUNSUPPORTED;
  const int jmax = c->cfg.joint_max_iter > 0 ? std::min(c->cfg.joint_max_iter, D2_JOINT_MAX_ITER)
                                             : 512;
  const double jtol = c->cfg.joint_tol > 0.0 && c->cfg.joint_tol < 1.0 ? c->cfg.joint_tol : 1e-9;
  bool uncertified = false;
  if (c->K == 0) return D2_ENOCENTROIDS;
  if (c->A > 0) return D2_EUNSUPPORTED;  // symbolic supports are not moved
  if (c->K != K || objs->dim != c->d || seg_size <= K) return D2_EINVAL;
  const long long N0 = objs->count;
  if (N0 < 1) return D2_EINVAL;
  cudaSetDevice(c->device);
  int rc = take_errors(c);  // errors left by earlier calls that did not wait
  if (rc != D2_OK) return rc;
  ObjView v;
  if ((rc = stage_bags(c, objs, kObjOff, kObjLoc, kObjW, &v))) return rc;
  int mmax = 0;
  if ((rc = bag_bound(c, objs, v, &mmax))) return rc;
  const double* om0;
  if ((rc = stage_in(c, omega, (size_t)N0, kOmega, &om0))) return rc;
  const int d = c->d;
  const long long Tc = c->Tc;
  // global labels C (identity), current omega
  int* C = static_cast<int*>(grow(c, kLvC, (size_t)N0 * 4, &rc));
  double* om = static_cast<double*>(grow(c, kLvOmega, (size_t)N0 * 8, &rc));
  if (rc != D2_OK) return rc;
  {
    std::vector<int> id(N0);
    for (long long i = 0; i < N0; ++i) id[i] = (int)i;
    CK(cudaMemcpyAsync(C, id.data(), (size_t)N0 * 4, cudaMemcpyHostToDevice, c->stream));
    if (om0) CK(cudaMemcpyAsync(om, om0, (size_t)N0 * 8, cudaMemcpyDeviceToDevice, c->stream));
    else {
      std::vector<double> ones(N0, 1.0);
      CK(cudaMemcpyAsync(om, ones.data(), (size_t)N0 * 8, cudaMemcpyHostToDevice, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
  }
  ObjView cur = v;
  int cur_mmax = mmax;
  for (int level = 0;; ++level) {
    const long long n_l = cur.count;
    cur.segof = nullptr;
    long long M = n_l <= seg_size ? 1 : (n_l + seg_size - 1) / seg_size;
    if (c->cfg.segmentation == D2_SEG_CONSTRAINED && n_l > seg_size) {
      // this level's segments from the binary constrained D2 splits
      int* segof = static_cast<int*>(grow(c, kLvSegof, (size_t)n_l * 4, &rc));
      if (rc != D2_OK) return rc;
      const int si = c->cfg.split_iters > 0 ? c->cfg.split_iters : 10;
      if ((rc = segment_impl(c, cur, cur_mmax, om, seg_size, si, segof, &M))) return rc;
      cur.segof = segof;
    }
    const long long seg = M == 1 ? n_l : seg_size;
    const long long KT = M * K;
    // centroid sets of this level: M copies of the resident set
    float* l32 = static_cast<float*>(grow(c, kLvCLoc32, (size_t)(M * Tc) * d * 4, &rc));
    double* l64 = static_cast<double*>(grow(c, kLvCLoc64, (size_t)(M * Tc) * d * 8, &rc));
    long long* lQ = static_cast<long long*>(grow(c, kLvCQ, (size_t)(M * Tc) * 8, &rc));
    double* lw = static_cast<double*>(grow(c, kLvCW, (size_t)(M * Tc) * 8, &rc));
    long long* loff = static_cast<long long*>(grow(c, kLvCOff, (size_t)(KT + 1) * 8, &rc));
    int* lab = static_cast<int*>(grow(c, kLvLab, (size_t)n_l * 4, &rc));
    double* ld2 = static_cast<double*>(grow(c, kLvD2, (size_t)n_l * 8, &rc));
    int* ct = static_cast<int*>(grow(c, kLvCT, (size_t)n_l * 4, &rc));
    double* wnew = static_cast<double*>(grow(c, kLvOmegaNew, (size_t)KT * 8, &rc));
    const long long stride = (long long)cur_mmax + c->nmax - 1;
    FlowOut fo;
    fo.stride = stride;
    fo.cell = static_cast<int*>(grow(c, kFlowCell, (size_t)(n_l * stride) * 4, &rc));
    fo.w = static_cast<double*>(grow(c, kFlowW, (size_t)(n_l * stride) * 8, &rc));
    void* scr = grow(c, kUpd, d2k::update_scratch_bytes(n_l, KT), &rc);
    const size_t lpart_n = d2k::update_part_bytes(n_l, KT, d);
    double* lpart = static_cast<double*>(grow(c, kLvPart, lpart_n, &rc));
    int* cand = static_cast<int*>(grow(c, kCand, (size_t)d2k::assign_scratch_ints(n_l, K, c->sms) * 4, &rc));
    if (rc != D2_OK) return rc;
    k_replicate<<<blocks_for(M * Tc), 256, 0, c->stream>>>(c->c_loc32, c->c_loc64, c->c_Q, c->c_w64,
                                                           c->c_off, K, Tc, d, M, l32, l64, lQ, lw,
                                                           loff);
    d2k::note_launches(1);
    CK(cudaGetLastError());
    CentView cv{l32, l64, lQ, loff, KT, d};
    const SolveCfg cfg = solve_cfg(c, mode_for(c, cur.ldt), cur_mmax);
    // Saved bases of all (object, centroid) pairs of this level: the rounds
    // re-solve the same pairs with the same marginals and moved centroid
    // locations, so each solve starts from its previous optimal basis.
    // A basis is its tree (parent, preorder position and subtree size
    // bytes per node: 3 B) plus its int64 flows (8 B per node).  The flows
    // are the tree's basic solution for the pair's marginals, which the
    // rounds do not change, so when the whole store does not fit only the
    // trees are kept and a reload recomputes the flows exactly (slower per
    // pair than reading them back, so only then).
    d2k::WarmStore ws{nullptr, nullptr, nullptr, nullptr, 0, 0};
    const long long npairs = n_l * (long long)K;
    const int ns = cur_mmax + c->nmax;
    const size_t meta_bytes = (size_t)npairs * ns * 3;
    const size_t flow_bytes = (size_t)npairs * ns * 8;
    // (not with Alg. 1 updates: the weights, so every pair's supplies, change each round)
    const size_t budget = (cfg.mode == 1 && iters > 1 && !alg1) ? warm_budget_bytes(c) : 0;
    // (a certify-all level keeps full bases or none: its screening kernel
    // carries no flow recomputation)
    const bool flows = meta_bytes + flow_bytes <= budget;
    if (flows || (meta_bytes <= budget && !cfg.certify)) {
      unsigned char* meta = static_cast<unsigned char*>(grow(c, kWarmMeta, meta_bytes, &rc));
      long long* wf = flows ? static_cast<long long*>(grow(c, kWarmFlow, flow_bytes, &rc)) : nullptr;
      if (rc != D2_OK) return rc;
      ws = d2k::WarmStore{meta, meta + (size_t)npairs * ns, meta + (size_t)npairs * ns * 2, wf, ns,
                          0};
    }
    Bins bins;
    if (want_bins(c, n_l, cur_mmax) && (rc = make_bins(c, cur, c->nmax, &bins))) return rc;
    // the pruning moments of this level's bags, once for all its rounds
    const bool moments = prunes(c, cfg, cv);
    if (moments && (rc = prune_moments(c, cur))) return rc;
    // Rounds 2.. repeat the same launches (same pairs, warm bases): round 1
    // is captured into a CUDA graph once and replayed.
    cudaGraphExec_t gexec = nullptr;
    long long glaunches = 0;
    const bool graphs = iters > 2 && !alg1 && c->stream != nullptr &&
                        c->stream != cudaStreamLegacy && c->stream != cudaStreamPerThread;
    // "until epsilon converges" (eps_tol > 0): the level objective of each
    // round's assignment, summed in a fixed order, read back before the next
    double* lterms = nullptr;
    double* leps = nullptr;
    const double etol = c->cfg.eps_tol;
    if (etol > 0.0) {
      lterms = static_cast<double*>(grow(c, kLvTerms, (size_t)n_l * 8, &rc));
      leps = static_cast<double*>(grow(c, kLvEps, 8, &rc));
      if (rc != D2_OK) return rc;
    }
    double eps_prev = -1.0;
    for (int it = 0; it < std::max(iters, 1); ++it) {
      d2k::TraceRange round_("level round");
      if (lterms && it >= 1) {
        CK(d2k::sum_fixed_order(lterms, n_l, leps, c->stream));
        double* he = reinterpret_cast<double*>(c->h_pin + 6);
        CK(cudaMemcpyAsync(he, leps, 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const double e = *he;
        if (eps_prev >= 0.0 && std::fabs(e - eps_prev) <= etol * e) break;
        eps_prev = e;
      }
      ws.warm = it > 0;
      if (gexec && it >= 2) {
        CK(cudaGraphLaunch(gexec, c->stream));
        d2k::note_launches(glaunches);
        continue;
      }
      const bool capture = graphs && it == 1;
      const long long l0 = d2k::launches();
      if (capture && cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
      }
      cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
      cudaStreamIsCapturing(c->stream, &cst);
      const bool capturing = cst == cudaStreamCaptureStatusActive;
      int rc2 = run_assign(c, cur, cv, seg, K, cfg.mode, cur_mmax, om, lab, ld2, lterms, fo, cand,
                           ws.par8 ? &ws : nullptr, bins, nullptr, false, nullptr, moments);
      cudaError_t ue = cudaSuccess;
      if (rc2 == D2_OK && it < iters && alg1) {
        // Alg. 1 Step 1: support weights of every cluster of the level by the
        // joint LP, then the assigned pairs' flows at those weights
        CentSet cs{l32, l64, lQ, lw, loff, KT, M * Tc};
        bool cert = true;
        rc2 = joint_core(c, cur, om, lab, seg, K, cs, cur_mmax, jmax, jtol, nullptr, nullptr, &cert);
        if (rc2 == D2_OK) {
          uncertified |= !cert;
          long long* po = static_cast<long long*>(grow(c, kJPObj, (size_t)n_l * 8, &rc));
          long long* pc = static_cast<long long*>(grow(c, kJPCen, (size_t)n_l * 8, &rc));
          double* dd = static_cast<double*>(grow(c, kJW, (size_t)n_l * 8, &rc));
          if (rc != D2_OK) return rc;
          k_pairs_global<<<blocks_for(n_l), 256, 0, c->stream>>>(lab, n_l, seg, cur.segof, K, po, pc);
          d2k::note_launches(1);
          CK(cudaGetLastError());
          const CentView cv2{l32, l64, lQ, loff, KT, d};
          SolveCfg cfg2 = cfg;
          if ((rc = attach_tree(c, &cfg2, n_l))) return rc;
          CK(d2k::mallows_pairs(cur, cv2, po, pc, n_l, cfg2, dd, fo, nullptr, c->d_err, c->stream));
        }
      }
      if (rc2 == D2_OK && it < iters)
        ue = d2k::update_locations(cur, om, lab, seg, K, fo, KT, loff, d, c->cent_ldt, l32, l64, scr,
                                   c->stream, lpart, lpart_n);
      if (capturing) {
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
        bool ok = ce == cudaSuccess && rc2 == D2_OK && ue == cudaSuccess && graph &&
                  cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        glaunches = d2k::launches() - l0;
        if (!ok) {
          cudaGetLastError();
          if (gexec) cudaGraphExecDestroy(gexec);
          gexec = nullptr;
          // run the round directly instead
          if ((rc = run_assign(c, cur, cv, seg, K, cfg.mode, cur_mmax, om, lab, ld2, lterms, fo,
                               cand, ws.par8 ? &ws : nullptr, bins, nullptr, false, nullptr,
                               moments)))
            return rc;
          if (it < iters)
            CK(d2k::update_locations(cur, om, lab, seg, K, fo, KT, loff, d, c->cent_ldt, l32, l64,
                                     scr, c->stream, lpart, lpart_n));
        } else {
          CK(cudaGraphLaunch(gexec, c->stream));
        }
        continue;
      }
      if (rc2 != D2_OK) return rc2;
      CK(ue);
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    // merge (Eq. (UpdateLabel), Eq. (UpdateGlobalLabel)) and member weights
    FlowOut sort_only{nullptr, nullptr, 0};
    CK(d2k::update_locations(cur, om, lab, seg, K, sort_only, KT, loff, d, c->cent_ldt, l32, l64,
                             scr, c->stream));
    CK(d2k::group_weight_sum(om, n_l, KT, scr, wnew, c->stream));
    k_merge_labels<<<blocks_for(n_l), 256, 0, c->stream>>>(lab, n_l, seg, cur.segof, K, ct);
    k_compose<<<blocks_for(N0), 256, 0, c->stream>>>(C, N0, ct);
    d2k::note_launches(2);
    CK(cudaGetLastError());
    if (M == 1) {
      CK(cudaMemcpyAsync(out_loc, l64, (size_t)Tc * d * 8, cudaMemcpyDefault, c->stream));
      if (out_support_w)
        CK(cudaMemcpyAsync(out_support_w, lw, (size_t)Tc * 8, cudaMemcpyDefault, c->stream));
      CK(cudaMemcpyAsync(out_cent_weight, wnew, (size_t)K * 8, cudaMemcpyDefault, c->stream));
      CK(cudaMemcpyAsync(labels, C, (size_t)N0 * 4, cudaMemcpyDefault, c->stream));
      break;
    }
    // the merged centroids become the next level's weighted data
    const bool f64 = c->cent_ldt == D2_F64;
    void* dloc = grow(c, kLvDataLoc, (size_t)(M * Tc) * d * (f64 ? 8 : 4), &rc);
    double* dw = static_cast<double*>(grow(c, kLvDataW, (size_t)(M * Tc) * 8, &rc));
    long long* doff = static_cast<long long*>(grow(c, kLvDataOff, (size_t)(KT + 1) * 8, &rc));
    double* om2 = static_cast<double*>(grow(c, kLvTmp, (size_t)KT * 8, &rc));
    if (rc != D2_OK) return rc;
    CK(cudaMemcpyAsync(dloc, f64 ? (const void*)l64 : (const void*)l32, (size_t)(M * Tc) * d * (f64 ? 8 : 4),
                       cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(dw, lw, (size_t)(M * Tc) * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(doff, loff, (size_t)(KT + 1) * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(om2, wnew, (size_t)KT * 8, cudaMemcpyDeviceToDevice, c->stream));
    // omega for the next level lives in kLvOmega (grown to KT)
    double* omn = static_cast<double*>(grow(c, kLvOmega, std::max<size_t>((size_t)KT * 8, (size_t)N0 * 8), &rc));
    if (rc != D2_OK) return rc;
    CK(cudaMemcpyAsync(omn, om2, (size_t)KT * 8, cudaMemcpyDeviceToDevice, c->stream));
    om = omn;
    cur.loc = dloc;
    cur.w = dw;
    cur.off = doff;
    cur.count = KT;
    cur.ldt = f64 ? D2_F64 : D2_F32;
    cur.wdt = D2_F64;
    cur_mmax = c->nmax;
    if (level > 64) return D2_EINVAL;
  }
  int bits = 0;
  if ((rc = read_err(c, &bits))) return rc;
  if (bits & d2k::kErrTimeout) return D2_ETIMEOUT;
  if (bits & d2k::kErrInvalid) return D2_EINVAL;
  if (bits & d2k::kErrNotConverged) return D2_ENOTCONVERGED;
  return uncertified ? D2_ENOTCONVERGED : D2_OK;
}

int d2_get_stats(d2_stats* out) {
  if (!out) return D2_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->kernel_launches = d2k::launches();
  d2k::joint_counters(&out->joint_rounds, &out->joint_master_pivots);
  long long v[6];
  if (d2k::solver_stats(v) == cudaSuccess) {
    out->pairs_screened = v[0];
    out->pivots_screened = v[1];
    out->pairs_exact = v[2];
    out->pivots_exact = v[3];
    out->pairs_certified = v[4];
    out->cells_checked = v[5];
  } else {
    cudaGetLastError();
  }
  return D2_OK;
}

}  // extern "C"
