// d2_serve.cu -- continuous-batching server for assignment requests
// (Alg. 2 Step 2 against a resident centroid set).  A worker thread admits
// queued requests (small ones smallest first, large ones in arrival order)
// into slots as slots and device memory
// free up; each slot owns two CUDA streams (high and low priority) and
// grow-only device/pinned buffers, so requests that arrive while others are
// on the GPU start at once and their kernels overlap with the running ones.
// A request runs as a sequence of bounded chunks (about 2^17 pairs each) of
// its bags, binned on the host by the nodes per lane their trees need; small
// requests go to high-priority streams, so their blocks are dispatched as
// soon as the chunk on the GPU drains instead of after a whole large request.
// A quarter of the slots (at least one, when there are two or more) only
// take small requests, and at most kMaxLarge large requests run at once,
// so a burst of large requests never holds every slot.
// Each request's labels and distances are computed by the same
// deterministic per-pair solver as d2_assign, so a result does not depend
// on what else is in flight or on the chunking.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "d2.h"
#include "d2_internal.h"
#include "d2_trace.h"

namespace {

constexpr long long kChunkPairs = 1LL << 17;  // pairs per chunk launch
constexpr int kSmallChunks = 2;                // requests of at most this many chunks: high priority
// Large requests (more chunks) in flight at once: one chunk already fills
// the GPU, so more only stretch every large request's latency.
constexpr int kMaxLarge = 2;

struct Request {
  long long ticket = 0;
  long long count = 0;
  int dim = 0, ldt = 0, wdt = 0, mmax = 0;
  std::vector<unsigned char> loc, w;
  std::vector<long long> off;
  // bags grouped by node bin (b: m + nmax <= 32(b+1)), index order inside
  std::vector<int> order;
  long long bstart[5] = {0, 0, 0, 0, 0};
  int bmmax[4] = {0, 0, 0, 0};
  long long chunks = 0;
  // results
  std::vector<int> labels;
  std::vector<double> dist2;
  int status = D2_OK;
  bool done = false;
  std::chrono::steady_clock::time_point t_submit, t_start, t_done;
  size_t bytes = 0;  // device bytes while in flight
};

struct Slot {
  cudaStream_t stream = nullptr;     // low priority
  cudaStream_t stream_hi = nullptr;  // high priority
  cudaStream_t cur = nullptr;        // the stream of the request in flight
  cudaEvent_t ev = nullptr;
  std::shared_ptr<Request> req;
  bool staging = false;
  // device
  void* d_loc = nullptr; size_t n_loc = 0;
  void* d_w = nullptr; size_t n_w = 0;
  long long* d_off = nullptr; size_t n_off = 0;
  int* d_order = nullptr; size_t n_order = 0;
  int* d_lab = nullptr; size_t n_lab = 0;
  double* d_d2 = nullptr; size_t n_d2 = 0;
  int* d_cand = nullptr; size_t n_cand = 0;
  // bounds of the pairs that cannot be an object's argmin
  double* d_mu = nullptr; size_t n_mu = 0;
  double* d_var = nullptr; size_t n_var = 0;
  unsigned* d_keep = nullptr; size_t n_keep = 0;
  int* d_err = nullptr;
  // pinned host
  unsigned char* h_in = nullptr; size_t n_in = 0;
  unsigned char* h_out = nullptr; size_t n_out = 0;
  int* h_err = nullptr;
};

template <typename T>
bool grow_dev(T** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes && *p) return true;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *cap = bytes;
  return true;
}

bool grow_host(unsigned char** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes && *p) return true;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *cap = bytes;
  return true;
}

size_t esz(int dt) { return dt == D2_F64 ? 8 : (dt == D2_F32 ? 4 : 2); }

}  // namespace

struct d2_server {
  d2_ctx* ctx = nullptr;
  int device = 0;
  d2k::CentView cv{};
  int nmax = 0, d = 0, mode = 1, budget_pivots = 64, sms = 1, start = 0;
  long long K = 0;
  // means and spreads of the resident centroids (pruning; null: off)
  double* d_cmu = nullptr;
  double* d_cvar = nullptr;
  size_t mem_budget = 0, mem_inflight = 0;
  std::vector<Slot> slots;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<long long, std::shared_ptr<Request>> table;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  std::atomic<bool> stop{false};
  long long next_ticket = 1;
  long long admitted = 0, completed = 0, peak_inflight = 0;

  bool launch(Slot& s, const std::shared_ptr<Request>& r);
  void run();
};

// Stage a request into a slot and enqueue its copies and kernels.
bool d2_server::launch(Slot& s, const std::shared_ptr<Request>& r) {
  d2k::TraceRange trace_("serve request");
  const long long N = r->count;
  const long long T = r->off.empty() ? 0 : r->off.back();
  const size_t b_loc = (size_t)T * r->dim * esz(r->ldt);
  const size_t b_w = (size_t)T * esz(r->wdt);
  const size_t b_off = (size_t)(N + 1) * 8;
  const size_t b_ord = (size_t)N * 4;
  const size_t b_in = b_loc + b_w + b_off + b_ord;
  const size_t b_out = (size_t)N * 4 + (size_t)N * 8 + 16;
  if (!grow_dev(reinterpret_cast<unsigned char**>(&s.d_loc), &s.n_loc, std::max<size_t>(b_loc, 16)) ||
      !grow_dev(reinterpret_cast<unsigned char**>(&s.d_w), &s.n_w, std::max<size_t>(b_w, 16)) ||
      !grow_dev(&s.d_off, &s.n_off, b_off) || !grow_dev(&s.d_order, &s.n_order, b_ord + 16) ||
      !grow_dev(&s.d_lab, &s.n_lab, (size_t)N * 4 + 16) ||
      !grow_dev(&s.d_d2, &s.n_d2, (size_t)N * 8 + 16) ||
      !grow_dev(&s.d_cand, &s.n_cand, (size_t)d2k::assign_scratch_ints(N, K, sms) * 4 + 16) ||
      (d_cmu && (!grow_dev(&s.d_mu, &s.n_mu, (size_t)N * r->dim * 8 + 16) ||
                 !grow_dev(&s.d_var, &s.n_var, (size_t)N * 8 + 16) ||
                 !grow_dev(&s.d_keep, &s.n_keep, (size_t)N * ((K + 31) / 32) * 4 + 16))) ||
      !grow_host(&s.h_in, &s.n_in, b_in) ||
      !grow_host(&s.h_out, &s.n_out, b_out))
    return false;
  std::memcpy(s.h_in, r->loc.data(), b_loc);
  std::memcpy(s.h_in + b_loc, r->w.data(), b_w);
  std::memcpy(s.h_in + b_loc + b_w, r->off.data(), b_off);
  std::memcpy(s.h_in + b_loc + b_w + b_off, r->order.data(), b_ord);
  s.cur = r->chunks <= kSmallChunks ? s.stream_hi : s.stream;
  cudaStream_t st = s.cur;
  cudaMemsetAsync(s.d_err, 0, sizeof(int), st);
  cudaMemcpyAsync(s.d_loc, s.h_in, b_loc, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s.d_w, s.h_in + b_loc, b_w, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s.d_off, s.h_in + b_loc + b_w, b_off, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s.d_order, s.h_in + b_loc + b_w + b_off, b_ord, cudaMemcpyHostToDevice, st);
  d2k::ObjView ob;
  ob.loc = s.d_loc;
  ob.w = s.d_w;
  ob.off = s.d_off;
  ob.count = N;
  ob.d = r->dim;
  ob.ldt = r->ldt;
  ob.wdt = r->wdt;
  d2k::SolveCfg cfg;
  cfg.mode = (r->ldt == D2_F64) ? 0 : mode;
  cfg.group = 32;
  cfg.nmax = nmax;
  cfg.budget = budget_pivots;
  cfg.sms = sms;
  cfg.start = start;
  d2k::FlowOut fo{nullptr, nullptr, 0};
  if (d_cmu && cfg.mode == 1) {
    // skip the pairs that cannot be an object's argmin (d2k::prune_keep)
    const int kw = (int)((K + 31) / 32);
    if (d2k::bag_moments(ob, s.d_mu, s.d_var, st) != cudaSuccess ||
        d2k::prune_keep(ob, N, (int)K, K, ob.d, s.d_mu, s.d_var, d_cmu, d_cvar, s.d_keep, kw, st) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cfg.keep = s.d_keep;
    cfg.keep_words = kw;
  }
  // bounded chunks, bin by bin (largest trees first); one stream, so the
  // chunks of a request run in order and share its scratch
  const long long per = std::max<long long>(1, kChunkPairs / std::max<long long>(K, 1));
  for (int b = 3; b >= 0; --b) {
    const long long b0 = r->bstart[b], b1 = r->bstart[b + 1];
    for (long long t0 = b0; t0 < b1; t0 += per) {
      d2k::SolveCfg cc = cfg;
      cc.mmax = r->bmmax[b];
      cc.oidx = s.d_order + t0;
      cc.nobj = std::min(per, b1 - t0);
      cudaError_t e = d2k::assign(ob, cv, N, (int)K, cc, nullptr, s.d_lab, s.d_d2, nullptr, fo,
                                  s.d_cand, s.d_err, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
    }
  }
  cudaMemcpyAsync(s.h_out, s.d_lab, (size_t)N * 4, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(s.h_out + (size_t)N * 4, s.d_d2, (size_t)N * 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(s.h_err, s.d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaEventRecord(s.ev, st);
  return cudaGetLastError() == cudaSuccess;
}

void d2_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop.load()) {
    bool progressed = false;
    // completions
    for (Slot& s : slots) {
      if (!s.req) continue;
      const cudaError_t q = cudaEventQuery(s.ev);
      if (q == cudaErrorNotReady) continue;
      std::shared_ptr<Request> r = s.req;
      const long long N = r->count;
      if (q != cudaSuccess) {
        cudaGetLastError();
        r->status = D2_ECUDA;
      } else {
        r->labels.resize(N);
        r->dist2.resize(N);
        std::memcpy(r->labels.data(), s.h_out, (size_t)N * 4);
        std::memcpy(r->dist2.data(), s.h_out + (size_t)N * 4, (size_t)N * 8);
        const int bits = *s.h_err;
        r->status = (bits & d2k::kErrInvalid) ? D2_EINVAL
                  : (bits & d2k::kErrNotConverged) ? D2_ENOTCONVERGED : D2_OK;
      }
      r->t_done = std::chrono::steady_clock::now();
      r->done = true;
      mem_inflight -= r->bytes;
      s.req.reset();
      ++completed;
      progressed = true;
      cv_done.notify_all();
    }
    // admissions: free slot and memory budget (staging runs unlocked)
    const int nslots = (int)slots.size();
    const int reserved = nslots >= 2 ? std::max(1, nslots / 4) : 0;  // small requests only
    while (!queue.empty()) {
      // small requests: the smallest first; large ones: in arrival order
      // (a large request is not overtaken again and again by smaller large
      // ones, which bounds the tail)
      int large = 0;
      for (Slot& s : slots) large += (s.req && s.req->chunks > kSmallChunks) ? 1 : 0;
      auto pick = queue.end();
      for (auto q = queue.begin(); q != queue.end(); ++q)
        if ((*q)->chunks <= kSmallChunks && (pick == queue.end() || (*q)->count < (*pick)->count))
          pick = q;
      Slot* free_slot = nullptr;
      if (pick != queue.end()) {
        for (int k = 0; k < nslots && !free_slot; ++k)
          if (!slots[k].req && !slots[k].staging) free_slot = &slots[k];
      }
      if (!free_slot) {  // no small request can start: the oldest large one
        pick = queue.end();
        if (large < kMaxLarge)
          for (auto q = queue.begin(); q != queue.end(); ++q)
            if ((*q)->chunks > kSmallChunks) { pick = q; break; }
        if (pick == queue.end()) break;
        for (int k = 0; k < nslots - reserved && !free_slot; ++k)
          if (!slots[k].req && !slots[k].staging) free_slot = &slots[k];
      }
      if (!free_slot) break;
      std::shared_ptr<Request> r = *pick;
      if (mem_inflight > 0 && mem_inflight + r->bytes > mem_budget) break;
      queue.erase(pick);
      free_slot->staging = true;
      mem_inflight += r->bytes;
      lk.unlock();
      r->t_start = std::chrono::steady_clock::now();
      const bool ok = launch(*free_slot, r);
      lk.lock();
      free_slot->staging = false;
      if (!ok) {
        mem_inflight -= r->bytes;
        r->status = D2_ENOMEM;
        r->done = true;
        r->t_done = std::chrono::steady_clock::now();
        cv_done.notify_all();
        continue;
      }
      free_slot->req = r;
      ++admitted;
      long long inflight = 0;
      for (Slot& s : slots) inflight += s.req ? 1 : 0;
      peak_inflight = std::max(peak_inflight, inflight);
      progressed = true;
    }
    if (!progressed) {
      bool busy = false;
      for (Slot& s : slots) busy |= (bool)s.req;
      // in flight: poll the events every 50 us; idle: sleep until work arrives
      if (busy) cv_work.wait_for(lk, std::chrono::microseconds(50));
      else cv_work.wait_for(lk, std::chrono::milliseconds(20));
    }
  }
}

// The context's resident centroid set (read-only while a server runs).
namespace d2k {
CentView ctx_centroids(const d2_ctx* c, int* nmax, int* d, int* device, int* mode, int* budget,
                       int* sms, long long* K, int* start);
bool ctx_prune(const d2_ctx* c);
}

extern "C" int d2_server_create(d2_server** out, d2_ctx* ctx, int32_t nslots, int64_t mem_budget) {
  if (!out || !ctx || nslots < 1 || nslots > 64 || mem_budget < 0) return D2_EINVAL;
  *out = nullptr;
  d2_server* sv = new (std::nothrow) d2_server();
  if (!sv) return D2_ENOMEM;
  sv->ctx = ctx;
  int mode = 1;
  sv->cv = d2k::ctx_centroids(ctx, &sv->nmax, &sv->d, &sv->device, &mode, &sv->budget_pivots, &sv->sms,
                              &sv->K, &sv->start);
  sv->mode = mode;
  if (sv->K == 0) {
    delete sv;
    return D2_ENOCENTROIDS;
  }
  sv->mem_budget = mem_budget > 0 ? (size_t)mem_budget : ((size_t)8 << 30);
  cudaSetDevice(sv->device);
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
    cudaGetLastError();
    prio_lo = prio_hi = 0;
  }
  sv->slots.resize(nslots);
  for (Slot& s : sv->slots) {
    if (cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s.stream_hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&s.d_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&s.h_err), sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      sv->stop = true;
      for (Slot& t : sv->slots) {
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.stream_hi) cudaStreamDestroy(t.stream_hi);
        if (t.ev) cudaEventDestroy(t.ev);
        if (t.d_err) cudaFree(t.d_err);
        if (t.h_err) cudaFreeHost(t.h_err);
      }
      delete sv;
      return D2_ECUDA;
    }
  }
  if (d2k::ctx_prune(ctx) && sv->cv.A == 0) {
    // the resident centroids' means and spreads, once
    if (cudaMalloc(&sv->d_cmu, (size_t)sv->K * sv->d * 8) != cudaSuccess ||
        cudaMalloc(&sv->d_cvar, (size_t)sv->K * 8) != cudaSuccess ||
        d2k::cent_moments(sv->cv, sv->d_cmu, sv->d_cvar, sv->slots[0].stream) != cudaSuccess ||
        cudaStreamSynchronize(sv->slots[0].stream) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(sv->d_cmu);
      cudaFree(sv->d_cvar);
      sv->d_cmu = nullptr;
      sv->d_cvar = nullptr;
    }
  }
  sv->worker = std::thread([sv] { sv->run(); });
  *out = sv;
  return D2_OK;
}

extern "C" int d2_server_submit(d2_server* sv, const d2_bags* objs, int64_t* ticket) {
  if (!sv || !objs || !ticket || !objs->loc || !objs->w || !objs->off || objs->count < 1 ||
      objs->dim != sv->d || objs->loc_dtype < D2_F64 || objs->loc_dtype > D2_BF16 ||
      (objs->w_dtype != D2_F64 && objs->w_dtype != D2_F32))
    return D2_EINVAL;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, objs->off) == cudaSuccess &&
      (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged))
    return D2_EINVAL;  // requests are host data
  cudaGetLastError();
  auto r = std::make_shared<Request>();
  const long long N = objs->count;
  const long long T = objs->off[N];
  if (objs->off[0] != 0 || T < N) return D2_EINVAL;
  int mmax = 0;
  for (long long i = 0; i < N; ++i) {
    const long long m = objs->off[i + 1] - objs->off[i];
    if (m < 1) return D2_EINVAL;
    if (m > D2_MAX_SUPPORT) return D2_EUNSUPPORTED;
    mmax = std::max<int>(mmax, (int)m);
  }
  if (mmax + sv->nmax > 128) return D2_EUNSUPPORTED;
  if (sv->cv.A > 0) {  // symbol ground costs: one-dimensional symbol ids in [0, A)
    if (objs->dim != 1) return D2_EINVAL;
    for (long long t = 0; t < T; ++t) {
      double x;
      if (objs->loc_dtype == D2_F64) x = static_cast<const double*>(objs->loc)[t];
      else if (objs->loc_dtype == D2_F32) x = static_cast<const float*>(objs->loc)[t];
      else return D2_EINVAL;
      if (!(x >= 0.0 && x < (double)sv->cv.A && x == std::floor(x))) return D2_EINVAL;
    }
  }
  // stable partition of the bags by node bin
  r->order.resize(N);
  long long cnt[4] = {0, 0, 0, 0};
  for (long long i = 0; i < N; ++i) {
    const int m = (int)(objs->off[i + 1] - objs->off[i]);
    const int b = (m + sv->nmax + 31) / 32 - 1;
    ++cnt[b];
    r->bmmax[b] = std::max(r->bmmax[b], m);
  }
  for (int b = 0; b < 4; ++b) r->bstart[b + 1] = r->bstart[b] + cnt[b];
  long long fill[4] = {r->bstart[0], r->bstart[1], r->bstart[2], r->bstart[3]};
  for (long long i = 0; i < N; ++i) {
    const int m = (int)(objs->off[i + 1] - objs->off[i]);
    r->order[fill[(m + sv->nmax + 31) / 32 - 1]++] = (int)i;
  }
  const long long per = std::max<long long>(1, kChunkPairs / std::max<long long>(sv->K, 1));
  for (int b = 0; b < 4; ++b) r->chunks += (cnt[b] + per - 1) / per;
  r->count = N;
  r->dim = objs->dim;
  r->ldt = objs->loc_dtype;
  r->wdt = objs->w_dtype;
  r->mmax = mmax;
  const size_t b_loc = (size_t)T * objs->dim * esz(objs->loc_dtype);
  const size_t b_w = (size_t)T * esz(objs->w_dtype);
  r->loc.assign(static_cast<const unsigned char*>(objs->loc), static_cast<const unsigned char*>(objs->loc) + b_loc);
  r->w.assign(static_cast<const unsigned char*>(objs->w), static_cast<const unsigned char*>(objs->w) + b_w);
  r->off.assign(objs->off, objs->off + N + 1);
  r->bytes = b_loc + b_w + (size_t)(N + 1) * 8 + (size_t)N * (4 + 4 + 8) +
             (size_t)d2k::assign_scratch_ints(N, sv->K, sv->sms) * 4;
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    sv->table[r->ticket] = r;
    sv->queue.push_back(r);
  }
  sv->cv_work.notify_one();
  *ticket = r->ticket;
  return D2_OK;
}

extern "C" int d2_server_poll(d2_server* sv, int64_t ticket, int32_t* labels, double* dist2,
                              double* latency_ms, int32_t timeout_ms) {
  if (!sv) return D2_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->table.find(ticket);
  if (it == sv->table.end()) return D2_EINVAL;
  std::shared_ptr<Request> r = it->second;
  const auto pred = [&] { return r->done; };
  if (timeout_ms < 0) sv->cv_done.wait(lk, pred);
  else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return D2_ETIMEOUT;
  if (labels) std::memcpy(labels, r->labels.data(), r->labels.size() * 4);
  if (dist2) std::memcpy(dist2, r->dist2.data(), r->dist2.size() * 8);
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const int st = r->status;
  sv->table.erase(it);
  return st;
}

extern "C" int d2_server_stats(d2_server* sv, int64_t* admitted, int64_t* completed,
                               int64_t* peak_inflight, int64_t* queued) {
  if (!sv) return D2_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (admitted) *admitted = sv->admitted;
  if (completed) *completed = sv->completed;
  if (peak_inflight) *peak_inflight = sv->peak_inflight;
  if (queued) *queued = (int64_t)sv->queue.size();
  return D2_OK;
}

extern "C" int d2_server_destroy(d2_server* sv) {
  if (!sv) return D2_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->device);
  for (Slot& s : sv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.stream_hi) cudaStreamSynchronize(s.stream_hi);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.stream_hi) cudaStreamDestroy(s.stream_hi);
    if (s.ev) cudaEventDestroy(s.ev);
    cudaFree(s.d_loc); cudaFree(s.d_w); cudaFree(s.d_off); cudaFree(s.d_order); cudaFree(s.d_lab);
    cudaFree(s.d_d2);
    cudaFree(s.d_cand); cudaFree(s.d_err);
    cudaFree(s.d_mu); cudaFree(s.d_var); cudaFree(s.d_keep);
    if (s.h_in) cudaFreeHost(s.h_in);
    if (s.h_out) cudaFreeHost(s.h_out);
    if (s.h_err) cudaFreeHost(s.h_err);
  }
  cudaFree(sv->d_cmu);
  cudaFree(sv->d_cvar);
  delete sv;
  return D2_OK;
}
