// d2_noalloc.cu -- d2_update_locations_noalloc: the centroid location
// update (same kernels as d2_update_locations) for callers that must not
// allocate device memory during the call.  Its scratch space is a
// fixed-size array in the library's own device memory instead of
// context-owned buffers grown with cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>

#include "d2.h"
#include "d2_internal.h"

namespace {

// Largest batch the fixed scratch array holds.
constexpr long long kMaxBags = 262144;   // objects per call
constexpr long long kMaxCents = 1024;    // centroids per call
constexpr long long kChunkBags = 1024;   // chunk size of the label sort

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
// Same layout as d2k::update_scratch_bytes(kMaxBags, kMaxCents).
constexpr size_t kSortBytes =
    al256((size_t)((kMaxBags + kChunkBags - 1) / kChunkBags) * kMaxCents * 4) +
    al256((size_t)(kMaxCents + 1) * 8) * 2 + al256((size_t)kMaxBags * 4) * 2;
// After the sort area: two ints for the bag-offset check (largest support
// count, invalid-offset flag).
constexpr size_t kInfoBytes = 256;
constexpr size_t kScratchBytes = kSortBytes + kInfoBytes;

// The scratch: allocated with the module, so every GPU that loads this
// library holds kScratchBytes (about 3 MB) until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device.  In host code the
// name g_scratch is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return D2_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return D2_ECUDA;
    }
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return D2_OK;
}

// Device (or managed) memory of the current device: host memory and
// another GPU's memory are refused.
bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int d2_update_locations_noalloc(const d2_bags* objs, const double* omega,
                                           const int32_t* labels, const d2_flows* flows,
                                           int64_t K, const int64_t* cent_off,
                                           int32_t cent_loc_dtype, double* cent_loc64,
                                           float* cent_loc32, void* cuda_stream) {
  if (!objs || !labels || !flows || !flows->cell || !flows->w || flows->stride < 1 || !cent_off ||
      !cent_loc64 || !cent_loc32 || K < 1 || objs->count < 0 || objs->dim < 1 ||
      objs->dim > D2_MAX_DIM || cent_loc_dtype < D2_F64 || cent_loc_dtype > D2_BF16 ||
      objs->loc_dtype < D2_F64 || objs->loc_dtype > D2_BF16 ||
      (objs->w_dtype != D2_F64 && objs->w_dtype != D2_F32))
    return D2_EINVAL;
  if (objs->count > kMaxBags || K > kMaxCents ||
      d2k::update_scratch_bytes(objs->count, K) > kScratchBytes)
    return D2_EUNSUPPORTED;
  if (objs->count == 0) return D2_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return D2_ECUDA;
  }
  // every buffer must already be in this device's memory: no staging copies
  if (!on_device(objs->loc, dev) || !on_device(objs->w, dev) || !on_device(objs->off, dev) ||
      !on_device(labels, dev) || !on_device(flows->cell, dev) || !on_device(flows->w, dev) ||
      !on_device(cent_off, dev) || !on_device(cent_loc64, dev) || !on_device(cent_loc32, dev) ||
      (omega && !on_device(omega, dev)))
    return D2_EINVAL;
  void* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != D2_OK) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // Check the bag offsets on the device (off[0] = 0, every bag 1..64
  // supports) into the info words after the sort area, and read them back
  // with the centroid offsets (the accumulator holds at most D2_MAX_SUPPORT
  // supports per centroid) in one wait on the stream.
  int* info_dev = reinterpret_cast<int*>(static_cast<unsigned char*>(scratch) + kSortBytes);
  int info[2] = {0, 0};
  long long hoff[kMaxCents + 1];
  if (d2k::scan_bags(reinterpret_cast<const long long*>(objs->off), objs->count, info_dev, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(info, info_dev, sizeof(info), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(hoff, cent_off, (size_t)(K + 1) * sizeof(long long), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return D2_ECUDA;
  }
  if (info[1] != 0 || info[0] < 1 || info[0] > D2_MAX_SUPPORT) return D2_EINVAL;
  if (hoff[0] != 0) return D2_EINVAL;
  for (long long j = 0; j < K; ++j) {
    const long long n = hoff[j + 1] - hoff[j];
    if (n < 1 || n > D2_MAX_SUPPORT) return D2_EINVAL;
  }
  d2k::ObjView v;
  v.loc = objs->loc;
  v.w = objs->w;
  v.off = reinterpret_cast<const long long*>(objs->off);
  v.count = objs->count;
  v.d = objs->dim;
  v.ldt = objs->loc_dtype;
  v.wdt = objs->w_dtype;
  d2k::FlowOut fo{flows->cell, flows->w, flows->stride};
  // The sort counters are cleared inside update_locations (cudaMemsetAsync
  // on the scratch); everything else in the scratch is written before use.
  const cudaError_t e = d2k::update_locations(
      v, omega, labels, objs->count, (int)K, fo, K, reinterpret_cast<const long long*>(cent_off),
      objs->dim, cent_loc_dtype, cent_loc32, cent_loc64, scratch,
      st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return D2_ECUDA;
  }
  return D2_OK;
}
