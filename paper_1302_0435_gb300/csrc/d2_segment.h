// d2_segment.h -- batched start centroids of the initial data segmentation
// (d2_segment.cu), used by the C ABI in d2_api.cu.
#pragma once

#include <cuda_runtime.h>

#include "d2_internal.h"

namespace d2k {

// Start centroids of many binary splits: centroid t is compact bag idx[t]
// of v (device ints, KT of them) with uniform weights, FP64 locations into
// cloc / cw, row offsets into coff [KT+1].
cudaError_t seg_cents_list(const ObjView& v, const int* idx, long long KT, double* cloc,
                           double* cw, long long* coff, cudaStream_t st);

}  // namespace d2k
