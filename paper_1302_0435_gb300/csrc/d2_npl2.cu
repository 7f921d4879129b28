// d2_npl2.cu -- the solver kernels (screen, certification, per-pair
// Mallows distance) instantiated for 2 tree nodes per lane.
#include "d2_solve.cuh"

namespace d2k {

cudaError_t assign_npl2(const ObjView& ob, const CentView& cv, long long seg_size, int K,
                         const SolveCfg& cfg, const double* omega, int* labels, double* dist2,
                         double* eps_terms, FlowOut fo, int* cand, int* d_err, cudaStream_t st,
                         const WarmStore* ws, const TcWork* tw) {
  return assign_st<32, 2>(ob, cv, seg_size, K, cfg, omega, labels, dist2, eps_terms, fo, cand,
                           d_err, st, ws, tw);
}

cudaError_t mallows_pairs_npl2(const ObjView& ob, const CentView& cv, const long long* pobj,
                                const long long* pcen, long long npairs, const SolveCfg& cfg,
                                double* dist2, FlowOut fo, int* status, int* d_err,
                                cudaStream_t st) {
  return mallows_pairs_st<32, 2>(ob, cv, pobj, pcen, npairs, cfg, dist2, fo, status, d_err, st);
}

cudaError_t stats_npl2(long long out[6]) { return read_unit_stats(out); }

}  // namespace d2k
