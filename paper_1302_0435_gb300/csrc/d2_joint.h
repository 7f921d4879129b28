// d2_joint.h -- declarations of the joint-weights solve of Alg. 1 Step 1
// (d2_joint.cu), used by the C ABI in d2_api.cu.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace d2k {

// Alg. 1 Step 1 (d2_joint.cu): per-cluster state of the cutting-plane
// solve of the joint LP of Eq. (WeightedD2).  Cuts per unit of the
// cluster's total omega, G member groups per round:
// cutA [K][itmax][G][nmax], cutB [K][itmax][G].
constexpr int kMaxJointN = 64;
constexpr int kMaxJointR = 80;  // master rows: groups + supports (shared memory)
// Target master size: more groups mean fewer cutting-plane rounds but a
// costlier FP64 master per round (200,000 image-like bags in 64 clusters of
// 16 supports: 16 / 32 / 64 groups take 120 / 86 / 60 rounds and 0.96 /
// 0.83 / 0.95 s).
#ifndef D2_JOINT_RTARGET
#define D2_JOINT_RTARGET 48
#endif
// Cut groups for centroids of up to nmax supports: a power of two dividing
// 128, at most 64, with groups + nmax <= max(target, nmax + 16), within
// kMaxJointR.
inline int joint_groups(int nmax) {
  int cap = D2_JOINT_RTARGET > nmax + 16 ? D2_JOINT_RTARGET : nmax + 16;
  if (cap > kMaxJointR) cap = kMaxJointR;
  int G = 64;
  while (G > 1 && G + nmax > cap) G >>= 1;
  return G;
}
struct JointView {
  double* cutA;
  double* cutB;
  int* bvar;        // [K][G+nmax] optimal basis of each cluster's master LP
  double* binv;     // [K][(G+nmax)^2] its inverse, kept between rounds
  int* since;       // [K] pivots since that inverse was last refactored
  int* nk;          // [K] cuts so far
  int* status;      // [K] 0 active, 1 certified, 2 round cap, 3 empty, 4 failed
  double* F;        // [K] F at this round's weights, per unit omega
  double* ub;       // [K] best F seen
  double* lb;       // [K] the master's lower bound
  double* omsum;    // [K] total omega of the cluster
  double* scale;    // [K] master scaling
  double* pbest;    // [Tc] weights of the best F
  double* wnext;    // [Tc] weights for the next round (final: the result)
  float* cutA32;    // [K][itmax][G][nmax] FP32 copies of the scaled cuts (pricing filter)
  float* cutB32;    // [K][itmax][G]
  unsigned long long* pivots;  // master pivots, summed
  long long K;
  int itmax;
  int nmax;
  int G;
  double tol;
};
size_t joint_state_bytes(long long K, long long Tc, int nmax, int itmax, int G);
JointView joint_view(void* mem, long long K, long long Tc, int nmax, int itmax, int G,
                     double tol);
JointView joint_sub(const JointView& v, long long k0, long long k1);
cudaError_t joint_init(const JointView& jv, const long long* start, const long long* coff,
                       const double* w64, cudaStream_t st);
// pair list (object, cluster) of the active clusters; pstart [K+1]
cudaError_t joint_list(const JointView& jv, const int* order, const long long* start,
                       long long* pstart, long long* pobj, long long* pcen, cudaStream_t st);
// cut of this round from the member solves (W, potentials, status per pair),
// then one master solve per active cluster: next weights into wnext
cudaError_t joint_round(const JointView& jv, const long long* pstart, const long long* pobj,
                        const double* omega, const double* W, const double* pot,
                        long long pstride, const int* pst, const long long* coff,
                        const double* w64, cudaStream_t st);
cudaError_t joint_finish(const JointView& jv, const long long* coff, double* eps, int* iters,
                         int* status, cudaStream_t st);
// process-wide counters of d2_update_weights: rounds and master pivots
void joint_note(long long rounds, long long pivots);
void joint_counters(int64_t* rounds, int64_t* pivots);

}  // namespace d2k
