// profile.cuh -- per-phase launch accounting (see profile.cu).
#pragma once
#include <cuda_runtime.h>

namespace mw {

enum Phase {
  kPhPanel = 0,
  kPhLaswp = 1,
  kPhTrsm = 2,
  kPhGemmPlain = 3,
  kPhGemmSplit = 4,
  kPhSolve = 5,
  kPhPerm = 6,
  kPhResidual = 7,
  kPhRefineAux = 8,
  kPhSplitAux = 9,
  kPhBatchLu = 10,
  kPhBatchSolve = 11,
  kPhPanelInner = 12,   // the split panel's inner tensor-core products
  kNumPhases = 13
};

bool prof_enabled();
void prof_count(int phase);

// Counts one launch of `phase`; when profiling is on, brackets the launches
// issued during its lifetime with events on stream s.
class ProfScope {
 public:
  ProfScope(int phase, cudaStream_t s);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int phase_;
  cudaStream_t s_;
  cudaEvent_t a_;
};

}  // namespace mw
