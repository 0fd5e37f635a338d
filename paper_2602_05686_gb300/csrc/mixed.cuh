// FP32 V-cycle on the symmetrically diagonal-scaled hierarchy, used inside
// FP64 flexible CG.
#pragma once

#include "common.cuh"

namespace sa {

struct MixedLevelIn {
  int64_t n = 0, nnz = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* v = nullptr;
  const double* diag = nullptr;
  double lmax = 0, lmin = 0;
  int64_t nc = 0, nnzP = 0;
  const int64_t* Prp = nullptr;
  const int32_t* Pci = nullptr;
  const double* Pv = nullptr;
  const int64_t* Rrp = nullptr;
  const int32_t* Rci = nullptr;
  const double* Rv = nullptr;
};

struct MixedHierarchy;

int mixed_build(Alloc& al, const MixedLevelIn* in, int nlev, int cheb_degree, const double* W, const double* WT,
                MixedHierarchy** out);
// z = D^-1/2 V~(D^-1/2 r): r FP64 fine residual; *z points to handle-owned FP64 memory
int mixed_vcycle(MixedHierarchy* m, cudaStream_t s, const double* r, double** z);
void mixed_free(MixedHierarchy* m);
// bytes streamed by one V-cycle (algorithmic: matrices + vectors), for the roofline
double mixed_vcycle_bytes(const MixedHierarchy* m);

}  // namespace sa
