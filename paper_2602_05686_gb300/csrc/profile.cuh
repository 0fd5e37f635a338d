// Optional per-launch timing of the solve-phase kernels with CUDA events
// recorded on the launching stream; off unless sa_profile_enable(1).
#pragma once

#include "common.cuh"

namespace sa {

enum ProfKind {
  PK_CHEB64 = 0,    // fused Chebyshev step, FP64 CSR
  PK_RESID64 = 1,   // residual, FP64 CSR
  PK_RESTRICT64 = 2,
  PK_PROLONG64 = 3,
  PK_FIRST64 = 4,   // first Chebyshev step from zero (no product)
  PK_CG_SPMV = 5,   // q = A p with the p.q partials (FP64 CSR)
  PK_CG_VEC = 6,    // CG vector updates and dot products
  PK_COARSE = 7,    // dense coarse solve
  PK_CHEB32 = 8,    // fused Chebyshev step, FP32 SELL
  PK_RESID32 = 9,
  PK_RESTRICT32 = 10,
  PK_PROLONG32 = 11,
  PK_FIRST32 = 12,
  PK_NKINDS = 13
};

bool prof_on();
// returns an event index to close with prof_end, or -1 when profiling is off
int prof_begin(cudaStream_t s, int kind, int level, double bytes);
void prof_end(cudaStream_t s, int idx);

}  // namespace sa
