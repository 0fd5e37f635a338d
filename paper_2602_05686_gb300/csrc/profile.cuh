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
  // setup phases (stream time between the phase's first and last launch)
  PK_S_NODAL = 13,     // a2 nodal tensors
  PK_S_STRENGTH = 14,  // a3/a4 strength + dropping (+ row counts)
  PK_S_GRAPH = 15,     // a5 filtered graph
  PK_S_MIS = 16,       // a6 MIS-2 rounds
  PK_S_AGG = 17,       // a7 aggregation, a8 tentative P
  PK_S_FILTER = 18,    // a10 filtered matrix, 1-norm diagonal
  PK_S_OMEGA = 19,     // a11 power method for omega
  PK_S_SMOOTHP = 20,   // a12 smoothed prolongator (SpGEMM + values)
  PK_S_TRANSPOSE = 21, // R = P^T
  PK_S_RAP = 22,       // a13 Galerkin product (two SpGEMMs + symmetrise)
  PK_S_AUX = 23,       // a9 coarse coordinates / tensors
  PK_S_CHEB = 24,      // a15 Chebyshev bounds
  PK_S_DENSE = 25,     // a15 coarse Cholesky + diagonal-block inverses
  PK_S_SELL = 26,      // a15 SELL packing of the scaled hierarchy
  PK_S_RAP_AP = 27,    // part of PK_S_RAP: the product A P
  PK_S_RAP_RAP = 28,   // part of PK_S_RAP: R (A P) and the mirror of its upper triangle
  // the multi-right-hand-side (K-column) kernels of block.cu and the block CG
  PK_B_CHEB64 = 29,
  PK_B_RESID64 = 30,
  PK_B_RESTRICT64 = 31,
  PK_B_PROLONG64 = 32,
  PK_B_FIRST64 = 33,
  PK_B_COARSE = 34,    // dense coarse solve on K columns (either form)
  PK_B_CHEB32 = 35,
  PK_B_RESID32 = 36,
  PK_B_RESTRICT32 = 37,
  PK_B_PROLONG32 = 38,
  PK_B_FIRST32 = 39,
  PK_B_CG_SPMV = 40,   // Q = A P on K columns with the p.q partials (FP64 SELL)
  PK_B_CG_VEC = 41,    // CG vector updates and dot products on K columns
  PK_NKINDS = 42
};

bool prof_on();
// returns an event index to close with prof_end, or -1 when profiling is off
int prof_begin(cudaStream_t s, int kind, int level, double bytes);
void prof_end(cudaStream_t s, int idx);

}  // namespace sa
