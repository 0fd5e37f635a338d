// Host-side launchers of the library's kernels (one declaration per step).
#pragma once

#include <functional>

#include "common.cuh"

namespace sa {

// ---- setup_exact.cu --------------------------------------------------------
// rows sorted, strictly ascending columns in [0, ncols), row pointers from 0
// to nnz; any violation ORs 32 into *err
int launch_validate_csr(cudaStream_t s, int64_t n, int64_t ncols, int64_t nnz, const int64_t* rp, const int32_t* ci,
                        int* err);
int launch_dirichlet_diag(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                          uint8_t* dir, double* diag, int* err);
int launch_nodal_tensors(Alloc& al, int dim, int64_t n, int tloc, const double* tensors, int64_t ne, int npe,
                         const int32_t* en, const double* meas, double* sigma, double* sinv, int* err);
int launch_strength_classical(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                              const double* diag, const uint8_t* dir, double theta, uint8_t* keep, int64_t* cnt);
int launch_strength_material(cudaStream_t s, int dim, int64_t n, const int64_t* rp, const int32_t* ci,
                             const double* x, const double* sinv, const uint8_t* dir, double theta, double* w,
                             double* D, uint8_t* keep, int64_t* cnt);
// cut-drop (replaces the pointwise mask in keep and the counts in cnt[i+1]);
// classical reads v/diag, material reads w/D
int launch_cut_drop(Alloc& al, int measure_classical, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci,
                    const double* v, const double* diag, const double* w, const double* D, const uint8_t* dir,
                    double theta, uint8_t* keep, int64_t* cnt);
int launch_filter(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                  const uint8_t* keep, const int64_t* rpF, int32_t* ciF, double* vF, double* Dt);
int launch_coarse_aux(cudaStream_t s, int64_t nc, int dim, const int64_t* mrp, const int32_t* mlist,
                      const double* x, const double* sigma, double* xc, double* sc, double* sic);
int launch_smooth_p_values(cudaStream_t s, int64_t n, const int64_t* rpT, const int32_t* ciT, const double* vT,
                           const int32_t* agg, const double* Dt, const double* omega_dev, double* vP);

// ---- graph.cu ----------------------------------------------------------------
// G_C row pointer from the filtered-matrix row pointer (one diagonal per row)
int launch_graph_rowptr(cudaStream_t s, int64_t n, const int64_t* rpF, int64_t* gcrp);
int launch_graph_compact(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, const uint8_t* keep,
                         const int64_t* gcrp, int32_t* gcci);
// MIS-2 by fixed-priority rounds; tag[n] is work space (on exit: roots hold
// ~0ull); returns the number of rounds in *rounds.
int run_mis2(Alloc& al, int64_t n, const int64_t* gcrp, const int32_t* gcci, const uint8_t* dir, int level,
             uint32_t seed, uint64_t* tag, int* rounds, int max_rounds);
// aggregates from the MIS-2 tags; writes agg[n] and *nc, roots (may be NULL)
int run_aggregate(Alloc& al, int64_t n, const int64_t* gcrp, const int32_t* gcci, const uint8_t* dir,
                  const uint64_t* tag, int32_t* agg, uint8_t* root, int64_t* nc, int* err);
int launch_tentative(cudaStream_t s, int64_t n, const int32_t* agg, const int64_t* rp, int32_t* ci, double* v);
int launch_tentative_count(cudaStream_t s, int64_t n, const int32_t* agg, int64_t* cnt);
// R = P^T (m x n) with each row of R sorted by source row; Rv may be NULL
// (pattern only).  Allocates Rrp/Rci/Rv.
int run_transpose(Alloc& al, int64_t n, int64_t m, const int64_t* rp, const int32_t* ci, const double* v,
                  Buf<int64_t>& Rrp, Buf<int32_t>& Rci, Buf<double>* Rv);

// ---- spgemm.cu -------------------------------------------------------------
// C = A * B (n x k times k x m) by count / fill with per-warp shared hash
// tables; rows of C have ascending columns and each entry accumulates its
// products in ascending A-column order (Gustavson order).  upper_only: the
// warp path leaves entries left of the diagonal at 0 (for a symmetric result
// whose lower triangle is mirrored from the upper one afterwards).  A is
// n x kdim, B is kdim x m.
int run_spgemm(Alloc& al, int64_t n, int64_t m, int64_t kdim, const int64_t* Arp, const int32_t* Aci,
               const double* Av, const int64_t* Brp, const int32_t* Bci, const double* Bv, Buf<int64_t>& Crp,
               Buf<int32_t>& Cci, Buf<double>& Cv, int64_t* nnzC, int upper_only = 0);
// lower triangle takes the value of the mirrored upper-triangle entry
int launch_symmetrize(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, double* v, int* err);

// ---- solve.cu -------------------------------------------------------------
struct PowerScratch;
// spectral-radius estimate of diag(s) A diag(s) by `steps` power steps from
// the hash-uniform start (tag, seed); result in *lam_dev (device scalar)
int run_power(Alloc& al, int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* s,
              int steps, uint32_t tag, uint32_t seed, double* lam_dev);
// the same iteration on an operator given by its product: apply(y, w)
// writes w = M y (the V-cycle's pre-scaled copy of D^-1/2 A D^-1/2)
int run_power_op(Alloc& al, int64_t n, int steps, uint32_t tag, uint32_t seed, double* lam_dev,
                 const std::function<int(const double*, double*)>& apply);
int launch_rsqrt_scale(cudaStream_t s, int64_t n, const double* d, double* out);  // 1/sqrt(d), inf -> 0
int launch_reciprocal(cudaStream_t s, int64_t n, const double* d, double* out);
int launch_omega(cudaStream_t s, const double* lam_dev, double omega_sym, double* omega_dev);

}  // namespace sa
