// Solve-phase launchers and the device-resident CG scalars.
#pragma once

#include "common.cuh"

namespace sa {

struct CsrView {
  int64_t n = 0, nnz = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* v = nullptr;
  int sw = 8;  // lanes per row
};

// right-hand sides one multi-vector solve carries (interleaved storage:
// element (i, c) of an n x k block at i*k + c)
constexpr int KMAX_BLOCK = 8;

struct CgScalars {
  double rz, pq, alpha, beta;
  int breakdown;
  int pad;
};

int pick_sw(int64_t n, int64_t nnz);
int launch_dots(cudaStream_t st, int64_t n, const double* a0, const double* b0, const double* a1, const double* b1,
                const double* a2, const double* b2, double* part, double* out);
int launch_finish(cudaStream_t st, const double* part, int np, double* out);
int launch_cg_alpha(cudaStream_t st, CgScalars* s, const double* dots);
int launch_cg_update(cudaStream_t st, int64_t n, const CgScalars* s, const double* p, const double* q, double* x,
                     double* r, double* rprev, double* part);
int launch_cg_beta(cudaStream_t st, CgScalars* s, const double* dots, int flexible);
int launch_cg_pupdate(cudaStream_t st, int64_t n, const CgScalars* s, const double* z, double* p, int first);

// k-column versions (k <= KMAX_BLOCK), each column summed in the one-vector
// order so that a column of a block solve equals the one-vector solve bitwise
int launch_bdots(cudaStream_t st, int64_t n, int k, const double* a0, const double* b0, const double* a1,
                 const double* b1, double* part, double* out);
int launch_bfinish(cudaStream_t st, const double* part, int np, int k, double* out);
int launch_bcg_alpha(cudaStream_t st, int k, CgScalars* s, const double* dots, const int* active);
int launch_bcg_update(cudaStream_t st, int64_t n, int k, const CgScalars* s, const int* active, const double* p,
                      const double* q, double* x, double* r, double* rprev, double* part);
int launch_bcg_beta(cudaStream_t st, int k, CgScalars* s, const double* dots, int flexible, const int* active);
int launch_bcg_pupdate(cudaStream_t st, int64_t n, int k, const CgScalars* s, const int* active, const double* z,
                       double* p, int first);
// column-major n x k <-> interleaved n x K (K >= k; columns k..K-1 zero)
int launch_interleave(cudaStream_t st, int64_t n, int k, int K, const double* src, double* dst, int to_interleaved);

// dense coarse level (dense.cu).  The coarse matrix A_c = L L^T (Cholesky)
// is solved by block substitution over diagonal blocks of COARSE_BS rows:
// L (row-major, lower triangle), LT = L^T, W = the inverses of the diagonal
// blocks L_KK (stored at their place in an n x n array; the rest unused) and
// WT = W^T.  Only the diagonal blocks are inverted (n COARSE_BS^2 / 3 flops
// instead of n^3 / 3 for the whole inverse).
constexpr int64_t COARSE_BS = 1024;

struct CoarseFactor {
  Buf<double> L, LT, W, WT;
};

struct CoarseView {
  int64_t n = 0;
  const double* L = nullptr;
  const double* LT = nullptr;
  const double* W = nullptr;
  const double* WT = nullptr;
};

inline CoarseView coarse_view(const CoarseFactor& F, int64_t n) {
  CoarseView v;
  v.n = n; v.L = F.L.p; v.LT = F.LT.p; v.W = F.W.p; v.WT = F.WT.p;
  return v;
}

// dense_start enqueues the whole factorisation on streams of its own, forked
// from al.stream after the dense copy of A; dense_finish makes al.stream wait
// for it and reports a pivot that was not positive (SA_ERR_NOT_SPD).  Work on
// al.stream in between must not read the factor.
struct DenseJob {
  Buf<double> Dinv;
  Buf<int> err;
  cudaStream_t main = nullptr, sd = nullptr, s2 = nullptr;
  cudaEvent_t e_fork = nullptr, e_done = nullptr, e_main = nullptr, e_side = nullptr;
  int64_t n = 0;
  int level = 0;         // for the setup-phase profile
  bool pending = false;  // forked and not yet joined
  DenseJob() = default;
  DenseJob(const DenseJob&) = delete;
  DenseJob& operator=(const DenseJob&) = delete;
  ~DenseJob();
};
int dense_start(Alloc& al, int64_t n, const int64_t* rp, const int32_t* ci, const double* v, CoarseFactor& F,
                DenseJob& job);
int dense_finish(DenseJob& job);
// x = A_c^-1 b = L^-T (L^-1 b); t and y: n-vector workspaces (t may not
// alias b, y or x).  The block form takes k in {2, 4, 8} interleaved columns.
int launch_coarse_solve(cudaStream_t st, const CoarseView& F, const double* b, double* t, double* y, double* x);
int launch_coarse_solve_block(cudaStream_t st, const CoarseView& F, int k, const double* b, double* t, double* y,
                              double* x);

}  // namespace sa
