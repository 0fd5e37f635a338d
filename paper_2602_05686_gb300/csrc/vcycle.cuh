// SELL-32 storage and the templated V-cycle on the scaled hierarchy.
#pragma once

#include <vector>

#include "common.cuh"
#include "solve.cuh"

namespace sa {

template <typename T>
struct Sell {
  int64_t n = 0, nslices = 0, stored = 0, nnz = 0;
  Buf<int64_t> sp;  // slice offsets (nslices + 1), in entries
  Buf<int32_t> ci;  // column indices (empty when compressed)
  Buf<T> v;
  // compressed columns: slice base + 16-bit offset, used when every slice's
  // column span fits in 16 bits
  int idx16 = 0;
  Buf<int32_t> base;
  Buf<uint16_t> c16;
  double idx_bytes() const { return idx16 ? 2.0 : 4.0; }
};

// per-level input of the scaled hierarchy (device pointers of the FP64 CSR
// hierarchy)
struct VLevelIn {
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

// a V-cycle matrix: SELL-32 (thread per row) when rows are short and padding
// small, else CSR with sw lanes per row; values scaled and stored in T
template <typename T>
struct Mat {
  int sw = 0;  // 0: SELL-32; else CSR with sw lanes per row
  int sell_lanes = 1;  // SELL-32: lanes per row (1 or 2)
  // CSR: rows with more than lt entries, taken by one warp each
  Buf<int32_t> lrows;
  int64_t nlong = 0, lt = INT64_MAX;
  int64_t n = 0, nnz = 0, nslices = 0;
  int64_t wmax = 0;  // longest row (SELL: widest slice)
  Sell<T> sell;
  Buf<int64_t> rp;
  Buf<int32_t> ci;
  Buf<T> v;
  // FP64 one-thread CSR (sw == 1): the rows grouped by length inside
  // windows of ROW_ORDER_WIN rows -- the order in which the several-column
  // kernels take them (else empty)
  Buf<int32_t> perm;
};

template <typename T>
struct VLevel {
  int64_t n = 0, nc = 0;
  double lmax = 0, lmin = 0;
  Mat<T> A, P, R;
  Buf<T> b, x, x2, r, d;
  Buf<double> sq;  // sqrt(diag) on the coarsest level
  Buf<T> kb, kx, kx2, kr, kd;  // k-column (interleaved) cycle vectors, n x KMAX_BLOCK, made on first use
};

template <typename T>
struct VHier {
  int deg = 2;
  std::vector<VLevel<T>*> lev;
  Buf<double> s0;  // fine-level D^-1/2
  Buf<double> z;   // FP64 output of the cycle
  Buf<double> ct, cs, cy, cx;       // coarse right-hand side and solve vectors
  CoarseView cf;                    // coarse factor
  int kready = 0;                   // k-column buffers allocated
  Buf<double> kz, kct, kcs, kcy, kcx;   // k-column output and coarse vectors
};

// algorithmic bytes: S-byte value + int32 (or 16-bit) column per stored entry
// of the unpadded matrix, 8-byte row pointers or slice offsets (+ slice
// bases), each vector element once
template <typename T>
inline double b_ptr(const Mat<T>& M) {  // row-pointer or slice-offset (+ slice base) bytes
  if (M.sw != 0) return 8.0 * (M.n + 1);
  return 8.0 * (M.nslices + 1) + (M.sell.idx16 ? 4.0 * M.nslices : 0.0);
}
template <typename T>
inline double b_idx(const Mat<T>& M) { return M.sw == 0 ? M.sell.idx_bytes() : 4.0; }
template <typename T>
inline double b_mat(const Mat<T>& M) { return (sizeof(T) + b_idx(M)) * M.nnz + b_ptr(M); }
template <typename T>
inline double b_cheb(const VLevel<T>* L) {
  const double S = sizeof(T);
  return (S + b_idx(L->A)) * L->A.nnz + b_ptr(L->A) + 5.0 * S * L->n;
}


// SELL-32 copy with values left_i * a_ij * right_j (scale vectors may be NULL = 1)
template <typename T>
int build_sell(Alloc& al, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* v,
               const double* left, const double* right, Sell<T>& S);
template <typename T>
int vh_build(Alloc& al, const VLevelIn* in, int nlev, int cheb_degree, const CoarseView& cf,
             VHier<T>** out);
// SA_OK, or SA_ERR_CUDA (error text set) when a staged several-column kernel's
// bounded wait ran out since the last call; synchronises `st`
int block_stage_status(cudaStream_t st);
// largest eigenvalue estimate of level l's scaled operator by power steps
// on the hierarchy's copy (result in the device scalar *lam_dev)
int vh_power(Alloc& al, VHier<double>* m, int l, int steps, uint32_t tag, uint32_t seed, double* lam_dev);
// z = D^-1/2 V~(D^-1/2 r); *z points to hierarchy-owned FP64 memory
template <typename T>
int vh_vcycle(VHier<T>* m, cudaStream_t s, const double* r, double** z);
template <typename T>
void vh_free(VHier<T>* m);
// K in {2, 4, 8} right-hand sides at once: R and *Z are interleaved n x K
// FP64 blocks; column c of *Z equals vh_vcycle of column c of R bitwise
template <typename T>
int vh_vcycle_block(Alloc& al, VHier<T>* m, cudaStream_t s, int k, const double* R, double** Z);

// outer CG on the unscaled fine operator in FP64 SELL
int launch_sell_spmv_dot(cudaStream_t st, const Sell<double>& A, const double* p, double* q, double* part,
                         int* nparts);
int launch_sell_residual64(cudaStream_t st, const Sell<double>& A, const double* b, const double* x, double* r);
// k-column forms (interleaved blocks); partials at part[c * np + cta]
int launch_bsell_spmv_dot(cudaStream_t st, const Sell<double>& A, int k, const double* P, double* Q, double* part,
                          int* nparts);
int launch_bsell_residual64(cudaStream_t st, const Sell<double>& A, int k, const double* B, const double* X,
                            double* R);

}  // namespace sa
