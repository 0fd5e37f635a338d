// Group solve: several independent problems (different operators, one
// right-hand side each) advanced together, every step of every problem in
// one launch per kernel kind.  A launch covers its problems one after
// another ("segments"): each segment gets the blocks its own one-problem
// launch would have, each block finds its segment, and runs that launch's
// arithmetic with its launch-local block index -- so a problem solved in a
// group ends bitwise where it ends solved alone.
#pragma once

#include "common.cuh"
#include "solve.cuh"
#include "vcycle.cuh"
#include "vkern.cuh"

namespace sa {

// at most this many problems per group
constexpr int GROUP_MAX = 64;

// matrix-row kernels of the V-cycle (T = float or double)
enum GMatOp { GM_CHEB = 0, GM_CHEB_OUT = 1, GM_RESID = 2, GM_SPMV = 3, GM_SPMV_ADD = 4 };

template <typename T>
struct GMat {
  uint32_t blk0;  // first block of this segment in the launch
  int fmt;        // -2 SELL two lanes, 0 SELL, 1 CSR one thread, CSR_LANES CSR lanes + long-row bin
  MatView<T> M;
  const T* b;
  const T* xin;
  T* xout;
  T* d;
  T* r;
  const double* s;
  double* z;
  T c1, c2;
  int first;
};

// elementwise kernels of the V-cycle
enum GVecOp { GV_FINE_IN = 0, GV_FIRST = 1, GV_COARSE_IN = 2, GV_COARSE_OUT = 3 };

template <typename T>
struct GVec {
  uint32_t blk0;
  int64_t n;
  const double* r64;  // fine entry: FP64 residual
  const double* s;    // fine entry: D^-1/2; coarse in/out: sqrt(diag)
  T c2;
  T* b;
  T* x;
  T* d;
  double* t;          // coarse in: t = sq * b; coarse out: x = (T)(sq * t)
};

// one row range of the coarse block substitution
struct GTri {
  uint32_t blk0;
  int64_t n, r0, r1;
  const double* M;
  const double* v;
  const double* rhs;
  double* out;
};

// outer FP64 CG of one problem
enum GCgOp {
  GC_RESID = 0,     // t = b - A x                 (rows)
  GC_SPMV_DOT = 1,  // q = A p, p.q partials       (rows)
  GC_DOTS = 2,      // dots of (a0,b0), (a1,b1)   (RED_BLOCKS per problem)
  GC_FINISH = 3,    // partials -> dots            (one block per problem)
  GC_ALPHA = 4,     //                             (one thread per problem)
  GC_UPDATE = 5,    // x, r, r_prev, r.r partials  (RED_BLOCKS per problem)
  GC_BETA = 6,      //                             (one thread per problem)
  GC_PUPDATE = 7,   // p = z + beta p              (RED_BLOCKS per problem)
  GC_GATHER = 8     // rr, breakdown -> host block (one thread per problem)
};

struct GCg {
  uint32_t blk0;    // rows geometry: first block of this problem
  int64_t n;
  // FP64 SELL fine operator
  const int64_t* sp;
  const int32_t* ci;
  const int32_t* base;
  const uint16_t* c16;
  const double* v;
  // operands (meaning per op)
  const double* a0;
  const double* b0;
  const double* a1;
  const double* b1;
  const double* in;   // x (GC_RESID), p (GC_SPMV_DOT), z (GC_PUPDATE)
  const double* bvec; // right-hand side (GC_RESID)
  double* out;        // t (GC_RESID), q (GC_SPMV_DOT), p (GC_PUPDATE)
  double* x;
  double* r;
  double* rprev;
  const double* p;
  const double* q;
  CgScalars* cg;
  double* part;
  double* dots;       // finish target / alpha, beta source
  int np, stride;     // finish: partial count and stride
  int flexible;       // beta: -1 initialise, 0 plain, 1 flexible
  int first;          // pupdate
  double* gather;     // GC_GATHER: 2 doubles per problem (r.r, breakdown)
};

template <typename T>
int launch_g_mat(cudaStream_t st, int op, const GMat<T>* d, int m, unsigned blocks);
template <typename T>
int launch_g_vec(cudaStream_t st, int op, const GVec<T>* d, int m, unsigned blocks);
int launch_g_tri(cudaStream_t st, int mode, const GTri* d, int m, unsigned blocks);
int launch_g_cg(cudaStream_t st, int op, const GCg* d, int m, unsigned blocks);

// launch geometry of one problem's matrix kernel (blocks of 256) and format code
template <typename T>
inline unsigned g_mat_blocks(const Mat<T>& M) { return mat_grid(M); }
template <typename T>
inline int g_mat_fmt(const Mat<T>& M) {
  if (M.sw == 0) return M.sell_lanes == 2 ? -2 : 0;
  return M.sw == 1 ? 1 : CSR_LANES;
}
// the coarse solve's row kernels use blocks of this many threads
int tri_threads();

}  // namespace sa
