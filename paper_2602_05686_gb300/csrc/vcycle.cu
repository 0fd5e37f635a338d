// The V-cycle of Algorithm 1 with Chebyshev smoothing (Sec. 4) on the
// symmetrically diagonal-scaled hierarchy
//   A~_l = D_l^-1/2 A_l D_l^-1/2,  P~_l = D_l^1/2 P_l D_{l+1}^-1/2,  R~_l = P~_l^T,
// which satisfies A~_{l+1} = R~_l A~_l P~_l in real arithmetic; Chebyshev on A~
// with a unit diagonal equals Chebyshev on D^-1 A in the original variables,
// and z = D_0^-1/2 V~(D_0^-1/2 r).  One templated code path serves both solve
// forms: T = double (FP64 PCG) and T = float (FP32 V-cycle inside FP64
// flexible CG).  Large matrices are SELL-32: slices of 32 consecutive rows
// stored column-major with one thread per row, so every warp load of values
// and column indices is one contiguous segment, and for finite-element
// stencils (consecutive rows share their stencil shape) the gathers of x are
// contiguous too; coarse levels with a few very long rows are CSR with a
// long-row bin (build_mat).  The coarsest level is solved in FP64 by block
// substitution with the dense coarse factor.
#include <math.h>

#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "solve.cuh"
#include "vcycle.cuh"
#include "vkern.cuh"

namespace sa {

// ---------------------------------------------------------------------------
// SELL-32 construction
// ---------------------------------------------------------------------------
// slice widths (longest row of each 32-row slice) x 32 into sz[sl + 1]; with
// mx, also the longest row overall (one atomic per warp)
__global__ void k_slice_width(int64_t n, const int64_t* __restrict__ rp, int64_t* __restrict__ sz,
                              unsigned int* __restrict__ mx) {
  const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ns = (n + 31) / 32;
  int64_t w = 0;
  if (sl < ns) {
    for (int64_t r = sl * 32; r < sl * 32 + 32 && r < n; ++r) {
      int64_t len = rp[r + 1] - rp[r];
      w = len > w ? len : w;
    }
    sz[sl + 1] = w * 32;
  }
  if (mx) {
    const unsigned int m = __reduce_max_sync(FULL, (unsigned int)w);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(mx, m);
  }
}

// out = left_i * a_ij * right_j with precomputed scale vectors (NULL = 1);
// padding entries point at column 0 with value 0
template <typename T>
__global__ void k_sell_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, const double* __restrict__ left,
                            const double* __restrict__ right, const int64_t* __restrict__ sp,
                            int32_t* __restrict__ oci, T* __restrict__ ov) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t sl = i / 32, r = i % 32;
  const int64_t base = sp[sl], width = (sp[sl + 1] - sp[sl]) / 32;
  const double li = left ? left[i] : 1.0;
  int64_t k = 0;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p, ++k) {
    int32_t j = ci[p];
    const double rj = right ? right[j] : 1.0;
    oci[base + k * 32 + r] = j;
    ov[base + k * 32 + r] = (T)(li * v[p] * rj);
  }
  for (; k < width; ++k) {
    oci[base + k * 32 + r] = 0;
    ov[base + k * 32 + r] = (T)0;
  }
}

// per slice: smallest column and the span of the real (unpadded) entries;
// one thread per row, the 32 rows of a slice form one warp
__global__ void k_slice_span(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             int32_t* __restrict__ base, unsigned int* __restrict__ maxspan) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lo = 0x7fffffff, hi = -1;
  if (r < n) {
    const int64_t b = rp[r], e = rp[r + 1];
    if (e > b) {  // columns ascend: first and last entry
      lo = ci[b];
      hi = ci[e - 1];
    }
  }
  lo = __reduce_min_sync(FULL, lo);
  hi = __reduce_max_sync(FULL, hi);
  if ((threadIdx.x & 31) == 0 && r < n) {
    if (hi < 0) lo = hi = 0;
    base[r >> 5] = lo;
    atomicMax(maxspan, (unsigned int)(hi - lo));
  }
}

// 16-bit offsets from the slice base (padding: offset 0, value 0)
__global__ void k_sell_compress(int64_t n, const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                                const int32_t* __restrict__ base, uint16_t* __restrict__ c16) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t sl = i / 32, r = i % 32;
  const int64_t b = sp[sl], width = (sp[sl + 1] - sp[sl]) / 32;
  const int32_t bs = base[sl];
  for (int64_t k = 0; k < width; ++k) {
    const int64_t q = b + k * 32 + r;
    int32_t c = ci[q] - bs;
    c16[q] = (uint16_t)(c < 0 ? 0 : c);  // padding held column 0
  }
}

__global__ void k_sqrt_vec(int64_t n, const double* __restrict__ d, double* __restrict__ out, int inv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = inv ? 1.0 / sqrt(d[i]) : sqrt(d[i]);
}

template <typename T>
int build_sell(Alloc& al, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* v,
               const double* left, const double* right, Sell<T>& S) {
  cudaStream_t s = al.stream;
  S.n = n;
  S.nnz = nnz;
  S.nslices = (n + 31) / 32;
  SA_TRY(S.sp.alloc(&al, S.nslices + 1));
  SA_TRY(memset_d(S.sp.p, 0, S.sp.bytes(), s));
  if (n <= 0) {
    SA_TRY(S.ci.alloc(&al, 0));
    SA_TRY(S.v.alloc(&al, 0));
    return SA_OK;
  }
  k_slice_width<<<blocks_for(S.nslices, 256), 256, 0, s>>>(n, rp, S.sp.p, nullptr);
  SA_LAUNCHED();
  SA_TRY(scan_inplace(al, S.sp.p + 1, S.nslices));
  SA_TRY(copy_d2h(&S.stored, S.sp.p + S.nslices, sizeof(int64_t), s));
  SA_TRY(S.ci.alloc(&al, S.stored));
  SA_TRY(S.v.alloc(&al, S.stored));
  k_sell_fill<T><<<blocks_for(n, 256), 256, 0, s>>>(n, rp, ci, v, left, right, S.sp.p, S.ci.p, S.v.p);
  SA_LAUNCHED();
  // compress the columns when every slice spans less than 2^16 columns
  Buf<unsigned int> span;
  SA_TRY(span.alloc(&al, 1));
  SA_TRY(memset_d(span.p, 0, sizeof(unsigned int), s));
  SA_TRY(S.base.alloc(&al, S.nslices));
  k_slice_span<<<blocks_for(n, 256), 256, 0, s>>>(n, rp, ci, S.base.p, span.p);
  SA_LAUNCHED();
  unsigned int h_span = 0;
  SA_TRY(copy_d2h(&h_span, span.p, sizeof(h_span), s));
  if (h_span < 65536u) {
    SA_TRY(S.c16.alloc(&al, S.stored));
    k_sell_compress<<<blocks_for(n, 256), 256, 0, s>>>(n, S.sp.p, S.ci.p, S.base.p, S.c16.p);
    SA_LAUNCHED();
    S.idx16 = 1;
    S.ci.release();
  } else {
    S.base.release();
  }
  return SA_OK;
}

template int build_sell<double>(Alloc&, int64_t, int64_t, const int64_t*, const int32_t*, const double*,
                                const double*, const double*, Sell<double>&);
template int build_sell<float>(Alloc&, int64_t, int64_t, const int64_t*, const int32_t*, const double*,
                               const double*, const double*, Sell<float>&);

// CSR copy with scaled values (precomputed scale vectors, NULL = 1)
template <typename T>
__global__ void k_csr_scale(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, const double* __restrict__ left,
                            const double* __restrict__ right, T* __restrict__ ov) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double li = left ? left[i] : 1.0;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) ov[p] = (T)(li * v[p] * (right ? right[ci[p]] : 1.0));
}

// rows with more than lt entries: flags, then their list (ascending)
__global__ void k_long_flag(int64_t n, const int64_t* __restrict__ rp, int64_t lt, int64_t* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i + 1] = (rp[i + 1] - rp[i] > lt) ? 1 : 0;
}

__global__ void k_long_fill(int64_t n, const int64_t* __restrict__ rp, int64_t lt, const int64_t* __restrict__ cnt,
                            int32_t* __restrict__ lrows) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && rp[i + 1] - rp[i] > lt) lrows[cnt[i]] = (int32_t)i;
}

// the row order of a one-thread CSR matrix: one block of ROW_ORDER_WIN
// threads per window of as many rows, a thread per row.  Key = the row's
// length (rows of ROW_ORDER_LEN - 1 or more entries share the last key; the
// threads past n take no key).  A row's place in the window is the number of
// rows with a smaller key, plus those with its key in lower warps, plus those
// with its key in lower lanes of its warp: a stable counting sort.
__global__ void __launch_bounds__(ROW_ORDER_WIN) k_row_order(int64_t n, const int64_t* __restrict__ rp,
                                                             int32_t* __restrict__ perm) {
  constexpr int NW = ROW_ORDER_WIN / 32;
  constexpr int PER_LANE = ROW_ORDER_LEN * NW / 32;
  __shared__ int s_cnt[ROW_ORDER_LEN * NW];  // [key][warp], then the exclusive prefix in that order
  const int64_t base = (int64_t)blockIdx.x * ROW_ORDER_WIN;
  const int64_t i = base + threadIdx.x;
  const int w = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  int key = ROW_ORDER_LEN;  // no row
  if (i < n) {
    const int64_t len = rp[i + 1] - rp[i];
    key = len < ROW_ORDER_LEN - 1 ? (int)len : ROW_ORDER_LEN - 1;
  }
  for (int t = threadIdx.x; t < ROW_ORDER_LEN * NW; t += blockDim.x) s_cnt[t] = 0;
  __syncthreads();
  const unsigned same = __match_any_sync(FULL, key);
  const int rank = __popc(same & ((1u << lane) - 1u));
  if (key < ROW_ORDER_LEN && rank == 0) s_cnt[key * NW + w] = __popc(same);
  __syncthreads();
  if (w == 0) {
    // lane l scans the PER_LANE consecutive counts from l * PER_LANE
    int loc[PER_LANE];
    int sum = 0;
#pragma unroll
    for (int q = 0; q < PER_LANE; ++q) {
      loc[q] = s_cnt[lane * PER_LANE + q];
      sum += loc[q];
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += u;
    }
    int run = inc - sum;
#pragma unroll
    for (int q = 0; q < PER_LANE; ++q) {
      s_cnt[lane * PER_LANE + q] = run;
      run += loc[q];
    }
  }
  __syncthreads();
  if (key < ROW_ORDER_LEN) perm[base + s_cnt[key * NW + w] + rank] = (int32_t)i;
}

// SELL-32 (one thread per row, one FMA per stored entry) if it stores at most
// 25 % padding; else CSR with CSR_LANES lanes per row (one for matrices of at
// most three entries per row on average), and the outlier rows -- longer than
// LONG_ROW_FACTOR times the mean row length and than LONG_ROW entries -- in
// the long-row bin (a warp per row, launched first).  On the coarse levels of
// the stretched battery stack a few rows are 10-40x longer than the rest: a
// few lanes per row keep the FP64 shuffle additions and idle lanes down (the
// FP64 pipe is the scarce unit), the bin keeps the long rows from holding the
// launch.  Measured on its material hierarchy against 8 lanes, 8 lanes with a
// bin, and 4 lanes with bins from 32 to 128 entries, 4 lanes with a bin was
// the fastest for both value types.  The bin's threshold is relative because
// of the several-column kernels: there a warp-per-row sum of eight columns
// adds about half again the FMAs in shuffle additions, and on the 320^3
// inclusions hierarchy a fixed 64 put 24-86 % of the coarse operators' rows
// and 74 % of the restriction's in the bin (measured on rows of 59 and 75
// entries: a thread per column took 0.43x and 0.61x the warp-per-row time).

template <typename T>
int build_mat(Alloc& al, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* v,
              const double* left, const double* right, Mat<T>& M) {
  cudaStream_t s = al.stream;
  M.n = n;
  M.nnz = nnz;
  M.nslices = (n + 31) / 32;
  int64_t stored = 0;
  unsigned int max_width = 0;
  if (n > 0) {
    Buf<int64_t> sz;
    Buf<unsigned int> mx;
    SA_TRY(sz.alloc(&al, M.nslices + 1));
    SA_TRY(mx.alloc(&al, 1));
    SA_TRY(memset_d(sz.p, 0, sz.bytes(), s));
    SA_TRY(memset_d(mx.p, 0, sizeof(unsigned int), s));
    k_slice_width<<<blocks_for(M.nslices, 256), 256, 0, s>>>(n, rp, sz.p, mx.p);
    SA_LAUNCHED();
    SA_TRY(scan_inplace(al, sz.p + 1, M.nslices));
    SA_TRY(copy_d2h(&stored, sz.p + M.nslices, sizeof(int64_t), s));
    SA_TRY(copy_d2h(&max_width, mx.p, sizeof(unsigned int), s));
  }
  // short rows (prolongators): SELL also above 25 % padding when its padding
  // costs fewer bytes than the CSR row pointers it saves (value + 32-bit
  // column per padded entry against 8 bytes per row less a slice pointer)
  const bool short_rows = (double)nnz <= (double)SHORT_ROW_MEAN * (double)n;
  const bool sell_smaller =
      short_rows && (double)(sizeof(T) + 4) * (double)(stored - nnz) < 8.0 * (double)(n - M.nslices);
  M.wmax = (int64_t)max_width;
  if (n == 0 || (double)stored <= 1.25 * (double)nnz || sell_smaller) {
    M.sw = 0;
    M.sell_lanes = n < SELL2_ROWS ? 2 : 1;
    return build_sell<T>(al, n, nnz, rp, ci, v, left, right, M.sell);
  }
  // prolongators hold 1-8 entries per row: one thread per row there (no
  // idle lanes, no shuffle additions, and one partial sum per column in the
  // several-column kernels: with four lanes' partial sums the FP64 level-0
  // prolongation of the 320^3 inclusions stack spent 2.5x its products in
  // FP64 instructions -- 88 % of the FP64 pipe in ncu)
  M.sw = short_rows ? 1 : CSR_LANES;
  M.nlong = 0;
  M.lt = INT64_MAX;
  const int64_t lt = std::max<int64_t>(LONG_ROW, LONG_ROW_FACTOR * ((nnz + n - 1) / n));
  if ((int64_t)max_width > lt) {
    M.lt = lt;
    Buf<int64_t> cnt;
    SA_TRY(cnt.alloc(&al, n + 1));
    SA_TRY(memset_d(cnt.p, 0, sizeof(int64_t), s));
    k_long_flag<<<blocks_for(n, 256), 256, 0, s>>>(n, rp, M.lt, cnt.p);
    SA_LAUNCHED();
    SA_TRY(scan_inplace(al, cnt.p + 1, n));
    SA_TRY(copy_d2h(&M.nlong, cnt.p + n, sizeof(int64_t), s));
    SA_TRY(M.lrows.alloc(&al, M.nlong));
    if (M.nlong > 0) {
      k_long_fill<<<blocks_for(n, 256), 256, 0, s>>>(n, rp, M.lt, cnt.p, M.lrows.p);
      SA_LAUNCHED();
    } else {
      M.lt = INT64_MAX;
    }
  }
  if (M.sw == 1 && sizeof(T) == 8) {  // FP64 rows only: see the several-column kernels
    SA_TRY(M.perm.alloc(&al, n));
    k_row_order<<<(unsigned)((n + ROW_ORDER_WIN - 1) / ROW_ORDER_WIN), ROW_ORDER_WIN, 0, s>>>(n, rp, M.perm.p);
    SA_LAUNCHED();
  }
  SA_TRY(M.rp.alloc(&al, n + 1));
  SA_TRY(M.ci.alloc(&al, nnz));
  SA_TRY(M.v.alloc(&al, nnz));
  SA_CUDA(cudaMemcpyAsync(M.rp.p, rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
  if (nnz > 0) SA_CUDA(cudaMemcpyAsync(M.ci.p, ci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
  k_csr_scale<T><<<blocks_for(n, 256), 256, 0, s>>>(n, rp, ci, v, left, right, M.v.p);
  SA_LAUNCHED();
  return SA_OK;
}

template <typename T>
int vh_build(Alloc& al, const VLevelIn* in, int nlev, int cheb_degree, const CoarseView& cf,
             VHier<T>** out) {
  VHier<T>* m = new VHier<T>();
  *out = m;
  m->deg = cheb_degree;
  m->cf = cf;
  cudaStream_t s = al.stream;
  // D_l^-1/2 and D_l^1/2 of every level, once (FP64 square roots are costly)
  std::vector<Buf<double>> isq(nlev), sq(nlev);
  for (int l = 0; l < nlev; ++l) {
    SA_TRY(isq[l].alloc(&al, in[l].n));
    SA_TRY(sq[l].alloc(&al, in[l].n));
    k_sqrt_vec<<<blocks_for(in[l].n, 256), 256, 0, s>>>(in[l].n, in[l].diag, isq[l].p, 1);
    SA_LAUNCHED();
    k_sqrt_vec<<<blocks_for(in[l].n, 256), 256, 0, s>>>(in[l].n, in[l].diag, sq[l].p, 0);
    SA_LAUNCHED();
  }
  for (int l = 0; l < nlev; ++l) {
    VLevel<T>* L = new VLevel<T>();
    m->lev.push_back(L);
    const VLevelIn& I = in[l];
    L->n = I.n;
    L->nc = I.nc;
    L->lmax = I.lmax;
    L->lmin = I.lmin;
    SA_TRY(L->b.alloc(&al, I.n));
    SA_TRY(L->x.alloc(&al, I.n));
    SA_TRY(L->x2.alloc(&al, I.n));
    SA_TRY(L->r.alloc(&al, I.n));
    SA_TRY(L->d.alloc(&al, I.n));
    if (l + 1 < nlev) {
      // A~ = D^-1/2 A D^-1/2, P~ = D_l^1/2 P D_{l+1}^-1/2, R~ = D_{l+1}^-1/2 R D_l^1/2
      SA_TRY(build_mat<T>(al, I.n, I.nnz, I.rp, I.ci, I.v, isq[l].p, isq[l].p, L->A));
      SA_TRY(build_mat<T>(al, I.n, I.nnzP, I.Prp, I.Pci, I.Pv, sq[l].p, isq[l + 1].p, L->P));
      SA_TRY(build_mat<T>(al, I.nc, I.nnzP, I.Rrp, I.Rci, I.Rv, isq[l + 1].p, sq[l].p, L->R));
    } else {
      L->sq = std::move(sq[l]);
      SA_TRY(m->ct.alloc(&al, I.n));
      SA_TRY(m->cs.alloc(&al, I.n));
      SA_TRY(m->cy.alloc(&al, I.n));
      SA_TRY(m->cx.alloc(&al, I.n));
    }
  }
  const int64_t n0 = in[0].n;
  SA_TRY(m->s0.alloc(&al, n0));
  SA_TRY(m->z.alloc(&al, n0));
  k_sqrt_vec<<<blocks_for(n0, 256), 256, 0, s>>>(n0, in[0].diag, m->s0.p, 1);
  SA_LAUNCHED();
  return SA_OK;
}

template int vh_build<double>(Alloc&, const VLevelIn*, int, int, const CoarseView&, VHier<double>**);
template int vh_build<float>(Alloc&, const VLevelIn*, int, int, const CoarseView&, VHier<float>**);

// ---------------------------------------------------------------------------
// kernels (one thread per row)
// ---------------------------------------------------------------------------
// x_out = x_in + d,  d = first ? c2 r : c1 d + c2 r,  r = b - A~ x_in
template <typename T, int SW>
__global__ void k_vc_cheb(MatView<T> A, const T* __restrict__ b, const T* __restrict__ xin, T* __restrict__ xout,
                          T* __restrict__ d, T c1, T c2, int first) {
  T y;
  int64_t i;
  if (!row_apply<T, SW>(A, xin, y, i)) return;
  const T dn = cheb_dir<T>(b[i], y, first ? (T)0 : d[i], c1, c2, first);
  d[i] = dn;
  xout[i] = xin[i] + dn;
}

template <typename T, int SW>
__global__ void k_vc_residual(MatView<T> A, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r) {
  T y;
  int64_t i;
  if (row_apply<T, SW>(A, x, y, i)) r[i] = b[i] - y;
}

template <typename T, int SW>
__global__ void k_vc_spmv(MatView<T> A, const T* __restrict__ x, T* __restrict__ out) {
  T y;
  int64_t i;
  if (row_apply<T, SW>(A, x, y, i)) out[i] = y;
}

template <typename T, int SW>
__global__ void k_vc_spmv_add(MatView<T> A, const T* __restrict__ x, T* __restrict__ out) {
  T y;
  int64_t i;
  if (row_apply<T, SW>(A, x, y, i)) out[i] += y;
}

// fine exit: the last post-smoothing step writes z = D^-1/2 x~ in FP64
template <typename T, int SW>
__global__ void k_vc_cheb_out(MatView<T> A, const T* __restrict__ b, const T* __restrict__ xin,
                              const T* __restrict__ d, T c1, T c2, int first, const double* __restrict__ s,
                              double* __restrict__ z) {
  T y;
  int64_t i;
  if (!row_apply<T, SW>(A, xin, y, i)) return;
  const T dn = cheb_dir<T>(b[i], y, first ? (T)0 : d[i], c1, c2, first);
  z[i] = s[i] * (double)(xin[i] + dn);
}

template <typename T>
__global__ void k_vc_first(int64_t n, const T* __restrict__ b, T c2, T* __restrict__ x, T* __restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    T dn = c2 * b[i];
    d[i] = dn;
    x[i] = dn;
  }
}

// fine entry b~ = D^-1/2 r (FP64 r), fused with the first Chebyshev step
template <typename T>
__global__ void k_vc_fine_in(int64_t n, const double* __restrict__ r, const double* __restrict__ s, T c2,
                             T* __restrict__ b, T* __restrict__ x, T* __restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    T bi = (T)(s[i] * r[i]);
    b[i] = bi;
    T dn = c2 * bi;
    d[i] = dn;
    x[i] = dn;
  }
}

// launch `K<T, sw>` over the rows of M (SELL: one thread per row; CSR: sw lanes)
#define LAUNCH_MAT(K, M, st, ...)                                                        \
  do {                                                                                   \
    const MatView<T> _mv = view(M);                                                      \
    const unsigned _g = mat_grid(M);                                                     \
    if ((M).sw == 0 && (M).sell_lanes == 2) K<T, -2><<<_g, 256, 0, st>>>(_mv, __VA_ARGS__); \
    else if ((M).sw == 0) K<T, 0><<<_g, 256, 0, st>>>(_mv, __VA_ARGS__);                 \
    else if ((M).sw == 1) K<T, 1><<<_g, 256, 0, st>>>(_mv, __VA_ARGS__);                 \
    else K<T, CSR_LANES><<<_g, 256, 0, st>>>(_mv, __VA_ARGS__);                          \
  } while (0)

// spectral-radius estimate of level l's operator D^-1/2 A D^-1/2 by `steps`
// power steps on the V-cycle's own (pre-scaled) copy, so the bounds come
// from the fastest form of the product (a15: Chebyshev bounds, Sec. 4)
int vh_power(Alloc& al, VHier<double>* m, int l, int steps, uint32_t tag, uint32_t seed, double* lam_dev) {
  using T = double;
  const Mat<T>& A = m->lev[l]->A;
  cudaStream_t st = al.stream;
  return run_power_op(al, m->lev[l]->n, steps, tag, seed, lam_dev, [&](const double* y, double* w) {
    LAUNCH_MAT(k_vc_spmv, A, st, y, w);
    SA_LAUNCHED();
    return SA_OK;
  });
}

template <typename T>
__global__ void k_coarse_in(int64_t n, const T* __restrict__ b, const double* __restrict__ sq,
                            double* __restrict__ t) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t[i] = sq[i] * (double)b[i];
}

template <typename T>
__global__ void k_coarse_out(int64_t n, const double* __restrict__ x, const double* __restrict__ sq,
                             T* __restrict__ xo) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xo[i] = (T)(sq[i] * x[i]);
}

// ---------------------------------------------------------------------------
// the cycle
// ---------------------------------------------------------------------------

#define PROFK(kind, level, bytes, launch)               \
  do {                                                  \
    int _pi = prof_begin(st, (kind), (level), (bytes)); \
    launch;                                             \
    prof_end(st, _pi);                                  \
    SA_LAUNCHED();                                      \
  } while (0)

template <typename T>
static int mv(VHier<T>* m, cudaStream_t st, int l, const double* r64, T** xo) {
  constexpr bool F64 = sizeof(T) == 8;
  const int K_CHEB = F64 ? PK_CHEB64 : PK_CHEB32, K_RES = F64 ? PK_RESID64 : PK_RESID32;
  const int K_RST = F64 ? PK_RESTRICT64 : PK_RESTRICT32, K_PRL = F64 ? PK_PROLONG64 : PK_PROLONG32;
  const int K_FST = F64 ? PK_FIRST64 : PK_FIRST32;
  const double S = sizeof(T);
  VLevel<T>* L = m->lev[l];
  const int nl = (int)m->lev.size();
  const int64_t n = L->n;
  if (l == nl - 1) {
    int pi = prof_begin(st, PK_COARSE, l, 8.0 * n * n + 48.0 * n);
    k_coarse_in<T><<<g256(n), 256, 0, st>>>(n, L->b.p, L->sq.p, m->ct.p);
    SA_LAUNCHED();
    SA_TRY(launch_coarse_solve(st, m->cf, m->ct.p, m->cs.p, m->cy.p, m->cx.p));
    k_coarse_out<T><<<g256(n), 256, 0, st>>>(n, m->cx.p, L->sq.p, L->x.p);
    prof_end(st, pi);
    SA_LAUNCHED();
    *xo = L->x.p;
    return SA_OK;
  }
  const int deg = m->deg;
  const double th = 0.5 * (L->lmax + L->lmin), de = 0.5 * (L->lmax - L->lmin);
  const double s1 = th / de;
  T* xa = L->x.p;
  T* xb = L->x2.p;
  const Mat<T>& A = L->A;
  if (l == 0) {
    PROFK(K_FST, l, 16.0 * n + 3.0 * S * n,
          (k_vc_fine_in<T><<<g256(n), 256, 0, st>>>(n, r64, m->s0.p, (T)(1.0 / th), L->b.p, xa, L->d.p)));
  } else {
    PROFK(K_FST, l, 3.0 * S * n, (k_vc_first<T><<<g256(n), 256, 0, st>>>(n, L->b.p, (T)(1.0 / th), xa, L->d.p)));
  }
  double rho = 1.0 / s1;
  for (int k = 1; k < deg; ++k) {
    double rn = 1.0 / (2.0 * s1 - rho);
    PROFK(K_CHEB, l, b_cheb(L),
          LAUNCH_MAT(k_vc_cheb, A, st, L->b.p, xa, xb, L->d.p, (T)(rn * rho), (T)(2.0 * rn / de), 0));
    T* t = xa; xa = xb; xb = t;
    rho = rn;
  }
  VLevel<T>* C = m->lev[l + 1];
  PROFK(K_RES, l, (S + b_idx(A)) * A.nnz + b_ptr(A) + 3.0 * S * n,
        LAUNCH_MAT(k_vc_residual, A, st, L->b.p, xa, L->r.p));
  PROFK(K_RST, l, (S + b_idx(L->R)) * L->R.nnz + b_ptr(L->R) + S * n + S * C->n,
        LAUNCH_MAT(k_vc_spmv, L->R, st, L->r.p, C->b.p));
  T* xc = nullptr;
  SA_TRY(mv(m, st, l + 1, nullptr, &xc));
  PROFK(K_PRL, l, (S + b_idx(L->P)) * L->P.nnz + b_ptr(L->P) + S * C->n + 2.0 * S * n,
        LAUNCH_MAT(k_vc_spmv_add, L->P, st, xc, xa));
  rho = 1.0 / s1;
  for (int k = 0; k < deg; ++k) {
    int first = (k == 0);
    T c1 = (T)0, c2 = (T)(1.0 / th);
    double rn = rho;
    if (!first) {
      rn = 1.0 / (2.0 * s1 - rho);
      c1 = (T)(rn * rho);
      c2 = (T)(2.0 * rn / de);
    }
    if (l == 0 && k == deg - 1) {
      PROFK(K_CHEB, l, b_cheb(L) + 16.0 * n - S * n,
            LAUNCH_MAT(k_vc_cheb_out, A, st, L->b.p, xa, L->d.p, c1, c2, first, m->s0.p, m->z.p));
    } else {
      PROFK(K_CHEB, l, b_cheb(L), LAUNCH_MAT(k_vc_cheb, A, st, L->b.p, xa, xb, L->d.p, c1, c2, first));
      T* t = xa; xa = xb; xb = t;
    }
    if (!first) rho = rn;
  }
  *xo = xa;
  return SA_OK;
}

template <typename T>
int vh_vcycle(VHier<T>* m, cudaStream_t st, const double* r, double** z) {
  if (m->lev.size() == 1) {
    // one level: the dense solve on r directly
    const int64_t n = m->lev[0]->n;
    int pi = prof_begin(st, PK_COARSE, 0, 8.0 * n * n + 32.0 * n);
    int s = launch_coarse_solve(st, m->cf, r, m->cs.p, m->cy.p, m->z.p);
    prof_end(st, pi);
    SA_TRY(s);
    *z = m->z.p;
    return SA_OK;
  }
  T* xo = nullptr;
  SA_TRY(mv<T>(m, st, 0, r, &xo));
  *z = m->z.p;
  return SA_OK;
}

template int vh_vcycle<double>(VHier<double>*, cudaStream_t, const double*, double**);
template int vh_vcycle<float>(VHier<float>*, cudaStream_t, const double*, double**);

template <typename T>
void vh_free(VHier<T>* m) {
  if (!m) return;
  for (VLevel<T>* L : m->lev) delete L;
  delete m;
}

template void vh_free<double>(VHier<double>*);
template void vh_free<float>(VHier<float>*);

// ---------------------------------------------------------------------------
// FP64 SELL kernels for the outer CG (unscaled fine operator)
// ---------------------------------------------------------------------------
// q = A p, partial sums of p.q per CTA (fixed order)
__global__ void k_sell_spmv_dot(int64_t n, const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                                const int32_t* __restrict__ base, const uint16_t* __restrict__ c16,
                                const double* __restrict__ v, const double* __restrict__ p, double* __restrict__ q,
                                double* __restrict__ part) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double c = 0.0;
  if (i < n) {
    double a = c16 ? sell_row16<double>(sp, base, c16, v, p, i) : sell_row<double>(sp, ci, v, p, i);
    q[i] = a;
    c = a * p[i];
  }
  c = warp_sum(c);
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = c;
  __syncthreads();
  if (w == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) part[blockIdx.x] = t;
  }
}

__global__ void k_sell_res64(int64_t n, const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                             const int32_t* __restrict__ base, const uint16_t* __restrict__ c16,
                             const double* __restrict__ v, const double* __restrict__ b,
                             const double* __restrict__ x, double* __restrict__ r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n)
    r[i] = b[i] - (c16 ? sell_row16<double>(sp, base, c16, v, x, i) : sell_row<double>(sp, ci, v, x, i));
}

int launch_sell_spmv_dot(cudaStream_t st, const Sell<double>& A, const double* p, double* q, double* part,
                         int* nparts) {
  *nparts = (int)g256(A.n);
  k_sell_spmv_dot<<<g256(A.n), 256, 0, st>>>(A.n, A.sp.p, A.ci.p, A.idx16 ? A.base.p : nullptr,
                                              A.idx16 ? A.c16.p : nullptr, A.v.p, p, q, part);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_sell_residual64(cudaStream_t st, const Sell<double>& A, const double* b, const double* x, double* r) {
  k_sell_res64<<<g256(A.n), 256, 0, st>>>(A.n, A.sp.p, A.ci.p, A.idx16 ? A.base.p : nullptr,
                                           A.idx16 ? A.c16.p : nullptr, A.v.p, b, x, r);
  SA_LAUNCHED();
  return SA_OK;
}


}  // namespace sa
