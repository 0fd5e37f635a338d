// Device helpers shared by the one- and multi-vector V-cycle kernels: the
// SELL-32 / CSR row products, the matrix view passed to the kernels and the
// Chebyshev row update (one definition, so both kernel families round alike).
#pragma once

#include "common.cuh"
#include "vcycle.cuh"

namespace sa {

// Row products of one thread: the entries of row i sit 32 apart inside its
// slice.  Several entries per iteration keep their value / column loads and
// gathers in flight together (the kernels are latency bound otherwise); the
// products are still added in entry order.  Values and
// columns are read once (evict-first loads), so the gathered x stays cached.
// entries per iteration: FP32 rows are latency bound and want more loads in
// flight; FP64 rows are bound by the FP64 pipe
template <typename T>
struct RowUnroll {
  static constexpr int U = sizeof(T) == 4 ? 8 : 4;
};

template <typename T, int U = RowUnroll<T>::U>
__device__ __forceinline__ T sell_row(const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                                      const T* __restrict__ v, const T* __restrict__ x, int64_t i) {
  const int64_t sl = i >> 5, r = i & 31;
  const int64_t b = sp[sl], e = sp[sl + 1];
  T acc = (T)0;
  int64_t p = b + r;
  for (; p + 32 * (U - 1) < e; p += 32 * U) {
    T vv[U], xx[U];
    int32_t cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      vv[u] = __ldcs(&v[p + 32 * u]);
      cc[u] = __ldcs(&ci[p + 32 * u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xx[u] = __ldg(&x[cc[u]]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc += vv[u] * xx[u];
  }
  for (; p < e; p += 32) acc += __ldcs(&v[p]) * __ldg(&x[__ldcs(&ci[p])]);
  return acc;
}

// compressed columns: x[base[slice] + offset]
template <typename T, int U = RowUnroll<T>::U>
__device__ __forceinline__ T sell_row16(const int64_t* __restrict__ sp, const int32_t* __restrict__ base,
                                        const uint16_t* __restrict__ c16, const T* __restrict__ v,
                                        const T* __restrict__ x, int64_t i) {
  const int64_t sl = i >> 5, r = i & 31;
  const int64_t b = sp[sl], e = sp[sl + 1];
  const T* __restrict__ xs = x + base[sl];
  T acc = (T)0;
  int64_t p = b + r;
  for (; p + 32 * (U - 1) < e; p += 32 * U) {
    T vv[U], xx[U];
    unsigned cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      vv[u] = __ldcs(&v[p + 32 * u]);
      cc[u] = __ldcs(&c16[p + 32 * u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xx[u] = __ldg(&xs[cc[u]]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc += vv[u] * xx[u];
  }
  for (; p < e; p += 32) acc += __ldcs(&v[p]) * __ldg(&xs[__ldcs(&c16[p])]);
  return acc;
}

// SELL-32 with two lanes per row: lanes 2r and 2r+1 of a warp take the even
// and the odd entries of row r of the slice (16 rows per warp), each summed in
// entry order; one shuffle adds the two
template <typename T, bool C16, int U = RowUnroll<T>::U>
__device__ __forceinline__ T sell2_lane(const int64_t* __restrict__ sp, const int32_t* __restrict__ base,
                                        const uint16_t* __restrict__ c16, const int32_t* __restrict__ ci,
                                        const T* __restrict__ v, const T* __restrict__ x, int64_t sl, int r, int h) {
  const int64_t b = sp[sl], e = sp[sl + 1];
  const T* __restrict__ xs = C16 ? x + base[sl] : x;
  T acc = (T)0;
  int64_t p = b + 32 * h + r;
  for (; p + 64 * (U - 1) < e; p += 64 * U) {
    T vv[U], xx[U];
    unsigned cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      vv[u] = __ldcs(&v[p + 64 * u]);
      cc[u] = C16 ? (unsigned)__ldcs(&c16[p + 64 * u]) : (unsigned)__ldcs(&ci[p + 64 * u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xx[u] = __ldg(&xs[cc[u]]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc += vv[u] * xx[u];
  }
  for (; p < e; p += 64) {
    const unsigned c = C16 ? (unsigned)__ldcs(&c16[p]) : (unsigned)__ldcs(&ci[p]);
    acc += __ldcs(&v[p]) * __ldg(&xs[c]);
  }
  return acc;
}

template <typename T>
struct MatView {
  int64_t n;
  const int64_t* p;  // SELL slice offsets or CSR row pointers
  const int32_t* ci;
  const T* v;
  const int32_t* base;   // compressed SELL columns (else NULL)
  const uint16_t* c16;
  // CSR long-row bin: rows with more than lt entries are listed in lrows and
  // taken by one warp each, in the first nlb blocks of the launch
  const int32_t* lrows;
  int64_t nlong;
  int64_t lt;
  unsigned nlb;
  // one-thread CSR rows: the launch order of the several-column kernels
  // (thread t takes row perm[t]; NULL: row t)
  const int32_t* perm;
};

// CSR storage of a V-cycle matrix: lanes per row; a row is in the long-row
// bin (a warp per row) above max(LONG_ROW, LONG_ROW_FACTOR x the mean row
// length) entries
constexpr int CSR_LANES = 4;
constexpr int64_t LONG_ROW = 64;
constexpr int64_t LONG_ROW_FACTOR = 4;
// CSR matrices with at most this many entries per row on average (the
// prolongators) take one thread per row
constexpr int64_t SHORT_ROW_MEAN = 8;
// their FP64 rows are taken by the several-column kernels grouped by length
// (0 .. ROW_ORDER_LEN - 2 entries, longer rows together) inside windows of
// ROW_ORDER_WIN consecutive rows, ascending row index within a length
constexpr int ROW_ORDER_WIN = 1024;
constexpr int ROW_ORDER_LEN = 16;
// SELL-32 matrices with fewer rows take two lanes per row (one thread per
// row leaves too few warps to cover the load latency)
constexpr int64_t SELL2_ROWS = int64_t(1) << 19;

// entries of one CSR lane loaded per round (added in entry order): rows
// of the regular bin, rows of the long-row bin
constexpr int CSR_UNROLL = 4;
constexpr int LONG_UNROLL = 8;

// the CSR lane sum of row i over entries b + sl, b + sl + W, ... (< e):
// U entries loaded per round, added in entry order
template <typename T, int W, int U>
__device__ __forceinline__ T csr_lane(const MatView<T>& M, const T* __restrict__ x, int64_t b, int64_t e, int sl) {
  T acc = (T)0;
  int64_t q = b + sl;
  for (; q + W * (U - 1) < e; q += W * U) {
    T vv[U], xx[U];
    int32_t cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      vv[u] = M.v[q + W * u];
      cc[u] = M.ci[q + W * u];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xx[u] = __ldg(&x[cc[u]]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc += vv[u] * xx[u];
  }
  for (; q < e; q += W) acc += M.v[q] * __ldg(&x[M.ci[q]]);
  return acc;
}

// blocks of 256 threads for nlong rows, a warp each
static inline unsigned long_blocks(int64_t nlong) { return blocks_for(nlong * 32, 256); }

template <typename T>
static MatView<T> view(const Mat<T>& M) {
  MatView<T> m;
  m.n = M.n;
  m.base = nullptr;
  m.c16 = nullptr;
  m.lrows = nullptr;
  m.nlong = 0;
  m.lt = INT64_MAX;
  m.nlb = 0;
  m.perm = nullptr;
  if (M.sw == 0) {
    m.p = M.sell.sp.p; m.ci = M.sell.ci.p; m.v = M.sell.v.p;
    if (M.sell.idx16) { m.base = M.sell.base.p; m.c16 = M.sell.c16.p; }
  } else {
    m.p = M.rp.p; m.ci = M.ci.p; m.v = M.v.p;
    if (M.sw == 1) m.perm = M.perm.p;
    if (M.nlong > 0) {
      m.lrows = M.lrows.p;
      m.nlong = M.nlong;
      m.lt = M.lt;
      m.nlb = long_blocks(M.nlong);
    }
  }
  return m;
}

// blocks of a launch: the long-row bin's, then the regular rows'
template <typename T>
static unsigned mat_grid(const Mat<T>& M) {
  const int64_t thr = M.sw == 0 ? (M.sell_lanes == 2 ? 64 * M.nslices : M.n) : M.n * (int64_t)M.sw;
  return blocks_for(thr, 256) + (M.sw != 0 && M.nlong > 0 ? long_blocks(M.nlong) : 0u);
}

// the row product of this thread's row; SW = 0: SELL-32, one thread per row;
// SW = -2: SELL-32, two lanes per row; SW > 0: CSR, SW lanes per row,
// reduced by shuffles (every lane of the warp reaches the shuffles), rows of
// the long-row bin by a warp each.  The sums do not depend on the unroll.
// Returns true for the thread that owns the row.
// row_apply_at takes the launch-local block index explicitly (blk), so a
// launch that covers several matrices one after another (the group solve)
// gives every row exactly the threads and arithmetic of its own launch.
template <typename T, int SW>
__device__ __forceinline__ bool row_apply_at(const MatView<T>& M, const T* __restrict__ x, T& out, int64_t& row,
                                             unsigned blk) {
  if constexpr (SW == -2) {
    const int64_t gt = (int64_t)blk * blockDim.x + threadIdx.x;
    const int64_t sl = gt >> 6;
    const int r = (int)((gt & 63) >> 1), h = (int)(gt & 1);
    const int64_t i = sl * 32 + r;
    row = i;
    T acc = (T)0;
    if (i < M.n)
      acc = M.c16 ? sell2_lane<T, true>(M.p, M.base, M.c16, M.ci, M.v, x, sl, r, h)
                  : sell2_lane<T, false>(M.p, M.base, M.c16, M.ci, M.v, x, sl, r, h);
    acc += __shfl_xor_sync(FULL, acc, 1);
    out = acc;
    return i < M.n && h == 0;
  } else if constexpr (SW == 0) {
    const int64_t gt = (int64_t)blk * blockDim.x + threadIdx.x;
    row = gt;
    if (gt >= M.n) return false;
    out = M.c16 ? sell_row16<T>(M.p, M.base, M.c16, M.v, x, gt) : sell_row<T>(M.p, M.ci, M.v, x, gt);
    return true;
  } else {
    if (blk < M.nlb) {
      // warp-uniform: one long row per warp
      const int64_t w = ((int64_t)blk * blockDim.x + threadIdx.x) >> 5;
      if (w >= M.nlong) return false;
      const int lane = (int)(threadIdx.x & 31);
      const int64_t i = M.lrows[w];
      row = i;
      T acc = csr_lane<T, 32, LONG_UNROLL>(M, x, M.p[i], M.p[i + 1], lane);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      out = acc;
      return lane == 0;
    }
    const int64_t gt = (int64_t)(blk - M.nlb) * blockDim.x + threadIdx.x;
    const int64_t i = gt / SW;
    const int sl = (int)(gt % SW);
    row = i;
    T acc = (T)0;
    bool own = false;
    if (i < M.n) {
      const int64_t b = M.p[i], e = M.p[i + 1];
      if (e - b <= M.lt) {
        own = sl == 0;
        acc = csr_lane<T, SW, CSR_UNROLL>(M, x, b, e, sl);
      }
    }
#pragma unroll
    for (int o = SW / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o, SW);
    out = acc;
    return own;
  }
}

template <typename T, int SW>
__device__ __forceinline__ bool row_apply(const MatView<T>& M, const T* __restrict__ x, T& out, int64_t& row) {
  return row_apply_at<T, SW>(M, x, out, row, blockIdx.x);
}

// Chebyshev direction d = first ? c2 r : c1 d + c2 r with r = b - y, written
// once and shared by the one- and multi-vector kernels (same rounding)
template <typename T>
__device__ __forceinline__ T cheb_dir(T b, T y, T d, T c1, T c2, int first) {
  const T r = b - y;
  return first ? c2 * r : fma(c1, d, c2 * r);
}

static inline unsigned g256(int64_t n) { return blocks_for(n, 256); }

}  // namespace sa
