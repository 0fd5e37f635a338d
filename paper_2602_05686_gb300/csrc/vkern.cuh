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

template <typename T>
__device__ __forceinline__ T sell_row(const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                                      const T* __restrict__ v, const T* __restrict__ x, int64_t i) {
  constexpr int U = RowUnroll<T>::U;
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
template <typename T>
__device__ __forceinline__ T sell_row16(const int64_t* __restrict__ sp, const int32_t* __restrict__ base,
                                        const uint16_t* __restrict__ c16, const T* __restrict__ v,
                                        const T* __restrict__ x, int64_t i) {
  constexpr int U = RowUnroll<T>::U;
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

template <typename T>
struct MatView {
  int64_t n;
  const int64_t* p;  // SELL slice offsets or CSR row pointers
  const int32_t* ci;
  const T* v;
  const int32_t* base;   // compressed SELL columns (else NULL)
  const uint16_t* c16;
};

template <typename T>
static MatView<T> view(const Mat<T>& M) {
  MatView<T> m;
  m.n = M.n;
  m.base = nullptr;
  m.c16 = nullptr;
  if (M.sw == 0) {
    m.p = M.sell.sp.p; m.ci = M.sell.ci.p; m.v = M.sell.v.p;
    if (M.sell.idx16) { m.base = M.sell.base.p; m.c16 = M.sell.c16.p; }
  } else {
    m.p = M.rp.p; m.ci = M.ci.p; m.v = M.v.p;
  }
  return m;
}

// the row product of this thread's row; SW = 0: SELL-32, one thread per row;
// SW > 0: CSR, SW lanes per row, reduced by shuffles (every lane of the warp
// reaches the shuffles).  Returns true for the thread that owns the row.
template <typename T, int SW>
__device__ __forceinline__ bool row_apply(const MatView<T>& M, const T* __restrict__ x, T& out, int64_t& row) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (SW == 0) {
    row = gt;
    if (gt >= M.n) return false;
    out = M.c16 ? sell_row16<T>(M.p, M.base, M.c16, M.v, x, gt) : sell_row<T>(M.p, M.ci, M.v, x, gt);
    return true;
  } else {
    const int64_t i = gt / SW;
    const int sl = (int)(gt % SW);
    row = i;
    T acc = (T)0;
    if (i < M.n) {
      const int64_t e = M.p[i + 1];
      for (int64_t q = M.p[i] + sl; q < e; q += SW) acc += M.v[q] * __ldg(&x[M.ci[q]]);
    }
#pragma unroll
    for (int o = SW / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o, SW);
    out = acc;
    return i < M.n && sl == 0;
  }
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
