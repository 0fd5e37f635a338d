// Iteration kernels: the power method on CSR matrices (sub-warp per row),
// fixed-order dot products, and the CG vector updates with device-resident
// scalars.  The V-cycle itself lives in vcycle.cu.
#include <math.h>

#include <functional>

#include "common.cuh"
#include "kernels.cuh"
#include "solve.cuh"

namespace sa {

// ---------------------------------------------------------------------------
// CSR row products with SW lanes per row (power method on the setup's CSR
// matrices); the result is valid in every lane of the group
// ---------------------------------------------------------------------------
#define ROW_SETUP(SW)                                                   \
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   \
  const int64_t i = gt / SW;                                            \
  const int sl = (int)(gt % SW);                                        \
  const bool valid = i < n;

// power method: y_j = s_j v_j with v_j = X_j * sc[4] (the previous product
// times the reciprocal of its norm; 1 for the start vector), formed once per
// step so that the product below costs one FP64 FMA per stored entry
__global__ void k_power_prep(int64_t n, const double* __restrict__ X, const double* __restrict__ s,
                             const double* __restrict__ sc, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = s ? s[i] * (X[i] * sc[4]) : X[i] * sc[4];  // s NULL: a pre-scaled operator
}

// w_i = s_i * sum_p a_p y_j
template <int SW>
__global__ void k_power_spmv(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, const double* __restrict__ s, const double* __restrict__ y,
                             double* __restrict__ w) {
  ROW_SETUP(SW)
  double acc = 0.0;
  if (valid) {
    const int64_t e = rp[i + 1];
    for (int64_t p = rp[i] + sl; p < e; p += SW) acc += v[p] * y[ci[p]];
  }
#pragma unroll
  for (int o = SW / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o, SW);
  if (valid && sl == 0) w[i] = s[i] * acc;
}

// ---------------------------------------------------------------------------
// fixed-order block reductions
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum_to(double (&val)[NV], double* __restrict__ out, int stride) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = warp_sum(val[k]);
    if (lane == 0) sh[k][w] = t;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sh[k][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) out[(int64_t)k * stride + blockIdx.x] = t;
    }
  }
}

// partial sums of up to three dot products over a fixed grid
__global__ void k_dots(int64_t n, const double* __restrict__ a0, const double* __restrict__ b0,
                       const double* __restrict__ a1, const double* __restrict__ b1, const double* __restrict__ a2,
                       const double* __restrict__ b2, double* __restrict__ part) {
  double acc[3] = {0.0, 0.0, 0.0};
  // two grid-stride elements per trip, their loads issued together and
  // added in the grid-stride order (the sums do not depend on the unroll)
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * st) {
    const int64_t j = i + st;
    const bool two = j < n;
    const double u0 = a0[i], v0 = b0[i], u1 = two ? a0[j] : 0.0, v1 = two ? b0[j] : 0.0;
    acc[0] = fma(u0, v0, acc[0]);
    if (two) acc[0] = fma(u1, v1, acc[0]);
    if (a1) {
      const double e0 = a1[i], f0 = b1[i], e1 = two ? a1[j] : 0.0, f1 = two ? b1[j] : 0.0;
      acc[1] = fma(e0, f0, acc[1]);
      if (two) acc[1] = fma(e1, f1, acc[1]);
    }
    if (a2) {
      const double e0 = a2[i], f0 = b2[i], e1 = two ? a2[j] : 0.0, f1 = two ? b2[j] : 0.0;
      acc[2] = fma(e0, f0, acc[2]);
      if (two) acc[2] = fma(e1, f1, acc[2]);
    }
  }
  block_sum_to<3>(acc, part, RED_BLOCKS);
}

// sums `np` partials of each of 3 dots in index order -> out[0..2]
__global__ void k_dots_finish(const double* __restrict__ part, int np, int stride, double* __restrict__ out) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < np; t += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] += part[(int64_t)k * stride + t];
  __shared__ double sh[3][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = warp_sum(acc[k]);
    if (lane == 0) sh[k][w] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int q = 0; q < nw; ++q) s += sh[k][q];
      out[k] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// power method (Sec. 2.2): spectral-radius estimate of diag(s) A diag(s)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fmix32_s(uint32_t h) {
  // MurmurHash3 32-bit finaliser (Appleby, public domain)
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__global__ void k_start_vector(int64_t n, uint32_t tag, uint32_t seed, double* __restrict__ v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    uint32_t h = fmix32_s((uint32_t)i ^ (0x7F4A7C15u * tag) ^ (seed * 0x2545F491u));
    double u = (double)h * (1.0 / 4294967296.0);
    v[i] = 2.0 * u - 1.0;
  }
}

// partial sums of w.w and v.v with v_j = X_j * sc[4]
__global__ void k_power_dots(int64_t n, const double* __restrict__ w, const double* __restrict__ X,
                             const double* __restrict__ sc, double* __restrict__ part) {
  const double inv = sc[4];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = X[i] * inv;
    acc[0] += w[i] * w[i];
    acc[1] += vi * vi;
  }
  block_sum_to<3>(acc, part, RED_BLOCKS);
}

// one CTA: sums the partials in index order, then lam = ||w|| / ||v||,
// sc[2] = ||w|| and sc[4] = 1 / ||w|| (the scale of the next iterate).  A zero product (every
// row unscaled) gives lam = 0 and stops the iteration (sc[3] = 1).
__global__ void k_power_finish(const double* __restrict__ part, double* __restrict__ sc, double* __restrict__ lam) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < RED_BLOCKS; t += blockDim.x)
#pragma unroll
    for (int k = 0; k < 2; ++k) acc[k] += part[(int64_t)k * RED_BLOCKS + t];
  __shared__ double sh[2][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    double t = warp_sum(acc[k]);
    if (lane == 0) sh[k][w] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ww = 0.0, vv = 0.0;
    for (int q = 0; q < nw; ++q) { ww += sh[0][q]; vv += sh[1][q]; }
    double nw2 = sqrt(ww);
    if (nw2 == 0.0 || sc[3] != 0.0) {
      sc[3] = 1.0;
      *lam = 0.0;
      return;
    }
    *lam = nw2 / sqrt(vv);
    sc[2] = nw2;
    sc[4] = 1.0 / nw2;
  }
}

__global__ void k_rsqrt_scale(int64_t n, const double* __restrict__ d, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = 1.0 / sqrt(d[i]);  // +inf -> 0
}

__global__ void k_reciprocal(int64_t n, const double* __restrict__ d, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = 1.0 / d[i];
}

__global__ void k_omega(const double* __restrict__ lam, double omega_sym, double* __restrict__ omega) {
  *omega = *lam > 0.0 ? omega_sym / *lam : 0.0;
}

int pick_sw(int64_t n, int64_t nnz) {
  double avg = n > 0 ? (double)nnz / (double)n : 1.0;
  if (avg <= 6) return 4;
  if (avg <= 40) return 8;
  if (avg <= 96) return 16;
  return 32;
}

#define DISPATCH_SW(sw, KERNEL, GRIDN, ...)                                                 \
  do {                                                                                       \
    const int _sw = (sw);                                                                    \
    const unsigned _g = blocks_for((GRIDN) * (int64_t)_sw, 256);                             \
    switch (_sw) {                                                                           \
      case 4: KERNEL<4><<<_g, 256, 0, st>>>(__VA_ARGS__); break;                             \
      case 8: KERNEL<8><<<_g, 256, 0, st>>>(__VA_ARGS__); break;                             \
      case 16: KERNEL<16><<<_g, 256, 0, st>>>(__VA_ARGS__); break;                           \
      default: KERNEL<32><<<_g, 256, 0, st>>>(__VA_ARGS__); break;                           \
    }                                                                                        \
  } while (0)

int launch_dots(cudaStream_t st, int64_t n, const double* a0, const double* b0, const double* a1,
                const double* b1, const double* a2, const double* b2, double* part, double* out) {
  k_dots<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, a0, b0, a1, b1, a2, b2, part);
  SA_LAUNCHED();
  k_dots_finish<<<1, 1024, 0, st>>>(part, RED_BLOCKS, RED_BLOCKS, out);
  SA_LAUNCHED();
  return SA_OK;
}

int run_power(Alloc& al, int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* s,
              int steps, uint32_t tag, uint32_t seed, double* lam_dev) {
  cudaStream_t st = al.stream;
  if (n <= 0) return SA_OK;
  Buf<double> x, w, y, part, sc;
  SA_TRY(x.alloc(&al, n));
  SA_TRY(w.alloc(&al, n));
  SA_TRY(y.alloc(&al, n));
  SA_TRY(part.alloc(&al, 3 * RED_BLOCKS));
  SA_TRY(sc.alloc(&al, 5));
  const double init[5] = {0.0, 0.0, 1.0, 0.0, 1.0};
  SA_CUDA(cudaMemcpyAsync(sc.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
  int64_t nnz = 0;
  SA_TRY(copy_d2h(&nnz, rp + n, sizeof(int64_t), st));
  const double avg = (double)nnz / (double)n;
  const int sw = avg <= 40.0 ? 4 : (avg <= 96.0 ? 8 : 16);
  k_start_vector<<<blocks_for(n, 256), 256, 0, st>>>(n, tag, seed, x.p);
  SA_LAUNCHED();
  double* X = x.p;  // previous product (the start vector at first)
  double* W = w.p;
  for (int it = 0; it < steps; ++it) {
    k_power_prep<<<blocks_for(n, 256), 256, 0, st>>>(n, X, s, sc.p, y.p);
    SA_LAUNCHED();
    DISPATCH_SW(sw, k_power_spmv, n, n, rp, ci, v, s, y.p, W);
    SA_LAUNCHED();
    k_power_dots<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, W, X, sc.p, part.p);
    SA_LAUNCHED();
    k_power_finish<<<1, 1024, 0, st>>>(part.p, sc.p, lam_dev);
    SA_LAUNCHED();
    double* t = X; X = W; W = t;
  }
  return SA_OK;
}

int run_power_op(Alloc& al, int64_t n, int steps, uint32_t tag, uint32_t seed, double* lam_dev,
                 const std::function<int(const double*, double*)>& apply) {
  cudaStream_t st = al.stream;
  if (n <= 0) return SA_OK;
  Buf<double> x, w, y, part, sc;
  SA_TRY(x.alloc(&al, n));
  SA_TRY(w.alloc(&al, n));
  SA_TRY(y.alloc(&al, n));
  SA_TRY(part.alloc(&al, 3 * RED_BLOCKS));
  SA_TRY(sc.alloc(&al, 5));
  const double init[5] = {0.0, 0.0, 1.0, 0.0, 1.0};
  SA_CUDA(cudaMemcpyAsync(sc.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
  k_start_vector<<<blocks_for(n, 256), 256, 0, st>>>(n, tag, seed, x.p);
  SA_LAUNCHED();
  double* X = x.p;
  double* W = w.p;
  for (int it = 0; it < steps; ++it) {
    k_power_prep<<<blocks_for(n, 256), 256, 0, st>>>(n, X, nullptr, sc.p, y.p);
    SA_LAUNCHED();
    SA_TRY(apply(y.p, W));
    k_power_dots<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, W, X, sc.p, part.p);
    SA_LAUNCHED();
    k_power_finish<<<1, 1024, 0, st>>>(part.p, sc.p, lam_dev);
    SA_LAUNCHED();
    double* t = X; X = W; W = t;
  }
  return SA_OK;
}

int launch_rsqrt_scale(cudaStream_t s, int64_t n, const double* d, double* out) {
  if (n <= 0) return SA_OK;
  k_rsqrt_scale<<<blocks_for(n, 256), 256, 0, s>>>(n, d, out);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_reciprocal(cudaStream_t s, int64_t n, const double* d, double* out) {
  if (n <= 0) return SA_OK;
  k_reciprocal<<<blocks_for(n, 256), 256, 0, s>>>(n, d, out);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_omega(cudaStream_t s, const double* lam_dev, double omega_sym, double* omega_dev) {
  k_omega<<<1, 1, 0, s>>>(lam_dev, omega_sym, omega_dev);
  SA_LAUNCHED();
  return SA_OK;
}

// ---------------------------------------------------------------------------
// CG with device-resident scalars (Sec. 4)
// ---------------------------------------------------------------------------
// alpha = rz / pq (pq = dots[0]); flags breakdown when pq <= 0 or NaN
__global__ void k_cg_alpha(CgScalars* __restrict__ s, const double* __restrict__ dots) {
  double pq = dots[0];
  s->pq = pq;
  if (!(pq > 0.0)) { s->breakdown = 1; s->alpha = 0.0; return; }
  s->alpha = s->rz / pq;
}

// x += alpha p; r -= alpha q; (r_prev = r before the update, if given);
// partial sums of r.r
__global__ void k_cg_update(int64_t n, const CgScalars* __restrict__ s, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                            double* __restrict__ rprev, double* __restrict__ part) {
  const double alpha = s->alpha;
  double acc[1] = {0.0};
  // two grid-stride elements per trip (loads together; r.r added in the
  // grid-stride order)
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * st) {
    const int64_t j = i + st;
    const bool two = j < n;
    double r0 = r[i];
    const double p0 = p[i], q0 = q[i], x0 = x[i];
    double r1 = 0.0, p1 = 0.0, q1 = 0.0, x1 = 0.0;
    if (two) {
      r1 = r[j];
      p1 = p[j];
      q1 = q[j];
      x1 = x[j];
    }
    if (rprev) {
      rprev[i] = r0;
      if (two) rprev[j] = r1;
    }
    x[i] = fma(alpha, p0, x0);
    r0 = fma(-alpha, q0, r0);
    r[i] = r0;
    acc[0] = fma(r0, r0, acc[0]);
    if (two) {
      x[j] = fma(alpha, p1, x1);
      r1 = fma(-alpha, q1, r1);
      r[j] = r1;
      acc[0] = fma(r1, r1, acc[0]);
    }
  }
  block_sum_to<1>(acc, part, 0);
}

// beta from the new r.z (and z.r_prev for flexible CG); flexible < 0
// initialises rz from dots[0]
__global__ void k_cg_beta(CgScalars* __restrict__ s, const double* __restrict__ dots, int flexible) {
  double rz_new = dots[0];
  if (flexible < 0) {
    s->rz = rz_new;
    s->beta = 0.0;
    s->breakdown = 0;
    return;
  }
  double num = flexible ? rz_new - dots[1] : rz_new;
  s->beta = num / s->rz;
  s->rz = rz_new;
}

__global__ void k_cg_pupdate(int64_t n, const CgScalars* __restrict__ s, const double* __restrict__ z,
                             double* __restrict__ p, int first) {
  const double beta = s->beta;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * st) {
    const int64_t j = i + st;
    const bool two = j < n;
    const double z0 = z[i], p0 = first ? 0.0 : p[i];
    const double z1 = two ? z[j] : 0.0, p1 = (two && !first) ? p[j] : 0.0;
    p[i] = first ? z0 : fma(beta, p0, z0);
    if (two) p[j] = first ? z1 : fma(beta, p1, z1);
  }
}

int launch_finish(cudaStream_t st, const double* part, int np, double* out) {
  k_dots_finish<<<1, 1024, 0, st>>>(part, np, 0, out);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_cg_alpha(cudaStream_t st, CgScalars* s, const double* dots) {
  k_cg_alpha<<<1, 1, 0, st>>>(s, dots);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_cg_update(cudaStream_t st, int64_t n, const CgScalars* s, const double* p, const double* q, double* x,
                     double* r, double* rprev, double* part) {
  k_cg_update<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, p, q, x, r, rprev, part);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_cg_beta(cudaStream_t st, CgScalars* s, const double* dots, int flexible) {
  k_cg_beta<<<1, 1, 0, st>>>(s, dots, flexible);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_cg_pupdate(cudaStream_t st, int64_t n, const CgScalars* s, const double* z, double* p, int first) {
  k_cg_pupdate<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, z, p, first);
  SA_LAUNCHED();
  return SA_OK;
}


// ---------------------------------------------------------------------------
// k-column CG (k independent solves in lockstep, interleaved n x k storage).
// Every column goes through the one-vector kernels' arithmetic in the same
// order (same grid, same per-thread stride, same reduction trees), so column
// c of a block solve equals the one-vector solve of that right-hand side.
// Columns that are done (converged, broken down) are frozen by `active`.
// ---------------------------------------------------------------------------
constexpr int KB = KMAX_BLOCK;

// Rows of an interleaved n x KK block move as whole vectors, in groups of
// G = 4 columns (one 256-bit access; rows on 32-byte boundaries) or G = 2
// (KK = 2: one 128-bit access).  Element-wise pieces at the row stride leave
// every warp store writing partial sectors.  The kernels keep the one-vector
// kernels' grid, per-thread stride and reduction trees (each column's
// arithmetic is theirs) and fit two 512-thread blocks per SM (64 registers):
// the per-column scalars are read from shared memory, not held.
template <int G>
__device__ __forceinline__ void ldgrp(const double* p, double (&v)[G]) {
  if constexpr (G == 4) {
    asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p) : "memory");
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  }
}
template <int G>
__device__ __forceinline__ void stgrp(double* p, const double (&v)[G]) {
  if constexpr (G == 4) {
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3]) : "memory");
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
}

// NV = KB: one dot per column (a1 unused); NV = 2 KB: two (a0.b0, a1.b1)
template <int KK, int NV>
__global__ void __launch_bounds__(RED_THREADS, 2) k_bdots(int64_t n, const double* __restrict__ a0,
                                                          const double* __restrict__ b0, const double* __restrict__ a1,
                                                          const double* __restrict__ b1, double* __restrict__ part) {
  constexpr int G = KK >= 4 ? 4 : 2;
  double acc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = i * KK;
#pragma unroll
    for (int g = 0; g < KK; g += G) {
      double a[G], b[G];
      ldgrp<G>(a0 + o + g, a);
      ldgrp<G>(b0 + o + g, b);
#pragma unroll
      for (int h = 0; h < G; ++h) acc[g + h] = fma(a[h], b[h], acc[g + h]);
      if constexpr (NV == 2 * KB) {
        ldgrp<G>(a1 + o + g, a);
        ldgrp<G>(b1 + o + g, b);
#pragma unroll
        for (int h = 0; h < G; ++h) acc[KB + g + h] = fma(a[h], b[h], acc[KB + g + h]);
      }
    }
  }
  block_sum_to<NV>(acc, part, RED_BLOCKS);
}

// out[v] = sum over np partials of value v (stride `stride`), in index order,
// with the reduction of k_dots_finish
template <int NV>
__global__ void k_bdots_finish(const double* __restrict__ part, int np, int stride, double* __restrict__ out) {
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += part[(int64_t)v * stride + t];
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double t = warp_sum(acc[v]);
    if (lane == 0) sh[v][w] = t;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += sh[threadIdx.x][q];
    out[threadIdx.x] = s;
  }
}

__global__ void k_bcg_alpha(int k, CgScalars* __restrict__ s, const double* __restrict__ dots,
                            const int* __restrict__ active) {
  const int c = threadIdx.x;
  if (c >= k) return;
  CgScalars& S = s[c];
  if (!active[c]) { S.alpha = 0.0; return; }
  const double pq = dots[c];
  S.pq = pq;
  if (!(pq > 0.0)) { S.breakdown = 1; S.alpha = 0.0; return; }
  S.alpha = S.rz / pq;
}

template <int KK>
__global__ void __launch_bounds__(RED_THREADS, 2)
    k_bcg_update(const int64_t n, const CgScalars* __restrict__ s, const int* __restrict__ active,
                 const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                 double* __restrict__ r, double* __restrict__ rprev, double* __restrict__ part) {
  constexpr int G = KK >= 4 ? 4 : 2;
  __shared__ double alpha[KB];
  __shared__ int on[KB];
  if (threadIdx.x < KB) {
    const int c = threadIdx.x;
    on[c] = c < KK && active[c];
    alpha[c] = c < KK ? s[c].alpha : 0.0;
  }
  __syncthreads();
  bool any = false;
#pragma unroll
  for (int c = 0; c < KK; ++c) any |= on[c] != 0;
  double acc[KB];
#pragma unroll
  for (int c = 0; c < KB; ++c) acc[c] = 0.0;
  // each column updated and summed exactly as in the one-vector kernel; a
  // frozen column's values are written back unchanged
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = i * KK;
#pragma unroll
    for (int g = 0; g < KK; g += G) {
      // r with q, then x with p: two groups live at a time
      double rv[G];
      ldgrp<G>(r + o + g, rv);
      if (any) {
        double u[G], v[G];
        if (rprev) stgrp<G>(rprev + o + g, rv);
        ldgrp<G>(q + o + g, u);
#pragma unroll
        for (int h = 0; h < G; ++h)
          if (on[g + h]) rv[h] = fma(-alpha[g + h], u[h], rv[h]);
        stgrp<G>(r + o + g, rv);
        ldgrp<G>(x + o + g, u);
        ldgrp<G>(p + o + g, v);
#pragma unroll
        for (int h = 0; h < G; ++h)
          if (on[g + h]) u[h] = fma(alpha[g + h], v[h], u[h]);
        stgrp<G>(x + o + g, u);
      }
#pragma unroll
      for (int h = 0; h < G; ++h) acc[g + h] = fma(rv[h], rv[h], acc[g + h]);
    }
  }
  block_sum_to<KB>(acc, part, RED_BLOCKS);
}

__global__ void k_bcg_beta(int k, CgScalars* __restrict__ s, const double* __restrict__ dots, int flexible,
                           const int* __restrict__ active) {
  const int c = threadIdx.x;
  if (c >= k || !active[c]) return;
  CgScalars& S = s[c];
  const double rz_new = dots[c];
  if (flexible < 0) {
    S.rz = rz_new;
    S.beta = 0.0;
    S.breakdown = 0;
    return;
  }
  const double num = flexible ? rz_new - dots[KB + c] : rz_new;
  S.beta = num / S.rz;
  S.rz = rz_new;
}

template <int KK>
__global__ void __launch_bounds__(RED_THREADS, 2)
    k_bcg_pupdate(int64_t n, const CgScalars* __restrict__ s, const int* __restrict__ active,
                  const double* __restrict__ z, double* __restrict__ p, int first) {
  constexpr int G = KK >= 4 ? 4 : 2;
  __shared__ double beta[KB];
  __shared__ int on[KB];
  if (threadIdx.x < KB) {
    const int c = threadIdx.x;
    on[c] = c < KK && active[c];
    beta[c] = c < KK ? s[c].beta : 0.0;
  }
  __syncthreads();
  bool any = false;
#pragma unroll
  for (int c = 0; c < KK; ++c) any |= on[c] != 0;
  if (!any) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = i * KK;
#pragma unroll
    for (int g = 0; g < KK; g += G) {
      double zv[G], pv[G];
      ldgrp<G>(z + o + g, zv);
      ldgrp<G>(p + o + g, pv);
#pragma unroll
      for (int h = 0; h < G; ++h)
        if (on[g + h]) pv[h] = first ? zv[h] : fma(beta[g + h], pv[h], zv[h]);
      stgrp<G>(p + o + g, pv);
    }
  }
}

// column-major n x k <-> interleaved n x K (columns k..K-1 of the block are zero)
__global__ void k_interleave(int64_t n, int k, int K, const double* __restrict__ src, double* __restrict__ dst,
                             int to_interleaved) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * K) return;
  const int64_t i = e / K;
  const int c = (int)(e % K);
  if (to_interleaved) dst[e] = c < k ? src[(int64_t)c * n + i] : 0.0;
  else if (c < k) dst[(int64_t)c * n + i] = src[e];
}

int launch_bdots(cudaStream_t st, int64_t n, int k, const double* a0, const double* b0, const double* a1,
                 const double* b1, double* part, double* out) {
  if (k != 2 && k != 4 && k != 8) return SA_ERR_INVALID_ARG;  // whole-row vectors
  // one dot per column, or two (a1 . b1 into out[KB + c])
  if (a1) {
    if (k == 2) k_bdots<2, 2 * KB><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, a0, b0, a1, b1, part);
    else if (k == 4) k_bdots<4, 2 * KB><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, a0, b0, a1, b1, part);
    else k_bdots<8, 2 * KB><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, a0, b0, a1, b1, part);
    SA_LAUNCHED();
    k_bdots_finish<2 * KB><<<1, 1024, 0, st>>>(part, RED_BLOCKS, RED_BLOCKS, out);
  } else {
    if (k == 2) k_bdots<2, KB><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, a0, b0, a1, b1, part);
    else if (k == 4) k_bdots<4, KB><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, a0, b0, a1, b1, part);
    else k_bdots<8, KB><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, a0, b0, a1, b1, part);
    SA_LAUNCHED();
    k_bdots_finish<KB><<<1, 1024, 0, st>>>(part, RED_BLOCKS, RED_BLOCKS, out);
  }
  SA_LAUNCHED();
  return SA_OK;
}

// partials laid out as part[c * np + b] (c < KB)
int launch_bfinish(cudaStream_t st, const double* part, int np, int k, double* out) {
  if (k < 1 || k > KB) return SA_ERR_INVALID_ARG;
  k_bdots_finish<KB><<<1, 1024, 0, st>>>(part, np, np, out);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_bcg_alpha(cudaStream_t st, int k, CgScalars* s, const double* dots, const int* active) {
  k_bcg_alpha<<<1, 32, 0, st>>>(k, s, dots, active);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_bcg_update(cudaStream_t st, int64_t n, int k, const CgScalars* s, const int* active, const double* p,
                      const double* q, double* x, double* r, double* rprev, double* part) {
  if (k != 2 && k != 4 && k != 8) return SA_ERR_INVALID_ARG;  // whole-row vectors
  if (k == 2) k_bcg_update<2><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, active, p, q, x, r, rprev, part);
  else if (k == 4) k_bcg_update<4><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, active, p, q, x, r, rprev, part);
  else k_bcg_update<8><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, active, p, q, x, r, rprev, part);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_bcg_beta(cudaStream_t st, int k, CgScalars* s, const double* dots, int flexible, const int* active) {
  k_bcg_beta<<<1, 32, 0, st>>>(k, s, dots, flexible, active);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_bcg_pupdate(cudaStream_t st, int64_t n, int k, const CgScalars* s, const int* active, const double* z,
                       double* p, int first) {
  if (k != 2 && k != 4 && k != 8) return SA_ERR_INVALID_ARG;  // whole-row vectors
  if (k == 2) k_bcg_pupdate<2><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, active, z, p, first);
  else if (k == 4) k_bcg_pupdate<4><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, active, z, p, first);
  else k_bcg_pupdate<8><<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, s, active, z, p, first);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_interleave(cudaStream_t st, int64_t n, int k, int K, const double* src, double* dst, int to_interleaved) {
  if (n * K <= 0) return SA_OK;
  k_interleave<<<blocks_for(n * K, 256), 256, 0, st>>>(n, k, K, src, dst, to_interleaved);
  SA_LAUNCHED();
  return SA_OK;
}

}  // namespace sa
