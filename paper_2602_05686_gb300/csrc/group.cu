// Kernels of the group solve (see group.cuh): the V-cycle's matrix-row and
// elementwise kernels and the outer CG kernels, each covering several
// problems in one launch.  Every kernel body repeats the arithmetic of its
// one-problem counterpart (vcycle.cu, solve.cu) with the launch-local block
// index of the segment, so the results are the one-problem results bit for
// bit.
#include "group.cuh"

namespace sa {

// the segment of this block: the last descriptor whose blk0 <= blockIdx.x
template <typename D>
__device__ __forceinline__ int seg_of(const D* __restrict__ d, int m) {
  __shared__ int s_seg;
  if (threadIdx.x == 0) {
    int lo = 0, hi = m - 1;
    const uint32_t b = blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (d[mid].blk0 <= b) lo = mid;
      else hi = mid - 1;
    }
    s_seg = lo;
  }
  __syncthreads();
  return s_seg;
}

// ---------------------------------------------------------------------------
// V-cycle: matrix-row kernels
// ---------------------------------------------------------------------------
template <typename T, int SW>
__device__ __forceinline__ void g_mat_row(int op, const GMat<T>& D, unsigned blk) {
  T y;
  int64_t i;
  switch (op) {
    case GM_CHEB: {
      if (!row_apply_at<T, SW>(D.M, D.xin, y, i, blk)) return;
      const T dn = cheb_dir<T>(D.b[i], y, D.first ? (T)0 : D.d[i], D.c1, D.c2, D.first);
      D.d[i] = dn;
      D.xout[i] = D.xin[i] + dn;
      return;
    }
    case GM_CHEB_OUT: {
      if (!row_apply_at<T, SW>(D.M, D.xin, y, i, blk)) return;
      const T dn = cheb_dir<T>(D.b[i], y, D.first ? (T)0 : D.d[i], D.c1, D.c2, D.first);
      D.z[i] = D.s[i] * (double)(D.xin[i] + dn);
      return;
    }
    case GM_RESID:
      if (row_apply_at<T, SW>(D.M, D.xin, y, i, blk)) D.r[i] = D.b[i] - y;
      return;
    case GM_SPMV:
      if (row_apply_at<T, SW>(D.M, D.xin, y, i, blk)) D.xout[i] = y;
      return;
    default:  // GM_SPMV_ADD
      if (row_apply_at<T, SW>(D.M, D.xin, y, i, blk)) D.xout[i] += y;
      return;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_g_mat(int op, const GMat<T>* __restrict__ d, int m) {
  const int k = seg_of(d, m);
  const GMat<T> D = d[k];
  const unsigned blk = blockIdx.x - D.blk0;
  // block-uniform branch: every thread of a block takes the same format
  switch (D.fmt) {
    case -2: g_mat_row<T, -2>(op, D, blk); break;
    case 0: g_mat_row<T, 0>(op, D, blk); break;
    case 1: g_mat_row<T, 1>(op, D, blk); break;
    default: g_mat_row<T, CSR_LANES>(op, D, blk); break;
  }
}

// ---------------------------------------------------------------------------
// V-cycle: elementwise kernels (blocks of 256, one element per thread)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_g_vec(int op, const GVec<T>* __restrict__ d, int m) {
  const int k = seg_of(d, m);
  const GVec<T>& D = d[k];
  const int64_t i = (int64_t)(blockIdx.x - D.blk0) * blockDim.x + threadIdx.x;
  if (i >= D.n) return;
  switch (op) {
    case GV_FINE_IN: {
      T bi = (T)(D.s[i] * D.r64[i]);
      D.b[i] = bi;
      T dn = D.c2 * bi;
      D.d[i] = dn;
      D.x[i] = dn;
      return;
    }
    case GV_FIRST: {
      T dn = D.c2 * D.b[i];
      D.d[i] = dn;
      D.x[i] = dn;
      return;
    }
    case GV_COARSE_IN:
      D.t[i] = D.s[i] * (double)D.b[i];
      return;
    default:  // GV_COARSE_OUT
      D.x[i] = (T)(D.s[i] * D.t[i]);
      return;
  }
}

template <typename T>
int launch_g_mat(cudaStream_t st, int op, const GMat<T>* d, int m, unsigned blocks) {
  if (m <= 0 || blocks == 0) return SA_OK;
  k_g_mat<T><<<blocks, 256, 0, st>>>(op, d, m);
  SA_LAUNCHED();
  return SA_OK;
}

template <typename T>
int launch_g_vec(cudaStream_t st, int op, const GVec<T>* d, int m, unsigned blocks) {
  if (m <= 0 || blocks == 0) return SA_OK;
  k_g_vec<T><<<blocks, 256, 0, st>>>(op, d, m);
  SA_LAUNCHED();
  return SA_OK;
}

template int launch_g_mat<double>(cudaStream_t, int, const GMat<double>*, int, unsigned);
template int launch_g_mat<float>(cudaStream_t, int, const GMat<float>*, int, unsigned);
template int launch_g_vec<double>(cudaStream_t, int, const GVec<double>*, int, unsigned);
template int launch_g_vec<float>(cudaStream_t, int, const GVec<float>*, int, unsigned);

// ---------------------------------------------------------------------------
// outer CG (FP64), the kernels of solve.cu / vcycle.cu per problem
// ---------------------------------------------------------------------------
// fixed-order block sum of NV values (the one-problem block_sum_to, with the
// output slot blk instead of blockIdx.x)
template <int NV>
__device__ __forceinline__ void g_block_sum_to(double (&val)[NV], double* __restrict__ out, int stride,
                                               unsigned blk) {
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
      if (lane == 0) out[(int64_t)k * stride + blk] = t;
    }
  }
}

__device__ __forceinline__ double g_sell_row(const GCg& D, const double* __restrict__ x, int64_t i) {
  return D.c16 ? sell_row16<double>(D.sp, D.base, D.c16, D.v, x, i) : sell_row<double>(D.sp, D.ci, D.v, x, i);
}

// rows geometry (blocks of 256): residual, operator product with p.q partials
__global__ void __launch_bounds__(256) k_g_cg_rows(int op, const GCg* __restrict__ d, int m) {
  const int k = seg_of(d, m);
  const GCg& D = d[k];
  const unsigned blk = blockIdx.x - D.blk0;
  const int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
  if (op == GC_RESID) {
    if (i < D.n) D.out[i] = D.bvec[i] - g_sell_row(D, D.in, i);
    return;
  }
  double c = 0.0;
  if (i < D.n) {
    double a = g_sell_row(D, D.in, i);
    D.out[i] = a;
    c = a * D.in[i];
  }
  c = warp_sum(c);
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = c;
  __syncthreads();
  if (w == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) D.part[blk] = t;
  }
}

// reduction geometry (RED_BLOCKS blocks of RED_THREADS per problem)
__global__ void __launch_bounds__(RED_THREADS) k_g_cg_red(int op, const GCg* __restrict__ d) {
  const int k = (int)(blockIdx.x / RED_BLOCKS);
  const unsigned blk = blockIdx.x % RED_BLOCKS;
  const GCg& D = d[k];
  const int64_t n = D.n;
  const int64_t stride = (int64_t)RED_BLOCKS * blockDim.x;
  if (op == GC_DOTS) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < n; i += stride) {
      acc[0] = fma(D.a0[i], D.b0[i], acc[0]);
      if (D.a1) acc[1] = fma(D.a1[i], D.b1[i], acc[1]);
    }
    g_block_sum_to<3>(acc, D.part, RED_BLOCKS, blk);
  } else if (op == GC_UPDATE) {
    const double alpha = D.cg->alpha;
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < n; i += stride) {
      double ri = D.r[i];
      if (D.rprev) D.rprev[i] = ri;
      D.x[i] = fma(alpha, D.p[i], D.x[i]);
      ri = fma(-alpha, D.q[i], ri);
      D.r[i] = ri;
      acc[0] = fma(ri, ri, acc[0]);
    }
    g_block_sum_to<1>(acc, D.part, 0, blk);
  } else {  // GC_PUPDATE
    const double beta = D.cg->beta;
    for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < n; i += stride)
      D.out[i] = D.first ? D.in[i] : fma(beta, D.out[i], D.in[i]);
  }
}

// one block of 1024 per problem: the partial sums in index order
__global__ void __launch_bounds__(1024) k_g_cg_finish(const GCg* __restrict__ d) {
  const GCg& D = d[blockIdx.x];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < D.np; t += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] += D.part[(int64_t)k * D.stride + t];
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
      D.dots[k] = s;
    }
  }
}

// one thread per problem: alpha, beta, the host gather
__global__ void k_g_cg_scalar(int op, const GCg* __restrict__ d, int m) {
  const int k = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (k >= m) return;
  const GCg& D = d[k];
  CgScalars* s = D.cg;
  if (op == GC_ALPHA) {
    double pq = D.dots[0];
    s->pq = pq;
    if (!(pq > 0.0)) { s->breakdown = 1; s->alpha = 0.0; return; }
    s->alpha = s->rz / pq;
  } else if (op == GC_BETA) {
    double rz_new = D.dots[0];
    if (D.flexible < 0) {
      s->rz = rz_new;
      s->beta = 0.0;
      s->breakdown = 0;
      return;
    }
    double num = D.flexible ? rz_new - D.dots[1] : rz_new;
    s->beta = num / s->rz;
    s->rz = rz_new;
  } else {  // GC_GATHER
    D.gather[2 * k] = D.dots[0];
    D.gather[2 * k + 1] = (double)s->breakdown;
  }
}

int launch_g_cg(cudaStream_t st, int op, const GCg* d, int m, unsigned blocks) {
  if (m <= 0) return SA_OK;
  switch (op) {
    case GC_RESID:
    case GC_SPMV_DOT:
      if (blocks == 0) return SA_OK;
      k_g_cg_rows<<<blocks, 256, 0, st>>>(op, d, m);
      break;
    case GC_DOTS:
    case GC_UPDATE:
    case GC_PUPDATE:
      k_g_cg_red<<<(unsigned)m * RED_BLOCKS, RED_THREADS, 0, st>>>(op, d);
      break;
    case GC_FINISH:
      k_g_cg_finish<<<(unsigned)m, 1024, 0, st>>>(d);
      break;
    default:
      k_g_cg_scalar<<<1, GROUP_MAX, 0, st>>>(op, d, m);
      break;
  }
  SA_LAUNCHED();
  return SA_OK;
}

}  // namespace sa
