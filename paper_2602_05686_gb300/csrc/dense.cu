// Coarsest level (Sec. 4: "the coarsest level is solved with a direct
// method").  A_L (n_L <= a few thousand) is densified and factored
// A_L = L L^T by a blocked right-looking Cholesky in FP64 (32 x 32 tiles);
// then W = L^-1 is formed by blocked forward substitution on the identity,
// so that every coarse solve is x = W^T (W b): two triangular matrix-vector
// products that use every SM, instead of two sequential triangular sweeps.
// W^T is stored explicitly so both products read contiguous rows.
#include <math.h>

#include "common.cuh"
#include "profile.cuh"
#include "solve.cuh"

namespace sa {

constexpr int NB = 32;

__global__ void k_densify(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ v, double* __restrict__ M) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) M[i * n + ci[p]] = v[p];
}

__global__ void k_set_identity(int64_t n, double* __restrict__ W) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * n) W[t] = (t / n == t % n) ? 1.0 : 0.0;
}

// factor the diagonal tile (k,k) in place (err = 1 on a non-positive pivot)
// and write the inverse of the factored tile, L_kk^-1 (lower triangular), to
// Dinv + k NB^2: the panel and inverse solves then become tile products
__global__ void k_potrf_diag(int64_t n, double* __restrict__ M, int k, int* __restrict__ err,
                             double* __restrict__ Dinv) {
  __shared__ double T[NB][NB + 1];
  __shared__ double rinv[NB];
  const int64_t o = (int64_t)k * NB;
  const int bs = (int)((n - o) < NB ? (n - o) : NB);
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    int r = t / NB, c = t % NB;
    T[r][c] = (r < bs && c < bs) ? M[(o + r) * n + o + c] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < bs; ++j) {
    if (threadIdx.x == 0) {
      double d = T[j][j];
      if (!(d > 0.0)) { atomicOr(err, 1); d = 1.0; }
      d = sqrt(d);
      T[j][j] = d;
      rinv[j] = 1.0 / d;
    }
    __syncthreads();
    const double ri = rinv[j];
    for (int r = j + 1 + threadIdx.x; r < bs; r += blockDim.x) T[r][j] *= ri;
    __syncthreads();
    const int m = bs - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      int r = j + 1 + t / m, c = j + 1 + t % m;
      if (c <= r) T[r][c] -= T[r][j] * T[c][j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < bs * bs; t += blockDim.x) {
    int r = t / bs, c = t % bs;
    M[(o + r) * n + o + c] = (c <= r) ? T[r][c] : 0.0;
  }
  // inverse by forward substitution, L y = e_c for every column c: eight
  // threads per column (one warp holds four columns) split each row's dot
  // product and combine it with shuffles
  __shared__ double Y[NB][NB + 1];
  {
    const int c = threadIdx.x >> 3, g = threadIdx.x & 7;
    for (int r = 0; r < NB; ++r) {
      double part = 0.0;
      if (r < bs && c < bs && r > c)
        for (int q = c + g; q < r; q += 8) part += T[r][q] * Y[q][c];
      part += __shfl_xor_sync(FULL, part, 4, 8);
      part += __shfl_xor_sync(FULL, part, 2, 8);
      part += __shfl_xor_sync(FULL, part, 1, 8);
      if (g == 0) {
        double y = 0.0;
        if (r < bs && c < bs && r >= c) y = ((r == c ? 1.0 : 0.0) - part) * rinv[r];
        Y[r][c] = y;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  double* D = Dinv + (int64_t)k * NB * NB;
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) D[t] = Y[t / NB][t % NB];
}

// L_ik = A_ik L_kk^-T for block rows i > k: a tile product with the stored
// L_kk^-1 (one CTA of 256 threads per block row, 4 outputs per thread)
__global__ void k_trsm_panel(int64_t n, double* __restrict__ M, int k, const double* __restrict__ Dinv) {
  __shared__ double Li[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  const int64_t ok = (int64_t)k * NB;
  const int bk = (int)((n - ok) < NB ? (n - ok) : NB);
  const int64_t oi = (int64_t)(k + 1 + blockIdx.x) * NB;
  const int bi = (int)((n - oi) < NB ? (n - oi) : NB);
  const double* D = Dinv + (int64_t)k * NB * NB;
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    int r = t / NB, c = t % NB;
    Li[r][c] = D[t];
    X[r][c] = (r < bi && c < bk) ? M[(oi + r) * n + ok + c] : 0.0;
  }
  __syncthreads();
  double out[NB * NB / 256];
#pragma unroll
  for (int u = 0; u < NB * NB / 256; ++u) {
    const int t = threadIdx.x + u * 256, r = t / NB, c = t % NB;
    double acc = 0.0;  // (L^-T)_qc = (L^-1)_cq, nonzero for q <= c
    for (int q = 0; q <= c; ++q) acc += X[r][q] * Li[c][q];
    out[u] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NB * NB / 256; ++u) {
    const int t = threadIdx.x + u * 256, r = t / NB, c = t % NB;
    if (r < bi && c < bk) M[(oi + r) * n + ok + c] = out[u];
  }
}

__device__ __forceinline__ void tri_index(int64_t idx, int* ti, int* tj) {
  // idx -> (ti, tj) with 0 <= tj <= ti, idx = ti (ti+1) / 2 + tj
  int t = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
  while ((int64_t)(t + 1) * (t + 2) / 2 <= idx) ++t;
  while ((int64_t)t * (t + 1) / 2 > idx) --t;
  *ti = t;
  *tj = (int)(idx - (int64_t)t * (t + 1) / 2);
}

// C -= A B^T on one NB x NB tile; 256 threads, 4 outputs each
__device__ __forceinline__ void tile_gemm_nt_sub(int64_t n, double* __restrict__ M, int64_t oc_r, int64_t oc_c,
                                                 int br, int bc, const double* __restrict__ Abase, int64_t oa_r,
                                                 int64_t oa_c, const double* __restrict__ Bbase, int64_t ob_r,
                                                 int64_t ob_c, int bkk, int64_t lda, int64_t ldb) {
  __shared__ double As[NB][NB + 1];
  __shared__ double Bs[NB][NB + 1];
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    int r = t / NB, c = t % NB;
    As[r][c] = (r < br && c < bkk) ? Abase[(oa_r + r) * lda + oa_c + c] : 0.0;
    Bs[r][c] = (r < bc && c < bkk) ? Bbase[(ob_r + r) * ldb + ob_c + c] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    int r = t / NB, c = t % NB;
    if (r < br && c < bc) {
      double s = 0.0;
#pragma unroll 8
      for (int m = 0; m < NB; ++m) s += As[r][m] * Bs[c][m];
      M[(oc_r + r) * n + oc_c + c] -= s;
    }
  }
}

// trailing update after panel k: A_ij -= L_ik L_jk^T for tiles first <= j <= i
// (col_only: the tiles of block column j = first only)
__global__ void k_syrk_update(int64_t n, double* __restrict__ M, int k, int first, int col_only) {
  int ti, tj;
  if (col_only) {
    ti = (int)blockIdx.x;
    tj = 0;
  } else {
    tri_index(blockIdx.x, &ti, &tj);
  }
  const int i = first + ti, j = first + tj;
  const int64_t oi = (int64_t)i * NB, oj = (int64_t)j * NB, ok = (int64_t)k * NB;
  const int bi = (int)((n - oi) < NB ? (n - oi) : NB);
  const int bj = (int)((n - oj) < NB ? (n - oj) : NB);
  const int bk = (int)((n - ok) < NB ? (n - ok) : NB);
  tile_gemm_nt_sub(n, M, oi, oj, bi, bj, M, oi, ok, M, oj, ok, bk, n, n);
}

// W_ij <- L_ii^-1 W_ij for block columns j <= i, a tile product with the
// stored L_ii^-1 (one CTA of 256 threads per j, 4 outputs per thread)
__global__ void k_trsm_lower_left(int64_t n, const double* __restrict__ Dinv, double* __restrict__ W, int i) {
  __shared__ double Li[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  const int j = blockIdx.x;
  const int64_t oi = (int64_t)i * NB, oj = (int64_t)j * NB;
  const int bi = (int)((n - oi) < NB ? (n - oi) : NB);
  const int bj = (int)((n - oj) < NB ? (n - oj) : NB);
  const double* D = Dinv + (int64_t)i * NB * NB;
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    int r = t / NB, c = t % NB;
    Li[r][c] = D[t];
    X[r][c] = (r < bi && c < bj) ? W[(oi + r) * n + oj + c] : 0.0;
  }
  __syncthreads();
  double out[NB * NB / 256];
#pragma unroll
  for (int u = 0; u < NB * NB / 256; ++u) {
    const int t = threadIdx.x + u * 256, r = t / NB, c = t % NB;
    double acc = 0.0;
    for (int q = 0; q <= r; ++q) acc += Li[r][q] * X[q][c];
    out[u] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NB * NB / 256; ++u) {
    const int t = threadIdx.x + u * 256, r = t / NB, c = t % NB;
    if (r < bi && c < bj) W[(oi + r) * n + oj + c] = out[u];
  }
}

// W_mj -= L_mi W_ij for block rows m >= m0 (m0 > i), j <= i
__global__ void k_gemm_left(int64_t n, const double* __restrict__ L, double* __restrict__ W, int i, int ncolb,
                            int m0) {
  const int m = m0 + blockIdx.x / ncolb;
  const int j = blockIdx.x % ncolb;
  const int64_t om = (int64_t)m * NB, oi = (int64_t)i * NB, oj = (int64_t)j * NB;
  const int bm = (int)((n - om) < NB ? (n - om) : NB);
  const int bi = (int)((n - oi) < NB ? (n - oi) : NB);
  const int bj = (int)((n - oj) < NB ? (n - oj) : NB);
  __shared__ double As[NB][NB + 1];
  __shared__ double Bs[NB][NB + 1];
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    int r = t / NB, c = t % NB;
    As[r][c] = (r < bm && c < bi) ? L[(om + r) * n + oi + c] : 0.0;   // L_mi
    Bs[r][c] = (r < bi && c < bj) ? W[(oi + r) * n + oj + c] : 0.0;   // W_ij
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    int r = t / NB, c = t % NB;
    if (r < bm && c < bj) {
      double s = 0.0;
#pragma unroll 8
      for (int q = 0; q < NB; ++q) s += As[r][q] * Bs[q][c];
      W[(om + r) * n + oj + c] -= s;
    }
  }
}

__global__ void k_transpose_dense(int64_t n, const double* __restrict__ W, double* __restrict__ WT) {
  __shared__ double t[32][33];
  int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  int x = threadIdx.x, y = threadIdx.y;
  for (int k = y; k < 32; k += 8) {
    int64_t r = by + k, c = bx + x;
    t[k][x] = (r < n && c < n) ? W[r * n + c] : 0.0;
  }
  __syncthreads();
  for (int k = y; k < 32; k += 8) {
    int64_t r = bx + k, c = by + x;
    if (r < n && c < n) WT[r * n + c] = t[x][k];
  }
}

DenseJob::~DenseJob() {
  // left without dense_finish (an error in between): the temporaries are
  // released on the caller's stream after this returns, so the dense
  // launches must have ended first
  if (pending) {
    if (sd) cudaStreamSynchronize(sd);
    if (s2) cudaStreamSynchronize(s2);
  }
  if (e_fork) cudaEventDestroy(e_fork);
  if (e_done) cudaEventDestroy(e_done);
  if (e_main) cudaEventDestroy(e_main);
  if (e_side) cudaEventDestroy(e_side);
  if (s2) cudaStreamDestroy(s2);   // pending work still completes
  if (sd) cudaStreamDestroy(sd);
}

int dense_start(Alloc& al, int64_t n, const int64_t* rp, const int32_t* ci, const double* v, Buf<double>& W,
                Buf<double>& WT, DenseJob& job) {
  cudaStream_t s = al.stream;
  job.main = s;
  job.n = n;
  if (n <= 0) return SA_OK;
  SA_TRY(job.M.alloc(&al, n * n));
  SA_TRY(W.alloc(&al, n * n));
  SA_TRY(WT.alloc(&al, n * n));
  SA_TRY(job.err.alloc(&al, 1));
  SA_TRY(memset_d(job.M.p, 0, job.M.bytes(), s));
  SA_TRY(memset_d(job.err.p, 0, sizeof(int), s));
  k_densify<<<blocks_for(n, 128), 128, 0, s>>>(n, rp, ci, v, job.M.p);
  SA_LAUNCHED();
  const int nb = (int)((n + NB - 1) / NB);
  SA_TRY(job.Dinv.alloc(&al, (int64_t)nb * NB * NB));
  // The factor runs on its own stream `sd`, forked from the caller's stream
  // after the dense copy; the caller goes on with work that does not read
  // W (Chebyshev bounds, SELL packing) and joins in dense_finish.  Within
  // it, look-ahead on a second stream: after panel k, `sd` updates only
  // block column k+1 and goes on to factor panel k+1, while `s2` updates
  // the rest of the trailing matrix (columns >= k+2); `sd` waits for that
  // before it updates column k+2.  The same for the inverse: row i+1 on `sd`,
  // rows >= i+2 on `s2`.  Without the extra streams everything runs on the
  // caller's stream in the same order.
  bool own = cudaStreamCreateWithFlags(&job.sd, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&job.e_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&job.e_done, cudaEventDisableTiming) == cudaSuccess;
  bool la = own && cudaStreamCreateWithFlags(&job.s2, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&job.e_main, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&job.e_side, cudaEventDisableTiming) == cudaSuccess;
  if (!la) cudaGetLastError();
  cudaStream_t m = s;
  if (own) {
    SA_CUDA(cudaEventRecord(job.e_fork, s));
    SA_CUDA(cudaStreamWaitEvent(job.sd, job.e_fork, 0));
    m = job.sd;
  }
  job.pending = own;
  cudaStream_t s2 = job.s2;
  double* M = job.M.p;
  double* D = job.Dinv.p;
  const int ph = prof_begin(m, PK_S_DENSE, job.level, 0.0);
  bool side_pending = false;
  for (int k = 0; k < nb; ++k) {
    k_potrf_diag<<<1, 256, 0, m>>>(n, M, k, job.err.p, D);
    count_launch();
    const int r = nb - k - 1;
    if (r > 0) {
      k_trsm_panel<<<r, 256, 0, m>>>(n, M, k, D);
      count_launch();
      if (la) {
        if (side_pending) SA_CUDA(cudaStreamWaitEvent(m, job.e_side, 0));
        k_syrk_update<<<r, 256, 0, m>>>(n, M, k, k + 1, 1);
        count_launch();
        if (r > 1) {
          SA_CUDA(cudaEventRecord(job.e_main, m));
          SA_CUDA(cudaStreamWaitEvent(s2, job.e_main, 0));
          k_syrk_update<<<(unsigned)((int64_t)(r - 1) * r / 2), 256, 0, s2>>>(n, M, k, k + 2, 0);
          count_launch();
          SA_CUDA(cudaEventRecord(job.e_side, s2));
          side_pending = true;
        } else {
          side_pending = false;
        }
      } else {
        k_syrk_update<<<(unsigned)((int64_t)r * (r + 1) / 2), 256, 0, m>>>(n, M, k, k + 1, 0);
        count_launch();
      }
    }
    SA_LAUNCHED();
  }
  if (la && side_pending) SA_CUDA(cudaStreamWaitEvent(m, job.e_side, 0));
  // W = L^-1 block row by block row.  A pivot that was not positive is
  // recorded in err and replaced by 1, so the inverse is computed on finite
  // data either way; dense_finish reports it.  The strict upper triangle of
  // M outside the diagonal tiles still holds A: W reads only the lower
  // triangle of L, so it is left as is.
  k_set_identity<<<blocks_for(n * n, 256), 256, 0, m>>>(n, W.p);
  count_launch();
  side_pending = false;
  for (int i = 0; i < nb; ++i) {
    k_trsm_lower_left<<<i + 1, 256, 0, m>>>(n, D, W.p, i);
    count_launch();
    const int r = nb - i - 1;
    if (r > 0) {
      if (la) {
        if (side_pending) SA_CUDA(cudaStreamWaitEvent(m, job.e_side, 0));
        k_gemm_left<<<(unsigned)(i + 1), 256, 0, m>>>(n, M, W.p, i, i + 1, i + 1);
        count_launch();
        if (r > 1) {
          SA_CUDA(cudaEventRecord(job.e_main, m));
          SA_CUDA(cudaStreamWaitEvent(s2, job.e_main, 0));
          k_gemm_left<<<(unsigned)((r - 1) * (i + 1)), 256, 0, s2>>>(n, M, W.p, i, i + 1, i + 2);
          count_launch();
          SA_CUDA(cudaEventRecord(job.e_side, s2));
          side_pending = true;
        } else {
          side_pending = false;
        }
      } else {
        k_gemm_left<<<(unsigned)(r * (i + 1)), 256, 0, m>>>(n, M, W.p, i, i + 1, i + 1);
        count_launch();
      }
    }
    SA_LAUNCHED();
  }
  if (la && side_pending) SA_CUDA(cudaStreamWaitEvent(m, job.e_side, 0));
  dim3 tb(32, 8), tg((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
  k_transpose_dense<<<tg, tb, 0, m>>>(n, W.p, WT.p);
  SA_LAUNCHED();
  prof_end(m, ph);
  if (own) SA_CUDA(cudaEventRecord(job.e_done, m));
  return SA_OK;
}

int dense_finish(DenseJob& job) {
  if (job.n <= 0) return SA_OK;
  if (job.pending) {
    SA_CUDA(cudaStreamWaitEvent(job.main, job.e_done, 0));
    job.pending = false;
  }
  int h_err = 0;
  SA_TRY(copy_d2h(&h_err, job.err.p, sizeof(int), job.main));
  return h_err ? SA_ERR_NOT_SPD : SA_OK;
}

// ---------------------------------------------------------------------------
// Coarse solve x = W^T (W b), W = L^-1 lower triangular (row-major), WT = W^T:
// y_i = sum_{j <= i} W_ij b_j, then x_j = sum_{i >= j} WT_ji y_i.  One CTA of
// TRI_WARPS warps per row: warp q takes the q-th of TRI_WARPS consecutive
// column segments of the row (segments of a multiple of 32 columns; lanes
// stride the segment with four loads in flight, each lane summing in column
// order; a shuffle tree adds the lanes), and the warps' sums are added in
// warp order.  A single warp per row left the longest rows (n entries) a
// chain of n/128 dependent load rounds.  The K-column forms run the same sums
// for every column as the one-column form (bitwise equal columns).
// ---------------------------------------------------------------------------
constexpr int TRI_WARPS = 4;

template <bool LOWER, int K>
__global__ void __launch_bounds__(TRI_WARPS * 32) k_tri_row(int64_t n, const double* __restrict__ M,
                                                            const double* __restrict__ v, double* __restrict__ out) {
  __shared__ double sh[TRI_WARPS][K];
  const int64_t i = blockIdx.x;
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  const int64_t lo = LOWER ? 0 : i, hi = LOWER ? i + 1 : n;
  const int64_t seg = (((hi - lo) + TRI_WARPS - 1) / TRI_WARPS + 31) & ~(int64_t)31;
  const int64_t b = lo + warp * seg;
  const int64_t e = b + seg < hi ? b + seg : hi;
  const double* __restrict__ Mi = M + i * n;
  double sum[K];
#pragma unroll
  for (int c = 0; c < K; ++c) sum[c] = 0.0;
  int64_t j = b + lane;
  for (; j + 96 < e; j += 128) {
    const double w0 = __ldcs(&Mi[j]), w1 = __ldcs(&Mi[j + 32]), w2 = __ldcs(&Mi[j + 64]), w3 = __ldcs(&Mi[j + 96]);
#pragma unroll
    for (int c = 0; c < K; ++c) {
      sum[c] += w0 * v[j * K + c];
      sum[c] += w1 * v[(j + 32) * K + c];
      sum[c] += w2 * v[(j + 64) * K + c];
      sum[c] += w3 * v[(j + 96) * K + c];
    }
  }
  for (; j < e; j += 32) {
    const double w = Mi[j];
#pragma unroll
    for (int c = 0; c < K; ++c) sum[c] += w * v[j * K + c];
  }
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const double t = warp_sum(sum[c]);
    if (lane == 0) sh[warp][c] = t;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    const int c = (int)threadIdx.x;
    double t = sh[0][c];
#pragma unroll
    for (int q = 1; q < TRI_WARPS; ++q) t += sh[q][c];
    out[i * K + c] = t;
  }
}

template <int K>
static int coarse_solve_k(cudaStream_t st, int64_t n, const double* W, const double* WT, const double* b, double* y,
                          double* x) {
  k_tri_row<true, K><<<(unsigned)n, TRI_WARPS * 32, 0, st>>>(n, W, b, y);
  SA_LAUNCHED();
  k_tri_row<false, K><<<(unsigned)n, TRI_WARPS * 32, 0, st>>>(n, WT, y, x);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_coarse_solve(cudaStream_t st, int64_t n, const double* W, const double* WT, const double* b, double* y,
                        double* x) {
  if (n <= 0) return SA_OK;
  return coarse_solve_k<1>(st, n, W, WT, b, y, x);
}

int launch_coarse_solve_block(cudaStream_t st, int64_t n, int k, const double* W, const double* WT, const double* b,
                              double* y, double* x) {
  if (n <= 0) return SA_OK;
  switch (k) {
    case 2: return coarse_solve_k<2>(st, n, W, WT, b, y, x);
    case 4: return coarse_solve_k<4>(st, n, W, WT, b, y, x);
    case 8: return coarse_solve_k<8>(st, n, W, WT, b, y, x);
    default: return SA_ERR_INVALID_ARG;
  }
}

}  // namespace sa
