// Coarsest level (Sec. 4: the coarsest level is solved directly).  A_L
// (n_L <= a few thousand) is densified and factored A_L = L L^T by a blocked
// right-looking Cholesky in FP64 (32 x 32 tiles); then the inverses of the
// diagonal blocks of COARSE_BS rows, W_KK = L_KK^-1, are formed by blocked
// forward substitution on the identity.  Every coarse solve is block
// substitution: per diagonal block a row-parallel product with the blocks
// already solved and one with W_KK (forward with L, backward with L^T and
// W_KK^T), so it uses every SM instead of running row-by-row sweeps.  L^T and
// W^T are stored explicitly so all products read contiguous rows.
#include <math.h>

#include "common.cuh"
#include "profile.cuh"
#include "group.cuh"
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
    // thread (warp w, lane r) owns T[r][w + 8q], q = 0..3 (256 threads)
    {
      const int r = (int)(threadIdx.x & 31), w = (int)(threadIdx.x >> 5);
      if (r > j && r < bs) {
        const double lrj = T[r][j];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = w + 8 * q;
          if (c > j && c <= r) T[r][c] -= lrj * T[c][j];
        }
      }
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

// W_ij <- L_ii^-1 W_ij for block columns j0 <= j <= i, a tile product with
// the stored L_ii^-1 (one CTA of 256 threads per j, 4 outputs per thread)
__global__ void k_trsm_lower_left(int64_t n, const double* __restrict__ Dinv, double* __restrict__ W, int i,
                                  int j0) {
  __shared__ double Li[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  const int j = j0 + (int)blockIdx.x;
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

// W_mj -= L_mi W_ij for block rows m >= m0 (m0 > i), block columns
// j0 <= j < j0 + ncolb (j <= i)
__global__ void k_gemm_left(int64_t n, const double* __restrict__ L, double* __restrict__ W, int i, int ncolb,
                            int m0, int j0) {
  const int m = m0 + (int)blockIdx.x / ncolb;
  const int j = j0 + (int)blockIdx.x % ncolb;
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

int dense_start(Alloc& al, int64_t n, const int64_t* rp, const int32_t* ci, const double* v, CoarseFactor& F,
                DenseJob& job) {
  cudaStream_t s = al.stream;
  job.main = s;
  job.n = n;
  if (n <= 0) return SA_OK;
  SA_TRY(F.L.alloc(&al, n * n));
  SA_TRY(F.LT.alloc(&al, n * n));
  SA_TRY(F.W.alloc(&al, n * n));
  SA_TRY(F.WT.alloc(&al, n * n));
  SA_TRY(job.err.alloc(&al, 1));
  SA_TRY(memset_d(F.L.p, 0, F.L.bytes(), s));
  SA_TRY(memset_d(job.err.p, 0, sizeof(int), s));
  k_densify<<<blocks_for(n, 128), 128, 0, s>>>(n, rp, ci, v, F.L.p);
  SA_LAUNCHED();
  const int nb = (int)((n + NB - 1) / NB);
  SA_TRY(job.Dinv.alloc(&al, (int64_t)nb * NB * NB));
  // The factor runs on its own stream `sd`, forked from the caller's stream
  // after the dense copy; the caller goes on with work that does not read
  // the factor (Chebyshev bounds, SELL packing) and joins in dense_finish.
  // Within it, look-ahead on a second stream: after panel k, `sd` updates
  // only block column k+1 and goes on to factor panel k+1, while `s2`
  // updates the rest of the trailing matrix (columns >= k+2); `sd` waits for
  // that before it updates column k+2.  The same for the diagonal-block
  // inverses: row i+1 on `sd`, rows >= i+2 of the same diagonal block on
  // `s2`.  Without the extra streams everything runs on the caller's stream
  // in the same order.
  // Both streams get the highest priority: the factor is the setup's
  // critical path (a chain of small panel launches), the work it overlaps
  // has slack, and the block scheduler then hands free SM slots to the
  // factor first.
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
    cudaGetLastError();
    prio_hi = 0;
  }
  bool own = cudaStreamCreateWithPriority(&job.sd, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
             cudaEventCreateWithFlags(&job.e_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&job.e_done, cudaEventDisableTiming) == cudaSuccess;
  bool la = own && cudaStreamCreateWithPriority(&job.s2, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
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
  double* M = F.L.p;
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
  // W_KK = L_KK^-1 for the diagonal blocks of COARSE_BS rows, block row by
  // block row (NB rows) inside each.  A pivot that was not positive is
  // recorded in err and replaced by 1, so the inverse is computed on finite
  // data either way; dense_finish reports it.  The strict upper triangle of
  // L outside the NB x NB diagonal tiles still holds A: the solve reads
  // only the lower triangle of L and the diagonal blocks of W.
  k_set_identity<<<blocks_for(n * n, 256), 256, 0, m>>>(n, F.W.p);
  count_launch();
  side_pending = false;
  constexpr int BB = (int)(COARSE_BS / NB);  // NB-blocks per diagonal block
  for (int i = 0; i < nb; ++i) {
    const int j0 = (i / BB) * BB;                   // first NB-block column of this diagonal block
    const int e = j0 + BB < nb ? j0 + BB : nb;      // end of its NB-block rows
    const int ncolb = i + 1 - j0;
    k_trsm_lower_left<<<(unsigned)ncolb, 256, 0, m>>>(n, D, F.W.p, i, j0);
    count_launch();
    const int r = e - i - 1;
    if (r > 0) {
      if (la) {
        if (side_pending) SA_CUDA(cudaStreamWaitEvent(m, job.e_side, 0));
        k_gemm_left<<<(unsigned)ncolb, 256, 0, m>>>(n, M, F.W.p, i, ncolb, i + 1, j0);
        count_launch();
        if (r > 1) {
          SA_CUDA(cudaEventRecord(job.e_main, m));
          SA_CUDA(cudaStreamWaitEvent(s2, job.e_main, 0));
          k_gemm_left<<<(unsigned)((r - 1) * ncolb), 256, 0, s2>>>(n, M, F.W.p, i, ncolb, i + 2, j0);
          count_launch();
          SA_CUDA(cudaEventRecord(job.e_side, s2));
          side_pending = true;
        } else {
          side_pending = false;
        }
      } else {
        k_gemm_left<<<(unsigned)(r * ncolb), 256, 0, m>>>(n, M, F.W.p, i, ncolb, i + 1, j0);
        count_launch();
      }
    }
    SA_LAUNCHED();
  }
  if (la && side_pending) SA_CUDA(cudaStreamWaitEvent(m, job.e_side, 0));
  dim3 tb(32, 8), tg((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
  k_transpose_dense<<<tg, tb, 0, m>>>(n, F.W.p, F.WT.p);
  SA_LAUNCHED();
  k_transpose_dense<<<tg, tb, 0, m>>>(n, F.L.p, F.LT.p);
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
// Coarse solve x = A_c^-1 b = L^-T (L^-1 b) by substitution over the diagonal
// blocks K (rows [r0, r1) of COARSE_BS):
//   forward   t_K = b_K - L_{K,<K} y_{<K};  y_K = W_KK t_K   (W_KK = L_KK^-1)
//   backward  t_K = y_K - (L^T)_{K,>K} x_{>K};  x_K = W_KK^T t_K
// Each step is a row-parallel product over one row range: one CTA of
// TRI_WARPS warps per row, warp q taking the q-th of TRI_WARPS consecutive
// column segments of the row's range (segments of a multiple of 32 columns;
// lanes stride the segment with four loads in flight, each lane summing in
// column order; a shuffle tree adds the lanes), the warps' sums added in warp
// order.  MODE: 0 sum over [r0, i] (lower triangle of a diagonal block),
// 1 over [i, r1) (upper), 2 rhs_i minus the sum over [0, r0), 3 rhs_i minus
// the sum over [r1, n).  The K-column forms run the same sums for every
// column as the one-column form (bitwise equal columns).
// ---------------------------------------------------------------------------
constexpr int TRI_WARPS = 4;

// the row i of one step (a block of TRI_WARPS warps per row)
template <int MODE, int K>
__device__ __forceinline__ void tri_row_at(int64_t n, int64_t r0, int64_t r1, const double* __restrict__ M,
                                           const double* __restrict__ v, const double* __restrict__ rhs,
                                           double* __restrict__ out, int64_t i) {
  __shared__ double sh[TRI_WARPS][K];
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  const int64_t lo = MODE == 0 ? r0 : (MODE == 1 ? i : (MODE == 2 ? 0 : r1));
  const int64_t hi = MODE == 0 ? i + 1 : (MODE == 1 ? r1 : (MODE == 2 ? r0 : n));
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
    out[i * K + c] = MODE >= 2 ? rhs[i * K + c] - t : t;
  }
}

template <int MODE, int K>
__global__ void __launch_bounds__(TRI_WARPS * 32) k_tri_row(int64_t n, int64_t r0, int64_t r1,
                                                            const double* __restrict__ M,
                                                            const double* __restrict__ v,
                                                            const double* __restrict__ rhs,
                                                            double* __restrict__ out) {
  tri_row_at<MODE, K>(n, r0, r1, M, v, rhs, out, r0 + blockIdx.x);
}

// the same step for several problems in one launch (group solve): block
// blockIdx.x - blk0 of a segment takes that segment's row r0 + (blockIdx.x -
// blk0), as its own launch would
template <int MODE>
__global__ void __launch_bounds__(TRI_WARPS * 32) k_g_tri(const GTri* __restrict__ d, int m) {
  __shared__ int s_seg;
  if (threadIdx.x == 0) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (d[mid].blk0 <= blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_seg = lo;
  }
  __syncthreads();
  const GTri& D = d[s_seg];
  tri_row_at<MODE, 1>(D.n, D.r0, D.r1, D.M, D.v, D.rhs, D.out, D.r0 + (int64_t)(blockIdx.x - D.blk0));
}

int launch_g_tri(cudaStream_t st, int mode, const GTri* d, int m, unsigned blocks) {
  if (m <= 0 || blocks == 0) return SA_OK;
  const unsigned T = TRI_WARPS * 32;
  switch (mode) {
    case 0: k_g_tri<0><<<blocks, T, 0, st>>>(d, m); break;
    case 1: k_g_tri<1><<<blocks, T, 0, st>>>(d, m); break;
    case 2: k_g_tri<2><<<blocks, T, 0, st>>>(d, m); break;
    default: k_g_tri<3><<<blocks, T, 0, st>>>(d, m); break;
  }
  SA_LAUNCHED();
  return SA_OK;
}

int tri_threads() { return TRI_WARPS * 32; }

template <int K>
static int coarse_solve_k(cudaStream_t st, const CoarseView& F, const double* b, double* t, double* y, double* x) {
  const int64_t n = F.n;
  const int nbk = (int)((n + COARSE_BS - 1) / COARSE_BS);
  const unsigned T = TRI_WARPS * 32;
  for (int q = 0; q < nbk; ++q) {
    const int64_t r0 = q * COARSE_BS, r1 = r0 + COARSE_BS < n ? r0 + COARSE_BS : n;
    const unsigned g = (unsigned)(r1 - r0);
    if (q > 0) {
      k_tri_row<2, K><<<g, T, 0, st>>>(n, r0, r1, F.L, y, b, t);
      SA_LAUNCHED();
    }
    k_tri_row<0, K><<<g, T, 0, st>>>(n, r0, r1, F.W, q > 0 ? t : b, nullptr, y);
    SA_LAUNCHED();
  }
  for (int q = nbk - 1; q >= 0; --q) {
    const int64_t r0 = q * COARSE_BS, r1 = r0 + COARSE_BS < n ? r0 + COARSE_BS : n;
    const unsigned g = (unsigned)(r1 - r0);
    if (q < nbk - 1) {
      k_tri_row<3, K><<<g, T, 0, st>>>(n, r0, r1, F.LT, x, y, t);
      SA_LAUNCHED();
    }
    k_tri_row<1, K><<<g, T, 0, st>>>(n, r0, r1, F.WT, q < nbk - 1 ? t : y, nullptr, x);
    SA_LAUNCHED();
  }
  return SA_OK;
}

int launch_coarse_solve(cudaStream_t st, const CoarseView& F, const double* b, double* t, double* y, double* x) {
  if (F.n <= 0) return SA_OK;
  return coarse_solve_k<1>(st, F, b, t, y, x);
}

int launch_coarse_solve_block(cudaStream_t st, const CoarseView& F, int k, const double* b, double* t, double* y,
                              double* x) {
  if (F.n <= 0) return SA_OK;
  switch (k) {
    case 2: return coarse_solve_k<2>(st, F, b, t, y, x);
    case 4: return coarse_solve_k<4>(st, F, b, t, y, x);
    case 8: return coarse_solve_k<8>(st, F, b, t, y, x);
    default: return SA_ERR_INVALID_ARG;
  }
}

}  // namespace sa
