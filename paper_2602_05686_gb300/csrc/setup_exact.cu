// Setup kernels whose floating-point results must be bitwise reproducible:
// Dirichlet detection, nodal tensors and their inverses, the two strength
// measures with pointwise dropping, the filtered matrix with lumping and the
// 1-norm diagonal, coarse auxiliary data, and the smoothed prolongator
// values.  This translation unit is compiled with -fmad=false: every
// expression below is evaluated with separately rounded IEEE operations in
// the order written, and every sum runs in ascending column / index order.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sa {

// ---------------------------------------------------------------------------
// a1. Dirichlet detection + diagonal (Sec. 3, Fig. 4 caption: Dirichlet
// nodes are isolated in the filtered graph).  Warp per row.  A row is
// Dirichlet iff every stored off-diagonal value is exactly zero.  err bit 1:
// a row without a stored diagonal.
// ---------------------------------------------------------------------------
__global__ void k_dirichlet_diag(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ v, uint8_t* __restrict__ dir,
                                 double* __restrict__ diag, int* __restrict__ err) {
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    const int64_t b = rp[i], e = rp[i + 1];
    bool offnz = false, has_d = false;
    double d = 0.0;
    for (int64_t p = b + lane; p < e; p += 32) {
      int32_t j = ci[p];
      double a = v[p];
      if (j == (int32_t)i) { d = a; has_d = true; }
      else if (a != 0.0) offnz = true;
    }
    unsigned anyoff = __ballot_sync(FULL, offnz);
    unsigned hd = __ballot_sync(FULL, has_d);
    // exactly one lane holds the diagonal
    double dd = hd ? __shfl_sync(FULL, d, __ffs(hd) - 1) : 0.0;
    if (lane == 0) {
      if (dir) dir[i] = anyoff ? 0 : 1;
      diag[i] = dd;
      if (!hd) atomicOr(err, 1);
    }
  }
}

// input check of the level-0 CSR: row pointers monotone from 0 to nnz,
// columns in [0, n) and strictly ascending in each row.  err bit 32.
__global__ void k_validate_csr(int64_t n, int64_t ncols, int64_t nnz, const int64_t* __restrict__ rp,
                               const int32_t* __restrict__ ci, int* __restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = rp[i], e = rp[i + 1];
  if ((i == 0 && b != 0) || (i == n - 1 && e != nnz) || e < b || b < 0 || e > nnz) {
    atomicOr(err, 32);
    return;
  }
  int32_t prev = -1;
  for (int64_t p = b; p < e; ++p) {
    int32_t j = ci[p];
    if (j <= prev || j < 0 || (int64_t)j >= ncols) { atomicOr(err, 32); return; }
    prev = j;
  }
}

// ---------------------------------------------------------------------------
// a2. nodal tensors and inverses (Sec. 3: Clement interpolant of an
// elementwise tensor; inverse by adjugate / determinant)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void invert_packed(int dim, const double* t, double* si) {
  if (dim == 2) {
    double det = t[0] * t[1] - t[2] * t[2];
    si[0] = t[1] / det;
    si[1] = t[0] / det;
    si[2] = -t[2] / det;
  } else {
    double a = t[0], b = t[1], c = t[2], d = t[3], e = t[4], f = t[5];
    double c00 = b * c - f * f;
    double c11 = a * c - e * e;
    double c22 = a * b - d * d;
    double c01 = e * f - d * c;
    double c02 = d * f - b * e;
    double c12 = d * e - a * f;
    double det = a * c00 + d * c01 + e * c02;
    si[0] = c00 / det;
    si[1] = c11 / det;
    si[2] = c22 / det;
    si[3] = c01 / det;
    si[4] = c02 / det;
    si[5] = c12 / det;
  }
}

__global__ void k_node_elem_count(int64_t ne, int npe, const int32_t* __restrict__ en, int64_t n,
                                  int64_t* __restrict__ cnt, int* __restrict__ err) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * npe) return;
  int32_t node = en[t];
  if (node < 0 || node >= n) { atomicOr(err, 2); return; }
  atomicAdd((unsigned long long*)&cnt[node + 1], 1ull);
}

__global__ void k_node_elem_fill(int64_t ne, int npe, const int32_t* __restrict__ en, int64_t n,
                                 const int64_t* __restrict__ off, int* __restrict__ cursor,
                                 int32_t* __restrict__ list) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * npe) return;
  int32_t node = en[t];
  if (node < 0 || node >= n) return;
  int pos = atomicAdd(&cursor[node], 1);
  list[off[node] + pos] = (int32_t)(t / npe);
}

// thread per node: sort incident elements ascending, average, invert
__global__ void k_node_tensor_from_elems(int64_t n, int dim, const int64_t* __restrict__ off,
                                         int32_t* __restrict__ list, const double* __restrict__ meas,
                                         const double* __restrict__ et, double* __restrict__ sigma,
                                         double* __restrict__ sinv, int* __restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int kp = dim == 3 ? 6 : 3;
  const int64_t b = off[i], e = off[i + 1];
  for (int64_t p = b + 1; p < e; ++p) {  // insertion sort of the node's own segment
    int32_t key = list[p];
    int64_t q = p - 1;
    while (q >= b && list[q] > key) { list[q + 1] = list[q]; --q; }
    list[q + 1] = key;
  }
  double num[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double den = 0.0;
  for (int64_t p = b; p < e; ++p) {
    int64_t el = list[p];
    double m = meas[el];
    for (int c = 0; c < kp; ++c) num[c] += m * et[el * kp + c];
    den += m;
  }
  if (den == 0.0) atomicOr(err, 4);
  double s[6];
  for (int c = 0; c < kp; ++c) {
    s[c] = num[c] / den;
    sigma[i * kp + c] = s[c];
  }
  double si[6];
  invert_packed(dim, s, si);
  for (int c = 0; c < kp; ++c) sinv[i * kp + c] = si[c];
}

// per-node tensors given (copy) or sigma = I (distance Laplacian); invert
__global__ void k_node_tensor_direct(int64_t n, int dim, const double* __restrict__ given,
                                     double* __restrict__ sigma, double* __restrict__ sinv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int kp = dim == 3 ? 6 : 3;
  double s[6];
  for (int c = 0; c < kp; ++c) {
    s[c] = given ? given[i * kp + c] : (c < dim ? 1.0 : 0.0);
    sigma[i * kp + c] = s[c];
  }
  double si[6];
  invert_packed(dim, s, si);
  for (int c = 0; c < kp; ++c) sinv[i * kp + c] = si[c];
}

// ---------------------------------------------------------------------------
// a3. classical measure + pointwise dropping (Sec. 2.1):
//   keep_ij <=> a_ij*a_ij >= (theta*theta) * |a_ii*a_jj|, diagonal kept,
//   Dirichlet nodes excluded.  Warp per row; also counts kept entries per
//   row (diagonal included) into cnt[i+1].
// ---------------------------------------------------------------------------
__global__ void k_strength_classical(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const double* __restrict__ v, const double* __restrict__ diag,
                                     const uint8_t* __restrict__ dir, double t2, uint8_t* __restrict__ keep,
                                     int64_t* __restrict__ cnt) {
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    const int64_t b = rp[i], e = rp[i + 1];
    const double di = diag[i];
    const bool diri = dir && dir[i];
    int kept = 0;
    for (int64_t p = b + lane; p < e; p += 32) {
      int32_t j = ci[p];
      uint8_t k;
      if (j == (int32_t)i) k = 1;
      else if (diri || (dir && dir[j])) k = 0;
      else {
        double a = v[p];
        k = (a * a >= t2 * fabs(di * diag[j])) ? 1 : 0;
      }
      keep[p] = k;
      kept += k;
    }
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(FULL, kept, o);
    if (lane == 0) cnt[i + 1] = kept;
  }
}

// ---------------------------------------------------------------------------
// a4. material-aware distance Laplacian (Sec. 2.1 distance Laplacian,
// Sec. 3 material distance with max symmetrisation):
//   w_ij = 1 / max(d^T sinv_i d, d^T sinv_j d), d = x_i - x_j,
//   D_i = sum_{j != i} w_ij (ascending column order).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double quad_form(int dim, const double* __restrict__ si, const double* d) {
  // t = sigma^-1 d, then d . t, as running sums of fused multiply-adds in
  // index order (explicit __fma_rn: one rounding per term even under
  // -fmad=false); even in d bit for bit
  if (dim == 2) {
    const double t0 = __fma_rn(si[2], d[1], si[0] * d[0]);
    const double t1 = __fma_rn(si[1], d[1], si[2] * d[0]);
    return __fma_rn(d[1], t1, d[0] * t0);
  }
  const double t0 = __fma_rn(si[4], d[2], __fma_rn(si[3], d[1], si[0] * d[0]));
  const double t1 = __fma_rn(si[5], d[2], __fma_rn(si[1], d[1], si[3] * d[0]));
  const double t2 = __fma_rn(si[2], d[2], __fma_rn(si[5], d[1], si[4] * d[0]));
  return __fma_rn(d[2], t2, __fma_rn(d[1], t1, d[0] * t0));
}

// w_ij = 1 / max(q_ij, q_ji) for the entries above the diagonal (j > i);
// the diagonal gets 0 and the lower entries are mirrored afterwards.  For
// (j, i) the difference vector is exactly -(x_i - x_j), and both quadratic
// forms are even in it with sign-symmetric rounding, so w_ji computed from row
// j would be the same bits: computing each pair once halves the FP64 work.
// One thread per row: the FP64 pipe issues a warp instruction whatever its
// active lanes, so the upper entries of 32 rows share each instruction.
template <int DIM>
__global__ void k_material_w(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ x, const double* __restrict__ sinv, double* __restrict__ w) {
  constexpr int KP = DIM == 3 ? 6 : 3;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = rp[i], e = rp[i + 1];
  double xi[3], si_i[KP];
#pragma unroll
  for (int c = 0; c < DIM; ++c) xi[c] = x[i * DIM + c];
#pragma unroll
  for (int c = 0; c < KP; ++c) si_i[c] = sinv[i * KP + c];
  for (int64_t p = b; p < e; ++p) {
    const int32_t j = ci[p];
    if (j < (int32_t)i) continue;  // mirrored by k_material_w_mirror
    double wv = 0.0;
    if (j != (int32_t)i) {
      double d[3], sj[KP];
#pragma unroll
      for (int c = 0; c < DIM; ++c) d[c] = xi[c] - x[(int64_t)j * DIM + c];
#pragma unroll
      for (int c = 0; c < KP; ++c) sj[c] = sinv[(int64_t)j * KP + c];
      double qij = quad_form(DIM, si_i, d);
      double qji = quad_form(DIM, sj, d);
      double m = qij > qji ? qij : qji;
      wv = 1.0 / m;
    }
    w[p] = wv;
  }
}

// the same per pair with a warp per row (lanes stride the row): on coarse
// levels a few rows are 10-40x longer than the rest, and a thread per row
// leaves them a long sequential tail.  Every w_ij comes from the same
// expression, so the values equal those of the thread-per-row form.
template <int DIM>
__global__ void k_material_w_warp(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                  const double* __restrict__ x, const double* __restrict__ sinv,
                                  double* __restrict__ w) {
  constexpr int KP = DIM == 3 ? 6 : 3;
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    double xi[3], si_i[KP];
#pragma unroll
    for (int c = 0; c < DIM; ++c) xi[c] = x[i * DIM + c];
#pragma unroll
    for (int c = 0; c < KP; ++c) si_i[c] = sinv[i * KP + c];
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const int32_t j = ci[p];
      if (j < (int32_t)i) continue;  // mirrored by k_material_w_mirror
      double wv = 0.0;
      if (j != (int32_t)i) {
        double d[3], sj[KP];
#pragma unroll
        for (int c = 0; c < DIM; ++c) d[c] = xi[c] - x[(int64_t)j * DIM + c];
#pragma unroll
        for (int c = 0; c < KP; ++c) sj[c] = sinv[(int64_t)j * KP + c];
        double qij = quad_form(DIM, si_i, d);
        double qji = quad_form(DIM, sj, d);
        double m = qij > qji ? qij : qji;
        wv = 1.0 / m;
      }
      w[p] = wv;
    }
  }
}

// lower entries: w_ij = w_ji, the (j, i) entry found by binary search in row
// j; a pattern without that entry (not structurally symmetric) gets w_ij
// computed here by the same expression
template <int DIM>
__global__ void k_material_w_mirror(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    const double* __restrict__ x, const double* __restrict__ sinv,
                                    double* __restrict__ w) {
  constexpr int KP = DIM == 3 ? 6 : 3;
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const int32_t j = ci[p];
      if (j >= (int32_t)i) break;  // columns ascend: the rest of the row is upper
      int64_t lo = rp[j], hi = rp[j + 1] - 1, f = -1;
      while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t c = ci[mid];
        if (c == (int32_t)i) { f = mid; break; }
        if (c < (int32_t)i) lo = mid + 1; else hi = mid - 1;
      }
      if (f >= 0) {
        w[p] = w[f];
      } else {
        double d[3], si[KP], sj[KP];
#pragma unroll
        for (int c = 0; c < DIM; ++c) d[c] = x[i * DIM + c] - x[(int64_t)j * DIM + c];
#pragma unroll
        for (int c = 0; c < KP; ++c) {
          si[c] = sinv[i * KP + c];
          sj[c] = sinv[(int64_t)j * KP + c];
        }
        double qij = quad_form(DIM, si, d);
        double qji = quad_form(DIM, sj, d);
        w[p] = 1.0 / (qij > qji ? qij : qji);
      }
    }
  }
}

// D_i = sum of the row's w in ascending column order (thread per row, so the
// sequential FP64 additions of 32 rows share one warp instruction).  The
// diagonal's w is +0, and adding +0 to a non-negative sum leaves it unchanged,
// so this equals the sum over the off-diagonal entries only.
__global__ void k_row_sum_ordered(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ w,
                                  double* __restrict__ D) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  const int64_t e = rp[i + 1];
  int64_t p = rp[i];
  // eight loads in flight per round (long coarse-level rows are otherwise a
  // chain of dependent load rounds); still added one by one in column order
  for (; p + 8 <= e; p += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = w[p + u];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  for (; p < e; ++p) acc += w[p];
  D[i] = acc;
}

// keep_ij <=> w_ij*w_ij >= (theta*theta) * (D_i*D_j)
__global__ void k_material_keep(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ w, const double* __restrict__ D,
                                const uint8_t* __restrict__ dir, double t2, uint8_t* __restrict__ keep,
                                int64_t* __restrict__ cnt) {
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    const int64_t b = rp[i], e = rp[i + 1];
    const double Di = D[i];
    const bool diri = dir && dir[i];
    int kept = 0;
    for (int64_t p = b + lane; p < e; p += 32) {
      int32_t j = ci[p];
      uint8_t k;
      if (j == (int32_t)i) k = 1;
      else if (diri || (dir && dir[j])) k = 0;
      else {
        double wv = w[p];
        k = (wv * wv >= t2 * (Di * D[j])) ? 1 : 0;
      }
      keep[p] = k;
      kept += k;
    }
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(FULL, kept, o);
    if (lane == 0 && cnt) cnt[i + 1] = kept;
  }
}

// ---------------------------------------------------------------------------
// Cut-drop criterion (Sec. 2.1, Eq. C^cut-drop) on squared strengths:
// classical s2 = a_ij^2 / |a_ii a_jj|, material s2 = w_ij^2 / (D_i D_j).
// Per row the off-diagonal strengths are ordered descending; the first k with
// theta^2 s2_k >= s2_{k+1} gives the threshold s2_k (no such k: keep all);
// an edge survives when both of its rows keep it.
// ---------------------------------------------------------------------------
__global__ void k_s2_classical(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ v, const double* __restrict__ diag,
                               double* __restrict__ s2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = diag[i];
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    int32_t j = ci[p];
    s2[p] = (j == (int32_t)i) ? 0.0 : (v[p] * v[p]) / fabs(di * diag[j]);
  }
}

__global__ void k_s2_material(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ w, const double* __restrict__ D, double* __restrict__ s2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double Di = D[i];
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    int32_t j = ci[p];
    s2[p] = (j == (int32_t)i) ? 0.0 : (w[p] * w[p]) / (Di * D[j]);
  }
}

constexpr int CUT_CAP = 256;   // row entries sorted in shared memory
constexpr int CUT_WARPS = 4;

// serial threshold for rows longer than CUT_CAP: walk the distinct values in
// descending order (ties form pairs of equal neighbours in the ordering)
__device__ double cut_threshold_serial(const int64_t b, const int64_t e, const int32_t* __restrict__ ci, int64_t i,
                                       const uint8_t* __restrict__ dir, const double* __restrict__ s2, double t2) {
  const bool diri = dir && dir[i];
  double cur = INFINITY, last = 0.0;
  bool any = false;
  for (;;) {
    double nxt = -1.0;
    int mult = 0;
    for (int64_t p = b; p < e; ++p) {
      int32_t j = ci[p];
      if (j == (int32_t)i || diri || (dir && dir[j])) continue;
      double x = s2[p];
      if (x < cur) {
        if (x > nxt) { nxt = x; mult = 1; }
        else if (x == nxt) ++mult;
      }
    }
    if (nxt < 0.0) return any ? last : 0.0;  // values exhausted: no gap, keep all
    if (any && t2 * last >= nxt) return last;
    if (mult >= 2 && t2 * nxt >= nxt) return nxt;
    any = true;
    last = nxt;
    cur = nxt;
  }
}

__global__ void __launch_bounds__(CUT_WARPS * 32)
k_cut_rows(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
           const uint8_t* __restrict__ dir, const double* __restrict__ s2, double t2,
           uint8_t* __restrict__ rowkeep) {
  __shared__ double vals_all[CUT_WARPS][CUT_CAP];
  __shared__ double srt_all[CUT_WARPS][CUT_CAP];
  const int w = threadIdx.x >> 5, lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  double* vals = vals_all[w];
  double* srt = srt_all[w];
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    const int64_t b = rp[i], e = rp[i + 1];
    const bool diri = dir && dir[i];
    // collect the row's valid strengths in column order
    int m = 0;
    for (int64_t p0 = b; p0 < e; p0 += 32) {
      int64_t p = p0 + lane;
      bool ok = false;
      double x = 0.0;
      if (p < e) {
        int32_t j = ci[p];
        ok = j != (int32_t)i && !diri && !(dir && dir[j]);
        x = s2[p];
      }
      unsigned bm = __ballot_sync(FULL, ok);
      if (ok && m + __popc(bm & lt) < CUT_CAP) vals[m + __popc(bm & lt)] = x;
      m += __popc(bm);
    }
    __syncwarp();
    double thr = 0.0;
    if (m > CUT_CAP) {
      if (lane == 0) thr = cut_threshold_serial(b, e, ci, i, dir, s2, t2);
      thr = __shfl_sync(FULL, thr, 0);
    } else if (m > 0) {
      // rank sort, descending (ties by position)
      for (int t = lane; t < m; t += 32) {
        const double x = vals[t];
        int r = 0;
        for (int u = 0; u < m; ++u) r += (vals[u] > x) || (vals[u] == x && u < t);
        srt[r] = x;
      }
      __syncwarp();
      thr = srt[m - 1];
      for (int k0 = 0; k0 < m - 1; k0 += 32) {
        const int k = k0 + lane;
        const bool gap = k < m - 1 && t2 * srt[k] >= srt[k + 1];
        const unsigned gm = __ballot_sync(FULL, gap);
        if (gm) {
          thr = srt[k0 + __ffs(gm) - 1];
          break;
        }
      }
    }
    for (int64_t p = b + lane; p < e; p += 32) {
      int32_t j = ci[p];
      bool ok = j != (int32_t)i && !diri && !(dir && dir[j]);
      rowkeep[p] = (ok && m > 0 && s2[p] >= thr) ? 1 : 0;
    }
    __syncwarp();
  }
}

// keep = diagonal, or kept by both rows; counts kept entries into cnt[i+1]
__global__ void k_cut_symmetrize(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const uint8_t* __restrict__ rowkeep, uint8_t* __restrict__ keep,
                                 int64_t* __restrict__ cnt) {
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    int kept = 0;
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      int32_t j = ci[p];
      uint8_t k;
      if (j == (int32_t)i) k = 1;
      else if (!rowkeep[p]) k = 0;
      else {
        int64_t lo = rp[j], hi = rp[j + 1] - 1, f = -1;
        while (lo <= hi) {
          int64_t mid = (lo + hi) >> 1;
          int32_t c = ci[mid];
          if (c == (int32_t)i) { f = mid; break; }
          if (c < (int32_t)i) lo = mid + 1; else hi = mid - 1;
        }
        k = (f >= 0 && rowkeep[f]) ? 1 : 0;
      }
      keep[p] = k;
      kept += k;
    }
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(FULL, kept, o);
    if (lane == 0) cnt[i + 1] = kept;
  }
}

// ---------------------------------------------------------------------------
// a10. filtered matrix A_F and 1-norm diagonal (Sec. 2.2, Eqs.
// filtered_matrix and 1_norm_diagonal).  rpF is the scan of
// the kept counts.  A row whose filtered 1-norm is <= 1e-12 times the 1-norm
// of its row of A (every off-diagonal dropped, lumped row sum ~ 0) gets
// Dt = +inf: it is not smoothed.
// ---------------------------------------------------------------------------
__global__ void k_filter(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const double* __restrict__ v, const uint8_t* __restrict__ keep,
                         const int64_t* __restrict__ rpF, int32_t* __restrict__ ciF, double* __restrict__ vF,
                         double* __restrict__ Dt) {
  // thread per row: the three ordered sums are sequential FP64 chains, so
  // one warp instruction advances 32 rows
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = rp[i], e = rp[i + 1];
  // lumped diagonal: a_ii, then the dropped entries in ascending order
  double dg = 0.0;
  for (int64_t p = b; p < e; ++p)
    if (ci[p] == (int32_t)i) dg = v[p];
  for (int64_t p = b; p < e; ++p)
    if (ci[p] != (int32_t)i && !keep[p]) dg += v[p];
  // the filtered row and both 1-norms in ascending order
  int64_t out = rpF[i];
  double s = 0.0, a1 = 0.0;
  for (int64_t p = b; p < e; ++p) {
    const int32_t j = ci[p];
    const double a = v[p];
    a1 += fabs(a);
    if (j == (int32_t)i || keep[p]) {
      const double fv = (j == (int32_t)i) ? dg : a;
      ciF[out] = j;
      vF[out] = fv;
      ++out;
      s += fabs(fv);
    }
  }
  Dt[i] = (s <= 1e-12 * a1) ? INFINITY : s;
}

// ---------------------------------------------------------------------------
// a9. coarse coordinates and tensors (Sec. 3, Eq. auxiliary_transfer):
// means over the aggregate members, summed in ascending fine index (mlist is
// sorted per aggregate); the coarse inverse tensors follow by inversion.
// ---------------------------------------------------------------------------
__global__ void k_coarse_aux(int64_t nc, int dim, const int64_t* __restrict__ mrp, const int32_t* __restrict__ mlist,
                             const double* __restrict__ x, const double* __restrict__ sigma,
                             double* __restrict__ xc, double* __restrict__ sc, double* __restrict__ sic) {
  int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nc) return;
  const int kp = dim == 3 ? 6 : 3;
  double sx[3] = {0.0, 0.0, 0.0}, ss[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double cnt = 0.0;
  for (int64_t p = mrp[a]; p < mrp[a + 1]; ++p) {
    int64_t i = mlist[p];
    for (int c = 0; c < dim; ++c) sx[c] += x[i * dim + c];
    for (int c = 0; c < kp; ++c) ss[c] += sigma[i * kp + c];
    cnt += 1.0;
  }
  for (int c = 0; c < dim; ++c) xc[a * dim + c] = sx[c] / cnt;
  double s[6];
  for (int c = 0; c < kp; ++c) {
    s[c] = ss[c] / cnt;
    sc[a * kp + c] = s[c];
  }
  double si[6];
  invert_packed(dim, s, si);
  for (int c = 0; c < kp; ++c) sic[a * kp + c] = si[c];
}

// ---------------------------------------------------------------------------
// a12. smoothed prolongator values from T = A_F P^ (Sec. 2.2):
//   c_i = omega / Dt_i,  P_ij = [j == agg(i)] - c_i * T_ij
// P shares the pattern of T.  omega is read from device memory.
// ---------------------------------------------------------------------------
__global__ void k_smooth_p_values(int64_t n, const int64_t* __restrict__ rpT, const int32_t* __restrict__ ciT,
                                  const double* __restrict__ vT, const int32_t* __restrict__ agg,
                                  const double* __restrict__ Dt, const double* __restrict__ omega_p,
                                  double* __restrict__ vP) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double omega = *omega_p;
  const double c = omega / Dt[i];
  const int32_t ai = agg[i];
  for (int64_t p = rpT[i]; p < rpT[i + 1]; ++p) {
    double t = vT[p];
    vP[p] = (ciT[p] == ai) ? 1.0 - c * t : -(c * t);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int launch_dirichlet_diag(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                          uint8_t* dir, double* diag, int* err) {
  if (n <= 0) return SA_OK;
  k_dirichlet_diag<<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, v, dir, diag, err);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_validate_csr(cudaStream_t s, int64_t n, int64_t ncols, int64_t nnz, const int64_t* rp, const int32_t* ci,
                        int* err) {
  if (n <= 0) return SA_OK;
  k_validate_csr<<<blocks_for(n, 256), 256, 0, s>>>(n, ncols, nnz, rp, ci, err);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_nodal_tensors(Alloc& al, int dim, int64_t n, int tloc, const double* tensors, int64_t ne, int npe,
                         const int32_t* en, const double* meas, double* sigma, double* sinv, int* err) {
  cudaStream_t s = al.stream;
  if (tloc == 1) {
    Buf<int64_t> off;
    Buf<int> cursor;
    Buf<int32_t> list;
    SA_TRY(off.alloc(&al, n + 1));
    SA_TRY(cursor.alloc(&al, n));
    SA_TRY(list.alloc(&al, ne * npe));
    SA_TRY(memset_d(off.p, 0, off.bytes(), s));
    SA_TRY(memset_d(cursor.p, 0, cursor.bytes(), s));
    k_node_elem_count<<<blocks_for(ne * npe, 256), 256, 0, s>>>(ne, npe, en, n, off.p, err);
    SA_LAUNCHED();
    SA_TRY(scan_inplace(al, off.p + 1, n));
    k_node_elem_fill<<<blocks_for(ne * npe, 256), 256, 0, s>>>(ne, npe, en, n, off.p, cursor.p, list.p);
    SA_LAUNCHED();
    k_node_tensor_from_elems<<<blocks_for(n, 128), 128, 0, s>>>(n, dim, off.p, list.p, meas, tensors, sigma, sinv,
                                                               err);
    SA_LAUNCHED();
  } else {
    k_node_tensor_direct<<<blocks_for(n, 256), 256, 0, s>>>(n, dim, tensors, sigma, sinv);
    SA_LAUNCHED();
  }
  return SA_OK;
}

int launch_strength_classical(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                              const double* diag, const uint8_t* dir, double theta, uint8_t* keep,
                              int64_t* cnt) {
  if (n <= 0) return SA_OK;
  const double t2 = theta * theta;
  k_strength_classical<<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, v, diag, dir, t2, keep, cnt);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_strength_material(cudaStream_t s, int dim, int64_t n, const int64_t* rp, const int32_t* ci,
                             const double* x, const double* sinv, const uint8_t* dir, double theta,
                             double* w, double* D, uint8_t* keep, int64_t* cnt) {
  if (n <= 0) return SA_OK;
  const double t2 = theta * theta;
  // a thread per row on large levels (uniform rows: 32 rows share each FP64
  // instruction), a warp per row below 2^19 rows (coarse levels, long rows)
  if (n >= (int64_t(1) << 19)) {
    if (dim == 3) k_material_w<3><<<blocks_for(n, 128), 128, 0, s>>>(n, rp, ci, x, sinv, w);
    else k_material_w<2><<<blocks_for(n, 128), 128, 0, s>>>(n, rp, ci, x, sinv, w);
  } else {
    if (dim == 3) k_material_w_warp<3><<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, x, sinv, w);
    else k_material_w_warp<2><<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, x, sinv, w);
  }
  SA_LAUNCHED();
  if (dim == 3) k_material_w_mirror<3><<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, x, sinv, w);
  else k_material_w_mirror<2><<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, x, sinv, w);
  SA_LAUNCHED();
  k_row_sum_ordered<<<blocks_for(n, 128), 128, 0, s>>>(n, rp, w, D);
  SA_LAUNCHED();
  k_material_keep<<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, w, D, dir, t2, keep, cnt);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_cut_drop(Alloc& al, int measure_classical, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci,
                    const double* v, const double* diag, const double* w, const double* D, const uint8_t* dir,
                    double theta, uint8_t* keep, int64_t* cnt) {
  cudaStream_t s = al.stream;
  if (n <= 0) return SA_OK;
  Buf<double> s2;
  Buf<uint8_t> rowkeep;
  SA_TRY(s2.alloc(&al, nnz));
  SA_TRY(rowkeep.alloc(&al, nnz));
  if (measure_classical) k_s2_classical<<<blocks_for(n, 128), 128, 0, s>>>(n, rp, ci, v, diag, s2.p);
  else k_s2_material<<<blocks_for(n, 128), 128, 0, s>>>(n, rp, ci, w, D, s2.p);
  SA_LAUNCHED();
  const double t2 = theta * theta;
  k_cut_rows<<<warp_rows_grid(n, CUT_WARPS * 32), CUT_WARPS * 32, 0, s>>>(n, rp, ci, dir, s2.p, t2, rowkeep.p);
  SA_LAUNCHED();
  k_cut_symmetrize<<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, rowkeep.p, keep, cnt);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_filter(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                  const uint8_t* keep, const int64_t* rpF, int32_t* ciF, double* vF, double* Dt) {
  if (n <= 0) return SA_OK;
  k_filter<<<blocks_for(n, 128), 128, 0, s>>>(n, rp, ci, v, keep, rpF, ciF, vF, Dt);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_coarse_aux(cudaStream_t s, int64_t nc, int dim, const int64_t* mrp, const int32_t* mlist,
                      const double* x, const double* sigma, double* xc, double* sc, double* sic) {
  if (nc <= 0) return SA_OK;
  k_coarse_aux<<<blocks_for(nc, 128), 128, 0, s>>>(nc, dim, mrp, mlist, x, sigma, xc, sc, sic);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_smooth_p_values(cudaStream_t s, int64_t n, const int64_t* rpT, const int32_t* ciT, const double* vT,
                           const int32_t* agg, const double* Dt, const double* omega_dev, double* vP) {
  if (n <= 0) return SA_OK;
  k_smooth_p_values<<<blocks_for(n, 256), 256, 0, s>>>(n, rpT, ciT, vT, agg, Dt, omega_dev, vP);
  SA_LAUNCHED();
  return SA_OK;
}

}  // namespace sa
