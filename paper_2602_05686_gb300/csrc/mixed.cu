// FP32 V-cycle (Algorithm 1 with Chebyshev smoothing) on the scaled
// hierarchy  A~_l = D_l^-1/2 A_l D_l^-1/2,  P~_l = D_l^1/2 P_l D_{l+1}^-1/2,
// R~_l = P~_l^T, which satisfies A~_{l+1} = R~_l A~_l P~_l exactly in real
// arithmetic, so the cycle is the FP64 cycle in scaled variables with a unit
// Jacobi diagonal.  Matrices are stored as FP32 SELL-32 (slices of 32
// consecutive rows, column-major inside a slice, one thread per row): every
// load of a warp is one contiguous 128-byte segment of values and one of
// column indices.  The coarsest level is solved in FP64 with the dense
// inverse factor.
#include <math.h>

#include <vector>

#include "common.cuh"
#include "mixed.cuh"
#include "profile.cuh"
#include "solve.cuh"

namespace sa {

struct Sell {
  int64_t n = 0, nslices = 0, stored = 0, nnz = 0;
  Buf<int64_t> sp;   // slice offsets (nslices + 1)
  Buf<int32_t> ci;
  Buf<float> v;
};

struct MLevel {
  int64_t n = 0, nc = 0;
  double lmax = 0, lmin = 0;
  Sell A, P, R;
  Buf<float> b, x, x2, r, d;
  Buf<double> sq;   // sqrt(diag) (coarsest level only)
};

struct MixedHierarchy {
  Alloc* al = nullptr;
  int deg = 2;
  std::vector<MLevel*> lev;
  Buf<double> s0;       // fine-level D^-1/2
  Buf<double> z;        // FP64 output
  Buf<double> ct, cy, cx;
  const double* W = nullptr;
  const double* WT = nullptr;
};

// ---------------------------------------------------------------------------
// construction: scaled values and SELL-32 packing
// ---------------------------------------------------------------------------
__global__ void k_slice_width(int64_t n, const int64_t* __restrict__ rp, int64_t* __restrict__ sz) {
  int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t ns = (n + 31) / 32;
  if (sl >= ns) return;
  int64_t w = 0;
  for (int64_t r = sl * 32; r < sl * 32 + 32 && r < n; ++r) {
    int64_t len = rp[r + 1] - rp[r];
    w = len > w ? len : w;
  }
  sz[sl + 1] = w * 32;
}

// value scaling: out = left[i] * a_ij * right[j]; left/right may be NULL (= 1)
__global__ void k_sell_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, const double* __restrict__ left,
                            const double* __restrict__ right, int left_sqrt, int right_sqrt,
                            const int64_t* __restrict__ sp, int32_t* __restrict__ oci, float* __restrict__ ov) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t sl = i / 32, r = i % 32;
  const int64_t base = sp[sl], width = (sp[sl + 1] - sp[sl]) / 32;
  double li = 1.0;
  if (left) li = left_sqrt ? sqrt(left[i]) : 1.0 / sqrt(left[i]);
  int64_t k = 0;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p, ++k) {
    int32_t j = ci[p];
    double rj = 1.0;
    if (right) rj = right_sqrt ? sqrt(right[j]) : 1.0 / sqrt(right[j]);
    oci[base + k * 32 + r] = j;
    ov[base + k * 32 + r] = (float)(li * v[p] * rj);
  }
  for (; k < width; ++k) {
    oci[base + k * 32 + r] = 0;
    ov[base + k * 32 + r] = 0.0f;
  }
}

__global__ void k_sqrt(int64_t n, const double* __restrict__ d, double* __restrict__ out, int inv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = inv ? 1.0 / sqrt(d[i]) : sqrt(d[i]);
}

static int build_sell(Alloc& al, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* v,
                      const double* left, int left_sqrt, const double* right, int right_sqrt, Sell& S) {
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
  k_slice_width<<<blocks_for(S.nslices, 256), 256, 0, s>>>(n, rp, S.sp.p);
  SA_LAUNCHED();
  SA_TRY(scan_inplace(al, S.sp.p + 1, S.nslices));
  SA_TRY(copy_d2h(&S.stored, S.sp.p + S.nslices, sizeof(int64_t), s));
  SA_TRY(S.ci.alloc(&al, S.stored));
  SA_TRY(S.v.alloc(&al, S.stored));
  k_sell_fill<<<blocks_for(n, 256), 256, 0, s>>>(n, rp, ci, v, left, right, left_sqrt, right_sqrt, S.sp.p, S.ci.p,
                                                 S.v.p);
  SA_LAUNCHED();
  return SA_OK;
}

int mixed_build(Alloc& al, const MixedLevelIn* in, int nlev, int cheb_degree, const double* W, const double* WT,
                MixedHierarchy** out) {
  MixedHierarchy* m = new MixedHierarchy();
  *out = m;
  m->al = &al;
  m->deg = cheb_degree;
  m->W = W;
  m->WT = WT;
  cudaStream_t s = al.stream;
  for (int l = 0; l < nlev; ++l) {
    MLevel* L = new MLevel();
    m->lev.push_back(L);
    const MixedLevelIn& I = in[l];
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
      // A~ = D^-1/2 A D^-1/2
      SA_TRY(build_sell(al, I.n, I.nnz, I.rp, I.ci, I.v, I.diag, 0, I.diag, 0, L->A));
      const double* dc = in[l + 1].diag;
      // P~ = D_l^1/2 P D_{l+1}^-1/2 (rows fine, columns coarse)
      SA_TRY(build_sell(al, I.n, I.nnzP, I.Prp, I.Pci, I.Pv, I.diag, 1, dc, 0, L->P));
      // R~ = D_{l+1}^-1/2 R D_l^1/2 (rows coarse, columns fine)
      SA_TRY(build_sell(al, I.nc, I.nnzP, I.Rrp, I.Rci, I.Rv, dc, 0, I.diag, 1, L->R));
    } else {
      SA_TRY(L->sq.alloc(&al, I.n));
      k_sqrt<<<blocks_for(I.n, 256), 256, 0, s>>>(I.n, I.diag, L->sq.p, 0);
      SA_LAUNCHED();
      SA_TRY(m->ct.alloc(&al, I.n));
      SA_TRY(m->cy.alloc(&al, I.n));
      SA_TRY(m->cx.alloc(&al, I.n));
    }
  }
  const int64_t n0 = in[0].n;
  SA_TRY(m->s0.alloc(&al, n0));
  SA_TRY(m->z.alloc(&al, n0));
  k_sqrt<<<blocks_for(n0, 256), 256, 0, s>>>(n0, in[0].diag, m->s0.p, 1);
  SA_LAUNCHED();
  return SA_OK;
}

void mixed_free(MixedHierarchy* m) {
  if (!m) return;
  for (MLevel* L : m->lev) delete L;
  delete m;
}

double mixed_vcycle_bytes(const MixedHierarchy* m) {
  // per level above the coarsest: 4 passes over A~ (1 pre, 1 residual, 2
  // post), one over P~ and R~, ~16 vector streams; coarsest: W and W^T halves
  double b = 0;
  const int nl = (int)m->lev.size();
  for (int l = 0; l < nl; ++l) {
    const MLevel* L = m->lev[l];
    if (l + 1 < nl) {
      b += 4.0 * L->A.stored * 8.0 + (double)(L->P.stored + L->R.stored) * 8.0 + 16.0 * L->n * 4.0;
    } else {
      b += (double)L->n * L->n * 8.0;
    }
  }
  return b;
}

// ---------------------------------------------------------------------------
// FP32 V-cycle kernels (one thread per row, SELL-32)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sell_row(const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                                          const float* __restrict__ v, const float* __restrict__ x, int64_t i) {
  const int64_t sl = i >> 5, r = i & 31;
  const int64_t b = sp[sl], e = sp[sl + 1];
  float acc = 0.0f;
  for (int64_t p = b + r; p < e; p += 32) acc += v[p] * __ldg(&x[ci[p]]);
  return acc;
}

// x_out = x_in + d,  d = first ? c2 r : c1 d + c2 r,  r = b - A~ x_in
__global__ void k_sell_cheb(int64_t n, const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                            const float* __restrict__ v, const float* __restrict__ b, const float* __restrict__ xin,
                            float* __restrict__ xout, float* __restrict__ d, float c1, float c2, int first) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r = b[i] - sell_row(sp, ci, v, xin, i);
  float dn = first ? c2 * r : c1 * d[i] + c2 * r;
  d[i] = dn;
  xout[i] = xin[i] + dn;
}

__global__ void k_cheb_first32(int64_t n, const float* __restrict__ b, float c2, float* __restrict__ x,
                               float* __restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float dn = c2 * b[i];
    d[i] = dn;
    x[i] = dn;
  }
}

// fine entry: b~ = D^-1/2 r (FP64 -> FP32), fused with the first Chebyshev step
__global__ void k_fine_in_first(int64_t n, const double* __restrict__ r, const double* __restrict__ s,
                                float c2, float* __restrict__ b, float* __restrict__ x, float* __restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float bi = (float)(s[i] * r[i]);
    b[i] = bi;
    float dn = c2 * bi;
    d[i] = dn;
    x[i] = dn;
  }
}

__global__ void k_sell_residual(int64_t n, const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                                const float* __restrict__ v, const float* __restrict__ b,
                                const float* __restrict__ x, float* __restrict__ r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = b[i] - sell_row(sp, ci, v, x, i);
}

__global__ void k_sell_spmv(int64_t n, const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                            const float* __restrict__ v, const float* __restrict__ x, float* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = sell_row(sp, ci, v, x, i);
}

__global__ void k_sell_spmv_add(int64_t n, const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                                const float* __restrict__ v, const float* __restrict__ x, float* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += sell_row(sp, ci, v, x, i);
}

// fine exit: z = D^-1/2 x~ in FP64 (fused into the last post-smoothing step)
__global__ void k_sell_cheb_out(int64_t n, const int64_t* __restrict__ sp, const int32_t* __restrict__ ci,
                                const float* __restrict__ v, const float* __restrict__ b,
                                const float* __restrict__ xin, float* __restrict__ d, float c1, float c2, int first,
                                const double* __restrict__ s, double* __restrict__ z) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r = b[i] - sell_row(sp, ci, v, xin, i);
  float dn = first ? c2 * r : c1 * d[i] + c2 * r;
  z[i] = s[i] * (double)(xin[i] + dn);
}

// coarsest: t = sqrt(d) b~ in FP64
__global__ void k_coarse_in(int64_t n, const float* __restrict__ b, const double* __restrict__ sq,
                            double* __restrict__ t) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t[i] = sq[i] * (double)b[i];
}

__global__ void k_coarse_out(int64_t n, const double* __restrict__ x, const double* __restrict__ sq,
                             float* __restrict__ xo) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xo[i] = (float)(sq[i] * x[i]);
}

static inline unsigned g256(int64_t n) { return blocks_for(n, 256); }

// algorithmic bytes: FP32 value + int32 column per stored entry of the
// unpadded matrix, 8-byte slice offsets, each vector element once
static double b_cheb32(const MLevel* L) { return 8.0 * L->A.nnz + 8.0 * (L->A.nslices + 1) + 20.0 * L->n; }

#define PROFK(kind, level, bytes, launch)               \
  do {                                                  \
    int _pi = prof_begin(st, (kind), (level), (bytes)); \
    launch;                                             \
    prof_end(st, _pi);                                  \
    SA_LAUNCHED();                                      \
  } while (0)

// V-cycle on level l with right-hand side L->b; result pointer in *xo.
// For l == 0 the FP64 output z is produced by the last smoothing step.
static int mv(MixedHierarchy* m, cudaStream_t st, int l, const double* r64, float** xo) {
  MLevel* L = m->lev[l];
  const int nl = (int)m->lev.size();
  const int64_t n = L->n;
  if (l == nl - 1) {
    int _pi = prof_begin(st, PK_COARSE, l, 8.0 * n * n + 48.0 * n);
    k_coarse_in<<<g256(n), 256, 0, st>>>(n, L->b.p, L->sq.p, m->ct.p);
    SA_LAUNCHED();
    SA_TRY(launch_coarse_solve(st, n, m->W, m->WT, m->ct.p, m->cy.p, m->cx.p));
    k_coarse_out<<<g256(n), 256, 0, st>>>(n, m->cx.p, L->sq.p, L->x.p);
    prof_end(st, _pi);
    SA_LAUNCHED();
    *xo = L->x.p;
    return SA_OK;
  }
  const int deg = m->deg;
  const double th = 0.5 * (L->lmax + L->lmin), de = 0.5 * (L->lmax - L->lmin);
  const double s1 = th / de;
  float* xa = L->x.p;
  float* xb = L->x2.p;
  const Sell& A = L->A;
  if (l == 0) {
    PROFK(PK_FIRST32, l, 28.0 * n,
          (k_fine_in_first<<<g256(n), 256, 0, st>>>(n, r64, m->s0.p, (float)(1.0 / th), L->b.p, xa, L->d.p)));
  } else {
    PROFK(PK_FIRST32, l, 12.0 * n, (k_cheb_first32<<<g256(n), 256, 0, st>>>(n, L->b.p, (float)(1.0 / th), xa, L->d.p)));
  }
  double rho = 1.0 / s1;
  for (int k = 1; k < deg; ++k) {
    double rn = 1.0 / (2.0 * s1 - rho);
    PROFK(PK_CHEB32, l, b_cheb32(L),
          (k_sell_cheb<<<g256(n), 256, 0, st>>>(n, A.sp.p, A.ci.p, A.v.p, L->b.p, xa, xb, L->d.p, (float)(rn * rho),
                                                (float)(2.0 * rn / de), 0)));
    float* t = xa; xa = xb; xb = t;
    rho = rn;
  }
  MLevel* C = m->lev[l + 1];
  PROFK(PK_RESID32, l, 8.0 * A.nnz + 8.0 * (A.nslices + 1) + 12.0 * n,
        (k_sell_residual<<<g256(n), 256, 0, st>>>(n, A.sp.p, A.ci.p, A.v.p, L->b.p, xa, L->r.p)));
  PROFK(PK_RESTRICT32, l, 8.0 * L->R.nnz + 8.0 * (L->R.nslices + 1) + 4.0 * n + 4.0 * C->n,
        (k_sell_spmv<<<g256(C->n), 256, 0, st>>>(C->n, L->R.sp.p, L->R.ci.p, L->R.v.p, L->r.p, C->b.p)));
  float* xc = nullptr;
  SA_TRY(mv(m, st, l + 1, nullptr, &xc));
  PROFK(PK_PROLONG32, l, 8.0 * L->P.nnz + 8.0 * (L->P.nslices + 1) + 4.0 * C->n + 8.0 * n,
        (k_sell_spmv_add<<<g256(n), 256, 0, st>>>(n, L->P.sp.p, L->P.ci.p, L->P.v.p, xc, xa)));
  // post-smoothing: deg steps from the corrected x
  rho = 1.0 / s1;
  for (int k = 0; k < deg; ++k) {
    int first = (k == 0);
    float c1 = 0.0f, c2 = (float)(1.0 / th);
    double rn = rho;
    if (!first) {
      rn = 1.0 / (2.0 * s1 - rho);
      c1 = (float)(rn * rho);
      c2 = (float)(2.0 * rn / de);
    }
    if (l == 0 && k == deg - 1) {
      PROFK(PK_CHEB32, l, b_cheb32(L) + 12.0 * n,
            (k_sell_cheb_out<<<g256(n), 256, 0, st>>>(n, A.sp.p, A.ci.p, A.v.p, L->b.p, xa, L->d.p, c1, c2, first,
                                                      m->s0.p, m->z.p)));
    } else {
      PROFK(PK_CHEB32, l, b_cheb32(L),
            (k_sell_cheb<<<g256(n), 256, 0, st>>>(n, A.sp.p, A.ci.p, A.v.p, L->b.p, xa, xb, L->d.p, c1, c2, first)));
      float* t = xa; xa = xb; xb = t;
    }
    if (!first) rho = rn;
  }
  *xo = xa;
  return SA_OK;
}

int mixed_vcycle(MixedHierarchy* m, cudaStream_t st, const double* r, double** z) {
  if (m->lev.size() == 1) {
    // single level: the coarse solve directly on D^-1/2 r
    MLevel* L = m->lev[0];
    const int64_t n = L->n;
    // b~ = s0 r, then x~ = D^1/2 A^-1 D^1/2 b~ = D^1/2 A^-1 r, z = s0 x~ = A^-1 r
    SA_TRY(launch_coarse_solve(st, n, m->W, m->WT, r, m->cy.p, m->z.p));
    *z = m->z.p;
    return SA_OK;
  }
  float* xo = nullptr;
  SA_TRY(mv(m, st, 0, r, &xo));
  *z = m->z.p;
  return SA_OK;
}

}  // namespace sa
