/*
 * Seeded synthetic input generator: bilinear (2D) / trilinear (3D) Lagrange
 * finite elements on a tensor-product box mesh, for the model problem
 *     -div(sigma(x) grad u) = f   with Dirichlet / Neumann boundaries
 * (the paper's Section 1, model problem and its variational form).
 *
 * This file is INPUT GENERATION ONLY.  It holds none of the AMG method's
 * arithmetic (no strength measure, aggregation, prolongator, Galerkin
 * product, smoother or Krylov iteration); both the CUDA library and the CPU
 * oracle consume what it writes.
 *
 * Node numbering: node (i,j,k) -> i + Nx*(j + Ny*k), Nx = nx+1, Ny = ny+1.
 * Element numbering: (ex,ey,ez) -> ex + nx*(ey + ny*ez).
 * Local element node a in [0, 2^dim): bit0 = +x, bit1 = +y, bit2 = +z.
 * Row pattern: the full Q1 stencil (9 points in 2D, 27 in 3D, truncated at
 * the boundary), columns ascending, explicit diagonal, stored even where a
 * value happens to be exactly zero.
 * Dirichlet nodes are eliminated symmetrically: their row keeps only the
 * diagonal (value 1, rhs = g), their column is removed from every other row
 * and the rhs is lifted by -a_ji * g_i.
 *
 * Element matrices use 2-point Gauss quadrature per axis, exact for the
 * products of Q1 gradients on axis-aligned boxes.  Entries of the element
 * matrix are computed for a <= b and mirrored, and the global sum runs over
 * elements in ascending order for both (i,j) and (j,i), so the assembled
 * matrix is bitwise symmetric.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

static int64_t node_id(int i, int j, int k, int Nx, int Ny) {
  return (int64_t)i + (int64_t)Nx * ((int64_t)j + (int64_t)Ny * (int64_t)k);
}

/* number of stored entries of the full Q1 pattern before Dirichlet elimination */
int64_t q1_pattern_nnz(int dim, int nx, int ny, int nz) {
  int64_t Nx = nx + 1, Ny = ny + 1, Nz = (dim == 3) ? nz + 1 : 1;
  int64_t cx = 3 * Nx - 2, cy = 3 * Ny - 2, cz = (dim == 3) ? 3 * Nz - 2 : 1;
  return cx * cy * cz;
}

/* position of column (i+dx, j+dy, k+dz) inside row (i,j,k) of the full pattern */
static inline int stencil_pos(int dim, int i, int j, int k, int nx, int ny, int nz,
                              int dx, int dy, int dz) {
  int cx = 1 + (i > 0) + (i < nx);
  int cy = 1 + (j > 0) + (j < ny);
  int ox = dx + (i > 0);
  int oy = dy + (j > 0);
  int oz = (dim == 3) ? dz + (k > 0) : 0;
  return (oz * cy + oy) * cx + ox;
}

/* element stiffness of an axis-aligned box with constant symmetric tensor K
 * (packed 2D: xx,yy,xy; 3D: xx,yy,zz,xy,xz,yz) */
static void elem_matrix(int dim, const double h[3], const double* K, double* Ke) {
  const int nl = 1 << dim;
  const double g = 1.0 / sqrt(3.0);
  const double gp[2] = {-g, g};
  double Kf[3][3] = {{0}};
  if (dim == 2) {
    Kf[0][0] = K[0]; Kf[1][1] = K[1]; Kf[0][1] = Kf[1][0] = K[2];
  } else {
    Kf[0][0] = K[0]; Kf[1][1] = K[1]; Kf[2][2] = K[2];
    Kf[0][1] = Kf[1][0] = K[3]; Kf[0][2] = Kf[2][0] = K[4]; Kf[1][2] = Kf[2][1] = K[5];
  }
  double detJ = 1.0;
  for (int d = 0; d < dim; ++d) detJ *= 0.5 * h[d];
  for (int a = 0; a < nl * nl; ++a) Ke[a] = 0.0;
  int nq = (dim == 3) ? 8 : 4;
  for (int q = 0; q < nq; ++q) {
    double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], (dim == 3) ? gp[(q >> 2) & 1] : 0.0};
    double grad[8][3];
    for (int a = 0; a < nl; ++a) {
      double s[3], ds[3];
      for (int d = 0; d < dim; ++d) {
        int bit = (a >> d) & 1;
        double sgn = bit ? 1.0 : -1.0;
        s[d] = 0.5 * (1.0 + sgn * xi[d]);
        ds[d] = 0.5 * sgn * (2.0 / h[d]);
      }
      for (int d = 0; d < dim; ++d) {
        double v = ds[d];
        for (int e = 0; e < dim; ++e) if (e != d) v *= s[e];
        grad[a][d] = v;
      }
    }
    for (int a = 0; a < nl; ++a)
      for (int b = a; b < nl; ++b) {
        double acc = 0.0;
        for (int d = 0; d < dim; ++d) {
          double kg = 0.0;
          for (int e = 0; e < dim; ++e) kg += Kf[d][e] * grad[b][e];
          acc += grad[a][d] * kg;
        }
        Ke[a * nl + b] += acc * detJ;
      }
  }
  for (int a = 0; a < nl; ++a)
    for (int b = 0; b < a; ++b) Ke[a * nl + b] = Ke[b * nl + a];
}

/* symmetric Dirichlet elimination in place: a Dirichlet row keeps only its
 * diagonal (value 1, rhs = g), the column of a Dirichlet node is removed from
 * every other row and that row's rhs is lifted by -a_ij * g_j */
static void eliminate_dirichlet(int64_t n, int64_t* row_ptr, int32_t* col, double* val, double* b,
                                const uint8_t* dir_mask, const double* dir_val) {
  for (int64_t r = 0; r < n; ++r) {
    if (dir_mask[r]) continue;
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
      int32_t c = col[p];
      if (dir_mask[c]) b[r] -= val[p] * (dir_val ? dir_val[c] : 0.0);
    }
  }
  int64_t w = 0, start = 0;
  for (int64_t r = 0; r < n; ++r) {
    int64_t end = row_ptr[r + 1];
    for (int64_t p = start; p < end; ++p) {
      int32_t c = col[p];
      int keepit = dir_mask[r] ? (c == r) : !dir_mask[c];
      if (keepit) {
        col[w] = c;
        val[w] = dir_mask[r] ? 1.0 : val[p];
        ++w;
      }
    }
    start = end;
    row_ptr[r + 1] = w;
    if (dir_mask[r]) b[r] = dir_val ? dir_val[r] : 0.0;
  }
}

/*
 * Assemble the Q1 system on the tensor-product mesh with node coordinates
 * xc[0..nx], yc[0..ny], zc[0..nz] (zc ignored in 2D).
 *   elem_K   : n_e * (3|6) packed tensors, elementwise constant
 *   elem_f   : n_e load density (constant per element), NULL -> 0
 *   dir_mask : n nodes, 1 = Dirichlet; dir_val: prescribed values (NULL -> 0)
 * Outputs (caller-allocated):
 *   row_ptr[n+1], col[nnz_max], val[nnz_max]  with nnz_max = q1_pattern_nnz
 *   b[n], coords[n*dim], elem_nodes[n_e * 2^dim], elem_measure[n_e]
 * Returns the number of stored entries after elimination (<= nnz_max), or -1.
 */
/* Element matrices depend only on the box edge lengths and the tensor, and a
 * workload has few distinct pairs (two tensors on a uniform grid for the
 * inclusions, one per layer for the stacks), so they are memoised in a small
 * hash table keyed by the exact bytes of (h, K): a hit returns the matrix the
 * same routine computed for the same inputs, bit for bit. */
#define EM_SLOTS 256
typedef struct { int used; double key[9]; double Ke[64]; } em_slot_t;

static void elem_matrix_cached(em_slot_t* cache, int dim, const double h[3], const double* K, double* Ke) {
  const int kp = (dim == 3) ? 6 : 3, nl = 1 << dim;
  double key[9] = {0};
  key[0] = h[0]; key[1] = h[1]; key[2] = h[2];
  memcpy(key + 3, K, sizeof(double) * (size_t)kp);
  uint64_t hs = 1469598103934665603ull;
  const unsigned char* kb = (const unsigned char*)key;
  for (size_t i = 0; i < sizeof(key); ++i) { hs ^= kb[i]; hs *= 1099511628211ull; }
  em_slot_t* sl = &cache[hs & (EM_SLOTS - 1)];
  if (sl->used && memcmp(sl->key, key, sizeof(key)) == 0) {
    memcpy(Ke, sl->Ke, sizeof(double) * (size_t)(nl * nl));
    return;
  }
  elem_matrix(dim, h, K, Ke);
  sl->used = 1;
  memcpy(sl->key, key, sizeof(key));
  memcpy(sl->Ke, Ke, sizeof(double) * (size_t)(nl * nl));
}

int64_t q1_assemble(int dim, int nx, int ny, int nz,
                    const double* xc, const double* yc, const double* zc,
                    const double* elem_K, const double* elem_f,
                    const uint8_t* dir_mask, const double* dir_val,
                    int64_t* row_ptr, int32_t* col, double* val, double* b,
                    double* coords, int32_t* elem_nodes, double* elem_measure) {
  if (dim != 2 && dim != 3) return -1;
  if (dim == 2) nz = 0;
  const int Nx = nx + 1, Ny = ny + 1, Nz = nz + 1;
  const int64_t n = (int64_t)Nx * Ny * Nz;
  const int nl = 1 << dim;
  const int kp = (dim == 3) ? 6 : 3;
  /* full pattern */
  row_ptr[0] = 0;
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        int64_t r = node_id(i, j, k, Nx, Ny);
        int cx = 1 + (i > 0) + (i < nx), cy = 1 + (j > 0) + (j < ny);
        int cz = (dim == 3) ? 1 + (k > 0) + (k < nz) : 1;
        row_ptr[r + 1] = (int64_t)cx * cy * cz;
      }
  for (int64_t r = 0; r < n; ++r) row_ptr[r + 1] += row_ptr[r];
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        int64_t r = node_id(i, j, k, Nx, Ny);
        int64_t p = row_ptr[r];
        int zlo = (dim == 3 && k > 0) ? -1 : 0, zhi = (dim == 3 && k < nz) ? 1 : 0;
        for (int dz = zlo; dz <= zhi; ++dz)
          for (int dy = (j > 0 ? -1 : 0); dy <= (j < ny ? 1 : 0); ++dy)
            for (int dx = (i > 0 ? -1 : 0); dx <= (i < nx ? 1 : 0); ++dx)
              col[p++] = (int32_t)node_id(i + dx, j + dy, k + dz, Nx, Ny);
      }
  const int64_t nnz_full = row_ptr[n];
  memset(val, 0, sizeof(double) * (size_t)nnz_full);
  memset(b, 0, sizeof(double) * (size_t)n);
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        int64_t r = node_id(i, j, k, Nx, Ny);
        coords[r * dim + 0] = xc[i];
        coords[r * dim + 1] = yc[j];
        if (dim == 3) coords[r * dim + 2] = zc[k];
      }
  const int ez_n = (dim == 3) ? nz : 1;
  double Ke[64];
  em_slot_t* cache = (em_slot_t*)calloc(EM_SLOTS, sizeof(em_slot_t));
  if (!cache) return -1;
  for (int ez = 0; ez < ez_n; ++ez)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        int64_t e = (int64_t)ex + (int64_t)nx * ((int64_t)ey + (int64_t)ny * ez);
        double h[3] = {xc[ex + 1] - xc[ex], yc[ey + 1] - yc[ey], (dim == 3) ? zc[ez + 1] - zc[ez] : 1.0};
        double meas = h[0] * h[1] * ((dim == 3) ? h[2] : 1.0);
        elem_measure[e] = meas;
        elem_matrix_cached(cache, dim, h, elem_K + e * kp, Ke);
        double fe = elem_f ? elem_f[e] * meas / (double)nl : 0.0;
        for (int a = 0; a < nl; ++a) {
          int ia = ex + (a & 1), ja = ey + ((a >> 1) & 1), ka = (dim == 3) ? ez + ((a >> 2) & 1) : 0;
          int64_t ga = node_id(ia, ja, ka, Nx, Ny);
          elem_nodes[e * nl + a] = (int32_t)ga;
          b[ga] += fe;
          for (int bb = 0; bb < nl; ++bb) {
            int ib = ex + (bb & 1), jb = ey + ((bb >> 1) & 1), kb = (dim == 3) ? ez + ((bb >> 2) & 1) : 0;
            int pos = stencil_pos(dim, ia, ja, ka, nx, ny, nz, ib - ia, jb - ja, kb - ka);
            val[row_ptr[ga] + pos] += Ke[a * nl + bb];
          }
        }
      }
  free(cache);
  if (dir_mask) eliminate_dirichlet(n, row_ptr, col, val, b, dir_mask, dir_val);
  return row_ptr[n];
}

/* SplitMix64 (Steele, Lea & Flood 2014), counter form: the k-th output for
 * a given seed is mix(seed + (k+1) * golden). */
static inline uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* out[k] = uniform double in [0,1) from the top 53 bits, k in [k0, k0+count) */
void q1_uniform(uint64_t seed, uint64_t k0, int64_t count, double* out) {
  for (int64_t k = 0; k < count; ++k)
    out[k] = (double)(splitmix64_at(seed, k0 + (uint64_t)k) >> 11) * (1.0 / 9007199254740992.0);
}

/* Nearest-seed (Voronoi) region of every element centroid of a uniform
 * n^3 element mesh on [0,1]^3; ties go to the lowest seed index. */
void q1_voronoi_regions(int nx, int ny, int nz, int nseeds, const double* seeds, int32_t* region) {
  for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        double cx = (ex + 0.5) / nx, cy = (ey + 0.5) / ny, cz = (ez + 0.5) / nz;
        double best = 1e300;
        int bi = 0;
        for (int s = 0; s < nseeds; ++s) {
          double dx = cx - seeds[3 * s], dy = cy - seeds[3 * s + 1], dz = cz - seeds[3 * s + 2];
          double d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < best) { best = d2; bi = s; }
        }
        region[(int64_t)ex + (int64_t)nx * ((int64_t)ey + (int64_t)ny * ez)] = bi;
      }
}

/* Mark the elements whose centroid lies inside a sphere (centre c, radius r,
 * in element units) of an n^3 uniform element grid; returns newly marked count. */
int64_t q1_mark_sphere(int nx, int ny, int nz, double cx, double cy, double cz, double r, uint8_t* inside) {
  int64_t added = 0;
  int x0 = (int)floor(cx - r), x1 = (int)ceil(cx + r);
  int y0 = (int)floor(cy - r), y1 = (int)ceil(cy + r);
  int z0 = (int)floor(cz - r), z1 = (int)ceil(cz + r);
  if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0; if (z0 < 0) z0 = 0;
  if (x1 > nx - 1) x1 = nx - 1; if (y1 > ny - 1) y1 = ny - 1; if (z1 > nz - 1) z1 = nz - 1;
  for (int ez = z0; ez <= z1; ++ez)
    for (int ey = y0; ey <= y1; ++ey)
      for (int ex = x0; ex <= x1; ++ex) {
        double dx = ex + 0.5 - cx, dy = ey + 0.5 - cy, dz = ez + 0.5 - cz;
        if (dx * dx + dy * dy + dz * dz <= r * r) {
          int64_t e = (int64_t)ex + (int64_t)nx * ((int64_t)ey + (int64_t)ny * ez);
          if (!inside[e]) { inside[e] = 1; ++added; }
        }
      }
  return added;
}

/* ------------------------------------------------------------------------
 * Annulus: trilinear hexahedra on r_i <= r <= r_o, 0 <= z <= t with nr x nt x
 * nz elements in the radial, circumferential and thickness directions,
 * periodic in the angle (nt >= 3).
 * Node (a, b, c) -> a + Nr*(b + nt*c), Nr = nr+1, Nz = nz+1, with coordinates
 * (r_a cos phi_b, r_a sin phi_b, z_c), r_a = r_i + a (r_o - r_i)/nr,
 * phi_b = 2 pi b / nt, z_c = c t / nz.  Local element node bits: bit0 = +r,
 * bit1 = +angle, bit2 = +z.  Element matrices use the isoparametric map with
 * 2x2x2 Gauss points (exact for the element volume, whose Jacobian is
 * polynomial of low degree on these straight-edged hexahedra).
 * Rows hold the full 27-point pattern with columns sorted ascending;
 * Dirichlet on a = 0 (value g_in) and a = nr (value g_out), natural
 * boundaries on z = 0 and z = t; elem_f (NULL -> 0) is a load density
 * constant per element, integrated against each shape function.
 * ------------------------------------------------------------------------ */
static void hex_matrix(const double X[8][3], const double* K, double* Ke, double* meas, double* Nint) {
  const double g = 1.0 / sqrt(3.0);
  const double Kf[3][3] = {{K[0], K[3], K[4]}, {K[3], K[1], K[5]}, {K[4], K[5], K[2]}};
  for (int a = 0; a < 64; ++a) Ke[a] = 0.0;
  for (int a = 0; a < 8; ++a) Nint[a] = 0.0;
  *meas = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double xi[3] = {(q & 1) ? g : -g, (q & 2) ? g : -g, (q & 4) ? g : -g};
    double dN[8][3], N[8];
    for (int a = 0; a < 8; ++a) {
      double s[3], sg[3];
      for (int d = 0; d < 3; ++d) {
        sg[d] = ((a >> d) & 1) ? 1.0 : -1.0;
        s[d] = 0.5 * (1.0 + sg[d] * xi[d]);
      }
      N[a] = s[0] * s[1] * s[2];
      dN[a][0] = 0.5 * sg[0] * s[1] * s[2];
      dN[a][1] = 0.5 * sg[1] * s[0] * s[2];
      dN[a][2] = 0.5 * sg[2] * s[0] * s[1];
    }
    double J[3][3] = {{0}};  /* J[d][e] = d x_d / d xi_e */
    for (int a = 0; a < 8; ++a)
      for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 3; ++e) J[d][e] += X[a][d] * dN[a][e];
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    /* inverse by the adjugate: Ji[e][d] = d xi_e / d x_d */
    double Ji[3][3];
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double gr[8][3];
    for (int a = 0; a < 8; ++a)
      for (int d = 0; d < 3; ++d) gr[a][d] = dN[a][0] * Ji[0][d] + dN[a][1] * Ji[1][d] + dN[a][2] * Ji[2][d];
    for (int a = 0; a < 8; ++a)
      for (int bb = a; bb < 8; ++bb) {
        double acc = 0.0;
        for (int d = 0; d < 3; ++d) {
          double kg = 0.0;
          for (int e = 0; e < 3; ++e) kg += Kf[d][e] * gr[bb][e];
          acc += gr[a][d] * kg;
        }
        Ke[a * 8 + bb] += acc * det;
      }
    *meas += det;
    for (int a = 0; a < 8; ++a) Nint[a] += N[a] * det;
  }
  for (int a = 0; a < 8; ++a)
    for (int bb = 0; bb < a; ++bb) Ke[a * 8 + bb] = Ke[bb * 8 + a];
}

static int64_t ann_id(int a, int b, int c, int Nr, int nt) {
  return (int64_t)a + (int64_t)Nr * ((int64_t)b + (int64_t)nt * (int64_t)c);
}

int64_t q1_annulus_nnz(int nr, int nt, int nz) {
  return (int64_t)(3 * (nr + 1) - 2) * (3 * (int64_t)nt) * (3 * (nz + 1) - 2);
}

int64_t q1_assemble_annulus(int nr, int nt, int nz, double ri, double ro, double t, const double* elem_K,
                            const double* elem_f, double g_in, double g_out, int64_t* row_ptr, int32_t* col, double* val, double* b,
                            double* coords, int32_t* elem_nodes, double* elem_measure, uint8_t* dir_mask) {
  if (nr < 1 || nt < 3 || nz < 1 || !(ro > ri) || !(ri > 0.0) || !(t > 0.0)) return -1;
  const double two_pi = 6.283185307179586476925286766559;
  const int Nr = nr + 1, Nz = nz + 1;
  const int64_t n = (int64_t)Nr * nt * Nz;
  /* pattern: 3 angle neighbours (periodic) x up to 3 radial x up to 3 thickness */
  row_ptr[0] = 0;
  for (int c = 0; c < Nz; ++c)
    for (int bq = 0; bq < nt; ++bq)
      for (int a = 0; a < Nr; ++a) {
        const int64_t r = ann_id(a, bq, c, Nr, nt);
        const int64_t p0 = row_ptr[r];
        int64_t p = p0;
        for (int dc = -1; dc <= 1; ++dc) {
          if (c + dc < 0 || c + dc > nz) continue;
          for (int db = -1; db <= 1; ++db) {
            const int bb = (bq + db + nt) % nt;
            for (int da = -1; da <= 1; ++da) {
              if (a + da < 0 || a + da > nr) continue;
              col[p++] = (int32_t)ann_id(a + da, bb, c + dc, Nr, nt);
            }
          }
        }
        for (int64_t x = p0 + 1; x < p; ++x) { /* insertion sort, <= 27 entries */
          int32_t v = col[x];
          int64_t y = x - 1;
          while (y >= p0 && col[y] > v) { col[y + 1] = col[y]; --y; }
          col[y + 1] = v;
        }
        row_ptr[r + 1] = p;
      }
  const int64_t nnz_full = row_ptr[n];
  memset(val, 0, sizeof(double) * (size_t)nnz_full);
  memset(b, 0, sizeof(double) * (size_t)n);
  for (int c = 0; c < Nz; ++c)
    for (int bq = 0; bq < nt; ++bq)
      for (int a = 0; a < Nr; ++a) {
        const int64_t r = ann_id(a, bq, c, Nr, nt);
        const double rad = ri + (ro - ri) * (double)a / (double)nr;
        const double phi = two_pi * (double)bq / (double)nt;
        coords[3 * r + 0] = rad * cos(phi);
        coords[3 * r + 1] = rad * sin(phi);
        coords[3 * r + 2] = t * (double)c / (double)nz;
        dir_mask[r] = (uint8_t)(a == 0 || a == nr);
      }
  /* The mesh and the tensor field are invariant under a rotation by
   * 2 pi / nt, so all elements of a ring (fixed ea, ec) share one element
   * matrix: it is computed once, from the element at angle index 0 and its
   * tensor, and reused around the ring. */
  const int64_t nring = (int64_t)nr * nz;
  double* Kr = (double*)malloc(sizeof(double) * (size_t)(nring * 64));
  double* Nr8 = (double*)malloc(sizeof(double) * (size_t)(nring * 8));
  double* Mr = (double*)malloc(sizeof(double) * (size_t)nring);
  if (!Kr || !Nr8 || !Mr) { free(Kr); free(Nr8); free(Mr); return -1; }
  double X[8][3];
  int64_t gid[8];
  for (int ec = 0; ec < nz; ++ec)
    for (int ea = 0; ea < nr; ++ea) {
      const int64_t e0 = (int64_t)ea + (int64_t)nr * ((int64_t)nt * ec);
      const int64_t q = (int64_t)ec * nr + ea;
      for (int l = 0; l < 8; ++l) {
        const int64_t gl = ann_id(ea + (l & 1), ((l >> 1) & 1) % nt, ec + ((l >> 2) & 1), Nr, nt);
        for (int d = 0; d < 3; ++d) X[l][d] = coords[3 * gl + d];
      }
      hex_matrix(X, elem_K + e0 * 6, Kr + q * 64, &Mr[q], Nr8 + q * 8);
    }
  for (int ec = 0; ec < nz; ++ec)
    for (int eb = 0; eb < nt; ++eb)
      for (int ea = 0; ea < nr; ++ea) {
        const int64_t e = (int64_t)ea + (int64_t)nr * ((int64_t)eb + (int64_t)nt * ec);
        const int64_t q = (int64_t)ec * nr + ea;
        const double* Ke = Kr + q * 64;
        const double* Nint = Nr8 + q * 8;
        elem_measure[e] = Mr[q];
        for (int l = 0; l < 8; ++l) {
          const int a = ea + (l & 1), bq = (eb + ((l >> 1) & 1)) % nt, c = ec + ((l >> 2) & 1);
          gid[l] = ann_id(a, bq, c, Nr, nt);
          elem_nodes[e * 8 + l] = (int32_t)gid[l];
        }
        for (int l = 0; l < 8; ++l) {
          if (elem_f) b[gid[l]] += elem_f[e] * Nint[l];  /* consistent load of a constant f */
          for (int m = 0; m < 8; ++m) {
            int64_t p = row_ptr[gid[l]];
            while (col[p] != (int32_t)gid[m]) ++p;  /* present by construction */
            val[p] += Ke[l * 8 + m];
          }
        }
      }
  free(Kr);
  free(Nr8);
  free(Mr);
  /* Dirichlet values: g_in on the inner ring, g_out on the outer ring */
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  if (!g) return -1;
  for (int64_t r = 0; r < n; ++r) g[r] = (r % Nr == 0) ? g_in : g_out;
  eliminate_dirichlet(n, row_ptr, col, val, b, dir_mask, g);
  free(g);
  return row_ptr[n];
}
