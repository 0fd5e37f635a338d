/*
 * sa.h -- C ABI of the GB300 smoothed-aggregation AMG library.
 *
 * Smoothed-aggregation algebraic multigrid (arXiv 2602.05686, Sec. 2) used as
 * the preconditioner of conjugate gradients (Sec. 4) for the material-weighted
 * Laplacian -div(sigma(x) grad u) = f discretised by finite elements
 * (Sec. 1, Eq. model_problem and linear_system).  Coarsening is driven by the
 * classical strength-of-connection measure S^sa = D^-1/2 A D^-1/2
 * (Sec. 2.1) or the material-aware distance Laplacian
 * S^dlap_sigma = D_sigma^-1/2 L_sigma D_sigma^-1/2 (Sec. 3), with pointwise
 * dropping.  Every step runs as a CUDA kernel on one GPU.
 *
 * Conventions for every call:
 *   - the return value is a status (SA_OK or a negative SA_ERR_*); no call
 *     aborts, traps or spins without a bound;
 *   - "device pointer" means memory of the current CUDA device; "host
 *     pointer" means ordinary or pinned host memory; calls that accept
 *     either copy with cudaMemcpyDefault (unified addressing);
 *   - all GPU work of a handle is ordered on options.stream (a
 *     cudaStream_t; NULL = the legacy default stream); a handle must not be
 *     used from two host threads at once;
 *   - indices are 0-based; CSR row pointers are int64, column indices int32.
 */
#ifndef SA_GB300_H
#define SA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sa_handle_s* sa_handle;

enum {
  SA_OK = 0,
  SA_ERR_INVALID_ARG = -1,    /* bad size, NULL pointer, unsupported option */
  SA_ERR_OOM = -2,            /* device allocation (or the allocator callback) failed */
  SA_ERR_CUDA = -3,           /* a CUDA runtime call failed; see sa_last_error() */
  SA_ERR_NOT_SPD = -4,        /* non-positive pivot in the coarse Cholesky factor */
  SA_ERR_STAGNATION = -5,     /* coarsening stagnated above the coarse-solve limit */
  SA_ERR_NO_CONVERGENCE = -6, /* maxit reached; x holds the last iterate */
  SA_ERR_BREAKDOWN = -7,      /* p^T A p <= 0 or NaN in CG */
  SA_ERR_CAPACITY = -8        /* an internal fixed-size table was exceeded */
};

typedef enum {
  SA_MEASURE_CLASSICAL = 0, /* |a_ij| / sqrt(|a_ii a_jj|) >= theta (Sec. 2.1) */
  SA_MEASURE_MATERIAL = 1,  /* material-weighted distance Laplacian (Sec. 3) */
  SA_MEASURE_DISTANCE = 2   /* Euclidean distance Laplacian (Sec. 2.1), sigma = I */
} sa_measure;

typedef enum {
  SA_DROP_POINTWISE = 0,  /* keep |S_ij| >= theta (Sec. 2.1, Eq. C^pw) */
  SA_DROP_CUT = 1         /* cut-drop (Sec. 2.1, Eq. C^cut-drop): per row, keep the entries above the
                             first gap where theta |S_(k)| >= |S_(k+1)| in descending order (no gap:
                             keep the row); an edge is kept only when both of its rows keep it */
} sa_drop;

typedef enum {
  SA_PREC_FP64 = 0,        /* FP64 PCG with an FP64 V-cycle */
  SA_PREC_FP32_VCYCLE = 1  /* FP64 flexible CG with an FP32 V-cycle on the
                              symmetrically diagonal-scaled hierarchy */
} sa_precision;

typedef enum {
  SA_TENSOR_NODE = 0,    /* tensors: n * kp values, one tensor per node */
  SA_TENSOR_ELEMENT = 1  /* tensors: n_elem * kp values, one per element,
                            averaged to nodes by the Clement interpolant (Sec. 3) */
} sa_tensor_loc;

/*
 * Problem statement (Sec. 1: A u = b from Q1/trilinear finite elements).
 * All arrays are caller-owned and only read during sa_setup; they may be
 * device or host pointers (one kind for all arrays, see `host`).
 *   A: SPD, structurally symmetric CSR, columns sorted ascending, diagonal
 *      stored.  Dirichlet rows carry only their diagonal and their columns
 *      are eliminated from the other rows (a row whose stored off-diagonals
 *      are all exactly zero is treated as Dirichlet and never aggregated).
 *   coords: n * dim node coordinates (row-major); required for the
 *      MATERIAL and DISTANCE measures, ignored for CLASSICAL.
 *   tensors: packed symmetric sigma, kp = 3 in 2D (xx, yy, xy), kp = 6 in
 *      3D (xx, yy, zz, xy, xz, yz); required for MATERIAL.
 *   elem_nodes / elem_measure: element connectivity (n_elem * nodes_per_elem)
 *      and element measures |e|, required for SA_TENSOR_ELEMENT.
 */
typedef struct {
  int dim;                 /* 2 or 3 */
  int host;                /* 1 if every array below is a host pointer */
  int64_t n, nnz;
  const int64_t* row_ptr;  /* n + 1 */
  const int32_t* col;      /* nnz */
  const double* val;       /* nnz */
  const double* coords;    /* n * dim */
  sa_tensor_loc tloc;
  const double* tensors;
  int64_t n_elem;
  int nodes_per_elem;
  const int32_t* elem_nodes;
  const double* elem_measure;
} sa_problem;

/*
 * Options.  sa_default_options fills the paper's settings (Sec. 4):
 *   theta = 0.08, measure MATERIAL, pointwise dropping, precision FP64, max_coarse = 5000,
 *   max_levels = 10, Chebyshev degree 2 with lambda_max boost 1.1 and ratio
 *   30, 10 power steps, omega_sym = 4/3, maxit = 500.
 * alloc/dealloc: optional device allocator (e.g. a caching allocator);
 *   NULL = stream-ordered cudaMallocAsync/cudaFreeAsync on `stream`, from the
 *   current device's default pool, whose release threshold the library raises
 *   so that freed memory stays cached for later setups in this process (pass
 *   an allocator to keep memory elsewhere).  A block the allocator returns
 *   must start on a 256-byte boundary (as cudaMalloc's do): the solve
 *   kernels move whole rows of their multi-column blocks with 32-byte
 *   vector accesses.  A misaligned block is handed back to `dealloc` and
 *   the call fails with SA_ERR_OOM and an error text saying so.
 */
typedef struct {
  double theta;
  sa_measure measure;
  sa_precision precision;
  int max_coarse, max_levels;
  int cheb_degree;
  double cheb_ratio, cheb_boost;
  int power_iters;
  double omega_sym;
  uint32_t seed;           /* salts the MIS-2 priorities and power-method starts */
  int maxit;
  void* stream;            /* cudaStream_t */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*dealloc)(void* ptr, void* ctx);
  void* alloc_ctx;
  int keep_setup_data;     /* 1: keep strength masks and roots for sa_export_strength */
  sa_drop drop;            /* dropping criterion (default pointwise) */
} sa_options;

typedef struct {
  int iters;               /* CG iterations (operator products with p) */
  double rel_res_true;     /* ||b - A x|| / ||b - A x0|| at exit, recomputed in FP64 */
  double setup_ms, solve_ms;
  int status;
} sa_solve_info;

/* fills *o with the defaults listed above; returns SA_OK */
int sa_default_options(sa_options* o);

/*
 * Builds the hierarchy (Sec. 2 and 3; steps a1-a15 of the hot path): copies
 * the inputs into handle-owned device memory, then per level computes the
 * strength mask, filtered graph, MIS-2 aggregates, tentative and smoothed
 * prolongators, coarse auxiliary data and the Galerkin product, then the
 * smoother and coarse-solve data.  *out receives the handle on SA_OK and is
 * NULL otherwise.  Blocks the calling thread until setup has finished
 * (sizes are read back between steps).
 */
int sa_setup(const sa_problem* prob, const sa_options* opt, sa_handle* out);

/*
 * Solves A x = b by CG preconditioned with one V(1,1) cycle per iteration
 * (Sec. 4; flexible CG for SA_PREC_FP32_VCYCLE) until
 * ||b - A x_k|| <= tol ||b - A x_0||.  b and x are n-vectors, both device or
 * both host pointers; x holds the initial guess on entry and the solution on
 * exit (also on SA_ERR_NO_CONVERGENCE).  info may be NULL.
 */
int sa_solve(sa_handle h, const double* b, double* x, double tol, sa_solve_info* info);

/*
 * k independent solves with the same hierarchy (several load cases of one
 * operator, Sec. 4.3: the setup is amortised over right-hand sides); B and X
 * are column-major n x k (column c starts at B + c*n), both device or both
 * host pointers; infos (may be NULL) receives k entries.  The columns run in
 * blocks of up to 8 that share every launch (operator products, V-cycle,
 * vector updates); each column follows the one-vector arithmetic in the same
 * order, so column c ends bitwise where sa_solve(b_c) ends (same iterations,
 * status and x).  Returns SA_OK, SA_ERR_NO_CONVERGENCE or SA_ERR_BREAKDOWN
 * (the first failing column's status; every column's status is in infos),
 * or an error of the whole call.  Block buffers (about 7 n x 8 doubles plus
 * the V-cycle's n_l x 8 vectors) are allocated on the first call.
 */
int sa_solve_batch(sa_handle h, int k, const double* B, double* X, double tol, sa_solve_info* infos);

/*
 * sa_solve_batch from the zero initial guess (the usual case of Sec. 4's
 * solves): X is output only -- nothing is read from it, and no host buffer
 * of zeros is filled or copied to the device; the device copy of the
 * initial guess is zero-filled in place.  Same arguments, statuses and
 * results as sa_solve_batch with X zero on entry (bitwise).  No counterpart
 * in the paper.
 */
int sa_solve_batch_zero(sa_handle h, int k, const double* B, double* X, double tol, sa_solve_info* infos);

/*
 * Switches the solve form of an existing hierarchy (the FP32 copies of the
 * scaled hierarchy are built on the first switch to SA_PREC_FP32_VCYCLE and
 * kept).  Blocks until that build has finished.
 */
int sa_set_precision(sa_handle h, sa_precision p);

/*
 * One application of the preconditioner z = M r (the V-cycle of
 * Algorithm 1 in the handle's precision); r, z device n-vectors.
 */
int sa_vcycle(sa_handle h, const double* r, double* z);

/*
 * Hierarchy statistics: *levels; n_l[levels], nnz_l[levels] (arrays of at
 * least 32 entries, may be NULL); *op_complexity = sum nnz(A_l) / nnz(A_1)
 * (Sec. 2.2); *device_bytes = device memory held by the handle.
 */
int sa_hierarchy_stats(sa_handle h, int* levels, int64_t* n_l, int64_t* nnz_l, double* op_complexity,
                       int64_t* device_bytes);

/*
 * Sizes of level l: out[0] = n_l, out[1] = nnz(A_l), out[2] = nnz(P_l),
 * out[3] = n_{l+1} (0 on the coarsest level), out[4] = nnz of the filtered graph.
 */
int sa_level_sizes(sa_handle h, int l, int64_t* out);

/*
 * Storage the FP64 V-cycle chose for the scaled operator of level l
 * (inspection only): out[0] = 0 for SELL-32, else the CSR lanes per row,
 * -1 on the coarsest (dense) level; out[1] = rows in the CSR long-row bin
 * (one warp each); out[2] = the entry count above which a row is in that
 * bin (-1: no bin); out[3] = stored entries (SELL: with padding); out[4] =
 * SELL-32 lanes per row (1 or 2; 0 otherwise).  out: 5 host int64.  Errors:
 * SA_ERR_INVALID_ARG for a NULL handle or out, or l out of range.
 */
int sa_level_format(sa_handle h, int l, int64_t* out);

/*
 * Copies level l to HOST arrays (any pointer may be NULL to skip it):
 * aggregate map agg[n_l] (-1 = Dirichlet), P_l in CSR (n_l x n_{l+1}) and A_l
 * in CSR.  Used by the parity tests.
 */
int sa_export_level(sa_handle h, int l, int32_t* agg, int64_t* P_rowptr, int32_t* P_col, double* P_val,
                    int64_t* A_rowptr, int32_t* A_col, double* A_val);

/*
 * Copies the strength data of level l to HOST arrays (NULL skips): keep mask
 * per stored entry of A_l, MIS-2 roots and Dirichlet flags per node (needs
 * options.keep_setup_data = 1), coordinates n_l*dim and inverse tensors
 * n_l*kp (material/distance measures), and scalars[4] = {omega,
 * lambda_omega, cheb_lambda_max, cheb_lambda_min}.
 */
int sa_export_strength(sa_handle h, int l, uint8_t* keep, uint8_t* root, uint8_t* dirichlet, double* coords,
                       double* sigma_inv, double* scalars);

/* releases every device buffer of the handle (stream-ordered) */
int sa_free(sa_handle h);

/*
 * Hierarchy store (no counterpart in the paper, which rebuilds the hierarchy
 * in every run; Sec. 4.3 notes that the setup cost is amortised over
 * right-hand sides, and a stored hierarchy carries that over to another
 * process or a later run).  The store holds the FP64 hierarchy: per level
 * A_l (CSR), its diagonal, P_l and R_l = P_l^T (CSR), the aggregate map and
 * the smoother scalars (omega, lambda_omega, Chebyshev bounds), plus the
 * options that built it.  Loading re-derives the rest deterministically
 * (reciprocal diagonals, the coarse Cholesky factor, the SELL copies of the
 * scaled hierarchy), so a loaded handle solves bit-identically to the one
 * that was stored.
 *
 * Format: a 112-byte header (magic "SAAMGH1", version 1, byte-order mark
 * 0x01020304, dim, levels, n, the setup options, payload bytes, FNV-1a-64
 * checksum over the payload's 64-bit words) followed by the levels, each a
 * 72-byte record {n, nnz, nc, nnzP, nnz_gc, omega, lambda_omega, lmax, lmin}
 * and its arrays in the order rp, col, val, diag [, P rp, P col, P val,
 * R rp, R col, R val, agg], every array zero-padded to 8 bytes.  Host byte
 * order; a store written on a machine of the other order is rejected.
 */

/* *bytes = size of the store of h (the buffer sa_serialize needs) */
int sa_serialized_size(sa_handle h, uint64_t* bytes);

/* writes the store of h into the caller-owned HOST buffer buf of `bytes`
 * bytes (>= sa_serialized_size, else SA_ERR_INVALID_ARG); synchronises the
 * handle's stream */
int sa_serialize(sa_handle h, void* buf, uint64_t bytes);

/*
 * Builds a handle from a store in the HOST buffer buf (`bytes` = its exact
 * size).  opt supplies the stream, the allocator callbacks, maxit and the
 * solve precision; every setup option is taken from the store.  Returns
 * SA_ERR_INVALID_ARG (with sa_last_error text) for a wrong magic, version,
 * byte order or size, a checksum mismatch, inconsistent level sizes or CSR
 * arrays whose row pointers or columns are out of range (checked on the
 * device before any use); SA_ERR_OOM when memory runs out.  The buffer is
 * only read and may be freed on return.
 */
int sa_deserialize(const void* buf, uint64_t bytes, const sa_options* opt, sa_handle* out);

/* static description of a status code */
const char* sa_status_string(int status);

/* text of the last CUDA error seen by this thread (empty if none) */
const char* sa_last_error(void);

/* number of kernel launches issued by this library in this process so far
 * (measurement support; no counterpart in the paper) */
int64_t sa_launch_count(void);

/*
 * sa_solve_group: m independent problems -- m different handles, one
 * right-hand side each -- solved together, every step in shared launches:
 * each operator product, V-cycle kernel (all levels; the dense coarse
 * solves of all problems together at the bottom of the cycle) and CG vector
 * update is one launch covering every problem still iterating.  This is the
 * continuous-batching form of the serving loop (requests for different
 * operators in flight together); no counterpart in the paper (a serving
 * extension; the method per problem is PCG / flexible CG as for sa_solve).
 *   - hs[m]: distinct handles with the same precision setting, Chebyshev
 *     degree and maxit, all on the current device; B[i], X[i]: n_i doubles
 *     (host or device pointers; X[i] in: initial guess, out: solution).
 *   - Each problem follows exactly the arithmetic of sa_solve: its iterations,
 *     status and solution are bitwise those of sa_solve on that handle alone.
 *   - Runs on hs[0]'s stream after the work already queued on every handle's
 *     stream; the handles must not be used elsewhere until the call returns
 *     (it synchronises before returning).  1 <= m <= 64.
 *   - Returns SA_OK when every problem converged, else the first non-OK
 *     problem status (per-problem status in infos[i].status; infos may be
 *     NULL); SA_ERR_INVALID_ARG for duplicate handles or mixed settings.
 */
int sa_solve_group(int m, sa_handle* hs, const double* const* B, double* const* X, double tol,
                   sa_solve_info* infos);

/*
 * Single steps on caller-provided DEVICE buffers, for stepwise parity checks
 * and for callers that build their own pipeline.  Ordered on `stream`.
 *
 * sa_strength: the per-edge strength filter of Sec. 2.1 / Sec. 3 with
 *   pointwise dropping on CSR (n, row_ptr, col, val).  keep[nnz] receives
 *   1 for the diagonal and for kept off-diagonals.  dirichlet[n] (may be
 *   NULL) excludes nodes.  CLASSICAL reads val; MATERIAL reads coords
 *   (n*dim) and sigma_inv (n*kp, inverse nodal tensors); DISTANCE reads
 *   coords only.  Scratch: the MATERIAL/DISTANCE measures need
 *   nnz + n doubles of device scratch, allocated and freed inside the call
 *   with cudaMallocAsync on `stream`.
 */
int sa_strength(sa_measure measure, int dim, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                const double* val, const double* coords, const double* sigma_inv, const uint8_t* dirichlet,
                double theta, uint8_t* keep, void* stream);

/*
 * sa_strength_material_noalloc: the material-aware strength filter of
 * sa_strength (SA_MEASURE_MATERIAL, same kernels, same bit-exact keep mask)
 * for callers that must not allocate device memory during the call: code
 * under an allocator or memory-pool policy that forbids new allocations, a
 * real-time or callback context where an allocation could block or fail, or
 * an application that owns all device memory and passes only inputs and
 * outputs.  (The paper has no counterpart; this is a deployment variant.)
 *   - Allocates nothing: its scratch (w and D, nnz + n doubles) is a fixed
 *     16 MiB static device array (plus one 256-byte line for an input-check
 *     flag) that every GPU loading this library holds until the process
 *     exits.  Sizes with nnz + n > 2,097,152 return SA_ERR_CAPACITY (see
 *     sa_last_error) without launching anything.
 *   - Inputs and outputs are caller-owned DEVICE buffers as for sa_strength:
 *     row_ptr[n+1], col[nnz], coords[n*dim], sigma_inv[n*kp] (inverse nodal
 *     tensors; identity tensors give the plain distance Laplacian),
 *     dirichlet[n] (may be NULL), keep[nnz] (output).  Ordered on `stream`.
 *   - The CSR is checked on the device before any weight is computed
 *     (row_ptr[0] = 0, monotone, row_ptr[n] = nnz, columns strictly
 *     ascending in [0, n)); the call waits for `stream` once to read that
 *     check, and a malformed CSR returns SA_ERR_INVALID_ARG with nothing
 *     written to keep or beyond the scratch array.
 *   - Each call looks up the device address of the array
 *     (cudaGetSymbolAddress) with the calling device current; the first
 *     call on a device loads the module there, so make that first call
 *     outside any stream capture.
 *   - All calls share the one array and every call overwrites it completely
 *     before reading it, so nothing carries over between calls; calls whose
 *     GPU work overlaps (different streams, host threads) race on it and
 *     must be serialised by the caller.
 */
int sa_strength_material_noalloc(int dim, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                 const double* coords, const double* sigma_inv, const uint8_t* dirichlet,
                                 double theta, uint8_t* keep, void* stream);

/*
 * Solve-phase kernel timing (no counterpart in the paper; measurement
 * support).  sa_profile_enable(1) clears the record and, until
 * sa_profile_enable(0), brackets every V-cycle and CG kernel launch with CUDA
 * events on the launching stream.  sa_profile_read synchronises on the
 * recorded events and fills up to max_rows rows, one per (kernel kind,
 * level): kind (0 FP64 Chebyshev step, 1 FP64 residual, 2 FP64 restriction,
 * 3 FP64 prolongation, 4 FP64 first Chebyshev step, 5 CG operator product,
 * 6 CG vector update / dot, 7 dense coarse solve, 8 FP32 Chebyshev step,
 * 9 FP32 residual, 10 FP32 restriction, 11 FP32 prolongation, 12 FP32 first
 * step; setup phases, stream time from the phase's first to last launch:
 * 13 nodal tensors, 14 strength, 15 filtered graph, 16 MIS-2, 17
 * aggregation, 18 filtered matrix, 19 omega, 20 smoothed P, 21 transpose,
 * 22 Galerkin product, 23 coarse aux data, 24 Chebyshev bounds, 25 dense
 * coarse factor, 26 SELL packing, 27 Galerkin A*P, 28 Galerkin R*(AP); the
 * K-column kernels of sa_solve_batch: 29-33 FP64 Chebyshev step, residual,
 * restriction, prolongation, first step, 34 dense coarse solve, 35-39 the
 * same five in FP32, 40 outer FP64 product with the p.q partials, 41 CG
 * vector updates and dot products on K columns), level,
 * launches, total milliseconds, and
 * total algorithmic bytes (bytes the kernel must move at least once; 0 for
 * the setup phases).  *rows receives the number of
 * rows available.  Host-side timing arrays, any may be NULL.
 */
int sa_profile_enable(int on);
int sa_profile_read(int max_rows, int* kind, int* level, int64_t* launches, double* total_ms, double* bytes,
                    int* rows);

#ifdef __cplusplus
}
#endif
#endif
