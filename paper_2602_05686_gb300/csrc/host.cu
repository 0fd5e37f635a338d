// Host orchestration behind the C ABI: hierarchy setup (Sec. 2-3), the
// V-cycle of Algorithm 1 with Chebyshev smoothing and the dense coarse
// solve, and (flexible) CG (Sec. 4).  Every numerical step is a kernel; the
// host only sequences launches and reads back sizes and convergence flags.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <type_traits>
#include <memory>
#include <vector>

#include "common.cuh"
#include "group.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "solve.cuh"
#include "vcycle.cuh"

namespace sa {

struct Level {
  int64_t n = 0, nnz = 0;
  Buf<int64_t> rp;
  Buf<int32_t> ci;
  Buf<double> v;
  Buf<double> diag, dinv;
  int sw = 8;
  // transfer operators (levels above the coarsest)
  int64_t nc = 0, nnzP = 0, nnz_gc = 0;
  int mis_rounds = 0;
  Buf<int32_t> agg;
  Buf<int64_t> Prp, Rrp;
  Buf<int32_t> Pci, Rci;
  Buf<double> Pv, Rv;
  // auxiliary data (material / distance measures)
  Buf<double> x, sigma, sinv;
  // optional diagnostics
  Buf<uint8_t> keep, root, dir;
  double omega = 0, lam_omega = 0, lmax = 0, lmin = 0;

};

}  // namespace sa

struct sa_handle_s {
  sa::Alloc al;
  sa_options opt;
  int dim = 0;
  int64_t n = 0;
  std::vector<std::unique_ptr<sa::Level>> lev;
  sa::CoarseFactor cf;  // coarse Cholesky factor and diagonal-block inverses
  int64_t nL = 0;
  sa::Sell<double> A0s;  // fine operator (unscaled) for the outer CG
  // Krylov workspace (FP64, fine level)
  sa::Buf<double> r, p, q, rprev, t, part, dots, xb, bb;
  sa::Buf<sa::CgScalars> cg;
  double* host_pin = nullptr;  // pinned readback buffer
  int zero_guess = 0;          // set for one sa_solve_batch_zero call: x is output only
  sa::VHier<double>* v64 = nullptr;  // FP64 V-cycle on the scaled hierarchy
  sa::VHier<float>* v32 = nullptr;   // FP32 V-cycle on the scaled hierarchy
  double setup_ms = 0;
  // device-driven CG loop: one captured graph per solve form
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int graph_failed = 0;
  long long body_launches[2] = {0, 0};  // kernels of one captured CG iteration
  sa::Buf<int> it_dev;
  sa::Buf<double> ctl;  // [0] tol * r0
  // k-column solve workspace (interleaved n x KMAX_BLOCK blocks), made on first use
  int kready = 0;
  sa::Buf<double> kR, kP, kQ, kRp, kT, kX, kB, kStage, kpart, kdots;
  sa::Buf<sa::CgScalars> kS;
  sa::Buf<int> kact;
};

namespace sa {

static int level_diag(sa_handle h, Level& L, uint8_t* dir, int* err) {
  SA_TRY(L.diag.alloc(&h->al, L.n));
  SA_TRY(launch_dirichlet_diag(h->al.stream, L.n, L.rp.p, L.ci.p, L.v.p, dir, L.diag.p, err));
  L.sw = pick_sw(L.n, L.nnz);
  return SA_OK;
}

static int read_i64(cudaStream_t s, const int64_t* d, int64_t* h) { return copy_d2h(h, d, sizeof(int64_t), s); }

// one coarsening step: level l -> level l+1.  *stop = 1 when level l is the
// coarsest (stagnation or nothing to coarsen).
#define PHASE_BEGIN(kind, level) int _ph_##kind = prof_begin(s, (kind), (level), 0.0)
#define PHASE_END(kind) prof_end(s, _ph_##kind)

static int coarsen(sa_handle h, int l, int* err, int* stop) {
  Alloc& al = h->al;
  cudaStream_t s = al.stream;
  const sa_options& o = h->opt;
  Level& L = *h->lev[l];
  const int64_t n = L.n, nnz = L.nnz;
  const uint8_t* dir = (l == 0) ? L.dir.p : nullptr;
  const bool aux = o.measure != SA_MEASURE_CLASSICAL;
  *stop = 0;

  // a3/a4: strength + pointwise dropping; kept counts per row -> rpF
  PHASE_BEGIN(PK_S_STRENGTH, l);
  Buf<uint8_t> keep;
  Buf<int64_t> rpF;
  SA_TRY(keep.alloc(&al, nnz));
  SA_TRY(rpF.alloc(&al, n + 1));
  SA_TRY(memset_d(rpF.p, 0, sizeof(int64_t), s));
  if (!aux) {
    SA_TRY(launch_strength_classical(s, n, L.rp.p, L.ci.p, L.v.p, L.diag.p, dir, o.theta, keep.p, rpF.p));
    if (o.drop == SA_DROP_CUT)
      SA_TRY(launch_cut_drop(al, 1, n, nnz, L.rp.p, L.ci.p, L.v.p, L.diag.p, nullptr, nullptr, dir, o.theta, keep.p,
                             rpF.p));
  } else {
    Buf<double> w, D;
    SA_TRY(w.alloc(&al, nnz));
    SA_TRY(D.alloc(&al, n));
    SA_TRY(launch_strength_material(s, h->dim, n, L.rp.p, L.ci.p, L.x.p, L.sinv.p, dir, o.theta, w.p, D.p, keep.p,
                                    rpF.p));
    if (o.drop == SA_DROP_CUT)
      SA_TRY(launch_cut_drop(al, 0, n, nnz, L.rp.p, L.ci.p, nullptr, nullptr, w.p, D.p, dir, o.theta, keep.p, rpF.p));
  }
  SA_TRY(scan_inplace(al, rpF.p + 1, n));
  int64_t nnzF = 0;
  SA_TRY(read_i64(s, rpF.p + n, &nnzF));
  PHASE_END(PK_S_STRENGTH);

  // a5: filtered graph
  PHASE_BEGIN(PK_S_GRAPH, l);
  Buf<int64_t> gcrp;
  Buf<int32_t> gcci;
  L.nnz_gc = nnzF - n;
  SA_TRY(gcrp.alloc(&al, n + 1));
  SA_TRY(gcci.alloc(&al, L.nnz_gc));
  SA_TRY(launch_graph_rowptr(s, n, rpF.p, gcrp.p));
  SA_TRY(launch_graph_compact(s, n, L.rp.p, L.ci.p, keep.p, gcrp.p, gcci.p));
  PHASE_END(PK_S_GRAPH);

  // a6/a7: MIS-2 and aggregates
  PHASE_BEGIN(PK_S_MIS, l);
  Buf<uint64_t> tag;
  SA_TRY(tag.alloc(&al, n));
  SA_TRY(run_mis2(al, n, gcrp.p, gcci.p, dir, l, o.seed, tag.p, &L.mis_rounds, 100000));
  PHASE_END(PK_S_MIS);
  PHASE_BEGIN(PK_S_AGG, l);
  SA_TRY(L.agg.alloc(&al, n));
  Buf<uint8_t> root;
  if (o.keep_setup_data) SA_TRY(root.alloc(&al, n));
  int64_t nc = 0;
  SA_TRY(run_aggregate(al, n, gcrp.p, gcci.p, dir, tag.p, L.agg.p, o.keep_setup_data ? root.p : nullptr, &nc, err));
  if (o.keep_setup_data) {
    L.keep = std::move(keep);
    L.root = std::move(root);
  }
  if (nc == 0 || (double)nc > 0.9 * (double)n) {
    L.agg.release();
    *stop = 1;
    return SA_OK;
  }
  L.nc = nc;

  // a8: tentative prolongator
  Buf<int64_t> Trp;
  Buf<int32_t> Tci;
  Buf<double> Tv;
  SA_TRY(Trp.alloc(&al, n + 1));
  SA_TRY(memset_d(Trp.p, 0, sizeof(int64_t), s));
  SA_TRY(launch_tentative_count(s, n, L.agg.p, Trp.p));
  SA_TRY(scan_inplace(al, Trp.p + 1, n));
  int64_t nnzT = 0;
  SA_TRY(read_i64(s, Trp.p + n, &nnzT));
  SA_TRY(Tci.alloc(&al, nnzT));
  SA_TRY(Tv.alloc(&al, nnzT));
  SA_TRY(launch_tentative(s, n, L.agg.p, Trp.p, Tci.p, Tv.p));
  PHASE_END(PK_S_AGG);

  // a10: filtered matrix and 1-norm diagonal
  PHASE_BEGIN(PK_S_FILTER, l);
  Buf<int32_t> ciF;
  Buf<double> vF, Dt, sc, scal;
  SA_TRY(ciF.alloc(&al, nnzF));
  SA_TRY(vF.alloc(&al, nnzF));
  SA_TRY(Dt.alloc(&al, n));
  const uint8_t* keep_p = o.keep_setup_data ? L.keep.p : keep.p;
  SA_TRY(launch_filter(s, n, L.rp.p, L.ci.p, L.v.p, keep_p, rpF.p, ciF.p, vF.p, Dt.p));
  PHASE_END(PK_S_FILTER);

  // a11: omega = omega_sym / rho(D~^-1 A_F)
  PHASE_BEGIN(PK_S_OMEGA, l);
  SA_TRY(sc.alloc(&al, n));
  SA_TRY(scal.alloc(&al, 2));
  SA_TRY(launch_rsqrt_scale(s, n, Dt.p, sc.p));
  SA_TRY(run_power(al, n, rpF.p, ciF.p, vF.p, sc.p, o.power_iters, (uint32_t)(2 * l + 1), o.seed, scal.p));
  SA_TRY(launch_omega(s, scal.p, o.omega_sym, scal.p + 1));
  PHASE_END(PK_S_OMEGA);

  // a12: P = P^ - omega D~^-1 A_F P^
  PHASE_BEGIN(PK_S_SMOOTHP, l);
  SA_TRY(run_spgemm(al, n, nc, n, rpF.p, ciF.p, vF.p, Trp.p, Tci.p, Tv.p, L.Prp, L.Pci, L.Pv, &L.nnzP));
  SA_TRY(launch_smooth_p_values(s, n, L.Prp.p, L.Pci.p, L.Pv.p, L.agg.p, Dt.p, scal.p + 1, L.Pv.p));
  PHASE_END(PK_S_SMOOTHP);
  double hs[2];
  SA_TRY(copy_d2h(hs, scal.p, sizeof(hs), s));
  L.lam_omega = hs[0];
  L.omega = hs[1];

  // a13: R = P^T, A_{l+1} = R (A P), exactly symmetric
  PHASE_BEGIN(PK_S_TRANSPOSE, l);
  SA_TRY(run_transpose(al, n, nc, L.Prp.p, L.Pci.p, L.Pv.p, L.Rrp, L.Rci, &L.Rv));
  PHASE_END(PK_S_TRANSPOSE);
  PHASE_BEGIN(PK_S_RAP, l);
  Buf<int64_t> APrp;
  Buf<int32_t> APci;
  Buf<double> APv;
  int64_t nnzAP = 0;
  PHASE_BEGIN(PK_S_RAP_AP, l);
  SA_TRY(run_spgemm(al, n, nc, n, L.rp.p, L.ci.p, L.v.p, L.Prp.p, L.Pci.p, L.Pv.p, APrp, APci, APv, &nnzAP));
  PHASE_END(PK_S_RAP_AP);
  std::unique_ptr<Level> N(new Level());
  N->n = nc;
  // R (A P) is symmetric: only its upper triangle is accumulated, the lower
  // one is mirrored from it
  PHASE_BEGIN(PK_S_RAP_RAP, l);
  SA_TRY(run_spgemm(al, nc, nc, n, L.Rrp.p, L.Rci.p, L.Rv.p, APrp.p, APci.p, APv.p, N->rp, N->ci, N->v, &N->nnz,
                    1));
  SA_TRY(launch_symmetrize(s, nc, N->rp.p, N->ci.p, N->v.p, err));
  PHASE_END(PK_S_RAP_RAP);
  SA_TRY(level_diag(h, *N, nullptr, err));
  PHASE_END(PK_S_RAP);

  // a9: coarse coordinates and tensors
  if (aux) {
    PHASE_BEGIN(PK_S_AUX, l);
    Buf<int64_t> Mrp;
    Buf<int32_t> Mci;
    SA_TRY(run_transpose(al, n, nc, Trp.p, Tci.p, nullptr, Mrp, Mci, nullptr));
    const int kp = h->dim == 3 ? 6 : 3;
    SA_TRY(N->x.alloc(&al, nc * h->dim));
    SA_TRY(N->sigma.alloc(&al, nc * kp));
    SA_TRY(N->sinv.alloc(&al, nc * kp));
    SA_TRY(launch_coarse_aux(s, nc, h->dim, Mrp.p, Mci.p, L.x.p, L.sigma.p, N->x.p, N->sigma.p, N->sinv.p));
    PHASE_END(PK_S_AUX);
  }
  h->lev.push_back(std::move(N));
  return SA_OK;
}

static int alloc_workspace(sa_handle h) {
  Alloc& al = h->al;
  const int64_t n = h->n;
  SA_TRY(h->r.alloc(&al, n));
  SA_TRY(h->p.alloc(&al, n));
  SA_TRY(h->q.alloc(&al, n));
  SA_TRY(h->rprev.alloc(&al, n));
  SA_TRY(h->t.alloc(&al, n));
  SA_TRY(h->xb.alloc(&al, n));
  SA_TRY(h->bb.alloc(&al, n));
  int64_t np = blocks_for(n * 32, 256) + RED_BLOCKS;
  SA_TRY(h->part.alloc(&al, 3 * np));
  SA_TRY(h->dots.alloc(&al, 8));
  SA_TRY(h->cg.alloc(&al, 1));
  SA_TRY(h->it_dev.alloc(&al, 1));
  SA_TRY(h->ctl.alloc(&al, 1));
  return SA_OK;
}

#define PROF(kind, level, bytes, call)                          \
  do {                                                          \
    int _pi = prof_begin(s, (kind), (level), (bytes));          \
    int _st = (call);                                           \
    prof_end(s, _pi);                                           \
    if (_st != SA_OK) return _st;                               \
  } while (0)

static int precondition(sa_handle h, const double* r, double** z) {
  if (h->opt.precision == SA_PREC_FP32_VCYCLE) return vh_vcycle<float>(h->v32, h->al.stream, r, z);
  return vh_vcycle<double>(h->v64, h->al.stream, r, z);
}

// outer-CG operator products on the FP64 SELL copy of the fine operator
static int op_spmv_dot(sa_handle h, const double* p, double* q, double* part, int* np) {
  return launch_sell_spmv_dot(h->al.stream, h->A0s, p, q, part, np);
}
static int op_residual(sa_handle h, const double* b, const double* x, double* r) {
  return launch_sell_residual64(h->al.stream, h->A0s, b, x, r);
}

struct HostScal {
  double rr, pad0, pad1;
};

// the initial guess into a device buffer: copied from x (host or device), or
// zero-filled on the device when the call has no initial guess
static int copy_in_guess(sa_handle h, double* dst, const double* x, size_t bytes) {
  if (h->zero_guess) SA_CUDA(cudaMemsetAsync(dst, 0, bytes, h->al.stream));
  else SA_CUDA(cudaMemcpyAsync(dst, x, bytes, cudaMemcpyDefault, h->al.stream));
  return SA_OK;
}

// CG / flexible CG on device buffers b, x (Sec. 4), host-driven: one
// readback per iteration.  Used when profiling (events bracket every launch).
static int cg_eager_dev(sa_handle h, const double* b, double* x, double tol, sa_solve_info* info);
static int cg_eager(sa_handle h, const double* b, double* x, double tol, sa_solve_info* info) {
  cudaStream_t s = h->al.stream;
  SA_CUDA(cudaMemcpyAsync(h->bb.p, b, sizeof(double) * h->n, cudaMemcpyDefault, s));
  SA_TRY(copy_in_guess(h, h->xb.p, x, sizeof(double) * h->n));
  int st = cg_eager_dev(h, h->bb.p, h->xb.p, tol, info);
  SA_CUDA(cudaMemcpyAsync(x, h->xb.p, sizeof(double) * h->n, cudaMemcpyDefault, s));
  SA_CUDA(cudaStreamSynchronize(s));
  return st;
}

static int cg_eager_dev(sa_handle h, const double* b, double* x, double tol, sa_solve_info* info) {
  cudaStream_t s = h->al.stream;
  Level& L0 = *h->lev[0];
  const int64_t n = h->n;
  const int flexible = h->opt.precision == SA_PREC_FP32_VCYCLE;
  double* hp = h->host_pin;
  auto t0 = std::chrono::steady_clock::now();
  int status = SA_ERR_NO_CONVERGENCE, it = 0;
  double r0 = 0.0;
  SA_TRY(op_residual(h, b, x, h->r.p));
  SA_TRY(launch_dots(s, n, h->r.p, h->r.p, nullptr, nullptr, nullptr, nullptr, h->part.p, h->dots.p));
  SA_CUDA(cudaMemcpyAsync(hp, h->dots.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  SA_CUDA(cudaStreamSynchronize(s));
  r0 = sqrt(hp[0]);
  if (r0 > 0.0) {
    double* z = nullptr;
    SA_TRY(precondition(h, h->r.p, &z));
    SA_TRY(launch_cg_pupdate(s, n, h->cg.p, z, h->p.p, 1));
    SA_TRY(launch_dots(s, n, h->r.p, z, nullptr, nullptr, nullptr, nullptr, h->part.p, h->dots.p));
    SA_TRY(launch_cg_beta(s, h->cg.p, h->dots.p, -1));
    const int maxit = h->opt.maxit;
    for (it = 1; it <= maxit; ++it) {
      int np = 0;
      PROF(PK_CG_SPMV, 0, (8.0 + h->A0s.idx_bytes()) * L0.nnz + 8.0 * (h->A0s.nslices + 1) + 16.0 * n,
           op_spmv_dot(h, h->p.p, h->q.p, h->part.p, &np));
      SA_TRY(launch_finish(s, h->part.p, np, h->dots.p));
      SA_TRY(launch_cg_alpha(s, h->cg.p, h->dots.p));
      PROF(PK_CG_VEC, 0, (flexible ? 56.0 : 48.0) * n,
           launch_cg_update(s, n, h->cg.p, h->p.p, h->q.p, x, h->r.p, flexible ? h->rprev.p : nullptr, h->part.p));
      SA_TRY(launch_finish(s, h->part.p, RED_BLOCKS, h->dots.p + 4));
      SA_CUDA(cudaMemcpyAsync(hp, h->dots.p + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
      SA_CUDA(cudaMemcpyAsync(hp + 1, &h->cg.p->breakdown, sizeof(int), cudaMemcpyDeviceToHost, s));
      SA_CUDA(cudaStreamSynchronize(s));
      int brk = 0;
      memcpy(&brk, hp + 1, sizeof(int));
      if (brk) { status = SA_ERR_BREAKDOWN; break; }
      if (sqrt(hp[0]) <= tol * r0) {
        SA_TRY(op_residual(h, b, x, h->t.p));
        SA_TRY(launch_dots(s, n, h->t.p, h->t.p, nullptr, nullptr, nullptr, nullptr, h->part.p, h->dots.p + 4));
        SA_CUDA(cudaMemcpyAsync(hp, h->dots.p + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
        SA_CUDA(cudaStreamSynchronize(s));
        if (sqrt(hp[0]) <= tol * r0) { status = SA_OK; break; }
        SA_CUDA(cudaMemcpyAsync(h->r.p, h->t.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      }
      SA_TRY(precondition(h, h->r.p, &z));
      PROF(PK_CG_VEC, 0, (flexible ? 24.0 : 16.0) * n,
           launch_dots(s, n, h->r.p, z, flexible ? z : nullptr, flexible ? h->rprev.p : nullptr, nullptr, nullptr,
                       h->part.p, h->dots.p));
      SA_TRY(launch_cg_beta(s, h->cg.p, h->dots.p, flexible));
      PROF(PK_CG_VEC, 0, 24.0 * n, launch_cg_pupdate(s, n, h->cg.p, z, h->p.p, 0));
    }
    if (it > maxit) it = maxit;
  } else {
    status = SA_OK;
  }
  // true residual at exit
  SA_TRY(op_residual(h, b, x, h->t.p));
  SA_TRY(launch_dots(s, n, h->t.p, h->t.p, nullptr, nullptr, nullptr, nullptr, h->part.p, h->dots.p + 4));
  SA_CUDA(cudaMemcpyAsync(hp, h->dots.p + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
  SA_CUDA(cudaStreamSynchronize(s));
  auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->iters = it;
    info->rel_res_true = r0 > 0.0 ? sqrt(hp[0]) / r0 : 0.0;
    info->setup_ms = h->setup_ms;
    info->solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->status = status;
  }
  return status;
}


// loop control inside the captured CG body: count the iteration and decide
// whether the WHILE node runs the body again
__global__ void k_loop_ctrl(cudaGraphConditionalHandle ch, int* __restrict__ it, const CgScalars* __restrict__ s,
                            const double* __restrict__ rr, const double* __restrict__ ctl, int maxit) {
  int k = *it + 1;
  *it = k;
  int cont = !s->breakdown && !(sqrt(*rr) <= ctl[0]) && k < maxit;
  cudaGraphSetConditional(ch, cont ? 1u : 0u);
}

// the second half of one CG iteration followed by the first half of the next:
// z = M r, beta, p = z + beta p, q = A p, alpha, x/r update, ||r||^2, control
static int cg_body(sa_handle h, cudaGraphConditionalHandle ch) {
  cudaStream_t s = h->al.stream;
  Level& L0 = *h->lev[0];
  const int64_t n = h->n;
  const int flexible = h->opt.precision == SA_PREC_FP32_VCYCLE;
  double* z = nullptr;
  SA_TRY(precondition(h, h->r.p, &z));
  SA_TRY(launch_dots(s, n, h->r.p, z, flexible ? z : nullptr, flexible ? h->rprev.p : nullptr, nullptr, nullptr,
                     h->part.p, h->dots.p));
  SA_TRY(launch_cg_beta(s, h->cg.p, h->dots.p, flexible));
  SA_TRY(launch_cg_pupdate(s, n, h->cg.p, z, h->p.p, 0));
  int np = 0;
  SA_TRY(op_spmv_dot(h, h->p.p, h->q.p, h->part.p, &np));
  SA_TRY(launch_finish(s, h->part.p, np, h->dots.p));
  SA_TRY(launch_cg_alpha(s, h->cg.p, h->dots.p));
  SA_TRY(launch_cg_update(s, n, h->cg.p, h->p.p, h->q.p, h->xb.p, h->r.p, flexible ? h->rprev.p : nullptr,
                          h->part.p));
  SA_TRY(launch_finish(s, h->part.p, RED_BLOCKS, h->dots.p + 4));
  k_loop_ctrl<<<1, 1, 0, s>>>(ch, h->it_dev.p, h->cg.p, h->dots.p + 4, h->ctl.p, h->opt.maxit);
  SA_LAUNCHED();
  return SA_OK;
}

static void drop_graph(sa_handle h, int form) {
  if (h->gexec[form]) cudaGraphExecDestroy(h->gexec[form]);
  if (h->graph[form]) cudaGraphDestroy(h->graph[form]);
  h->gexec[form] = nullptr;
  h->graph[form] = nullptr;
}

// captures the body into a graph with a conditional WHILE node; on any
// failure the handle falls back to host-driven iterations
static int capture_loop(sa_handle h, int form) {
  if (h->gexec[form]) return SA_OK;
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return SA_ERR_CUDA;
  }
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle ch;
  cudaGraphNodeParams p = {};
  cudaGraphNode_t node;
  if (cudaGraphCreate(&g, 0) != cudaSuccess ||
      cudaGraphConditionalHandleCreate(&ch, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return SA_ERR_CUDA;
  }
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = ch;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return SA_ERR_CUDA;
  }
  cudaGraph_t body = p.conditional.phGraph_out[0];
  cudaStream_t user = h->al.stream;
  h->al.stream = h->cap_stream;  // every launch of the body goes to the capture stream
  int st = SA_OK;
  if (cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess) {
    st = SA_ERR_CUDA;
  } else {
    const long long c0 = launch_counter();
    st = cg_body(h, ch);
    h->body_launches[form] = launch_counter() - c0;
    count_launches(-h->body_launches[form]);  // captured, not run: counted per replayed iteration
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(h->cap_stream, &out) != cudaSuccess) st = SA_ERR_CUDA;
  }
  h->al.stream = user;
  if (st == SA_OK && cudaGraphInstantiate(&h->gexec[form], g, 0) != cudaSuccess) st = SA_ERR_CUDA;
  cudaGetLastError();
  if (st != SA_OK) {
    h->gexec[form] = nullptr;
    cudaGraphDestroy(g);
    return st;
  }
  h->graph[form] = g;
  return SA_OK;
}

// CG with the iterations after the first run inside one graph launch; the
// host reads back once per launch (convergence candidate, maxit or
// breakdown) and confirms convergence with the true residual.
static int cg_graph(sa_handle h, const double* b, double* x, double tol, sa_solve_info* info) {
  cudaStream_t s = h->al.stream;
  Level& L0 = *h->lev[0];
  const int64_t n = h->n;
  const int form = h->opt.precision == SA_PREC_FP32_VCYCLE ? 1 : 0;
  const int flexible = form;
  double* hp = h->host_pin;
  auto t0 = std::chrono::steady_clock::now();
  SA_CUDA(cudaMemcpyAsync(h->bb.p, b, sizeof(double) * n, cudaMemcpyDefault, s));
  SA_TRY(copy_in_guess(h, h->xb.p, x, sizeof(double) * n));
  int status = SA_ERR_NO_CONVERGENCE, it = 0;
  SA_TRY(op_residual(h, h->bb.p, h->xb.p, h->r.p));
  SA_TRY(launch_dots(s, n, h->r.p, h->r.p, nullptr, nullptr, nullptr, nullptr, h->part.p, h->dots.p));
  SA_CUDA(cudaMemcpyAsync(hp, h->dots.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  SA_CUDA(cudaStreamSynchronize(s));
  const double r0 = sqrt(hp[0]);
  if (r0 > 0.0) {
    hp[2] = tol * r0;
    SA_CUDA(cudaMemcpyAsync(h->ctl.p, hp + 2, sizeof(double), cudaMemcpyHostToDevice, s));
    // first iteration (host-driven)
    double* z = nullptr;
    SA_TRY(precondition(h, h->r.p, &z));
    SA_TRY(launch_cg_pupdate(s, n, h->cg.p, z, h->p.p, 1));
    SA_TRY(launch_dots(s, n, h->r.p, z, nullptr, nullptr, nullptr, nullptr, h->part.p, h->dots.p));
    SA_TRY(launch_cg_beta(s, h->cg.p, h->dots.p, -1));
    int np = 0;
    SA_TRY(op_spmv_dot(h, h->p.p, h->q.p, h->part.p, &np));
    SA_TRY(launch_finish(s, h->part.p, np, h->dots.p));
    SA_TRY(launch_cg_alpha(s, h->cg.p, h->dots.p));
    SA_TRY(launch_cg_update(s, n, h->cg.p, h->p.p, h->q.p, h->xb.p, h->r.p, flexible ? h->rprev.p : nullptr,
                            h->part.p));
    SA_TRY(launch_finish(s, h->part.p, RED_BLOCKS, h->dots.p + 4));
    int one = 1;
    SA_CUDA(cudaMemcpyAsync(h->it_dev.p, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    bool graph_launched = false;
    for (;;) {
      SA_CUDA(cudaMemcpyAsync(hp, h->dots.p + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
      SA_CUDA(cudaMemcpyAsync(hp + 1, &h->cg.p->breakdown, sizeof(int), cudaMemcpyDeviceToHost, s));
      SA_CUDA(cudaMemcpyAsync((char*)(hp + 1) + sizeof(int), h->it_dev.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      SA_CUDA(cudaStreamSynchronize(s));
      int brk = 0;
      memcpy(&brk, hp + 1, sizeof(int));
      memcpy(&it, (char*)(hp + 1) + sizeof(int), sizeof(int));
      if (brk) { status = SA_ERR_BREAKDOWN; break; }
      if (sqrt(hp[0]) <= tol * r0) {
        SA_TRY(op_residual(h, h->bb.p, h->xb.p, h->t.p));
        SA_TRY(launch_dots(s, n, h->t.p, h->t.p, nullptr, nullptr, nullptr, nullptr, h->part.p, h->dots.p + 6));
        SA_CUDA(cudaMemcpyAsync(hp + 3, h->dots.p + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
        SA_CUDA(cudaStreamSynchronize(s));
        if (sqrt(hp[3]) <= tol * r0) { status = SA_OK; break; }
        SA_CUDA(cudaMemcpyAsync(h->r.p, h->t.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      }
      if (it >= h->opt.maxit) break;
      SA_CUDA(cudaGraphLaunch(h->gexec[form], s));
      graph_launched = true;
    }
    if (graph_launched && it > 1) count_launches((long long)(it - 1) * h->body_launches[form]);
  } else {
    status = SA_OK;
  }
  SA_TRY(op_residual(h, h->bb.p, h->xb.p, h->t.p));
  SA_TRY(launch_dots(s, n, h->t.p, h->t.p, nullptr, nullptr, nullptr, nullptr, h->part.p, h->dots.p + 6));
  SA_CUDA(cudaMemcpyAsync(hp + 3, h->dots.p + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
  SA_CUDA(cudaMemcpyAsync(x, h->xb.p, sizeof(double) * n, cudaMemcpyDefault, s));
  SA_CUDA(cudaStreamSynchronize(s));
  auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->iters = it;
    info->rel_res_true = r0 > 0.0 ? sqrt(hp[3]) / r0 : 0.0;
    info->setup_ms = h->setup_ms;
    info->solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->status = status;
  }
  return status;
}

// SA_CG_GRAPH=0 in the environment keeps every CG iteration host-driven (the
// same kernels in the same order, launched one by one): for tools that do not
// look inside conditional graph nodes, such as per-kernel profilers
static bool graphs_allowed() {
  const char* e = getenv("SA_CG_GRAPH");
  return !(e && e[0] == '0');
}

static int cg_device(sa_handle h, const double* b, double* x, double tol, sa_solve_info* info) {
  const int form = h->opt.precision == SA_PREC_FP32_VCYCLE ? 1 : 0;
  if (!prof_on() && !h->graph_failed && graphs_allowed()) {
    if (!h->gexec[form] && capture_loop(h, form) != SA_OK) h->graph_failed = 1;
    if (h->gexec[form]) return cg_graph(h, b, x, tol, info);
  }
  return cg_eager(h, b, x, tol, info);
}


// ---------------------------------------------------------------------------
// k right-hand sides in lockstep (sa_solve_batch): every operator product,
// cycle and vector update is one launch for all k columns, each column
// following the one-vector CG's arithmetic in the same order, so column c
// ends bitwise where sa_solve on that right-hand side ends.  One host
// readback per iteration (squared residual norms and breakdown flags).
// ---------------------------------------------------------------------------
static int block_workspace(sa_handle h) {
  if (h->kready) return SA_OK;
  Alloc& al = h->al;
  const int64_t nk = h->n * KMAX_BLOCK;
  SA_TRY(h->kR.alloc(&al, nk));
  SA_TRY(h->kP.alloc(&al, nk));
  SA_TRY(h->kQ.alloc(&al, nk));
  SA_TRY(h->kRp.alloc(&al, nk));
  SA_TRY(h->kT.alloc(&al, nk));
  SA_TRY(h->kX.alloc(&al, nk));
  SA_TRY(h->kB.alloc(&al, nk));
  SA_TRY(h->kStage.alloc(&al, nk));
  const int64_t np = blocks_for(h->n, 256) + RED_BLOCKS;
  SA_TRY(h->kpart.alloc(&al, 2 * KMAX_BLOCK * np));
  SA_TRY(h->kdots.alloc(&al, 6 * KMAX_BLOCK));  // [0, 2K) dots, [2K, 3K) r.r, [3K, 5K) true residuals
  SA_TRY(h->kS.alloc(&al, KMAX_BLOCK));
  SA_TRY(h->kact.alloc(&al, KMAX_BLOCK));
  h->kready = 1;
  return SA_OK;
}

static int precondition_block(sa_handle h, int k, const double* R, double** Z) {
  if (h->opt.precision == SA_PREC_FP32_VCYCLE) return vh_vcycle_block<float>(h->al, h->v32, h->al.stream, k, R, Z);
  return vh_vcycle_block<double>(h->al, h->v64, h->al.stream, k, R, Z);
}

static int cg_block(sa_handle h, int k, const double* B, double* X, double tol, sa_solve_info* infos, int* statuses) {
  // the block carries K in {2, 4, 8} columns; columns k..K-1 are zero and
  // never active
  const int K = k <= 2 ? 2 : (k <= 4 ? 4 : KMAX_BLOCK);
  cudaStream_t s = h->al.stream;
  const int64_t n = h->n;
  const int flexible = h->opt.precision == SA_PREC_FP32_VCYCLE;
  const int maxit = h->opt.maxit;
  auto t0 = std::chrono::steady_clock::now();
  SA_TRY(block_workspace(h));
  double* R = h->kR.p; double* P = h->kP.p; double* Q = h->kQ.p; double* Rp = h->kRp.p;
  double* T = h->kT.p; double* Xb = h->kX.p; double* Bb = h->kB.p;
  double* part = h->kpart.p; double* dots = h->kdots.p;
  const double vb = 8.0 * (double)n * K;  // bytes of one n x K block
  // inputs: column-major (host or device) -> interleaved
  SA_CUDA(cudaMemcpyAsync(h->kStage.p, B, sizeof(double) * n * k, cudaMemcpyDefault, s));
  SA_TRY(launch_interleave(s, n, k, K, h->kStage.p, Bb, 1));
  if (h->zero_guess) {
    SA_CUDA(cudaMemsetAsync(Xb, 0, sizeof(double) * n * K, s));  // what interleaving zeros gives
  } else {
    SA_CUDA(cudaMemcpyAsync(h->kStage.p, X, sizeof(double) * n * k, cudaMemcpyDefault, s));
    SA_TRY(launch_interleave(s, n, k, K, h->kStage.p, Xb, 1));
  }
  // host view of the columns
  double r0[KMAX_BLOCK], hb[2 * KMAX_BLOCK];
  int act[KMAX_BLOCK], its[KMAX_BLOCK], st[KMAX_BLOCK];
  struct { double rr[KMAX_BLOCK]; CgScalars S[KMAX_BLOCK]; } hr;
  SA_TRY(launch_bsell_residual64(s, h->A0s, K, Bb, Xb, R));
  PROF(PK_B_CG_VEC, 0, 2 * vb, launch_bdots(s, n, K, R, R, nullptr, nullptr, part, dots));
  SA_CUDA(cudaMemcpyAsync(hb, dots, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
  SA_CUDA(cudaStreamSynchronize(s));
  int nact = 0;
  for (int c = 0; c < K; ++c) {
    r0[c] = sqrt(hb[c]);
    act[c] = c < k && r0[c] > 0.0;
    its[c] = 0;
    st[c] = act[c] ? SA_ERR_NO_CONVERGENCE : SA_OK;
    nact += act[c];
  }
  SA_CUDA(cudaMemcpyAsync(h->kact.p, act, sizeof(int) * K, cudaMemcpyHostToDevice, s));
  if (nact > 0) {
    // first iteration
    double* Z = nullptr;
    SA_TRY(precondition_block(h, K, R, &Z));
    PROF(PK_B_CG_VEC, 0, 2 * vb, launch_bcg_pupdate(s, n, K, h->kS.p, h->kact.p, Z, P, 1));
    PROF(PK_B_CG_VEC, 0, 2 * vb, launch_bdots(s, n, K, R, Z, nullptr, nullptr, part, dots));
    SA_TRY(launch_bcg_beta(s, K, h->kS.p, dots, -1, h->kact.p));
    for (int it = 1;; ++it) {
      int np = 0;
      SA_TRY(launch_bsell_spmv_dot(s, h->A0s, K, P, Q, part, &np));
      SA_TRY(launch_bfinish(s, part, np, K, dots));
      SA_TRY(launch_bcg_alpha(s, K, h->kS.p, dots, h->kact.p));
      PROF(PK_B_CG_VEC, 0, (flexible ? 7 : 6) * vb,
           launch_bcg_update(s, n, K, h->kS.p, h->kact.p, P, Q, Xb, R, flexible ? Rp : nullptr, part));
      SA_TRY(launch_bfinish(s, part, RED_BLOCKS, K, dots + 2 * KMAX_BLOCK));
      SA_CUDA(cudaMemcpyAsync(hr.rr, dots + 2 * KMAX_BLOCK, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
      SA_CUDA(cudaMemcpyAsync(hr.S, h->kS.p, sizeof(CgScalars) * K, cudaMemcpyDeviceToHost, s));
      SA_CUDA(cudaStreamSynchronize(s));
      // per column: breakdown, convergence candidate (confirmed on the true
      // residual, which replaces r when it does not confirm), maxit
      bool cand = false;
      for (int c = 0; c < K; ++c) {
        if (!act[c]) continue;
        its[c] = it;
        if (hr.S[c].breakdown) { st[c] = SA_ERR_BREAKDOWN; act[c] = 0; continue; }
        if (sqrt(hr.rr[c]) <= tol * r0[c]) cand = true;
      }
      if (cand) {
        SA_TRY(launch_bsell_residual64(s, h->A0s, K, Bb, Xb, T));
        SA_TRY(launch_bdots(s, n, K, T, T, nullptr, nullptr, part, dots + 3 * KMAX_BLOCK));
        SA_CUDA(cudaMemcpyAsync(hb, dots + 3 * KMAX_BLOCK, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
        SA_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < K; ++c) {
          if (!act[c] || !(sqrt(hr.rr[c]) <= tol * r0[c])) continue;
          if (sqrt(hb[c]) <= tol * r0[c]) {
            st[c] = SA_OK;
            act[c] = 0;
          } else {
            SA_CUDA(cudaMemcpy2DAsync(R + c, sizeof(double) * K, T + c, sizeof(double) * K, sizeof(double), n,
                                      cudaMemcpyDeviceToDevice, s));
          }
        }
      }
      nact = 0;
      for (int c = 0; c < K; ++c) {
        if (act[c] && it >= maxit) act[c] = 0;  // status stays SA_ERR_NO_CONVERGENCE
        nact += act[c];
      }
      SA_CUDA(cudaMemcpyAsync(h->kact.p, act, sizeof(int) * K, cudaMemcpyHostToDevice, s));
      if (nact == 0) break;
      SA_TRY(precondition_block(h, K, R, &Z));
      PROF(PK_B_CG_VEC, 0, (flexible ? 3 : 2) * vb,
           launch_bdots(s, n, K, R, Z, flexible ? Z : nullptr, flexible ? Rp : nullptr, part, dots));
      SA_TRY(launch_bcg_beta(s, K, h->kS.p, dots, flexible, h->kact.p));
      PROF(PK_B_CG_VEC, 0, 3 * vb, launch_bcg_pupdate(s, n, K, h->kS.p, h->kact.p, Z, P, 0));
    }
  }
  // true residuals at exit and the solutions
  SA_TRY(launch_bsell_residual64(s, h->A0s, K, Bb, Xb, T));
  SA_TRY(launch_bdots(s, n, K, T, T, nullptr, nullptr, part, dots + 3 * KMAX_BLOCK));
  SA_CUDA(cudaMemcpyAsync(hb, dots + 3 * KMAX_BLOCK, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
  SA_TRY(launch_interleave(s, n, k, K, Xb, h->kStage.p, 0));
  SA_CUDA(cudaMemcpyAsync(X, h->kStage.p, sizeof(double) * n * k, cudaMemcpyDefault, s));
  SA_CUDA(cudaStreamSynchronize(s));
  SA_TRY(block_stage_status(s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int c = 0; c < k; ++c) {
    statuses[c] = st[c];
    if (infos) {
      infos[c].iters = its[c];
      infos[c].rel_res_true = r0[c] > 0.0 ? sqrt(hb[c]) / r0[c] : 0.0;
      infos[c].setup_ms = h->setup_ms;
      infos[c].solve_ms = ms;
      infos[c].status = st[c];
    }
  }
  return SA_OK;
}

template <typename T>
static int upload(Alloc& al, Buf<T>& dst, const T* src, int64_t count) {
  SA_TRY(dst.alloc(&al, count));
  if (count > 0) SA_CUDA(cudaMemcpyAsync(dst.p, src, sizeof(T) * (size_t)count, cudaMemcpyDefault, al.stream));
  return SA_OK;
}

static std::vector<VLevelIn> vlevel_inputs(sa_handle h) {
  const int nlev = (int)h->lev.size();
  std::vector<VLevelIn> in(nlev);
  for (int l = 0; l < nlev; ++l) {
    Level& L = *h->lev[l];
    in[l].n = L.n; in[l].nnz = L.nnz; in[l].rp = L.rp.p; in[l].ci = L.ci.p; in[l].v = L.v.p;
    in[l].diag = L.diag.p; in[l].lmax = L.lmax; in[l].lmin = L.lmin;
    in[l].nc = (l + 1 < nlev) ? L.nc : 0; in[l].nnzP = L.nnzP;
    in[l].Prp = L.Prp.p; in[l].Pci = L.Pci.p; in[l].Pv = L.Pv.p;
    in[l].Rrp = L.Rrp.p; in[l].Rci = L.Rci.p; in[l].Rv = L.Rv.p;
  }
  return in;
}

// FP32 copies of the scaled hierarchy for the mixed-precision form
static int build_mixed(sa_handle h) {
  if (h->v32) return SA_OK;
  std::vector<VLevelIn> in = vlevel_inputs(h);
  return vh_build<float>(h->al, in.data(), (int)in.size(), h->opt.cheb_degree, sa::coarse_view(h->cf, h->nL),
                         &h->v32);
}

static int setup_impl(const sa_problem* P, const sa_options* o, sa_handle h) {
  Alloc& al = h->al;
  cudaStream_t s = al.stream;
  auto t0 = std::chrono::steady_clock::now();
  h->dim = P->dim;
  h->n = P->n;
  Buf<int> err;
  SA_TRY(err.alloc(&al, 1));
  SA_TRY(memset_d(err.p, 0, sizeof(int), s));
  std::unique_ptr<Level> L0(new Level());
  L0->n = P->n;
  L0->nnz = P->nnz;
  SA_TRY(upload(al, L0->rp, P->row_ptr, P->n + 1));
  SA_TRY(upload(al, L0->ci, P->col, P->nnz));
  SA_TRY(upload(al, L0->v, P->val, P->nnz));
  SA_TRY(launch_validate_csr(s, P->n, P->n, P->nnz, L0->rp.p, L0->ci.p, err.p));
  {
    int e0 = 0;
    SA_TRY(copy_d2h(&e0, err.p, sizeof(int), s));
    if (e0) {
      set_error_text("row pointers or column indices invalid (range, order)");
      return SA_ERR_INVALID_ARG;
    }
  }
  SA_TRY(L0->dir.alloc(&al, P->n));
  SA_TRY(level_diag(h, *L0, L0->dir.p, err.p));
  {
    int e0 = 0;
    SA_TRY(copy_d2h(&e0, err.p, sizeof(int), s));
    if (e0) {
      set_error_text("a row has no stored diagonal");
      return SA_ERR_INVALID_ARG;
    }
  }
  const int kp = P->dim == 3 ? 6 : 3;
  PHASE_BEGIN(PK_S_NODAL, 0);
  if (o->measure != SA_MEASURE_CLASSICAL) {
    SA_TRY(upload(al, L0->x, P->coords, P->n * P->dim));
    SA_TRY(L0->sigma.alloc(&al, P->n * kp));
    SA_TRY(L0->sinv.alloc(&al, P->n * kp));
    if (o->measure == SA_MEASURE_DISTANCE) {
      SA_TRY(launch_nodal_tensors(al, P->dim, P->n, 0, nullptr, 0, 0, nullptr, nullptr, L0->sigma.p, L0->sinv.p,
                                  err.p));
    } else if (P->tloc == SA_TENSOR_NODE) {
      Buf<double> t;
      SA_TRY(upload(al, t, P->tensors, P->n * kp));
      SA_TRY(launch_nodal_tensors(al, P->dim, P->n, 0, t.p, 0, 0, nullptr, nullptr, L0->sigma.p, L0->sinv.p, err.p));
    } else {
      Buf<double> t, m;
      Buf<int32_t> en;
      SA_TRY(upload(al, t, P->tensors, P->n_elem * kp));
      SA_TRY(upload(al, m, P->elem_measure, P->n_elem));
      SA_TRY(upload(al, en, P->elem_nodes, P->n_elem * P->nodes_per_elem));
      SA_TRY(launch_nodal_tensors(al, P->dim, P->n, 1, t.p, P->n_elem, P->nodes_per_elem, en.p, m.p, L0->sigma.p,
                                  L0->sinv.p, err.p));
    }
  }
  PHASE_END(PK_S_NODAL);
  h->lev.push_back(std::move(L0));
  for (int l = 0;; ++l) {
    Level& L = *h->lev[l];
    if (L.n <= o->max_coarse || l + 1 >= o->max_levels) break;
    int stop = 0;
    SA_TRY(coarsen(h, l, err.p, &stop));
    if (stop) break;
  }
  int h_err = 0;
  SA_TRY(copy_d2h(&h_err, err.p, sizeof(int), s));
  if (h_err) {
    char msg[64];
    snprintf(msg, sizeof(msg), "setup validation flags 0x%x", h_err);
    set_error_text(msg);
    return SA_ERR_INVALID_ARG;
  }
  const int nlev = (int)h->lev.size();
  Level& Lc = *h->lev[nlev - 1];
  if (Lc.n > 16384) return SA_ERR_STAGNATION;
  h->nL = Lc.n;
  // a15: the coarse Cholesky factor and its diagonal-block inverses, on
  // streams of their own: the Chebyshev bounds and the packing of the
  // hierarchy below overlap it (the packing stores the addresses of the
  // factor's arrays, not their contents)
  DenseJob dj;
  dj.level = nlev - 1;
  SA_TRY(dense_start(al, Lc.n, Lc.rp.p, Lc.ci.p, Lc.v.p, h->cf, dj));
  // a15: smoother data: the V-cycle's copies of every level (values
  // D^-1/2 A D^-1/2, SELL-32 or CSR), then the Chebyshev bounds from 10
  // power steps on those copies (the product in its fastest form)
  for (int l = 0; l < nlev; ++l) {
    Level& L = *h->lev[l];
    SA_TRY(L.dinv.alloc(&al, L.n));
    SA_TRY(launch_reciprocal(s, L.n, L.diag.p, L.dinv.p));
  }
  SA_TRY(alloc_workspace(h));
  PHASE_BEGIN(PK_S_SELL, 0);
  {
    Level& L0 = *h->lev[0];
    SA_TRY(build_sell<double>(al, L0.n, L0.nnz, L0.rp.p, L0.ci.p, L0.v.p, nullptr, nullptr, h->A0s));
    std::vector<VLevelIn> in = vlevel_inputs(h);
    SA_TRY(vh_build<double>(al, in.data(), nlev, o->cheb_degree, coarse_view(h->cf, h->nL), &h->v64));
  }
  PHASE_END(PK_S_SELL);
  for (int l = 0; l + 1 < nlev; ++l) {
    PHASE_BEGIN(PK_S_CHEB, l);
    Level& L = *h->lev[l];
    Buf<double> lam;
    SA_TRY(lam.alloc(&al, 1));
    SA_TRY(vh_power(al, h->v64, l, o->power_iters, (uint32_t)(2 * l + 2), o->seed, lam.p));
    double hl = 0;
    SA_TRY(copy_d2h(&hl, lam.p, sizeof(double), s));
    L.lmax = o->cheb_boost * hl;
    L.lmin = L.lmax / o->cheb_ratio;
    h->v64->lev[l]->lmax = L.lmax;
    h->v64->lev[l]->lmin = L.lmin;
    PHASE_END(PK_S_CHEB);
  }
  if (o->precision == SA_PREC_FP32_VCYCLE) SA_TRY(build_mixed(h));
  SA_TRY(dense_finish(dj));
  SA_CUDA(cudaStreamSynchronize(s));
  auto t1 = std::chrono::steady_clock::now();
  h->setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  return SA_OK;
}

}  // namespace sa

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int sa_default_options(sa_options* o) {
  if (!o) return SA_ERR_INVALID_ARG;
  memset(o, 0, sizeof(*o));
  o->theta = 0.08;
  o->measure = SA_MEASURE_MATERIAL;
  o->precision = SA_PREC_FP64;
  o->max_coarse = 5000;
  o->max_levels = 10;
  o->cheb_degree = 2;
  o->cheb_ratio = 30.0;
  o->cheb_boost = 1.1;
  o->power_iters = 10;
  o->omega_sym = 4.0 / 3.0;
  o->seed = 0;
  o->maxit = 500;
  return SA_OK;
}

static int validate(const sa_problem* P, const sa_options* o) {
  if (!P || !o) return SA_ERR_INVALID_ARG;
  if (P->dim != 2 && P->dim != 3) return SA_ERR_INVALID_ARG;
  if (P->n <= 0 || P->nnz < P->n || P->n >= (int64_t)0x7fffffff) return SA_ERR_INVALID_ARG;
  if (!P->row_ptr || !P->col || !P->val) return SA_ERR_INVALID_ARG;
  if ((int)o->measure < 0 || (int)o->measure > 2) return SA_ERR_INVALID_ARG;
  if ((int)o->drop < 0 || (int)o->drop > 1) return SA_ERR_INVALID_ARG;
  if ((int)o->precision < 0 || (int)o->precision > 1) return SA_ERR_INVALID_ARG;
  if (o->measure != SA_MEASURE_CLASSICAL && !P->coords) return SA_ERR_INVALID_ARG;
  if (o->measure == SA_MEASURE_MATERIAL) {
    if (!P->tensors) return SA_ERR_INVALID_ARG;
    if (P->tloc == SA_TENSOR_ELEMENT &&
        (P->n_elem <= 0 || P->nodes_per_elem <= 0 || !P->elem_nodes || !P->elem_measure))
      return SA_ERR_INVALID_ARG;
  }
  if (!(o->theta >= 0.0) || o->cheb_degree < 1 || o->power_iters < 1 || o->max_levels < 1 || o->maxit < 1 ||
      !(o->cheb_ratio > 1.0) || !(o->cheb_boost > 0.0) || o->max_coarse < 1)
    return SA_ERR_INVALID_ARG;
  return SA_OK;
}

int sa_setup(const sa_problem* prob, const sa_options* opt, sa_handle* out) {
  if (!out) return SA_ERR_INVALID_ARG;
  *out = nullptr;
  int st = validate(prob, opt);
  if (st) return st;
  sa_handle h = new (std::nothrow) sa_handle_s();
  if (!h) return SA_ERR_OOM;
  h->opt = *opt;
  h->al.stream = (cudaStream_t)opt->stream;
  h->al.fn_alloc = opt->alloc;
  h->al.fn_free = opt->dealloc;
  h->al.ctx = opt->alloc_ctx;
  if (cudaMallocHost(&h->host_pin, 64) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SA_ERR_OOM;
  }
  st = sa::setup_impl(prob, opt, h);
  if (st != SA_OK) {
    cudaStreamSynchronize(h->al.stream);
    sa_free(h);
    return st;
  }
  *out = h;
  return SA_OK;
}

int sa_solve(sa_handle h, const double* b, double* x, double tol, sa_solve_info* info) {
  if (!h || !b || !x || !(tol > 0.0)) return SA_ERR_INVALID_ARG;
  // b and x are copied into handle-owned buffers (cudaMemcpyDefault: host or
  // device), so the captured CG loop always sees the same addresses
  return sa::cg_device(h, b, x, tol, info);
}

int sa_solve_batch(sa_handle h, int k, const double* B, double* X, double tol, sa_solve_info* infos) {
  if (!h || k < 0 || (k > 0 && (!B || !X)) || !(tol > 0.0)) return SA_ERR_INVALID_ARG;
  int worst = SA_OK;
  for (int c0 = 0; c0 < k; c0 += sa::KMAX_BLOCK) {
    const int kk = (k - c0) < sa::KMAX_BLOCK ? (k - c0) : sa::KMAX_BLOCK;
    int sts[sa::KMAX_BLOCK];
    const int64_t off = (int64_t)c0 * h->n;
    int st = kk == 1 ? sa_solve(h, B + off, X + off, tol, infos ? infos + c0 : nullptr)
                     : sa::cg_block(h, kk, B + off, X + off, tol, infos ? infos + c0 : nullptr, sts);
    if (kk == 1) sts[0] = st;
    else if (st != SA_OK) return st;  // a CUDA or allocation failure of the whole block
    for (int c = 0; c < kk; ++c) {
      if (sts[c] != SA_OK && worst == SA_OK) worst = sts[c];
      if (sts[c] != SA_OK && sts[c] != SA_ERR_NO_CONVERGENCE && kk == 1) return sts[c];
    }
  }
  return worst;
}

int sa_solve_batch_zero(sa_handle h, int k, const double* B, double* X, double tol, sa_solve_info* infos) {
  if (!h) return SA_ERR_INVALID_ARG;
  h->zero_guess = 1;
  const int st = sa_solve_batch(h, k, B, X, tol, infos);
  h->zero_guess = 0;
  return st;
}

int sa_set_precision(sa_handle h, sa_precision p) {
  if (!h || ((int)p != 0 && (int)p != 1)) return SA_ERR_INVALID_ARG;
  if (p == SA_PREC_FP32_VCYCLE) {
    int st = sa::build_mixed(h);
    if (st != SA_OK) return st;
    SA_CUDA(cudaStreamSynchronize(h->al.stream));
  }
  h->opt.precision = p;
  return SA_OK;
}

int sa_vcycle(sa_handle h, const double* r, double* z) {
  if (!h || !r || !z) return SA_ERR_INVALID_ARG;
  double* zz = nullptr;
  SA_TRY(sa::precondition(h, r, &zz));
  SA_CUDA(cudaMemcpyAsync(z, zz, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->al.stream));
  SA_CUDA(cudaStreamSynchronize(h->al.stream));
  return SA_OK;
}

int sa_hierarchy_stats(sa_handle h, int* levels, int64_t* n_l, int64_t* nnz_l, double* op_complexity,
                       int64_t* device_bytes) {
  if (!h) return SA_ERR_INVALID_ARG;
  const int nlev = (int)h->lev.size();
  if (levels) *levels = nlev;
  double tot = 0;
  for (int l = 0; l < nlev && l < 32; ++l) {
    if (n_l) n_l[l] = h->lev[l]->n;
    if (nnz_l) nnz_l[l] = h->lev[l]->nnz;
    tot += (double)h->lev[l]->nnz;
  }
  if (op_complexity) *op_complexity = tot / (double)h->lev[0]->nnz;
  if (device_bytes) *device_bytes = h->al.live_bytes;
  return SA_OK;
}

int sa_level_sizes(sa_handle h, int l, int64_t* out) {
  if (!h || !out || l < 0 || l >= (int)h->lev.size()) return SA_ERR_INVALID_ARG;
  const sa::Level& L = *h->lev[l];
  const bool has_p = l + 1 < (int)h->lev.size();
  out[0] = L.n;
  out[1] = L.nnz;
  out[2] = has_p ? L.nnzP : 0;
  out[3] = has_p ? L.nc : 0;
  out[4] = L.nnz_gc;
  return SA_OK;
}

int sa_level_format(sa_handle h, int l, int64_t* out) {
  if (!h || !out || !h->v64 || l < 0 || l >= (int)h->v64->lev.size()) return SA_ERR_INVALID_ARG;
  if (l + 1 == (int)h->v64->lev.size()) {
    out[0] = -1; out[1] = 0; out[2] = -1; out[3] = h->v64->lev[l]->n * h->v64->lev[l]->n; out[4] = 0;
    return SA_OK;
  }
  const sa::Mat<double>& A = h->v64->lev[l]->A;
  out[0] = A.sw;
  out[1] = A.sw == 0 ? 0 : A.nlong;
  out[2] = (A.sw == 0 || A.nlong == 0) ? -1 : A.lt;
  out[3] = A.sw == 0 ? A.sell.stored : A.nnz;
  out[4] = A.sw == 0 ? A.sell_lanes : 0;
  return SA_OK;
}

int sa_export_level(sa_handle h, int l, int32_t* agg, int64_t* P_rowptr, int32_t* P_col, double* P_val,
                    int64_t* A_rowptr, int32_t* A_col, double* A_val) {
  if (!h || l < 0 || l >= (int)h->lev.size()) return SA_ERR_INVALID_ARG;
  const sa::Level& L = *h->lev[l];
  cudaStream_t s = h->al.stream;
  const bool has_p = l + 1 < (int)h->lev.size();
  auto d2h = [&](void* dst, const void* src, size_t bytes) -> int {
    if (dst && src && bytes) SA_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    return SA_OK;
  };
  SA_TRY(d2h(A_rowptr, L.rp.p, sizeof(int64_t) * (L.n + 1)));
  SA_TRY(d2h(A_col, L.ci.p, sizeof(int32_t) * L.nnz));
  SA_TRY(d2h(A_val, L.v.p, sizeof(double) * L.nnz));
  if (has_p) {
    SA_TRY(d2h(agg, L.agg.p, sizeof(int32_t) * L.n));
    SA_TRY(d2h(P_rowptr, L.Prp.p, sizeof(int64_t) * (L.n + 1)));
    SA_TRY(d2h(P_col, L.Pci.p, sizeof(int32_t) * L.nnzP));
    SA_TRY(d2h(P_val, L.Pv.p, sizeof(double) * L.nnzP));
  }
  SA_CUDA(cudaStreamSynchronize(s));
  return SA_OK;
}

int sa_export_strength(sa_handle h, int l, uint8_t* keep, uint8_t* root, uint8_t* dirichlet, double* coords,
                       double* sigma_inv, double* scalars) {
  if (!h || l < 0 || l >= (int)h->lev.size()) return SA_ERR_INVALID_ARG;
  const sa::Level& L = *h->lev[l];
  cudaStream_t s = h->al.stream;
  const int kp = h->dim == 3 ? 6 : 3;
  auto d2h = [&](void* dst, const void* src, size_t bytes) -> int {
    if (dst && src && bytes) SA_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    return SA_OK;
  };
  if ((keep && !L.keep.p) || (root && !L.root.p)) {
    if (l + 1 < (int)h->lev.size() || keep || root) {
      // diagnostics were not kept (keep_setup_data = 0) or l is the coarsest
      if (!h->opt.keep_setup_data) return SA_ERR_INVALID_ARG;
    }
  }
  SA_TRY(d2h(keep, L.keep.p, L.nnz));
  SA_TRY(d2h(root, L.root.p, L.n));
  if (dirichlet) {
    if (L.dir.p) SA_TRY(d2h(dirichlet, L.dir.p, L.n));
    else memset(dirichlet, 0, (size_t)L.n);
  }
  SA_TRY(d2h(coords, L.x.p, sizeof(double) * L.n * h->dim));
  SA_TRY(d2h(sigma_inv, L.sinv.p, sizeof(double) * L.n * kp));
  SA_CUDA(cudaStreamSynchronize(s));
  if (scalars) {
    scalars[0] = L.omega;
    scalars[1] = L.lam_omega;
    scalars[2] = L.lmax;
    scalars[3] = L.lmin;
  }
  return SA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// hierarchy store: the FP64 hierarchy (A_l, D_l, P_l, R_l, aggregates and the
// smoother scalars) in one host buffer, reloaded without re-running the setup
// ---------------------------------------------------------------------------
namespace {

const char kStoreMagic[8] = {'S', 'A', 'A', 'M', 'G', 'H', '1', '\0'};
const uint32_t kStoreVersion = 1;
const uint32_t kStoreOrder = 0x01020304u;

struct StoreHeader {
  char magic[8];
  uint32_t version, order;
  int32_t dim, nlev;
  int64_t n;
  double theta, cheb_ratio, cheb_boost, omega_sym;
  int32_t measure, drop, max_coarse, max_levels, cheb_degree, power_iters;
  uint32_t seed, reserved;
  uint64_t payload, checksum;
};

struct StoreLevel {
  int64_t n, nnz, nc, nnzP, nnz_gc;
  double omega, lam_omega, lmax, lmin;
};

static_assert(sizeof(StoreHeader) == 112, "store header layout");
static_assert(sizeof(StoreLevel) == 72, "store level record layout");

uint64_t pad8(uint64_t b) { return (b + 7) & ~(uint64_t)7; }

// payload bytes of one level (arrays padded to 8 bytes)
uint64_t level_bytes(const StoreLevel& L, bool last) {
  uint64_t b = sizeof(StoreLevel);
  b += pad8(8ull * (uint64_t)(L.n + 1)) + pad8(4ull * (uint64_t)L.nnz) + pad8(8ull * (uint64_t)L.nnz) +
       pad8(8ull * (uint64_t)L.n);
  if (!last)
    b += pad8(8ull * (uint64_t)(L.n + 1)) + pad8(4ull * (uint64_t)L.nnzP) + pad8(8ull * (uint64_t)L.nnzP) +
         pad8(8ull * (uint64_t)(L.nc + 1)) + pad8(4ull * (uint64_t)L.nnzP) + pad8(8ull * (uint64_t)L.nnzP) +
         pad8(4ull * (uint64_t)L.n);
  return b;
}

// FNV-1a over 64-bit words (the payload is a whole number of words)
uint64_t store_checksum(const unsigned char* p, uint64_t bytes) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (uint64_t o = 0; o + 8 <= bytes; o += 8) {
    uint64_t w;
    memcpy(&w, p + o, 8);
    h ^= w;
    h *= 0x100000001b3ull;
  }
  return h;
}

StoreLevel store_level_of(const sa::Level& L, bool last) {
  StoreLevel d;
  memset(&d, 0, sizeof(d));
  d.n = L.n; d.nnz = L.nnz; d.nnz_gc = L.nnz_gc;
  d.nc = last ? 0 : L.nc;
  d.nnzP = last ? 0 : L.nnzP;
  d.omega = L.omega; d.lam_omega = L.lam_omega; d.lmax = L.lmax; d.lmin = L.lmin;
  return d;
}

}  // namespace

namespace sa {

static uint64_t store_size(sa_handle h) {
  const int nlev = (int)h->lev.size();
  uint64_t b = sizeof(StoreHeader);
  for (int l = 0; l < nlev; ++l) b += level_bytes(store_level_of(*h->lev[l], l + 1 == nlev), l + 1 == nlev);
  return b;
}

// rebuild what the solve needs from a loaded FP64 hierarchy: reciprocal
// diagonals, the coarse factor, the Krylov workspace and the SELL copies
static int finish_loaded(sa_handle h) {
  Alloc& al = h->al;
  cudaStream_t s = al.stream;
  const int nlev = (int)h->lev.size();
  for (int l = 0; l < nlev; ++l) {
    Level& L = *h->lev[l];
    SA_TRY(L.dinv.alloc(&al, L.n));
    SA_TRY(launch_reciprocal(s, L.n, L.diag.p, L.dinv.p));
    L.sw = pick_sw(L.n, L.nnz);
  }
  Level& Lc = *h->lev[nlev - 1];
  h->nL = Lc.n;
  // the coarse factorisation overlaps the packing below (which stores the
  // addresses of the factor's arrays, not their contents)
  DenseJob dj;
  dj.level = nlev - 1;
  SA_TRY(dense_start(al, Lc.n, Lc.rp.p, Lc.ci.p, Lc.v.p, h->cf, dj));
  SA_TRY(alloc_workspace(h));
  Level& L0 = *h->lev[0];
  SA_TRY(build_sell<double>(al, L0.n, L0.nnz, L0.rp.p, L0.ci.p, L0.v.p, nullptr, nullptr, h->A0s));
  std::vector<VLevelIn> in = vlevel_inputs(h);
  SA_TRY(vh_build<double>(al, in.data(), nlev, h->opt.cheb_degree, coarse_view(h->cf, h->nL), &h->v64));
  if (h->opt.precision == SA_PREC_FP32_VCYCLE) SA_TRY(build_mixed(h));
  return dense_finish(dj);
}

static int load_impl(const unsigned char* buf, uint64_t bytes, sa_handle h) {
  Alloc& al = h->al;
  cudaStream_t s = al.stream;
  auto t0 = std::chrono::steady_clock::now();
  StoreHeader H;
  memcpy(&H, buf, sizeof(H));
  const unsigned char* p = buf + sizeof(H);
  const unsigned char* end = buf + bytes;
  h->dim = H.dim;
  h->n = H.n;
  Buf<int> err;
  SA_TRY(err.alloc(&al, 1));
  SA_TRY(memset_d(err.p, 0, sizeof(int), s));
  auto take = [&](void* dst, uint64_t nb) -> bool {
    if ((uint64_t)(end - p) < pad8(nb)) return false;
    if (dst) memcpy(dst, p, nb);
    p += pad8(nb);
    return true;
  };
  auto up = [&](auto& B, int64_t count) -> int {
    using T = typename std::remove_reference<decltype(*B.p)>::type;
    const uint64_t nb = sizeof(T) * (uint64_t)count;
    if ((uint64_t)(end - p) < pad8(nb)) return SA_ERR_INVALID_ARG;
    SA_TRY(upload(al, B, reinterpret_cast<const T*>(p), count));
    p += pad8(nb);
    return SA_OK;
  };
  int64_t expect_n = H.n;
  for (int l = 0; l < H.nlev; ++l) {
    const bool last = l + 1 == H.nlev;
    StoreLevel d;
    if (!take(&d, sizeof(d))) return SA_ERR_INVALID_ARG;
    if (d.n != expect_n || d.n <= 0 || d.n >= (int64_t)0x7fffffff || d.nnz < d.n || d.nnz_gc < 0 ||
        (!last && (d.nc <= 0 || d.nc >= d.n || d.nnzP < 0)) || (last && (d.nc != 0 || d.nnzP != 0)))
      return SA_ERR_INVALID_ARG;
    std::unique_ptr<Level> L(new Level());
    L->n = d.n; L->nnz = d.nnz; L->nnz_gc = d.nnz_gc;
    L->omega = d.omega; L->lam_omega = d.lam_omega; L->lmax = d.lmax; L->lmin = d.lmin;
    SA_TRY(up(L->rp, d.n + 1));
    SA_TRY(up(L->ci, d.nnz));
    SA_TRY(up(L->v, d.nnz));
    SA_TRY(up(L->diag, d.n));
    SA_TRY(launch_validate_csr(s, d.n, d.n, d.nnz, L->rp.p, L->ci.p, err.p));
    if (!last) {
      L->nc = d.nc; L->nnzP = d.nnzP;
      SA_TRY(up(L->Prp, d.n + 1));
      SA_TRY(up(L->Pci, d.nnzP));
      SA_TRY(up(L->Pv, d.nnzP));
      SA_TRY(up(L->Rrp, d.nc + 1));
      SA_TRY(up(L->Rci, d.nnzP));
      SA_TRY(up(L->Rv, d.nnzP));
      SA_TRY(up(L->agg, d.n));
      SA_TRY(launch_validate_csr(s, d.n, d.nc, d.nnzP, L->Prp.p, L->Pci.p, err.p));
      SA_TRY(launch_validate_csr(s, d.nc, d.n, d.nnzP, L->Rrp.p, L->Rci.p, err.p));
      expect_n = d.nc;
    }
    h->lev.push_back(std::move(L));
  }
  if (p != end) return SA_ERR_INVALID_ARG;
  int e0 = 0;
  SA_TRY(copy_d2h(&e0, err.p, sizeof(int), s));
  if (e0) {
    set_error_text("stored hierarchy has invalid row pointers or column indices");
    return SA_ERR_INVALID_ARG;
  }
  if (h->lev.back()->n > 16384) return SA_ERR_INVALID_ARG;
  SA_TRY(finish_loaded(h));
  SA_CUDA(cudaStreamSynchronize(s));
  h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return SA_OK;
}

}  // namespace sa

extern "C" {

int sa_serialized_size(sa_handle h, uint64_t* bytes) {
  if (!h || !bytes) return SA_ERR_INVALID_ARG;
  *bytes = sa::store_size(h);
  return SA_OK;
}

int sa_serialize(sa_handle h, void* buf, uint64_t bytes) {
  if (!h || !buf) return SA_ERR_INVALID_ARG;
  const uint64_t need = sa::store_size(h);
  if (bytes < need) {
    sa::set_error_text("buffer smaller than sa_serialized_size");
    return SA_ERR_INVALID_ARG;
  }
  unsigned char* out = static_cast<unsigned char*>(buf);
  cudaStream_t s = h->al.stream;
  StoreHeader H;
  memset(&H, 0, sizeof(H));
  memcpy(H.magic, kStoreMagic, 8);
  H.version = kStoreVersion;
  H.order = kStoreOrder;
  H.dim = h->dim;
  H.nlev = (int32_t)h->lev.size();
  H.n = h->n;
  H.theta = h->opt.theta; H.cheb_ratio = h->opt.cheb_ratio; H.cheb_boost = h->opt.cheb_boost;
  H.omega_sym = h->opt.omega_sym;
  H.measure = (int32_t)h->opt.measure; H.drop = (int32_t)h->opt.drop; H.max_coarse = h->opt.max_coarse;
  H.max_levels = h->opt.max_levels; H.cheb_degree = h->opt.cheb_degree; H.power_iters = h->opt.power_iters;
  H.seed = h->opt.seed;
  H.payload = need - sizeof(H);
  uint64_t o = sizeof(H);
  memset(out + o, 0, (size_t)H.payload);  // padding bytes are part of the checksum
  auto put = [&](const void* src, uint64_t nb, bool dev) -> int {
    if (nb) {
      if (dev) SA_CUDA(cudaMemcpyAsync(out + o, src, (size_t)nb, cudaMemcpyDeviceToHost, s));
      else memcpy(out + o, src, (size_t)nb);
    }
    o += pad8(nb);
    return SA_OK;
  };
  for (int l = 0; l < H.nlev; ++l) {
    const bool last = l + 1 == H.nlev;
    const sa::Level& L = *h->lev[l];
    const StoreLevel d = store_level_of(L, last);
    SA_TRY(put(&d, sizeof(d), false));
    SA_TRY(put(L.rp.p, 8ull * (uint64_t)(L.n + 1), true));
    SA_TRY(put(L.ci.p, 4ull * (uint64_t)L.nnz, true));
    SA_TRY(put(L.v.p, 8ull * (uint64_t)L.nnz, true));
    SA_TRY(put(L.diag.p, 8ull * (uint64_t)L.n, true));
    if (!last) {
      SA_TRY(put(L.Prp.p, 8ull * (uint64_t)(L.n + 1), true));
      SA_TRY(put(L.Pci.p, 4ull * (uint64_t)L.nnzP, true));
      SA_TRY(put(L.Pv.p, 8ull * (uint64_t)L.nnzP, true));
      SA_TRY(put(L.Rrp.p, 8ull * (uint64_t)(L.nc + 1), true));
      SA_TRY(put(L.Rci.p, 4ull * (uint64_t)L.nnzP, true));
      SA_TRY(put(L.Rv.p, 8ull * (uint64_t)L.nnzP, true));
      SA_TRY(put(L.agg.p, 4ull * (uint64_t)L.n, true));
    }
  }
  SA_CUDA(cudaStreamSynchronize(s));
  H.checksum = store_checksum(out + sizeof(H), H.payload);
  memcpy(out, &H, sizeof(H));
  return SA_OK;
}

int sa_deserialize(const void* buf, uint64_t bytes, const sa_options* opt, sa_handle* out) {
  if (!out) return SA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!buf || !opt || bytes < sizeof(StoreHeader)) return SA_ERR_INVALID_ARG;
  if ((int)opt->precision < 0 || (int)opt->precision > 1 || opt->maxit < 1) return SA_ERR_INVALID_ARG;
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  StoreHeader H;
  memcpy(&H, in, sizeof(H));
  if (memcmp(H.magic, kStoreMagic, 8) != 0 || H.version != kStoreVersion || H.order != kStoreOrder ||
      (H.dim != 2 && H.dim != 3) || H.nlev < 1 || H.nlev > 32 || H.payload != bytes - sizeof(H) ||
      H.cheb_degree < 1 || H.payload % 8 != 0) {
    sa::set_error_text("not a stored hierarchy of this version");
    return SA_ERR_INVALID_ARG;
  }
  if (store_checksum(in + sizeof(H), H.payload) != H.checksum) {
    sa::set_error_text("stored hierarchy checksum mismatch");
    return SA_ERR_INVALID_ARG;
  }
  sa_handle h = new (std::nothrow) sa_handle_s();
  if (!h) return SA_ERR_OOM;
  h->opt = *opt;
  h->opt.theta = H.theta; h->opt.cheb_ratio = H.cheb_ratio; h->opt.cheb_boost = H.cheb_boost;
  h->opt.omega_sym = H.omega_sym; h->opt.measure = (sa_measure)H.measure; h->opt.drop = (sa_drop)H.drop;
  h->opt.max_coarse = H.max_coarse; h->opt.max_levels = H.max_levels; h->opt.cheb_degree = H.cheb_degree;
  h->opt.power_iters = H.power_iters; h->opt.seed = H.seed; h->opt.keep_setup_data = 0;
  h->al.stream = (cudaStream_t)opt->stream;
  h->al.fn_alloc = opt->alloc;
  h->al.fn_free = opt->dealloc;
  h->al.ctx = opt->alloc_ctx;
  if (cudaMallocHost(&h->host_pin, 64) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SA_ERR_OOM;
  }
  int st = sa::load_impl(in, bytes, h);
  if (st != SA_OK) {
    cudaStreamSynchronize(h->al.stream);
    sa_free(h);
    return st;
  }
  *out = h;
  return SA_OK;
}

}  // extern "C"

extern "C" {

int sa_free(sa_handle h) {
  if (!h) return SA_OK;
  sa::drop_graph(h, 0);
  sa::drop_graph(h, 1);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->v64) sa::vh_free<double>(h->v64);
  if (h->v32) sa::vh_free<float>(h->v32);
  h->A0s.sp.release();
  h->A0s.ci.release();
  h->A0s.v.release();
  h->lev.clear();
  h->cf.L.release();
  h->cf.LT.release();
  h->cf.W.release();
  h->cf.WT.release();
  h->r.release(); h->p.release(); h->q.release(); h->rprev.release(); h->t.release();
  h->part.release(); h->dots.release(); h->xb.release(); h->bb.release(); h->cg.release();
  h->it_dev.release(); h->ctl.release();
  h->kR.release(); h->kP.release(); h->kQ.release(); h->kRp.release(); h->kT.release(); h->kX.release();
  h->kB.release(); h->kStage.release(); h->kpart.release(); h->kdots.release(); h->kS.release(); h->kact.release();
  cudaStreamSynchronize(h->al.stream);
  if (h->host_pin) cudaFreeHost(h->host_pin);
  delete h;
  return SA_OK;
}

const char* sa_status_string(int st) {
  switch (st) {
    case SA_OK: return "ok";
    case SA_ERR_INVALID_ARG: return "invalid argument";
    case SA_ERR_OOM: return "out of device memory";
    case SA_ERR_CUDA: return "CUDA error";
    case SA_ERR_NOT_SPD: return "coarse operator not SPD";
    case SA_ERR_STAGNATION: return "coarsening stagnated";
    case SA_ERR_NO_CONVERGENCE: return "no convergence within maxit";
    case SA_ERR_BREAKDOWN: return "CG breakdown";
    case SA_ERR_CAPACITY: return "internal capacity exceeded";
    default: return "unknown status";
  }
}

int sa_strength(sa_measure measure, int dim, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                const double* val, const double* coords, const double* sigma_inv, const uint8_t* dirichlet,
                double theta, uint8_t* keep, void* stream) {
  if (n < 0 || nnz < 0 || !row_ptr || !col || !keep || (dim != 2 && dim != 3)) return SA_ERR_INVALID_ARG;
  if (measure == SA_MEASURE_CLASSICAL && !val) return SA_ERR_INVALID_ARG;
  if (measure != SA_MEASURE_CLASSICAL && !coords) return SA_ERR_INVALID_ARG;
  if (measure == SA_MEASURE_MATERIAL && !sigma_inv) return SA_ERR_INVALID_ARG;
  if ((int)measure < 0 || (int)measure > 2) return SA_ERR_INVALID_ARG;
  sa::Alloc al;
  al.stream = (cudaStream_t)stream;
  cudaStream_t s = al.stream;
  sa::Buf<int64_t> cnt;
  SA_TRY(cnt.alloc(&al, n + 1));
  if (measure == SA_MEASURE_CLASSICAL) {
    sa::Buf<double> diag;
    sa::Buf<int> err;
    SA_TRY(diag.alloc(&al, n));
    SA_TRY(err.alloc(&al, 1));
    SA_TRY(sa::memset_d(err.p, 0, sizeof(int), s));
    SA_TRY(sa::launch_dirichlet_diag(s, n, row_ptr, col, val, nullptr, diag.p, err.p));
    SA_TRY(sa::launch_strength_classical(s, n, row_ptr, col, val, diag.p, dirichlet, theta, keep, cnt.p));
  } else {
    sa::Buf<double> w, D, si, sg;
    sa::Buf<int> err;
    SA_TRY(w.alloc(&al, nnz));
    SA_TRY(D.alloc(&al, n));
    const double* sinv = sigma_inv;
    if (measure == SA_MEASURE_DISTANCE) {
      const int kp = dim == 3 ? 6 : 3;
      SA_TRY(si.alloc(&al, n * kp));
      SA_TRY(sg.alloc(&al, n * kp));
      SA_TRY(err.alloc(&al, 1));
      SA_TRY(sa::launch_nodal_tensors(al, dim, n, 0, nullptr, 0, 0, nullptr, nullptr, sg.p, si.p, err.p));
      sinv = si.p;
    }
    SA_TRY(sa::launch_strength_material(s, dim, n, row_ptr, col, coords, sinv, dirichlet, theta, w.p, D.p, keep,
                                        cnt.p));
  }
  return SA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// group solve (sa_solve_group): m problems with different operators, one
// right-hand side each, advanced together.  Every step is one launch for all
// problems still iterating (group.cuh); the arithmetic of each problem is the
// host-driven one-vector CG's (cg_eager_dev), so a problem ends bitwise where
// sa_solve ends.  The coarse solves of all problems run together at the
// bottom of the group V-cycle.
// ---------------------------------------------------------------------------
namespace sa {

// descriptor arrays of one group solve: built on the host, copied to the
// device in one transfer whenever the set of iterating problems changes
struct GArena {
  std::vector<unsigned char> img;
  Buf<unsigned char> dev;
  Alloc* al = nullptr;
  void clear() { img.clear(); }
  template <typename D>
  size_t put(const std::vector<D>& v) {
    size_t off = (img.size() + 63) & ~size_t(63);
    img.resize(off + sizeof(D) * v.size());
    if (!v.empty()) memcpy(img.data() + off, v.data(), sizeof(D) * v.size());
    return off;
  }
  int upload(cudaStream_t s) {
    if (img.empty()) return SA_OK;
    if ((size_t)dev.n < img.size()) {
      dev.release();
      SA_TRY(dev.alloc(al, (int64_t)img.size() + 4096));
    }
    SA_CUDA(cudaMemcpyAsync(dev.p, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    return SA_OK;
  }
  template <typename D>
  const D* at(size_t off) const { return reinterpret_cast<const D*>(dev.p + off); }
};

struct GLaunch {
  int kind;  // 0 matrix rows, 1 elementwise, 2 coarse substitution
  int op;    // op or substitution mode
  size_t off;
  int m;
  unsigned blocks;
};

template <typename T>
struct GroupVcycle {
  std::vector<sa_handle> hs;
  std::vector<VHier<T>*> vh;
  std::vector<const double*> r64;  // cycle input per problem (the outer residual)
  std::vector<GLaunch> launches;
  std::vector<std::pair<int, int>> pending;  // (problem, coarsest level) waiting for the shared coarse solve

  // level l for the problems `segs` that have it; returns per problem the
  // level's output vector
  void plan_level(GArena& ar, int l, const std::vector<int>& segs, std::vector<T*>& xout) {
    std::vector<int> D;
    for (int i : segs) {
      if (l == (int)vh[i]->lev.size() - 1) {
        pending.emplace_back(i, l);
        xout[i] = vh[i]->lev[l]->x.p;  // written by the shared coarse solve
      } else {
        D.push_back(i);
      }
    }
    if (D.empty()) {
      flush_coarse(ar);
      return;
    }
    const int deg = vh[D[0]]->deg;
    std::vector<T*> xa(hs.size()), xb(hs.size());
    std::vector<double> th(hs.size()), de(hs.size()), s1(hs.size()), rho(hs.size());
    for (int i : D) {
      VLevel<T>* L = vh[i]->lev[l];
      th[i] = 0.5 * (L->lmax + L->lmin);
      de[i] = 0.5 * (L->lmax - L->lmin);
      s1[i] = th[i] / de[i];
      xa[i] = L->x.p;
      xb[i] = L->x2.p;
    }
    {  // first step from zero (fine level: entry from the FP64 residual)
      std::vector<GVec<T>> v;
      uint32_t blk = 0;
      for (int i : D) {
        VLevel<T>* L = vh[i]->lev[l];
        GVec<T> g = {};
        g.blk0 = blk;
        g.n = L->n;
        g.r64 = r64[i];
        g.s = vh[i]->s0.p;
        g.c2 = (T)(1.0 / th[i]);
        g.b = L->b.p;
        g.x = xa[i];
        g.d = L->d.p;
        v.push_back(g);
        blk += g256(L->n);
      }
      launches.push_back({1, l == 0 ? GV_FINE_IN : GV_FIRST, ar.put(v), (int)v.size(), blk});
    }
    for (int i : D) rho[i] = 1.0 / s1[i];
    for (int q = 1; q < deg; ++q) {
      std::vector<GMat<T>> v;
      uint32_t blk = 0;
      for (int i : D) {
        VLevel<T>* L = vh[i]->lev[l];
        const double rn = 1.0 / (2.0 * s1[i] - rho[i]);
        v.push_back(mat_desc(L->A, blk, L->b.p, xa[i], xb[i], L->d.p, (T)(rn * rho[i]), (T)(2.0 * rn / de[i]), 0));
        std::swap(xa[i], xb[i]);
        rho[i] = rn;
      }
      launches.push_back({0, GM_CHEB, ar.put(v), (int)v.size(), blk});
    }
    {
      std::vector<GMat<T>> v;
      uint32_t blk = 0;
      for (int i : D) {
        VLevel<T>* L = vh[i]->lev[l];
        GMat<T> g = mat_desc(L->A, blk, L->b.p, xa[i], nullptr, nullptr, (T)0, (T)0, 0);
        g.r = L->r.p;
        v.push_back(g);
      }
      launches.push_back({0, GM_RESID, ar.put(v), (int)v.size(), blk});
    }
    {
      std::vector<GMat<T>> v;
      uint32_t blk = 0;
      for (int i : D) {
        VLevel<T>* L = vh[i]->lev[l];
        v.push_back(mat_desc(L->R, blk, nullptr, L->r.p, vh[i]->lev[l + 1]->b.p, nullptr, (T)0, (T)0, 0));
      }
      launches.push_back({0, GM_SPMV, ar.put(v), (int)v.size(), blk});
    }
    std::vector<T*> xc(hs.size(), nullptr);
    plan_level(ar, l + 1, D, xc);
    {
      std::vector<GMat<T>> v;
      uint32_t blk = 0;
      for (int i : D) {
        VLevel<T>* L = vh[i]->lev[l];
        v.push_back(mat_desc(L->P, blk, nullptr, xc[i], xa[i], nullptr, (T)0, (T)0, 0));
      }
      launches.push_back({0, GM_SPMV_ADD, ar.put(v), (int)v.size(), blk});
    }
    for (int i : D) rho[i] = 1.0 / s1[i];
    for (int q = 0; q < deg; ++q) {
      const int first = (q == 0);
      const bool out = (l == 0 && q == deg - 1);
      std::vector<GMat<T>> v;
      uint32_t blk = 0;
      for (int i : D) {
        VLevel<T>* L = vh[i]->lev[l];
        T c1 = (T)0, c2 = (T)(1.0 / th[i]);
        double rn = rho[i];
        if (!first) {
          rn = 1.0 / (2.0 * s1[i] - rho[i]);
          c1 = (T)(rn * rho[i]);
          c2 = (T)(2.0 * rn / de[i]);
        }
        GMat<T> g = mat_desc(L->A, blk, L->b.p, xa[i], out ? nullptr : xb[i], L->d.p, c1, c2, first);
        if (out) {
          g.s = vh[i]->s0.p;
          g.z = vh[i]->z.p;
        } else {
          std::swap(xa[i], xb[i]);
        }
        if (!first) rho[i] = rn;
        v.push_back(g);
      }
      launches.push_back({0, out ? GM_CHEB_OUT : GM_CHEB, ar.put(v), (int)v.size(), blk});
    }
    for (int i : D) xout[i] = xa[i];
  }

  GMat<T> mat_desc(const Mat<T>& M, uint32_t& blk, const T* b, const T* xin, T* xo, T* d, T c1, T c2, int first) {
    GMat<T> g = {};
    g.blk0 = blk;
    g.fmt = g_mat_fmt(M);
    g.M = view(M);
    g.b = b;
    g.xin = xin;
    g.xout = xo;
    g.d = d;
    g.c1 = c1;
    g.c2 = c2;
    g.first = first;
    blk += g_mat_blocks(M);
    return g;
  }

  // the coarse solves of every pending problem, together (block substitution
  // of dense.cu, one launch per step for all problems that have the step)
  void flush_coarse(GArena& ar) {
    if (pending.empty()) return;
    struct C { int i, l; bool direct; int64_t n; int nbk; const double* bin; double *t, *y, *x; CoarseView F; };
    std::vector<C> cs;
    int maxnbk = 0;
    {
      std::vector<GVec<T>> v;
      uint32_t blk = 0;
      for (auto& pr : pending) {
        const int i = pr.first, l = pr.second;
        VHier<T>* m = vh[i];
        C c;
        c.i = i; c.l = l; c.direct = (m->lev.size() == 1); c.F = m->cf; c.n = m->cf.n;
        c.nbk = (int)((c.n + COARSE_BS - 1) / COARSE_BS);
        c.bin = c.direct ? r64[i] : m->ct.p;
        c.t = m->cs.p; c.y = m->cy.p; c.x = c.direct ? m->z.p : m->cx.p;
        cs.push_back(c);
        maxnbk = c.nbk > maxnbk ? c.nbk : maxnbk;
        if (!c.direct) {
          VLevel<T>* L = m->lev[l];
          GVec<T> g = {};
          g.blk0 = blk; g.n = L->n; g.s = L->sq.p; g.b = L->b.p; g.t = m->ct.p;
          v.push_back(g);
          blk += g256(L->n);
        }
      }
      launches.push_back({1, GV_COARSE_IN, ar.put(v), (int)v.size(), blk});
    }
    for (int q = 0; q < maxnbk; ++q) {   // forward: t_K = b_K - L_{K,<K} y; y_K = W_KK t_K
      for (int mode : {2, 0}) {
        if (mode == 2 && q == 0) continue;
        std::vector<GTri> v;
        uint32_t blk = 0;
        for (auto& c : cs) {
          if (c.nbk <= q) continue;
          const int64_t r0 = q * COARSE_BS, r1 = r0 + COARSE_BS < c.n ? r0 + COARSE_BS : c.n;
          GTri g = {};
          g.blk0 = blk; g.n = c.n; g.r0 = r0; g.r1 = r1;
          if (mode == 2) { g.M = c.F.L; g.v = c.y; g.rhs = c.bin; g.out = c.t; }
          else { g.M = c.F.W; g.v = q > 0 ? c.t : c.bin; g.rhs = nullptr; g.out = c.y; }
          v.push_back(g);
          blk += (uint32_t)(r1 - r0);
        }
        launches.push_back({2, mode, ar.put(v), (int)v.size(), blk});
      }
    }
    for (int t = 0; t < maxnbk; ++t) {   // backward: t_K = y_K - L^T_{K,>K} x; x_K = W_KK^T t_K
      for (int mode : {3, 1}) {
        if (mode == 3 && t == 0) continue;
        std::vector<GTri> v;
        uint32_t blk = 0;
        for (auto& c : cs) {
          if (c.nbk <= t) continue;
          const int q = c.nbk - 1 - t;
          const int64_t r0 = q * COARSE_BS, r1 = r0 + COARSE_BS < c.n ? r0 + COARSE_BS : c.n;
          GTri g = {};
          g.blk0 = blk; g.n = c.n; g.r0 = r0; g.r1 = r1;
          if (mode == 3) { g.M = c.F.LT; g.v = c.x; g.rhs = c.y; g.out = c.t; }
          else { g.M = c.F.WT; g.v = t > 0 ? c.t : c.y; g.rhs = nullptr; g.out = c.x; }
          v.push_back(g);
          blk += (uint32_t)(r1 - r0);
        }
        launches.push_back({2, mode, ar.put(v), (int)v.size(), blk});
      }
    }
    {
      std::vector<GVec<T>> v;
      uint32_t blk = 0;
      for (auto& c : cs) {
        if (c.direct) continue;
        VLevel<T>* L = vh[c.i]->lev[c.l];
        GVec<T> g = {};
        g.blk0 = blk; g.n = L->n; g.s = L->sq.p; g.x = L->x.p; g.t = vh[c.i]->cx.p;
        v.push_back(g);
        blk += g256(L->n);
      }
      launches.push_back({1, GV_COARSE_OUT, ar.put(v), (int)v.size(), blk});
    }
    pending.clear();
  }

  void plan(GArena& ar, const std::vector<int>& act) {
    launches.clear();
    pending.clear();
    std::vector<T*> xo(hs.size(), nullptr);
    plan_level(ar, 0, act, xo);
  }

  int run(const GArena& ar, cudaStream_t st) const {
    for (const GLaunch& g : launches) {
      if (g.m == 0) continue;
      if (g.kind == 0) SA_TRY(launch_g_mat<T>(st, g.op, ar.at<GMat<T>>(g.off), g.m, g.blocks));
      else if (g.kind == 1) SA_TRY(launch_g_vec<T>(st, g.op, ar.at<GVec<T>>(g.off), g.m, g.blocks));
      else SA_TRY(launch_g_tri(st, g.op, ar.at<GTri>(g.off), g.m, g.blocks));
    }
    return SA_OK;
  }
};

template <typename T>
static int cg_group(std::vector<sa_handle>& hs, std::vector<VHier<T>*>& vh, const double* const* B, double* const* X,
                    double tol, sa_solve_info* infos, int* statuses) {
  const int m = (int)hs.size();
  cudaStream_t s = hs[0]->al.stream;
  const int flexible = hs[0]->opt.precision == SA_PREC_FP32_VCYCLE;
  const int maxit = hs[0]->opt.maxit;
  auto t0 = std::chrono::steady_clock::now();
  GArena ar;
  ar.al = &hs[0]->al;
  Buf<double> gath;
  SA_TRY(gath.alloc(&hs[0]->al, 2 * GROUP_MAX));
  std::vector<double> hg(2 * GROUP_MAX);
  GroupVcycle<T> V;
  V.hs = hs;
  V.vh = vh;
  for (int i = 0; i < m; ++i) V.r64.push_back(hs[i]->r.p);
  for (int i = 0; i < m; ++i) {
    SA_CUDA(cudaMemcpyAsync(hs[i]->bb.p, B[i], sizeof(double) * hs[i]->n, cudaMemcpyDefault, s));
    SA_CUDA(cudaMemcpyAsync(hs[i]->xb.p, X[i], sizeof(double) * hs[i]->n, cudaMemcpyDefault, s));
  }
  // descriptor arrays for a set of problems
  struct Ops {
    size_t resid_r, resid_t, dots_rr, fin_dots, dots_tt, fin_dots4, spmv, fin_spmv, alpha, update, fin_upd, beta0,
        beta, pup1, pup, dots_rz, gather;
    unsigned rows;
    int m;
  };
  auto build = [&](const std::vector<int>& set, Ops& o) {
    std::vector<GCg> base;
    uint32_t blk = 0;
    for (int i : set) {
      sa_handle h = hs[i];
      GCg g = {};
      g.blk0 = blk;
      g.n = h->n;
      g.sp = h->A0s.sp.p; g.ci = h->A0s.ci.p; g.v = h->A0s.v.p;
      g.base = h->A0s.idx16 ? h->A0s.base.p : nullptr;
      g.c16 = h->A0s.idx16 ? h->A0s.c16.p : nullptr;
      g.cg = h->cg.p;
      g.part = h->part.p;
      base.push_back(g);
      blk += g256(h->n);
    }
    o.rows = blk;
    o.m = (int)set.size();
    auto var = [&](auto fn) {
      std::vector<GCg> v = base;
      for (size_t k = 0; k < set.size(); ++k) fn(v[k], hs[set[k]], vh[set[k]]);
      return ar.put(v);
    };
    o.resid_r = var([](GCg& g, sa_handle h, VHier<T>*) { g.in = h->xb.p; g.bvec = h->bb.p; g.out = h->r.p; });
    o.resid_t = var([](GCg& g, sa_handle h, VHier<T>*) { g.in = h->xb.p; g.bvec = h->bb.p; g.out = h->t.p; });
    o.dots_rr = var([](GCg& g, sa_handle h, VHier<T>*) { g.a0 = h->r.p; g.b0 = h->r.p; });
    o.dots_tt = var([](GCg& g, sa_handle h, VHier<T>*) { g.a0 = h->t.p; g.b0 = h->t.p; });
    o.dots_rz = var([&](GCg& g, sa_handle h, VHier<T>* w) {
      g.a0 = h->r.p; g.b0 = w->z.p;
      if (flexible) { g.a1 = w->z.p; g.b1 = h->rprev.p; }
    });
    o.fin_dots = var([](GCg& g, sa_handle h, VHier<T>*) { g.np = RED_BLOCKS; g.stride = RED_BLOCKS; g.dots = h->dots.p; });
    o.fin_dots4 = var([](GCg& g, sa_handle h, VHier<T>*) { g.np = RED_BLOCKS; g.stride = RED_BLOCKS; g.dots = h->dots.p + 4; });
    o.spmv = var([](GCg& g, sa_handle h, VHier<T>*) { g.in = h->p.p; g.out = h->q.p; });
    o.fin_spmv = var([](GCg& g, sa_handle h, VHier<T>*) { g.np = (int)g256(h->n); g.stride = 0; g.dots = h->dots.p; });
    o.alpha = var([](GCg& g, sa_handle h, VHier<T>*) { g.dots = h->dots.p; });
    o.update = var([&](GCg& g, sa_handle h, VHier<T>*) {
      g.x = h->xb.p; g.r = h->r.p; g.rprev = flexible ? h->rprev.p : nullptr; g.p = h->p.p; g.q = h->q.p;
    });
    o.fin_upd = var([](GCg& g, sa_handle h, VHier<T>*) { g.np = RED_BLOCKS; g.stride = 0; g.dots = h->dots.p + 4; });
    o.beta0 = var([](GCg& g, sa_handle h, VHier<T>*) { g.dots = h->dots.p; g.flexible = -1; });
    o.beta = var([&](GCg& g, sa_handle h, VHier<T>*) { g.dots = h->dots.p; g.flexible = flexible; });
    o.pup1 = var([](GCg& g, sa_handle h, VHier<T>* w) { g.in = w->z.p; g.out = h->p.p; g.first = 1; });
    o.pup = var([](GCg& g, sa_handle h, VHier<T>* w) { g.in = w->z.p; g.out = h->p.p; g.first = 0; });
    o.gather = var([&](GCg& g, sa_handle h, VHier<T>*) { g.dots = h->dots.p + 4; g.gather = gath.p; });
  };
  auto L = [&](int op, size_t off, const Ops& o, unsigned blocks) {
    return launch_g_cg(s, op, ar.at<GCg>(off), o.m, blocks);
  };
  // host copy of the gathered (r.r, breakdown) pairs of the problems in `set`
  auto gather = [&](const Ops& o, size_t off) -> int {
    SA_TRY(L(GC_GATHER, off, o, 0));
    SA_CUDA(cudaMemcpyAsync(hg.data(), gath.p, sizeof(double) * 2 * o.m, cudaMemcpyDeviceToHost, s));
    SA_CUDA(cudaStreamSynchronize(s));
    return SA_OK;
  };

  std::vector<int> all(m);
  for (int i = 0; i < m; ++i) all[i] = i;
  std::vector<double> r0(m, 0.0);
  std::vector<int> its(m, 0), st(m, SA_ERR_NO_CONVERGENCE), act;
  Ops o;
  ar.clear();
  build(all, o);
  SA_TRY(ar.upload(s));
  SA_TRY(L(GC_RESID, o.resid_r, o, o.rows));
  SA_TRY(L(GC_DOTS, o.dots_rr, o, 0));
  SA_TRY(L(GC_FINISH, o.fin_dots, o, 0));
  // gather reads dots + 4; the initial r.r sits in dots[0]: gather it by a
  // finish into dots + 4 as well (the same sum)
  SA_TRY(L(GC_FINISH, o.fin_dots4, o, 0));
  SA_TRY(gather(o, o.gather));
  for (int i = 0; i < m; ++i) {
    r0[i] = sqrt(hg[2 * i]);
    if (r0[i] > 0.0) act.push_back(i);
    else st[i] = SA_OK;
  }
  int it = 0;
  if (!act.empty()) {
    ar.clear();
    build(act, o);
    V.plan(ar, act);
    SA_TRY(ar.upload(s));
    SA_TRY(V.run(ar, s));
    SA_TRY(L(GC_PUPDATE, o.pup1, o, 0));
    SA_TRY(L(GC_DOTS, o.dots_rz, o, 0));
    SA_TRY(L(GC_FINISH, o.fin_dots, o, 0));
    SA_TRY(L(GC_BETA, o.beta0, o, 0));
    for (it = 1; it <= maxit && !act.empty(); ++it) {
      SA_TRY(L(GC_SPMV_DOT, o.spmv, o, o.rows));
      SA_TRY(L(GC_FINISH, o.fin_spmv, o, 0));
      SA_TRY(L(GC_ALPHA, o.alpha, o, 0));
      SA_TRY(L(GC_UPDATE, o.update, o, 0));
      SA_TRY(L(GC_FINISH, o.fin_upd, o, 0));
      SA_TRY(gather(o, o.gather));
      std::vector<int> cand, keep;
      for (size_t k = 0; k < act.size(); ++k) {
        const int i = act[k];
        its[i] = it;
        if (hg[2 * k + 1] != 0.0) { st[i] = SA_ERR_BREAKDOWN; continue; }
        if (sqrt(hg[2 * k]) <= tol * r0[i]) cand.push_back(i);
        keep.push_back(i);
      }
      if (!cand.empty()) {
        // confirm on the true residual; where it does not confirm, it
        // replaces the recursive one
        Ops oc;
        const size_t mark = ar.img.size();
        build(cand, oc);  // appended to the image of the iterating set and uploaded with it
        SA_TRY(ar.upload(s));
        SA_TRY(L(GC_RESID, oc.resid_t, oc, oc.rows));
        SA_TRY(L(GC_DOTS, oc.dots_tt, oc, 0));
        SA_TRY(L(GC_FINISH, oc.fin_dots4, oc, 0));
        SA_TRY(gather(oc, oc.gather));
        std::vector<int> still;
        for (size_t k = 0; k < cand.size(); ++k) {
          const int i = cand[k];
          if (sqrt(hg[2 * k]) <= tol * r0[i]) st[i] = SA_OK;
          else SA_CUDA(cudaMemcpyAsync(hs[i]->r.p, hs[i]->t.p, sizeof(double) * hs[i]->n, cudaMemcpyDeviceToDevice, s));
        }
        for (int i : keep)
          if (st[i] != SA_OK) still.push_back(i);
        keep.swap(still);
        ar.img.resize(mark);  // the device copy of the prefix is unchanged
      }
      std::vector<int> next;
      for (int i : keep)
        if (it < maxit) next.push_back(i);  // at maxit the status stays SA_ERR_NO_CONVERGENCE
      if (next.empty()) { act.clear(); break; }
      if (next != act) {
        act.swap(next);
        ar.clear();
        build(act, o);
        V.plan(ar, act);
        SA_TRY(ar.upload(s));
      }
      SA_TRY(V.run(ar, s));
      SA_TRY(L(GC_DOTS, o.dots_rz, o, 0));
      SA_TRY(L(GC_FINISH, o.fin_dots, o, 0));
      SA_TRY(L(GC_BETA, o.beta, o, 0));
      SA_TRY(L(GC_PUPDATE, o.pup, o, 0));
    }
  }
  // true residuals at exit, the solutions
  ar.clear();
  build(all, o);
  SA_TRY(ar.upload(s));
  SA_TRY(L(GC_RESID, o.resid_t, o, o.rows));
  SA_TRY(L(GC_DOTS, o.dots_tt, o, 0));
  SA_TRY(L(GC_FINISH, o.fin_dots4, o, 0));
  SA_TRY(gather(o, o.gather));
  for (int i = 0; i < m; ++i)
    SA_CUDA(cudaMemcpyAsync(X[i], hs[i]->xb.p, sizeof(double) * hs[i]->n, cudaMemcpyDefault, s));
  SA_CUDA(cudaStreamSynchronize(s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < m; ++i) {
    statuses[i] = st[i];
    if (infos) {
      infos[i].iters = its[i];
      infos[i].rel_res_true = r0[i] > 0.0 ? sqrt(hg[2 * i]) / r0[i] : 0.0;
      infos[i].setup_ms = hs[i]->setup_ms;
      infos[i].solve_ms = ms;
      infos[i].status = st[i];
    }
  }
  return SA_OK;
}

}  // namespace sa

extern "C" {

int sa_solve_group(int m, sa_handle* hs, const double* const* B, double* const* X, double tol,
                   sa_solve_info* infos) {
  if (m < 0 || m > sa::GROUP_MAX || (m > 0 && (!hs || !B || !X)) || !(tol > 0.0)) return SA_ERR_INVALID_ARG;
  if (m == 0) return SA_OK;
  std::vector<sa_handle> h(hs, hs + m);
  for (int i = 0; i < m; ++i) {
    if (!h[i] || !B[i] || !X[i]) return SA_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (h[j] == h[i]) {
        sa::set_error_text("sa_solve_group: a handle appears twice (one right-hand side per handle)");
        return SA_ERR_INVALID_ARG;
      }
    if (h[i]->opt.precision != h[0]->opt.precision || h[i]->opt.cheb_degree != h[0]->opt.cheb_degree ||
        h[i]->opt.maxit != h[0]->opt.maxit) {
      sa::set_error_text("sa_solve_group: handles differ in precision, Chebyshev degree or maxit");
      return SA_ERR_INVALID_ARG;
    }
  }
  // the group runs on the first handle's stream, after the other handles' work
  cudaStream_t s = h[0]->al.stream;
  for (int i = 1; i < m; ++i) {
    if (h[i]->al.stream == s) continue;
    cudaEvent_t e;
    SA_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    SA_CUDA(cudaEventRecord(e, h[i]->al.stream));
    SA_CUDA(cudaStreamWaitEvent(s, e, 0));
    cudaEventDestroy(e);
  }
  std::vector<int> sts(m, SA_OK);
  int st;
  if (h[0]->opt.precision == SA_PREC_FP32_VCYCLE) {
    std::vector<sa::VHier<float>*> v;
    for (auto x : h) {
      if (!x->v32) return SA_ERR_INVALID_ARG;
      v.push_back(x->v32);
    }
    st = sa::cg_group<float>(h, v, B, X, tol, infos, sts.data());
  } else {
    std::vector<sa::VHier<double>*> v;
    for (auto x : h) {
      if (!x->v64) return SA_ERR_INVALID_ARG;
      v.push_back(x->v64);
    }
    st = sa::cg_group<double>(h, v, B, X, tol, infos, sts.data());
  }
  if (st != SA_OK) return st;
  int worst = SA_OK;
  for (int i = 0; i < m; ++i)
    if (sts[i] != SA_OK && worst == SA_OK) worst = sts[i];
  return worst;
}

}  // extern "C"
