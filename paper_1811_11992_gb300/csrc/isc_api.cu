// Host implementation of the isc.h C ABI: handle lifecycle, Newton and time
// step drivers, Krylov solvers (GMRES(m) and BiCGSTAB, both right
// preconditioned), exports and per-kernel timing.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "isc_internal.cuh"

using namespace isc;

struct isc_handle : public Handle {
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};

namespace {

// scalar slots in Handle::scal
constexpr int S_NORM = 0;     // 3 norms (bit patterns of doubles, atomicMax) and the wells' |F_w| / |target|
constexpr int S_H0 = 8;       // 72 Gram-Schmidt coefficients
constexpr int S_H1 = 80;      // 72 re-orthogonalisation coefficients
constexpr int S_NRM = 152;    // squared norm
constexpr int S_Y = 160;      // 72 solution coefficients
constexpr int S_BICG = 232;   // BiCGSTAB scalars
constexpr int NSCAL = 256;
constexpr int MAX_RESTART = 64;

int set_err(isc_handle* h, int code, const std::string& msg) {
  if (h) h->last_error = msg;
  return code;
}

#define CUDA_TRY(h, expr)                                                                       \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) return set_err(h, ISC_ERR_CUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
  } while (0)

cudaEvent_t take_event(isc_handle* h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct Region {
  isc_handle* h;
  int cls;
  cudaEvent_t b = nullptr;
  cudaEvent_t a = nullptr;
  Region(isc_handle* h_, int cls_, int launches) : h(h_), cls(cls_) {
    h->stats.launches[cls] += launches;
    h->stats.calls[cls] += 1;
    if (h->opt.profile) {
      a = take_event(h);
      b = take_event(h);
      cudaEventRecord(a, h->stream);
    }
  }
  ~Region() {
    if (a) {
      cudaEventRecord(b, h->stream);
      h->recs.push_back({cls, a, b});
    }
  }
};

void resolve_timers(isc_handle* h) {
  if (h->recs.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (auto& r : h->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) h->stats.ms[r.cls] += ms;
    h->pool.push_back(r.a);
    h->pool.push_back(r.b);
  }
  h->recs.clear();
}

int check_device_status(isc_handle* h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->h_status, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  int s = *h->h_status;
  if (s == 0) return ISC_OK;
  CUDA_TRY(h, cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->stream));
  if (s & DS_SINGULAR) return set_err(h, ISC_ERR_SINGULAR_BLOCK, "zero pivot in a diagonal block");
  if (s & DS_COKE) return set_err(h, ISC_ERR_COKE, "coke equation did not converge in a cell");
  if (s & DS_NONFINITE) return set_err(h, ISC_ERR_NONFINITE, "non-finite residual");
  if (s & DS_TIMEOUT) return set_err(h, ISC_ERR_TIMEOUT, "bounded device wait gave up");
  return set_err(h, ISC_ERR_CUDA, "unknown device status");
}

template <typename T>
int dalloc(isc_handle* h, T** p, size_t count) {
  const size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) return set_err(h, ISC_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->dev_sizes[(void*)*p] = bytes;
  return ISC_OK;
}

// frees an allocation made by dalloc before the handle's end
void dfree(isc_handle* h, void* p) {
  if (!p) return;
  h->dev_sizes.erase(p);
  cudaFree(p);
}

void free_all(isc_handle* h) {
  void* ptrs[] = {h->rowptr, h->col, h->level_cells, h->phi_ref, h->depth, h->tx, h->ty, h->tz, h->well_slot,
                  h->slots, h->u, h->coke, h->u_n, h->coke_n, h->acc_n, h->props, h->fbuf, h->R, h->J, h->ntot, h->du,
                  h->rhs, h->dinv, h->uhat, h->J32, h->dinv32, h->uhat32, h->vec32, h->V32, h->Z32, h->w32, h->gm_in, h->scal_in, h->V, h->Z, h->w, h->tmp, h->partial, h->scal, h->dstatus, h->pipe, h->red_counter, h->gmres,
                  h->wx, h->wy, h->wz, h->cw, h->bhp, h->bhp_n, h->Dw, h->Bv, h->Cv, h->Fq, h->Dq, h->adj.store, h->adj.ubar, h->adj.cbar, h->adj.lam, h->adj.glnk, h->adj.grx,
                  h->adj.scond, h->adj.kd, h->adj.loss_cell, h->adj.sums, h->adj.inj_first, h->adj.inj_count, h->u_prev, h->run_max};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->dev_sizes.clear();
  cpr_free(*h);
  if (h->h_scal) cudaFreeHost(h->h_scal);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->h_ring) cudaFreeHost(h->h_ring);
  for (auto& ev : h->gm_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& r : h->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
}

double host_dot(isc_handle* h, const double* a, const double* b, int off) {
  launch_mdot(*h, a, 1, b, off, h->stream);
  cudaMemcpyAsync(h->h_scal + off, h->scal + off, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  return h->h_scal[off];
}

void spmv(isc_handle* h, const double* x, double* y) {
  Region rg(h, ISC_K_SPMV, h->nwc ? 3 : 1);
  launch_spmv(h->n, h->rowptr, h->col, h->J, x, y, h->decoupled ? 1 : 0, h->stream);
  launch_well_border_spmv(*h, x, y, h->stream);
}

void prec_cells(isc_handle* h, const double* r, double* z);

// block lower-triangular: the cells' preconditioner, then the coupled wells' rows
void prec(isc_handle* h, const double* r, double* z) {
  prec_cells(h, r, z);
  if (h->nwc) {
    Region rg(h, ISC_K_PREC_APPLY, 1);
    launch_well_prec(*h, r, z, h->stream);
  }
}

int inner_solve(isc_handle* h, const double* r, double* z);

void prec_cells(isc_handle* h, const double* r, double* z) {
  if (h->opt.precision == ISC_PRECISION_MIXED_FGMRES) {
    inner_solve(h, r, z);
    return;
  }
  if (h->opt.prec == ISC_PREC_CPR) {
    {
      Region rg(h, ISC_K_CPR, cpr_pressure_launches(*h));
      launch_cpr_pressure(*h, r, h->stream);
    }
    {
      Region rg(h, ISC_K_PREC_APPLY, 2);
      launch_ilu_apply_pipe(*h, h->cpr.r1, z, h->stream);
    }
    Region rg(h, ISC_K_CPR, 1);
    launch_cpr_finish(*h, z, h->stream);
    return;
  }
  int launches = h->opt.prec == ISC_PREC_BILU0 ? 2 : 1;
  Region rg(h, ISC_K_PREC_APPLY, launches);
  launch_prec_apply(*h, r, z, h->stream);
}

// z ~ A^-1 r by inner_its iterations of right-preconditioned GMRES in FP32 on the
// FP32 copy of the (decoupled) matrix with the FP32 block ILU(0) (or CPR-PF with the
// FP32 pressure multigrid and FP32 ILU(0)),
// classical Gram-Schmidt applied twice, x0 = 0; the rotations and the final
// back-substitution run on the device, so the whole solve is a fixed launch
// sequence with no host round trip. A fixed iteration count keeps it cheap to
// schedule; the outer GMRES is flexible, so the resulting operator may vary.
int inner_solve(isc_handle* h, const double* r, double* z) {
  const int m = h->opt.inner_its;
  const int len = h->n * 8;
  const size_t vs = (size_t)len;
  cudaStream_t s = h->stream;
  float* V = h->V32;
  float* Z = h->Z32;
  double* G = h->gm_in;
  double* sc = h->scal_in;  // [0, 64) h0, [64, 128) h1, 128 ||w||^2, [136, 200) y
  {
    Region rg(h, ISC_K_BLAS1, 3);
    launch_f32_nrm(*h, len, r, V, sc + 128, s);
    launch_gmres_start_dev(G, m, sc + 128, s);
    launch_scale_dev32(G, len, V, V, s);
  }
  for (int j = 0; j < m; ++j) {
    float* Vj = V + (size_t)j * vs;
    float* Zj = Z + (size_t)j * vs;
    if (h->opt.prec == ISC_PREC_CPR) {
      // CPR-PF on FP32 vectors: FP32 pressure multigrid, r1 = r - A E p (in w32, free until
      // the SpMV below), FP32 ILU(0) on r1, z += E p
      {
        Region rg(h, ISC_K_CPR, cpr_pressure_launches(*h));
        launch_cpr_pressure32(*h, Vj, h->w32, s);
      }
      {
        Region rg(h, ISC_K_PREC_APPLY, 2);
        launch_ilu_apply_f32(*h, h->w32, Zj, s);
      }
      Region rg(h, ISC_K_CPR, 1);
      launch_cpr_finish32(*h, Zj, s);
    } else {
      Region rg(h, ISC_K_PREC_APPLY, 2);
      launch_ilu_apply_f32(*h, Vj, Zj, s);
    }
    {
      Region rg(h, ISC_K_SPMV32, 1);
      launch_spmv32(h->n, h->rowptr, h->col, h->J32, Zj, h->w32, h->decoupled ? 1 : 0, s);
    }
    Region rg(h, ISC_K_BLAS1, j + 1 < m ? 5 : 4);
    launch_mdot32(*h, len, vs, V, j + 1, h->w32, sc, s);
    launch_maxpy_mdot32(*h, len, vs, h->w32, V, j + 1, sc, sc + 64, s);
    launch_maxpy_norm32(*h, len, vs, h->w32, V, j + 1, sc + 64, sc + 128, s);
    launch_gmres_givens_at(G, j, m, sc, sc + 64, sc + 128, s);
    if (j + 1 < m) launch_scale_dev32(G, len, h->w32, V + (size_t)(j + 1) * vs, s);
  }
  Region rg(h, ISC_K_BLAS1, 2);
  launch_gmres_backsub_at(G, m, m, sc + 136, s);
  launch_comb_out32(len, Z, vs, m, sc + 136, z, s);
  return ISC_OK;
}

int build_prec(isc_handle* h) {
  if (h->opt.prec == ISC_PREC_CPR) {
    // (re)allocates when the precision of the multigrid arrays changed
    int st = cpr_setup_levels(*h);
    if (st) return set_err(h, st, "CPR multigrid workspace");
    Region rg(h, ISC_K_CPR, h->cpr.nlev);
    launch_cpr_setup(*h, h->stream);
  }
  if (h->opt.prec == ISC_PREC_BILU0 || h->opt.prec == ISC_PREC_CPR) {
    const bool mixed = h->opt.precision != ISC_PRECISION_FP64;
    if (mixed && !h->J32) {
      // first mixed-precision use: FP32 copies of the blocks and D^-1, two FP32 sweep vectors
      int e = 0;
      e |= dalloc(h, &h->J32, (size_t)h->nnzb * BB);
      e |= dalloc(h, &h->dinv32, (size_t)h->n * BB);
      e |= dalloc(h, &h->uhat32, (size_t)h->n * 3 * BB);
      e |= dalloc(h, &h->vec32, (size_t)h->n * 16);
      if (e) return ISC_ERR_NOMEM;
    }
    if (h->opt.precision == ISC_PRECISION_MIXED_FGMRES && h->inner_alloc < h->opt.inner_its) {
      // inner FP32 GMRES workspace, (re)allocated when inner_its grows
      for (void* q : {(void*)h->V32, (void*)h->Z32, (void*)h->w32, (void*)h->gm_in, (void*)h->scal_in}) dfree(h, q);
      h->V32 = h->Z32 = h->w32 = nullptr;
      h->gm_in = h->scal_in = nullptr;
      const size_t n8 = (size_t)h->n * 8;
      int e = 0;
      e |= dalloc(h, &h->V32, n8 * (h->opt.inner_its + 1));
      e |= dalloc(h, &h->Z32, n8 * h->opt.inner_its);
      e |= dalloc(h, &h->w32, n8);
      e |= dalloc(h, &h->gm_in, GMRES_STATE);
      e |= dalloc(h, &h->scal_in, 256);
      if (e) return ISC_ERR_NOMEM;
      h->inner_alloc = h->opt.inner_its;
    }
    // mixed precision: FP32 copy of the blocks, then the factorisation in FP32
    Region rg(h, ISC_K_ILU_FACTOR, mixed ? 2 : 1);
    launch_ilu_factor(*h, h->stream);
  } else if (h->opt.prec == ISC_PREC_BJACOBI) {
    Region rg(h, ISC_K_ILU_FACTOR, 1);
    launch_bjacobi_factor(*h, h->stream);
  }
  h->prec_built = true;
  return check_device_status(h);
}

// Right-preconditioned restarted GMRES(m), classical Gram-Schmidt applied twice.
// Solves A x = b, x0 = 0. The Hessenberg column, the Givens rotations and the
// next basis vector's scaling are computed on the device; the host reads the
// residual estimate one iteration behind (it has already queued the next
// iteration when it waits), so the GPU never idles on a host round trip. At
// convergence the one speculative iteration is discarded: the solution uses
// the columns up to the converged one.
int gmres(isc_handle* h, const double* b, double* x, int* its_out, double* rel_out) {
  const int len = h->vlen;
  const int m = std::min(h->opt.restart, h->restart_alloc);
  cudaStream_t s = h->stream;
  double* V = h->V;
  double* Z = h->Z;
  cudaMemsetAsync(x, 0, sizeof(double) * len, s);
  double bnorm;
  {
    Region rg(h, ISC_K_BLAS1, 2);
    bnorm = sqrt(host_dot(h, b, b, S_NRM));
  }
  *its_out = 0;
  *rel_out = 0.0;
  if (bnorm == 0.0) return ISC_OK;
  if (!isfinite(bnorm)) return set_err(h, ISC_ERR_NONFINITE, "non-finite right-hand side");
  int its = 0;
  double rel = 1.0;
  bool first = true;
  // single classical Gram-Schmidt leaves the second set of coefficients at zero
  if (h->opt.orth == ISC_ORTH_CGS1) cudaMemsetAsync(h->scal + S_H1, 0, sizeof(double) * (MAX_RESTART + 8), s);
  while (its < h->opt.maxit_lin) {
    double beta;
    if (first) {
      cudaMemcpyAsync(V, b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
      beta = bnorm;
    } else {
      spmv(h, x, h->w);
      Region rg(h, ISC_K_BLAS1, 3);
      cudaMemcpyAsync(V, b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
      launch_axpby(len, -1.0, h->w, 1.0, V, s);
      beta = sqrt(host_dot(h, V, V, S_NRM));
    }
    first = false;
    rel = beta / bnorm;
    if (rel <= h->opt.tol_lin) break;
    {
      Region rg(h, ISC_K_BLAS1, 2);
      launch_scale_copy(len, 1.0 / beta, V, V, s);
      launch_gmres_start(*h, m, beta, s);
    }
    const int jmax = std::min(m, h->opt.maxit_lin - its);
    int jdone = 0;
    bool stop = false;
    // the status of iteration j: (rel, 1/h, h) in ring slot j % 2
    auto status = [&](int j, double* r, double* hn) -> int {
      if (cudaEventSynchronize(h->gm_ev[j & 1]) != cudaSuccess) return ISC_ERR_CUDA;
      *r = h->h_ring[3 * (j & 1)];
      *hn = h->h_ring[3 * (j & 1) + 2];
      if (!isfinite(*r) || !isfinite(*hn)) return set_err(h, ISC_ERR_NONFINITE, "non-finite Krylov vector");
      return ISC_OK;
    };
    // residual estimates of the iterations read so far (to predict convergence)
    double r_prev2 = -1.0, r_prev1 = -1.0;
    bool read_prev = false;  // the status of iteration j - 1 was read before launching j
    for (int j = 0; j < jmax; ++j) {
      // when the observed reduction rate predicts that iteration j - 1 has converged,
      // wait for its status instead of launching a speculative iteration
      read_prev = false;
      if (j >= 1 && r_prev2 > 0.0 && r_prev1 > 0.0 && r_prev1 * (r_prev1 / r_prev2) <= 4.0 * h->opt.tol_lin) {
        double r, hn;
        int st = status(j - 1, &r, &hn);
        if (st) return st;
        rel = r;
        r_prev2 = r_prev1;
        r_prev1 = r;
        read_prev = true;
        if (r <= h->opt.tol_lin || hn == 0.0) {
          jdone = j;
          stop = true;
          break;
        }
      }
      double* Vj = V + (size_t)j * h->vstride;
      double* Zj = Z + (size_t)j * h->vstride;
      prec(h, Vj, Zj);
      spmv(h, Zj, h->w);
      if (h->opt.orth == ISC_ORTH_CGS1) {
        // classical Gram-Schmidt once: h0 = V^T w; w -= V h0 fused with ||w||^2 (h1 stays 0)
        Region rg(h, ISC_K_BLAS1, 4);
        launch_mdot(*h, V, j + 1, h->w, S_H0, s);
        launch_maxpy_norm(*h, h->w, V, j + 1, S_H0, S_NRM, s);
        launch_gmres_givens(*h, j, m, bnorm, S_H0, S_H1, S_NRM, s);
        launch_scale_dev(*h, h->w, V + (size_t)(j + 1) * h->vstride, s);
        cudaMemcpyAsync(h->h_ring + 3 * (j & 1), gmres_status(*h), 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaEventRecord(h->gm_ev[j & 1], s);
      } else {
        // classical Gram-Schmidt applied twice: h0 = V^T w; w -= V h0 fused with h1 = V^T w;
        // w -= V h1 fused with ||w||^2
        Region rg(h, ISC_K_BLAS1, j + 1 <= 32 ? 5 : 6);
        launch_mdot(*h, V, j + 1, h->w, S_H0, s);
        launch_maxpy_mdot(*h, h->w, V, j + 1, S_H0, S_H1, s);
        launch_maxpy_norm(*h, h->w, V, j + 1, S_H1, S_NRM, s);
        launch_gmres_givens(*h, j, m, bnorm, S_H0, S_H1, S_NRM, s);
        launch_scale_dev(*h, h->w, V + (size_t)(j + 1) * h->vstride, s);
        cudaMemcpyAsync(h->h_ring + 3 * (j & 1), gmres_status(*h), 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaEventRecord(h->gm_ev[j & 1], s);
      }
      if (j >= 1 && !read_prev) {
        double r, hn;
        int st = status(j - 1, &r, &hn);
        if (st) return st;
        rel = r;
        r_prev2 = r_prev1;
        r_prev1 = r;
        if (r <= h->opt.tol_lin || hn == 0.0) {
          jdone = j;  // iteration j is speculative: discarded
          stop = true;
          break;
        }
      }
    }
    if (!stop) {
      double r, hn;
      int st = status(jmax - 1, &r, &hn);
      if (st) return st;
      rel = r;
      jdone = jmax;
    }
    its += jdone;
    {
      Region rg(h, ISC_K_BLAS1, 2);
      launch_gmres_backsub(*h, jdone, m, S_Y, s);
      launch_maxpy(*h, x, Z, jdone, S_Y, 1.0, s);
    }
    if (rel <= h->opt.tol_lin) {
      spmv(h, x, h->w);
      Region rg(h, ISC_K_BLAS1, 3);
      cudaMemcpyAsync(h->tmp, b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
      launch_axpby(len, -1.0, h->w, 1.0, h->tmp, s);
      rel = sqrt(host_dot(h, h->tmp, h->tmp, S_NRM)) / bnorm;
      if (rel <= h->opt.tol_lin) break;
    }
  }
  *its_out = its;
  *rel_out = rel;
  if (rel > h->opt.tol_lin) return set_err(h, ISC_ERR_KRYLOV_NOCONV, "GMRES did not reach tol_lin");
  return ISC_OK;
}

// Right-preconditioned BiCGSTAB, x0 = 0.
int bicgstab(isc_handle* h, const double* b, double* x, int* its_out, double* rel_out) {
  const int len = h->vlen;
  cudaStream_t s = h->stream;
  const size_t vs = h->vstride;
  double* r = h->V;
  double* rhat = r + vs;
  double* p = rhat + vs;
  double* v = p + vs;
  double* sv = v + vs;
  double* t = sv + vs;
  double* phat = h->Z;
  double* shat = phat + vs;
  cudaMemsetAsync(x, 0, sizeof(double) * len, s);
  double bnorm;
  {
    Region rg(h, ISC_K_BLAS1, 2);
    bnorm = sqrt(host_dot(h, b, b, S_NRM));
  }
  *its_out = 0;
  *rel_out = 0.0;
  if (bnorm == 0.0) return ISC_OK;
  cudaMemcpyAsync(r, b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(rhat, b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(p, 0, sizeof(double) * len, s);
  cudaMemsetAsync(v, 0, sizeof(double) * len, s);
  double rho_old = 1.0, alpha = 1.0, omega = 1.0, rel = 1.0;
  int it;
  for (it = 1; it <= h->opt.maxit_lin; ++it) {
    double rho;
    {
      Region rg(h, ISC_K_BLAS1, 2);
      rho = host_dot(h, rhat, r, S_BICG);
    }
    if (rho == 0.0) break;
    {
      Region rg(h, ISC_K_BLAS1, 2);
      if (it == 1) {
        cudaMemcpyAsync(p, r, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
      } else {
        double beta = (rho / rho_old) * (alpha / omega);
        launch_axpby(len, -omega, v, 1.0, p, s);
        launch_axpby(len, 1.0, r, beta, p, s);
      }
    }
    prec(h, p, phat);
    spmv(h, phat, v);
    double rv;
    {
      Region rg(h, ISC_K_BLAS1, 2);
      rv = host_dot(h, rhat, v, S_BICG + 1);
    }
    alpha = rho / rv;
    double snorm;
    {
      Region rg(h, ISC_K_BLAS1, 4);
      cudaMemcpyAsync(sv, r, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
      launch_axpby(len, -alpha, v, 1.0, sv, s);
      snorm = sqrt(host_dot(h, sv, sv, S_BICG + 2));
    }
    if (snorm / bnorm <= h->opt.tol_lin) {
      Region rg(h, ISC_K_BLAS1, 1);
      launch_axpby(len, alpha, phat, 1.0, x, s);
      rel = snorm / bnorm;
      break;
    }
    prec(h, sv, shat);
    spmv(h, shat, t);
    double ts, tt;
    {
      Region rg(h, ISC_K_BLAS1, 4);
      ts = host_dot(h, t, sv, S_BICG + 3);
      tt = host_dot(h, t, t, S_BICG + 4);
    }
    omega = tt > 0.0 ? ts / tt : 0.0;
    {
      Region rg(h, ISC_K_BLAS1, 5);
      launch_axpby(len, alpha, phat, 1.0, x, s);
      launch_axpby(len, omega, shat, 1.0, x, s);
      cudaMemcpyAsync(r, sv, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
      launch_axpby(len, -omega, t, 1.0, r, s);
      rel = sqrt(host_dot(h, r, r, S_BICG + 5)) / bnorm;
    }
    rho_old = rho;
    if (!isfinite(rel)) return set_err(h, ISC_ERR_NONFINITE, "non-finite BiCGSTAB residual");
    if (rel <= h->opt.tol_lin || omega == 0.0) break;
  }
  *its_out = std::min(it, h->opt.maxit_lin);
  *rel_out = rel;
  if (rel > h->opt.tol_lin) return set_err(h, ISC_ERR_KRYLOV_NOCONV, "BiCGSTAB did not reach tol_lin");
  return ISC_OK;
}

// Transmissibilities (harmonic average of A k / h of the two cells, Sec. 3.1),
// the face weights d ln T / d ln k_lo = t_hi / (t_lo + t_hi), the well
// indices and the injector shares at the current ln k multipliers; uploaded
// on the handle's stream (the host vectors live until the copies finish).
int refresh_parameters(isc_handle* h) {
  const int n = h->n, nx = h->nx, ny = h->ny, nz = h->nz;
  std::vector<double> tx(n, 0.0), ty(n, 0.0), tz(n, 0.0), wx(n, 0.0), wy(n, 0.0), wz(n, 0.0);
  std::vector<double> k(3 * (size_t)n);
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < n; ++c) k[(size_t)d * n + c] = h->h_perm0[(size_t)d * n + c] * exp(h->h_lnk[c]);
  const double* kx = k.data();
  const double* ky = kx + n;
  const double* kz = ky + n;
  auto harm = [](double a, double b) { return 2.0 * a * b / (a + b); };
  const double ax = h->face_area[0], ay = h->face_area[1], az = h->face_area[2];
  for (int c = 0; c < n; ++c) {
    int ix = c % nx, iy = (c / nx) % ny, iz = c / (nx * ny);
    if (ix < nx - 1) {
      tx[c] = harm(ax * kx[c], ax * kx[c + 1]);
      wx[c] = kx[c + 1] / (kx[c] + kx[c + 1]);
    }
    if (iy < ny - 1) {
      ty[c] = harm(ay * ky[c], ay * ky[c + nx]);
      wy[c] = ky[c + nx] / (ky[c] + ky[c + nx]);
    }
    if (iz < nz - 1) {
      tz[c] = harm(az * kz[c], az * kz[c + nx * ny]);
      wz[c] = kz[c + nx * ny] / (kz[c] + kz[c + nx * ny]);
    }
  }
  // well indices scale with the cell's permeability (Peaceman WI is linear in k)
  for (const WellInfo& W : h->h_wells) {
    double wsum = 0.0;
    for (int q = 0; q < W.count; ++q) {
      WellSlot& sl = h->h_slots[W.first + q];
      sl.WI = h->h_WI0[W.first + q] * exp(h->h_lnk[sl.cell]);
      wsum += sl.WI;
    }
    if (W.kind == ISC_WELL_COUPLED_INJECTOR) {
      // the stream's composition and molar enthalpy; the rate follows the bottom-hole pressure
      for (int q = 0; q < W.count; ++q) {
        WellSlot& sl = h->h_slots[W.first + q];
        for (int c = 0; c < 6; ++c) sl.src[c] = W.inj_y[c];
        sl.src[6] = W.Hinj;
      }
    }
    if (W.kind != ISC_WELL_RATE_INJECTOR) continue;
    for (int q = 0; q < W.count; ++q) {
      WellSlot& sl = h->h_slots[W.first + q];
      sl.share = sl.WI / wsum;
      for (int c = 0; c < 6; ++c) sl.src[c] = sl.share * W.target * W.inj_y[c];
      sl.src[6] = sl.share * W.target * W.Hinj;
    }
  }
  cudaStream_t s = h->stream;
  CUDA_TRY(h, cudaMemcpyAsync(h->tx, tx.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(h, cudaMemcpyAsync(h->ty, ty.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(h, cudaMemcpyAsync(h->tz, tz.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(h, cudaMemcpyAsync(h->wx, wx.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(h, cudaMemcpyAsync(h->wy, wy.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(h, cudaMemcpyAsync(h->wz, wz.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  if (h->nslots)
    CUDA_TRY(h, cudaMemcpyAsync(h->slots, h->h_slots.data(), sizeof(WellSlot) * h->nslots, cudaMemcpyHostToDevice, s));
  CUDA_TRY(h, cudaStreamSynchronize(s));
  return ISC_OK;
}

int validate_options(isc_handle* h, const isc_options& o) {
  if (o.restart < 1 || o.restart > MAX_RESTART) return set_err(h, ISC_ERR_INVALID_ARG, "restart must be 1..64");
  if (o.krylov != ISC_KRYLOV_GMRES && o.krylov != ISC_KRYLOV_BICGSTAB)
    return set_err(h, ISC_ERR_INVALID_ARG, "unknown krylov method");
  if (o.prec < ISC_PREC_NONE || o.prec > ISC_PREC_CPR) return set_err(h, ISC_ERR_INVALID_ARG, "unknown preconditioner");
  if (o.precision != ISC_PRECISION_FP64 && o.precision != ISC_PRECISION_MIXED &&
      o.precision != ISC_PRECISION_MIXED_FGMRES)
    return set_err(h, ISC_ERR_INVALID_ARG, "unknown precision");
  if (o.precision == ISC_PRECISION_MIXED_FGMRES) {
    if (o.krylov != ISC_KRYLOV_GMRES || (o.prec != ISC_PREC_BILU0 && o.prec != ISC_PREC_CPR))
      return set_err(h, ISC_ERR_INVALID_ARG, "mixed_fgmres needs krylov = GMRES and prec = BILU0 or CPR");
    if (o.inner_its < 1 || o.inner_its > 32) return set_err(h, ISC_ERR_INVALID_ARG, "inner_its must be 1..32");
  }
  if (o.orth != ISC_ORTH_CGS2 && o.orth != ISC_ORTH_CGS1) return set_err(h, ISC_ERR_INVALID_ARG, "unknown orth");
  if (!(o.tol_lin > 0.0) || o.maxit_lin < 1 || !(o.tol_newton >= 0.0) || o.maxit_newton < 1)
    return set_err(h, ISC_ERR_INVALID_ARG, "tolerances must be positive and iteration limits >= 1");
  return ISC_OK;
}

}  // namespace

// The forward sweep of the discrete adjoint: the time loop with the frozen step
// sizes, the loss, and the states kept for the reverse sweep (every K-th state
// as a checkpoint plus the last segment's states). Records the step sizes so
// that adjoint_backward can run later on the same store.
static int adjoint_forward(isc_handle* h, const isc_adjoint_spec* spec, double* loss, isc_adjoint_info* info) {
  const int N = spec->n_steps, K = spec->checkpoint_every;
  if (N < 1 || K < 1 || !spec->dt) return set_err(h, ISC_ERR_INVALID_ARG, "n_steps and checkpoint_every must be >= 1");
  for (int q = 0; q < N; ++q)
    if (!(spec->dt[q] > 0.0) || !isfinite(spec->dt[q])) return set_err(h, ISC_ERR_INVALID_ARG, "step sizes must be > 0");
  if (!(spec->tol_adjoint >= 0.0)) return set_err(h, ISC_ERR_INVALID_ARG, "tol_adjoint must be >= 0");
  if (!h->have_acc) return set_err(h, ISC_ERR_STATE, "isc_begin_step (or isc_init_equilibrium) must come first");
  const int n = h->n;
  // a stored state: u (8N), C_c (N), the coupled wells' bottom-hole pressures
  const size_t len = (size_t)n * 8, SN = (size_t)n * 9 + h->nwc;
  const int ncp = (N + K - 1) / K;
  const int need = ncp + K + 2;                 // checkpoints, K+1 segment states, the final state
  const int traj0 = ncp, fin = ncp + K + 1;
  AdjointWork& A = h->adj;
  cudaStream_t s = h->stream;
  A.ready = false;
  // workspace
  if (!A.ubar) {
    int e = 0;
    // ubar and lambda hold the cells' 8N entries and the coupled wells' rows (Krylov vector length)
    e |= dalloc(h, &A.ubar, (size_t)h->vstride);
    e |= dalloc(h, &A.cbar, n);
    e |= dalloc(h, &A.lam, (size_t)h->vstride);
    e |= dalloc(h, &A.glnk, n);
    e |= dalloc(h, &A.grx, (size_t)2 * ISC_MAX_RXN * n);
    e |= dalloc(h, &A.scond, n);
    e |= dalloc(h, &A.kd, n);
    e |= dalloc(h, &A.loss_cell, n);
    e |= dalloc(h, &A.sums, 1 + 2 * ISC_MAX_RXN);
    if (e) return ISC_ERR_NOMEM;
  }
  if (A.cap_states < need) {
    dfree(h, A.store);
    A.store = nullptr;
    A.cap_states = 0;
    if (dalloc(h, &A.store, (size_t)need * SN)) return ISC_ERR_NOMEM;
    A.cap_states = need;
  }
  auto slot = [&](int k) { return A.store + (size_t)k * SN; };
  auto save = [&](int k) -> int {
    CUDA_TRY(h, cudaMemcpyAsync(slot(k), h->u, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(slot(k) + len, h->coke, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (h->nwc)
      CUDA_TRY(h, cudaMemcpyAsync(slot(k) + len + n, h->bhp, sizeof(double) * h->nwc, cudaMemcpyDeviceToDevice, s));
    return ISC_OK;
  };
  int st;
  CUDA_TRY(h, cudaMemsetAsync(A.loss_cell, 0, sizeof(double) * n, s));
  if ((st = save(0)) || (st = save(traj0))) return st;
  int seg0 = 0;
  for (int q = 1; q <= N; ++q) {
    isc_step_info si;
    st = isc_timestep(h, spec->dt[q - 1], &si);
    info->newton_iterations += si.newton_iterations;
    info->krylov_iterations_forward += si.krylov_iterations;
    if (st) return info->status = st;
    {
      Region rg(h, ISC_K_ADJOINT, 1);
      launch_oil_rate(*h, spec->dt[q - 1], s);
    }
    const int j = q - seg0;
    if ((st = save(traj0 + j))) return st;
    if (j == K && q < N) {
      seg0 = q;
      if ((st = save(q / K)) || (st = save(traj0))) return st;
    }
  }
  if ((st = save(fin))) return st;
  launch_row_sums(1, n, A.loss_cell, A.sums, s);
  double Lsum = 0.0;
  CUDA_TRY(h, cudaMemcpyAsync(&Lsum, A.sums, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaStreamSynchronize(s));
  info->loss = Lsum;
  if (loss) *loss = Lsum;
  A.dts.assign(spec->dt, spec->dt + N);
  A.K = K;
  A.tol_adjoint = spec->tol_adjoint;
  A.loss = Lsum;
  A.traj_used = false;
  A.ready = true;
  return ISC_OK;
}

// The reverse sweep over the states the last adjoint_forward kept: per step
// (last to first) one transposed solve and the gradient parts, each earlier
// segment recomputed from its checkpoint. Leaves the handle at the loop's final state.
static int adjoint_backward(isc_handle* h, double* g_log_k, double* g_Ea, double* g_lnA, isc_adjoint_info* info) {
  AdjointWork& A = h->adj;
  if (!A.ready) return set_err(h, ISC_ERR_STATE, "run the forward sweep (isc_adjoint_forward) first");
  const int N = (int)A.dts.size(), K = A.K;
  const int n = h->n, nr = h->P.nr;
  const size_t len = (size_t)n * 8, SN = (size_t)n * 9 + h->nwc, vlen = (size_t)h->vlen;
  const int ncp = (N + K - 1) / K;
  const int traj0 = ncp, fin = ncp + K + 1;
  cudaStream_t s = h->stream;
  info->loss = A.loss;
  auto slot = [&](int k) { return A.store + (size_t)k * SN; };
  auto save = [&](int k) -> int {
    CUDA_TRY(h, cudaMemcpyAsync(slot(k), h->u, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(slot(k) + len, h->coke, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (h->nwc)
      CUDA_TRY(h, cudaMemcpyAsync(slot(k) + len + n, h->bhp, sizeof(double) * h->nwc, cudaMemcpyDeviceToDevice, s));
    return ISC_OK;
  };
  auto load_accepted = [&](int k) -> int {
    CUDA_TRY(h, cudaMemcpyAsync(h->u, slot(k), sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->coke, slot(k) + len, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (h->nwc)
      CUDA_TRY(h, cudaMemcpyAsync(h->bhp, slot(k) + len + n, sizeof(double) * h->nwc, cudaMemcpyDeviceToDevice, s));
    return isc_begin_step(h);
  };
  CUDA_TRY(h, cudaMemsetAsync(A.ubar, 0, sizeof(double) * vlen, s));
  CUDA_TRY(h, cudaMemsetAsync(A.cbar, 0, sizeof(double) * n, s));
  CUDA_TRY(h, cudaMemsetAsync(A.glnk, 0, sizeof(double) * n, s));
  CUDA_TRY(h, cudaMemsetAsync(A.grx, 0, sizeof(double) * 2 * ISC_MAX_RXN * n, s));
  const double tol_saved = h->opt.tol_lin;
  const double tol_adj = A.tol_adjoint > 0.0 ? A.tol_adjoint : tol_saved;
  int result = ISC_OK;
  // the last segment's states are still in the trajectory slots from the forward sweep;
  // a second backward over the same forward recomputes it too
  for (int seg = ncp - 1; seg >= 0 && result == ISC_OK; --seg) {
    const int s0 = seg * K, s1 = std::min(s0 + K, N);
    if (seg < ncp - 1 || A.traj_used) {
      // recompute the segment's states from its checkpoint (the Newton path is deterministic)
      if ((result = load_accepted(seg))) break;
      if ((result = save(traj0))) break;
      for (int q = s0 + 1; q <= s1 && result == ISC_OK; ++q) {
        isc_step_info si;
        result = isc_timestep(h, A.dts[q - 1], &si);
        info->newton_iterations += si.newton_iterations;
        info->krylov_iterations_forward += si.krylov_iterations;
        info->recomputed_steps++;
        if (!result) result = save(traj0 + q - s0);
      }
      if (result) break;
    }
    for (int q = s1; q > s0; --q) {
      const double dt = A.dts[q - 1];
      const double* old = slot(traj0 + q - 1 - s0);
      const double* cur = slot(traj0 + q - s0);
      cudaMemcpyAsync(h->u_n, old, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(h->coke_n, old + len, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
      launch_old_accumulation(*h, s);
      h->have_acc = true;
      cudaMemcpyAsync(h->u, cur, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
      if (h->nwc) cudaMemcpyAsync(h->bhp, cur + len + n, sizeof(double) * h->nwc, cudaMemcpyDeviceToDevice, s);
      {
        Region rg(h, ISC_K_ADJOINT, h->nwc ? 2 : 1);
        launch_adj_pre(*h, dt, s);
      }
      if ((result = isc_assemble(h, dt))) break;
      {
        Region rg(h, ISC_K_ADJOINT, 1);
        launch_bsr_transpose(*h, s);
      }
      // [J C^T-border; B^T D]: the transposed bordered system exchanges the border
      // column (dF/d bhp per perforation) and the well rows (dF_w/du); D is its own transpose
      std::swap(h->Bv, h->Cv);
      // J^T lambda = ubar (the transposed system is decoupled and preconditioned like J);
      // the wells' rows take dP/d bhp
      cudaMemcpyAsync(h->R, A.ubar, sizeof(double) * vlen, cudaMemcpyDeviceToDevice, s);
      int its = 0;
      double rel = 0.0;
      if (!(h->opt.decouple && (result = isc_decouple(h))) && !(result = build_prec(h))) {
        {
          Region rg(h, ISC_K_BLAS1, 1);
          launch_scale_copy((int)vlen, 1.0, h->R, h->rhs, s);
        }
        h->opt.tol_lin = tol_adj;
        if (h->opt.krylov == ISC_KRYLOV_GMRES)
          result = gmres(h, h->rhs, A.lam, &its, &rel);
        else
          result = bicgstab(h, h->rhs, A.lam, &its, &rel);
        h->opt.tol_lin = tol_saved;
      }
      std::swap(h->Bv, h->Cv);
      info->krylov_iterations_adjoint += its;
      info->adjoint_rel_residual = std::max(info->adjoint_rel_residual, rel);
      if (result) break;
      {
        Region rg(h, ISC_K_ADJOINT, (q > 1 ? 4 : 3) + (h->nwc ? 1 : 0));
        launch_adj_post(*h, q > 1, s);
      }
      CUDA_TRY(h, cudaGetLastError());
    }
  }
  A.traj_used = true;
  h->opt.tol_lin = tol_saved;
  h->assembled = h->decoupled = h->prec_built = false;
  if (result == ISC_OK) result = check_device_status(h);
  // leave the handle at the final state of the time loop
  int st2 = load_accepted(fin);
  if (result) return info->status = result;
  if (st2) return info->status = st2;
  if (g_log_k) CUDA_TRY(h, cudaMemcpyAsync(g_log_k, A.glnk, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (nr > 0) {
    launch_row_sums(2 * nr, n, A.grx, A.sums + 1, s);
    double sums[2 * ISC_MAX_RXN];
    CUDA_TRY(h, cudaMemcpyAsync(sums, A.sums + 1, sizeof(double) * 2 * nr, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    for (int r = 0; r < nr; ++r) {
      if (g_lnA) g_lnA[r] = sums[r];
      if (g_Ea) g_Ea[r] = sums[nr + r];
    }
  }
  CUDA_TRY(h, cudaStreamSynchronize(s));
  return ISC_OK;
}

extern "C" {

void isc_default_options(isc_options* o) {
  memset(o, 0, sizeof(*o));
  o->krylov = ISC_KRYLOV_GMRES;
  o->restart = 30;
  o->prec = ISC_PREC_BILU0;
  o->decouple = 1;
  o->tol_lin = 1e-6;
  o->maxit_lin = 600;
  o->tol_newton = 1e-6;
  o->maxit_newton = 25;
  o->max_dp_frac = 0.2;
  o->max_dT = 50.0;
  o->profile = 0;
  o->precision = ISC_PRECISION_FP64;
  o->stream = nullptr;
  o->inner_its = 10;
  o->orth = ISC_ORTH_CGS2;
}

const char* isc_status_string(int st) {
  switch (st) {
    case ISC_OK: return "ok";
    case ISC_ERR_INVALID_ARG: return "invalid argument";
    case ISC_ERR_CUDA: return "CUDA error";
    case ISC_ERR_NOMEM: return "out of device memory";
    case ISC_ERR_SINGULAR_BLOCK: return "singular diagonal block";
    case ISC_ERR_KRYLOV_NOCONV: return "Krylov solver did not converge";
    case ISC_ERR_NEWTON_NOCONV: return "Newton did not converge";
    case ISC_ERR_NONFINITE: return "non-finite value";
    case ISC_ERR_COKE: return "coke equation did not converge";
    case ISC_ERR_TIMEOUT: return "device wait timed out";
    case ISC_ERR_UNIMPLEMENTED: return "not implemented";
    case ISC_ERR_STATE: return "call order violated";
    default: return "unknown status";
  }
}

const char* isc_last_error(const isc_handle* h) { return h ? h->last_error.c_str() : "null handle"; }
int32_t isc_num_cells(const isc_handle* h) { return h ? h->n : 0; }
int32_t isc_nnzb(const isc_handle* h) { return h ? h->nnzb : 0; }

int isc_create(const isc_grid* grid, const isc_rock* rock, const isc_fluid* fl, const isc_reactions* rx,
               const isc_wells* wells, const isc_options* opts, isc_handle** out) {
  if (!out) return ISC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grid || !rock || !fl || !rx || !wells) return ISC_ERR_INVALID_ARG;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0))
    return ISC_ERR_INVALID_ARG;
  long long nll = (long long)grid->nx * grid->ny * grid->nz;
  if (nll * 7 * 64 > (long long)INT32_MAX * 64LL || nll > (1LL << 28)) return ISC_ERR_INVALID_ARG;
  if (!rock->phi_ref || !rock->perm) return ISC_ERR_INVALID_ARG;
  if (rx->nr < 0 || rx->nr > ISC_MAX_RXN) return ISC_ERR_INVALID_ARG;
  isc_handle* h = new (std::nothrow) isc_handle();
  if (!h) return ISC_ERR_NOMEM;
  isc_options o;
  if (opts)
    o = *opts;
  else
    isc_default_options(&o);
  int st = validate_options(h, o);
  if (st) {
    delete h;
    return st;
  }
  h->opt = o;
  h->stream = (cudaStream_t)o.stream;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz, n = (int)nll;
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->n = n;
  // N M = 0 check of every reaction (Sec. 2.1)
  double Mfull[7];
  for (int c = 0; c < 6; ++c) Mfull[c] = fl->M[c];
  Mfull[6] = fl->coke_M;
  for (int r = 0; r < rx->nr; ++r) {
    double s = 0, a = 0;
    for (int c = 0; c < 7; ++c) {
      s += rx->stoich[r][c] * Mfull[c];
      a += fabs(rx->stoich[r][c]) * Mfull[c];
    }
    if (fabs(s) > 1e-12 * a) {
      int e = set_err(h, ISC_ERR_INVALID_ARG, "reaction " + std::to_string(r) + " violates N M = 0");
      *out = nullptr;
      delete h;
      return e;
    }
    if (rx->kind[r] < 0 || rx->kind[r] > 2 || (rx->kind[r] != ISC_RXN_COKE_OXIDATION && rx->comp[r] != 1 && rx->comp[r] != 2)) {
      delete h;
      return ISC_ERR_INVALID_ARG;
    }
  }
  // parameters
  Params& P = h->P;
  P.nx = nx;
  P.ny = ny;
  P.nz = nz;
  P.n = n;
  P.V = grid->dx * grid->dy * grid->dz;
  P.gx = grid->dy * grid->dz / grid->dx;
  P.gy = grid->dx * grid->dz / grid->dy;
  P.gz = grid->dx * grid->dy / grid->dz;
  for (int c = 0; c < 6; ++c) {
    P.M[c] = fl->M[c];
    P.a_rk[c] = pow(fl->Tc[c], 1.25) / sqrt(fl->pc[c]);
    P.b_rk[c] = fl->Tc[c] / fl->pc[c];
    P.sqM[c] = sqrt(fl->M[c]);
    P.avg[c] = fl->avg[c];
    P.bvg[c] = fl->bvg[c];
    for (int k = 0; k < 4; ++k) P.cpg[c][k] = fl->cpg[c][k];
  }
  for (int c = 0; c < 3; ++c) {
    P.rho_ref[c] = fl->rho_ref[c];
    P.cp[c] = fl->cp[c];
    P.ct1[c] = fl->ct1[c];
    P.ct2[c] = fl->ct2[c];
    P.cpt[c] = fl->cpt[c];
    P.hvr[c] = fl->hvr[c];
    P.ev[c] = fl->ev[c];
    P.Tc[c] = fl->Tc[c];
    P.ln_avisc[c] = log(fl->avisc[c]);
    P.bvisc[c] = fl->bvisc[c];
    for (int k = 0; k < 5; ++k) P.kv[c][k] = fl->kv[c][k];
    P.K_phase[c] = fl->K_phase[c];
  }
  P.p_ref = fl->p_ref;
  P.T_ref = fl->T_ref;
  P.coke_rho = fl->coke_rho;
  P.coke_cp = fl->coke_cp;
  P.coke_K = fl->coke_K;
  P.Swc = fl->Swc;
  P.Sorw = fl->Sorw;
  P.Sgc = fl->Sgc;
  P.Sorg = fl->Sorg;
  P.per_eps = fl->per_eps;
  P.gravity = fl->gravity;
  P.cpor = rock->cpor;
  P.ctpor = rock->ctpor;
  P.cptpor = rock->cptpor;
  P.rock_p_ref = rock->p_ref;
  P.rock_T_ref = rock->T_ref;
  P.cv1 = rock->cv1;
  P.cv2 = rock->cv2;
  P.K_rock = rock->K_rock;
  P.cv_scale = rock->cv1;
  P.nr = rx->nr;
  for (int r = 0; r < rx->nr; ++r) {
    P.kind[r] = rx->kind[r];
    P.comp[r] = rx->comp[r];
    for (int c = 0; c < 7; ++c) P.stoich[r][c] = rx->stoich[r][c];
    P.A[r] = rx->A[r];
    P.EaR[r] = rx->Ea[r] / R_GAS;
    P.dH[r] = rx->dH[r];
  }
  P.coke_max = rx->coke_max;
  // BSR pattern of the 7-point stencil (columns sorted) and hyperplane levels
  h->h_rowptr.resize(n + 1);
  h->h_col.reserve((size_t)n * 7);
  h->h_rowptr[0] = 0;
  for (int c = 0; c < n; ++c) {
    int ix = c % nx, iy = (c / nx) % ny, iz = c / (nx * ny);
    if (iz > 0) h->h_col.push_back(c - nx * ny);
    if (iy > 0) h->h_col.push_back(c - nx);
    if (ix > 0) h->h_col.push_back(c - 1);
    h->h_col.push_back(c);
    if (ix < nx - 1) h->h_col.push_back(c + 1);
    if (iy < ny - 1) h->h_col.push_back(c + nx);
    if (iz < nz - 1) h->h_col.push_back(c + nx * ny);
    h->h_rowptr[c + 1] = (int32_t)h->h_col.size();
  }
  h->nnzb = (int)h->h_col.size();
  h->nlevels = nx + ny + nz - 2;
  std::vector<int32_t> level_cells(n);
  h->h_level_ptr.assign(h->nlevels + 1, 0);
  for (int c = 0; c < n; ++c) {
    int L = c % nx + (c / nx) % ny + c / (nx * ny);
    h->h_level_ptr[L + 1]++;
  }
  for (int L = 0; L < h->nlevels; ++L) h->h_level_ptr[L + 1] += h->h_level_ptr[L];
  {
    std::vector<int32_t> fill(h->h_level_ptr.begin(), h->h_level_ptr.end() - 1);
    for (int c = 0; c < n; ++c) {
      int L = c % nx + (c / nx) % ny + c / (nx * ny);
      level_cells[fill[L]++] = c;
    }
  }
  // permeabilities and depths (the transmissibilities follow from the ln k
  // multipliers, all zero at creation, in refresh_parameters)
  const double* kx = rock->perm;
  const double* ky = rock->perm + n;
  const double* kz = rock->perm + 2 * (size_t)n;
  std::vector<double> depth(n);
  for (int c = 0; c < n; ++c) {
    int iz = c / (nx * ny);
    depth[c] = grid->depth ? grid->depth[c] : (iz + 0.5) * grid->dz;
    if (!(rock->phi_ref[c] > 0.0) || !(kx[c] > 0) || !(ky[c] > 0) || !(kz[c] > 0)) {
      delete h;
      return ISC_ERR_INVALID_ARG;
    }
  }
  h->h_perm0.assign(rock->perm, rock->perm + 3 * (size_t)n);
  h->h_lnk.assign(n, 0.0);
  h->face_area[0] = grid->dy * grid->dz / grid->dx;
  h->face_area[1] = grid->dx * grid->dz / grid->dy;
  h->face_area[2] = grid->dx * grid->dy / grid->dz;
  h->area_xy = grid->dx * grid->dy;
  for (int r = 0; r < rx->nr; ++r) {
    h->h_Ea[r] = rx->Ea[r];
    h->h_lnA[r] = log(rx->A[r]);
  }
  // well slots
  std::vector<int32_t> well_slot(n, -1);
  std::vector<int32_t> inj_first, inj_count;
  std::vector<CoupledWell> coupled;
  for (int w = 0; w < wells->nw; ++w) {
    const isc_well& W = wells->wells[w];
    if (W.n_perf < 1 || !W.cells || !W.WI || W.kind < ISC_WELL_RATE_INJECTOR || W.kind > ISC_WELL_COUPLED_INJECTOR) {
      delete h;
      return ISC_ERR_INVALID_ARG;
    }
    const bool is_coupled = W.kind == ISC_WELL_COUPLED_PRODUCER || W.kind == ISC_WELL_COUPLED_INJECTOR;
    const bool injects = W.kind == ISC_WELL_RATE_INJECTOR || W.kind == ISC_WELL_COUPLED_INJECTOR;
    if (is_coupled) {
      const int ctl = W.control;
      // a coupled injector fixes its bottom-hole pressure or its total injected rate
      const bool ctl_ok = W.kind == ISC_WELL_COUPLED_PRODUCER ? (ctl >= ISC_CTRL_BHP && ctl <= ISC_CTRL_TOTAL_RATE)
                                                              : (ctl == ISC_CTRL_BHP || ctl == ISC_CTRL_TOTAL_RATE);
      const bool ok = ctl_ok && W.target == W.target && W.target != 0.0 && W.bhp_init > 0.0;
      if (!ok) {
        delete h;
        return ISC_ERR_INVALID_ARG;
      }
      CoupledWell cw{};
      cw.control = ctl;
      cw.first = (int)h->h_slots.size();
      cw.count = W.n_perf;
      cw.target = W.target;
      coupled.push_back(cw);
      h->h_bhp_init.push_back(W.bhp_init);
    }
    WellInfo info{};
    info.kind = W.kind;
    info.first = (int)h->h_slots.size();
    info.count = W.n_perf;
    info.target = W.target;
    for (int c = 0; c < 6; ++c) info.inj_y[c] = W.inj_y[c];
    if (injects) {
      // molar enthalpy of the injected stream at T_inj
      double T = W.inj_T, Tr = fl->T_ref, Hinj = 0.0;
      for (int c = 0; c < 6; ++c) {
        double hg = 0, tk = T, trk = Tr;
        for (int k = 0; k < 4; ++k) {
          hg += fl->cpg[c][k] / (k + 1) * (tk - trk);
          tk *= T;
          trk *= Tr;
        }
        if (W.inj_phase == 0) {
          if (c == 0) {
            double hv = (fl->Tc[0] > T) ? fl->hvr[0] * pow(fl->Tc[0] - T, fl->ev[0]) : 0.0;
            Hinj += W.inj_y[0] * (hg - hv);
          }
        } else {
          Hinj += W.inj_y[c] * hg;
        }
      }
      info.Hinj = Hinj;
      if (W.kind == ISC_WELL_RATE_INJECTOR) {
        inj_first.push_back(info.first);
        inj_count.push_back(info.count);
      }
    }
    for (int q = 0; q < W.n_perf; ++q) {
      int c = W.cells[q];
      if (c < 0 || c >= n || well_slot[c] >= 0) {
        delete h;
        return ISC_ERR_INVALID_ARG;
      }
      WellSlot sl{};
      sl.kind = W.kind;
      sl.cell = c;
      sl.bhp = W.target;
      sl.wc = is_coupled ? (int)coupled.size() - 1 : -1;
      sl.control = W.control;
      sl.zref = W.ref_depth;
      sl.phase = W.inj_phase == 0 ? 0 : 2;
      well_slot[c] = (int32_t)h->h_slots.size();
      h->h_slots.push_back(sl);
      h->h_WI0.push_back(W.WI[q]);
    }
    h->h_wells.push_back(info);
  }
  h->nslots = (int)h->h_slots.size();
  h->adj.n_inj = (int)inj_first.size();
  h->nwc = (int)coupled.size();
  // device memory; Krylov vectors hold the cells' 8N unknowns and the coupled wells' bottom-hole pressures
  h->restart_alloc = std::max(o.restart, 8);
  h->vlen = n * 8 + h->nwc;
  // vectors start on 64-byte boundaries (the sweeps and SpMV use 16-byte vector accesses)
  h->vstride = (h->vlen + 7) / 8 * 8;
  const size_t len = (size_t)h->vstride;
  h->red_blocks = 304;
  int e = 0;
  e |= dalloc(h, &h->rowptr, n + 1);
  e |= dalloc(h, &h->col, h->nnzb);
  e |= dalloc(h, &h->level_cells, n);
  e |= dalloc(h, &h->phi_ref, n);
  e |= dalloc(h, &h->depth, n);
  e |= dalloc(h, &h->tx, n);
  e |= dalloc(h, &h->ty, n);
  e |= dalloc(h, &h->tz, n);
  e |= dalloc(h, &h->wx, n);
  e |= dalloc(h, &h->wy, n);
  e |= dalloc(h, &h->wz, n);
  e |= dalloc(h, &h->adj.inj_first, std::max(h->adj.n_inj, 1));
  e |= dalloc(h, &h->adj.inj_count, std::max(h->adj.n_inj, 1));
  e |= dalloc(h, &h->well_slot, n);
  e |= dalloc(h, &h->slots, std::max(h->nslots, 1));
  e |= dalloc(h, &h->cw, std::max(h->nwc, 1));
  e |= dalloc(h, &h->bhp, std::max(h->nwc, 1));
  e |= dalloc(h, &h->bhp_n, std::max(h->nwc, 1));
  e |= dalloc(h, &h->Dw, std::max(h->nwc, 1));
  e |= dalloc(h, &h->Bv, (size_t)std::max(h->nslots, 1) * 8);
  e |= dalloc(h, &h->Cv, (size_t)std::max(h->nslots, 1) * 8);
  e |= dalloc(h, &h->Fq, std::max(h->nslots, 1));
  e |= dalloc(h, &h->Dq, std::max(h->nslots, 1));
  e |= dalloc(h, &h->u, (size_t)n * 8);
  e |= dalloc(h, &h->coke, n);
  e |= dalloc(h, &h->u_n, (size_t)n * 8);
  e |= dalloc(h, &h->coke_n, n);
  e |= dalloc(h, &h->acc_n, (size_t)n * 7);
  e |= dalloc(h, &h->props, (size_t)n * NQD);
  e |= dalloc(h, &h->fbuf, (size_t)n * 3 * 7);
  e |= dalloc(h, &h->R, len);
  e |= dalloc(h, &h->J, (size_t)h->nnzb * BB);
  e |= dalloc(h, &h->ntot, n);
  e |= dalloc(h, &h->du, len);
  e |= dalloc(h, &h->rhs, len);
  e |= dalloc(h, &h->dinv, (size_t)n * BB);
  e |= dalloc(h, &h->uhat, (size_t)n * 3 * BB);
  e |= dalloc(h, &h->V, (size_t)(h->restart_alloc + 1) * len);
  e |= dalloc(h, &h->Z, (size_t)h->restart_alloc * len);
  e |= dalloc(h, &h->w, len);
  e |= dalloc(h, &h->tmp, len);
  e |= dalloc(h, &h->partial, (size_t)h->red_blocks * (MAX_RESTART + 8));
  e |= dalloc(h, &h->scal, NSCAL);
  e |= dalloc(h, &h->dstatus, 1);
  e |= dalloc(h, &h->pipe, 2);
  e |= dalloc(h, &h->red_counter, 1);
  e |= dalloc(h, &h->gmres, GMRES_STATE);
  if (e) {
    std::string msg = h->last_error;
    free_all(h);
    delete h;
    return ISC_ERR_NOMEM;
  }
  if (cudaMallocHost((void**)&h->h_scal, sizeof(double) * NSCAL) != cudaSuccess ||
      cudaMallocHost((void**)&h->h_status, sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&h->h_ring, sizeof(double) * 6) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->gm_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->gm_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    free_all(h);
    delete h;
    return ISC_ERR_NOMEM;
  }
  cudaStream_t s = h->stream;
  cudaMemcpyAsync(h->rowptr, h->h_rowptr.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->col, h->h_col.data(), sizeof(int32_t) * h->nnzb, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->level_cells, level_cells.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->phi_ref, rock->phi_ref, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->depth, depth.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->well_slot, well_slot.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
  if (h->nwc) {
    cudaMemcpyAsync(h->cw, coupled.data(), sizeof(CoupledWell) * h->nwc, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->bhp, h->h_bhp_init.data(), sizeof(double) * h->nwc, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->bhp_n, h->h_bhp_init.data(), sizeof(double) * h->nwc, cudaMemcpyHostToDevice, s);
  }
  cudaMemsetAsync(h->Bv, 0, sizeof(double) * std::max(h->nslots, 1) * 8, s);
  cudaMemsetAsync(h->Cv, 0, sizeof(double) * std::max(h->nslots, 1) * 8, s);
  if (h->adj.n_inj) {
    cudaMemcpyAsync(h->adj.inj_first, inj_first.data(), sizeof(int32_t) * h->adj.n_inj, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->adj.inj_count, inj_count.data(), sizeof(int32_t) * h->adj.n_inj, cudaMemcpyHostToDevice, s);
  }
  if (refresh_parameters(h) != ISC_OK) {
    free_all(h);
    delete h;
    return ISC_ERR_CUDA;
  }
  cudaMemsetAsync(h->dstatus, 0, sizeof(int), s);
  cudaMemsetAsync(h->red_counter, 0, sizeof(unsigned), s);
  cudaMemsetAsync(h->u, 0, sizeof(double) * (size_t)n * 8, s);
  cudaMemsetAsync(h->coke, 0, sizeof(double) * n, s);
  cudaMemsetAsync(h->coke_n, 0, sizeof(double) * n, s);
  cudaError_t ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    free_all(h);
    delete h;
    return ISC_ERR_CUDA;
  }
  *out = h;
  return ISC_OK;
}

void isc_destroy(isc_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

int isc_set_options(isc_handle* h, const isc_options* o) {
  if (!h || !o) return ISC_ERR_INVALID_ARG;
  int st = validate_options(h, *o);
  if (st) return st;
  if (o->restart > h->restart_alloc) return set_err(h, ISC_ERR_INVALID_ARG, "restart larger than at creation");
  if ((cudaStream_t)o->stream != h->stream) cudaStreamSynchronize(h->stream);
  h->opt = *o;
  h->stream = (cudaStream_t)o->stream;
  h->prec_built = false;
  h->adj.ready = false;  // a reverse sweep recomputes states with the options of its forward sweep
  return ISC_OK;
}

int isc_init_equilibrium(isc_handle* h, double p0, double T0, double Sw0, double So0, double x_LO0,
                         const double y_rest[3], int32_t n_ignited, const int32_t* ignited, double T_ignite) {
  if (!h || !y_rest || n_ignited < 0 || (n_ignited > 0 && !ignited)) return ISC_ERR_INVALID_ARG;
  launch_init_equilibrium(*h, p0, T0, Sw0, So0, x_LO0, y_rest, h->stream);
  if (h->nwc)
    CUDA_TRY(h, cudaMemcpyAsync(h->bhp, h->h_bhp_init.data(), sizeof(double) * h->nwc, cudaMemcpyHostToDevice,
                                h->stream));
  for (int q = 0; q < n_ignited; ++q) {
    int c = ignited[q];
    if (c < 0 || c >= h->n) return set_err(h, ISC_ERR_INVALID_ARG, "ignited cell out of range");
    CUDA_TRY(h, cudaMemcpyAsync(h->u + (size_t)5 * h->n + c, &T_ignite, sizeof(double), cudaMemcpyHostToDevice,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return isc_begin_step(h);
}

int isc_set_state(isc_handle* h, const double* u, const double* coke) {
  if (!h || !u) return ISC_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(h->u, u, sizeof(double) * 8 * h->n, cudaMemcpyHostToDevice, h->stream));
  if (coke) CUDA_TRY(h, cudaMemcpyAsync(h->coke, coke, sizeof(double) * h->n, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->assembled = h->decoupled = h->prec_built = false;
  return ISC_OK;
}

int isc_get_state(isc_handle* h, double* u, double* coke) {
  if (!h || !u) return ISC_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(u, h->u, sizeof(double) * 8 * h->n, cudaMemcpyDeviceToHost, h->stream));
  if (coke) CUDA_TRY(h, cudaMemcpyAsync(coke, h->coke, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ISC_OK;
}

int isc_set_state_device(isc_handle* h, const double* d_u, const double* d_coke) {
  if (!h || !d_u) return ISC_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(h->u, d_u, sizeof(double) * 8 * h->n, cudaMemcpyDeviceToDevice, h->stream));
  if (d_coke) CUDA_TRY(h, cudaMemcpyAsync(h->coke, d_coke, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  h->assembled = h->decoupled = h->prec_built = false;
  return ISC_OK;
}

int isc_get_state_device(isc_handle* h, double* d_u, double* d_coke) {
  if (!h || !d_u) return ISC_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(d_u, h->u, sizeof(double) * 8 * h->n, cudaMemcpyDeviceToDevice, h->stream));
  if (d_coke) CUDA_TRY(h, cudaMemcpyAsync(d_coke, h->coke, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  return ISC_OK;
}

int isc_begin_step(isc_handle* h) {
  if (!h) return ISC_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(h->u_n, h->u, sizeof(double) * 8 * h->n, cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->coke_n, h->coke, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  if (h->nwc)
    CUDA_TRY(h, cudaMemcpyAsync(h->bhp_n, h->bhp, sizeof(double) * h->nwc, cudaMemcpyDeviceToDevice, h->stream));
  launch_old_accumulation(*h, h->stream);
  CUDA_TRY(h, cudaGetLastError());
  h->have_acc = true;
  return ISC_OK;
}

int isc_assemble(isc_handle* h, double dt) {
  if (!h || !(dt > 0.0)) return ISC_ERR_INVALID_ARG;
  if (!h->have_acc) return set_err(h, ISC_ERR_STATE, "isc_begin_step (or isc_init_equilibrium) must come first");
  h->P.dt = dt;
  h->P.inv_dt = 1.0 / dt;
  {
    Region rg(h, ISC_K_PROPS, 1);
    launch_props(*h, h->stream);
  }
  {
    Region rg(h, ISC_K_FLUX, 2);  // face pass and gather
    launch_flux(*h, h->stream);
  }
  if (h->nwc) {
    Region rg(h, ISC_K_PROPS, 1);
    launch_well_equations(*h, h->stream);
  }
  CUDA_TRY(h, cudaGetLastError());
  h->assembled = true;
  h->decoupled = false;
  h->prec_built = false;
  h->last_dt = dt;
  return ISC_OK;
}

int isc_decouple(isc_handle* h) {
  if (!h) return ISC_ERR_INVALID_ARG;
  if (!h->assembled) return set_err(h, ISC_ERR_STATE, "assemble first");
  if (h->decoupled) return ISC_OK;
  {
    Region rg(h, ISC_K_GJ, 1);
    launch_gj(*h, h->stream);
  }
  CUDA_TRY(h, cudaGetLastError());
  int st = check_device_status(h);
  if (st) return st;
  h->decoupled = true;
  h->prec_built = false;
  return ISC_OK;
}

int isc_build_preconditioner(isc_handle* h) {
  if (!h) return ISC_ERR_INVALID_ARG;
  if (!h->assembled) return set_err(h, ISC_ERR_STATE, "assemble first");
  return build_prec(h);
}

int isc_solve(isc_handle* h, isc_newton_info* info) {
  if (!h) return ISC_ERR_INVALID_ARG;
  if (!h->assembled) return set_err(h, ISC_ERR_STATE, "assemble first");
  int st = ISC_OK;
  if (!h->prec_built) {
    st = build_prec(h);
    if (st) return st;
  }
  const int len = h->vlen;
  {
    Region rg(h, ISC_K_BLAS1, 1);
    launch_scale_copy(len, -1.0, h->R, h->rhs, h->stream);
  }
  int its = 0;
  double rel = 0.0;
  if (h->opt.krylov == ISC_KRYLOV_GMRES)
    st = gmres(h, h->rhs, h->du, &its, &rel);
  else
    st = bicgstab(h, h->rhs, h->du, &its, &rel);
  if (info) {
    info->krylov_iterations = its;
    info->krylov_rel_residual = rel;
    info->status = st;
  }
  CUDA_TRY(h, cudaGetLastError());
  return st;
}

int isc_update(isc_handle* h) {
  if (!h) return ISC_ERR_INVALID_ARG;
  {
    Region rg(h, ISC_K_UPDATE, h->nwc ? 2 : 1);
    launch_update(*h, h->stream);
    launch_well_update(*h, h->stream);
  }
  CUDA_TRY(h, cudaGetLastError());
  h->assembled = h->decoupled = h->prec_built = false;
  return ISC_OK;
}

int isc_newton_step(isc_handle* h, double dt, isc_newton_info* info) {
  if (!h) return ISC_ERR_INVALID_ARG;
  isc_newton_info loc{};
  if (!info) info = &loc;
  memset(info, 0, sizeof(*info));
  int st = isc_assemble(h, dt);
  if (st) return st;
  {
    Region rg(h, ISC_K_NORM, 2);
    launch_norms(*h, h->stream);
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->h_scal + S_NORM, h->scal + S_NORM, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
  st = check_device_status(h);  // synchronises
  if (st) {
    info->status = st;
    return st;
  }
  info->norm_mass = h->h_scal[S_NORM] * dt;
  info->norm_energy = h->h_scal[S_NORM + 1] * dt;
  info->norm_gs = h->h_scal[S_NORM + 2];
  info->norm = std::max(info->norm_mass, std::max(info->norm_energy, info->norm_gs));
  if (h->nwc) info->norm = std::max(info->norm, h->h_scal[S_NORM + 3]);  // coupled wells: max |F_w| / |target|
  if (!isfinite(info->norm)) {
    info->status = ISC_ERR_NONFINITE;
    return set_err(h, ISC_ERR_NONFINITE, "non-finite residual norm");
  }
  if (info->norm <= h->opt.tol_newton) {
    info->converged = 1;
    return ISC_OK;
  }
  if (h->opt.decouple) {
    st = isc_decouple(h);
    if (st) {
      info->status = st;
      return st;
    }
  }
  st = isc_solve(h, info);
  if (st) {
    info->status = st;
    return st;
  }
  st = isc_update(h);
  info->status = st;
  return st;
}

int isc_timestep(isc_handle* h, double dt, isc_step_info* info) {
  if (!h || !(dt > 0.0)) return ISC_ERR_INVALID_ARG;
  isc_step_info loc{};
  if (!info) info = &loc;
  memset(info, 0, sizeof(*info));
  if (!h->have_acc) return set_err(h, ISC_ERR_STATE, "isc_begin_step (or isc_init_equilibrium) must come first");
  int st = ISC_OK;
  bool conv = false;
  for (int it = 0; it <= h->opt.maxit_newton; ++it) {
    isc_newton_info ni;
    st = isc_newton_step(h, dt, &ni);
    info->final_norm = ni.norm;
    if (st) break;
    if (ni.converged) {
      conv = true;
      break;
    }
    info->newton_iterations++;
    info->krylov_iterations += ni.krylov_iterations;
  }
  if (conv) {
    st = isc_begin_step(h);
    info->status = st;
    return st;
  }
  // restore the accepted state
  cudaMemcpyAsync(h->u, h->u_n, sizeof(double) * 8 * h->n, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(h->coke, h->coke_n, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->stream);
  if (h->nwc) cudaMemcpyAsync(h->bhp, h->bhp_n, sizeof(double) * h->nwc, cudaMemcpyDeviceToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  h->assembled = h->decoupled = h->prec_built = false;
  if (st == ISC_OK) st = set_err(h, ISC_ERR_NEWTON_NOCONV, "Newton did not converge within maxit_newton");
  info->status = st;
  return st;
}

namespace {
// failures of a time step that a shorter step can cure (the state is restored)
bool cut_cures(int st) {
  return st == ISC_ERR_NEWTON_NOCONV || st == ISC_ERR_KRYLOV_NOCONV || st == ISC_ERR_NONFINITE ||
         st == ISC_ERR_COKE || st == ISC_ERR_SINGULAR_BLOCK;
}
}  // namespace

int isc_run(isc_handle* h, double t_end, double dt0, double dt_max, double dT_target, double dS_target,
            int32_t max_cuts, int32_t max_steps, double* dt_history, isc_run_info* info) {
  if (!h || !(t_end >= 0.0) || !isfinite(t_end) || !(dt0 > 0.0) || !isfinite(dt0) || !(dt_max > 0.0) ||
      !(dT_target > 0.0) || !(dS_target > 0.0) || max_cuts < 0 || max_steps < 1)
    return ISC_ERR_INVALID_ARG;
  isc_run_info loc{};
  if (!info) info = &loc;
  memset(info, 0, sizeof(*info));
  if (!h->have_acc) return set_err(h, ISC_ERR_STATE, "isc_begin_step (or isc_init_equilibrium) must come first");
  const int n = h->n;
  if (!h->u_prev) {
    int e = dalloc(h, &h->u_prev, (size_t)3 * n);
    e |= dalloc(h, &h->run_max, 2);
    if (e) return ISC_ERR_NOMEM;
  }
  cudaStream_t s = h->stream;
  double t = 0.0, dt = dt0;
  while (t < t_end * (1.0 - 1e-12) && info->steps < max_steps) {
    dt = std::min(dt, t_end - t);
    // T, S_w, S_g of the accepted state (rows 5..7 of the SoA state, contiguous)
    CUDA_TRY(h, cudaMemcpyAsync(h->u_prev, h->u_n + (size_t)5 * n, sizeof(double) * 3 * n,
                                cudaMemcpyDeviceToDevice, s));
    int st = ISC_OK;
    for (int c = 0;; ++c) {
      isc_step_info si{};
      st = isc_timestep(h, dt, &si);  // on failure the accepted state is restored
      info->newton_iterations += si.newton_iterations;
      info->krylov_iterations += si.krylov_iterations;
      if (st == ISC_OK || !cut_cures(st) || c == max_cuts) break;
      info->cuts++;
      dt *= 0.5;
    }
    if (st != ISC_OK) {
      info->status = st;
      info->t = t;
      info->dt_next = dt;
      if (cut_cures(st))
        set_err(h, st, "time step at t = " + std::to_string(t) + " s failed after " + std::to_string(max_cuts) +
                           " halvings: " + h->last_error);
      return st;
    }
    // the controller: the largest changes of T and of S_w, S_g over the accepted step
    CUDA_TRY(h, cudaMemsetAsync(h->run_max, 0, 2 * sizeof(unsigned long long), s));
    launch_max_change(n, h->u + (size_t)5 * n, h->u_prev, h->run_max, s);
    CUDA_TRY(h, cudaGetLastError());
    unsigned long long mx[2];
    CUDA_TRY(h, cudaMemcpyAsync(mx, h->run_max, sizeof(mx), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    double dT, dS;
    memcpy(&dT, &mx[0], sizeof(double));
    memcpy(&dS, &mx[1], sizeof(double));
    if (dt_history) dt_history[info->steps] = dt;
    info->steps++;
    t += dt;
    const double f = std::min(dT_target / std::max(dT, 1e-12), dS_target / std::max(dS, 1e-12));
    dt = std::min(dt * std::min(std::max(f, 0.5), 2.0), dt_max);
  }
  info->t = t;
  info->dt_next = dt;
  info->status = ISC_OK;
  return ISC_OK;
}

int isc_set_heat_loss(isc_handle* h, double K_ob, double d, double T_ini, double rho, int32_t faces) {
  if (!h || !(K_ob >= 0.0) || !(d > 0.0) || !(T_ini > 0.0) || !isfinite(K_ob) || !isfinite(d) || !isfinite(rho) ||
      faces < 0 || faces > 3)
    return ISC_ERR_INVALID_ARG;
  h->P.hl_AK = (faces == 0) ? 0.0 : h->area_xy * K_ob;
  h->P.hl_inv_d = 1.0 / d;
  h->P.hl_Tini = T_ini;
  h->P.hl_rho = rho;
  h->P.hl_faces = faces;
  h->adj.ready = false;  // the stored forward sweep no longer matches the model
  h->assembled = h->decoupled = h->prec_built = false;  // the next residual includes it
  return ISC_OK;
}

int isc_set_system(isc_handle* h, const double* val, const double* F, int32_t decoupled) {
  if (!h || !val || !F || (decoupled != 0 && decoupled != 1)) return ISC_ERR_INVALID_ARG;
  if (h->nwc)
    return set_err(h, ISC_ERR_UNIMPLEMENTED, "a caller's system cannot carry the coupled producers' border");
  if (decoupled) {
    // the unit-diagonal SpMV and the sweeps skip the diagonal blocks: they must be I exactly
    for (int i = 0; i < h->n; ++i)
      for (int b = h->h_rowptr[i]; b < h->h_rowptr[i + 1]; ++b)
        if (h->h_col[b] == i)
          for (int e = 0; e < BB; ++e)
            if (val[(size_t)b * BB + e] != ((e % 9 == 0) ? 1.0 : 0.0))
              return set_err(h, ISC_ERR_INVALID_ARG, "decoupled system: a diagonal block is not the identity");
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->J, val, sizeof(double) * BB * (size_t)h->nnzb, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->R, F, sizeof(double) * 8 * (size_t)h->n, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->assembled = true;
  h->decoupled = decoupled != 0;
  h->prec_built = false;
  return ISC_OK;
}

int isc_solve_external(isc_handle* h, const int32_t* rowptr, const int32_t* col, const double* val, const double* b,
                       double* x, isc_newton_info* info) {
  if (!h || !rowptr || !col || !val || !b || !x) return ISC_ERR_INVALID_ARG;
  if (memcmp(rowptr, h->h_rowptr.data(), sizeof(int32_t) * (h->n + 1)) != 0 ||
      memcmp(col, h->h_col.data(), sizeof(int32_t) * h->nnzb) != 0)
    return set_err(h, ISC_ERR_INVALID_ARG, "the matrix must have the handle's 7-point BSR pattern");
  std::vector<double> F((size_t)8 * h->n);
  for (size_t k = 0; k < F.size(); ++k) F[k] = -b[k];  // isc_solve solves J du = -F
  int st = isc_set_system(h, val, F.data(), 0);
  if (st) return st;
  if (h->opt.decouple) {
    st = isc_decouple(h);
    if (st) return st;
  }
  st = isc_solve(h, info);
  if (st) return st;
  return isc_get_update(h, x);
}

int isc_get_residual(isc_handle* h, double* F) {
  if (!h || !F) return ISC_ERR_INVALID_ARG;
  if (!h->assembled) return set_err(h, ISC_ERR_STATE, "assemble first");
  CUDA_TRY(h, cudaMemcpyAsync(F, h->R, sizeof(double) * 8 * h->n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ISC_OK;
}

int isc_get_jacobian_bsr(isc_handle* h, int32_t* rowptr, int32_t* col, double* val) {
  if (!h) return ISC_ERR_INVALID_ARG;
  if (rowptr) memcpy(rowptr, h->h_rowptr.data(), sizeof(int32_t) * (h->n + 1));
  if (col) memcpy(col, h->h_col.data(), sizeof(int32_t) * h->nnzb);
  if (val) {
    if (!h->assembled) return set_err(h, ISC_ERR_STATE, "assemble first");
    CUDA_TRY(h, cudaMemcpyAsync(val, h->J, sizeof(double) * BB * h->nnzb, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return ISC_OK;
}

int isc_get_update(isc_handle* h, double* du) {
  if (!h || !du) return ISC_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(du, h->du, sizeof(double) * 8 * h->n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ISC_OK;
}

int isc_get_coke(isc_handle* h, double* coke) {
  if (!h || !coke) return ISC_ERR_INVALID_ARG;
  CUDA_TRY(h, cudaMemcpyAsync(coke, h->coke, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ISC_OK;
}

int isc_spmv(isc_handle* h, const double* x, double* y) {
  if (!h || !x || !y) return ISC_ERR_INVALID_ARG;
  if (!h->assembled) return set_err(h, ISC_ERR_STATE, "assemble first");
  const size_t len = (size_t)h->vlen;
  CUDA_TRY(h, cudaMemcpyAsync(h->w, x, sizeof(double) * len, cudaMemcpyHostToDevice, h->stream));
  spmv(h, h->w, h->tmp);
  CUDA_TRY(h, cudaMemcpyAsync(y, h->tmp, sizeof(double) * len, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return ISC_OK;
}

int isc_check_reciprocal(int32_t n, const double* x, double* y, double* z) {
  if (n < 0 || (n > 0 && (!x || !y || !z))) return ISC_ERR_INVALID_ARG;
  if (n == 0) return ISC_OK;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 3 * (size_t)n) != cudaSuccess) return ISC_ERR_NOMEM;
  int st = ISC_OK;
  if (cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess) st = ISC_ERR_CUDA;
  if (st == ISC_OK) {
    launch_recip_check(n, d, d + n, d + 2 * (size_t)n, 0);
    if (cudaMemcpy(y, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(z, d + 2 * (size_t)n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      st = ISC_ERR_CUDA;
  }
  cudaFree(d);
  return st;
}

int isc_precond_apply(isc_handle* h, const double* r, double* z) {
  if (!h || !r || !z) return ISC_ERR_INVALID_ARG;
  if (!h->prec_built) return set_err(h, ISC_ERR_STATE, "build the preconditioner first");
  const size_t len = (size_t)h->vlen;
  CUDA_TRY(h, cudaMemcpyAsync(h->w, r, sizeof(double) * len, cudaMemcpyHostToDevice, h->stream));
  prec(h, h->w, h->V);
  CUDA_TRY(h, cudaMemcpyAsync(z, h->V, sizeof(double) * len, cudaMemcpyDeviceToHost, h->stream));
  return check_device_status(h);  // synchronises; reports a sweep whose bounded wait gave up
}

int isc_get_ilu_diag(isc_handle* h, double* dinv) {
  if (!h || !dinv) return ISC_ERR_INVALID_ARG;
  if (!h->prec_built || (h->opt.prec != ISC_PREC_BILU0 && h->opt.prec != ISC_PREC_CPR))
    return set_err(h, ISC_ERR_STATE, "build the block ILU(0) (or CPR-PF) preconditioner first");
  const size_t cnt = (size_t)h->n * BB;
  if (h->opt.precision == ISC_PRECISION_FP64) {
    CUDA_TRY(h, cudaMemcpyAsync(dinv, h->dinv, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return ISC_OK;
  }
  std::vector<float> f(cnt);
  CUDA_TRY(h, cudaMemcpyAsync(f.data(), h->dinv32, sizeof(float) * cnt, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (size_t k = 0; k < cnt; ++k) dinv[k] = (double)f[k];
  return ISC_OK;
}

int isc_get_stats(isc_handle* h, isc_stats* st) {
  if (!h || !st) return ISC_ERR_INVALID_ARG;
  resolve_timers(h);
  *st = h->stats;
  return ISC_OK;
}

int isc_get_device_bytes(isc_handle* h, uint64_t* bytes) {
  if (!h || !bytes) return ISC_ERR_INVALID_ARG;
  uint64_t t = h->cpr.bytes;
  for (const auto& kv : h->dev_sizes) t += kv.second;
  *bytes = t;
  return ISC_OK;
}

int isc_reset_stats(isc_handle* h) {
  if (!h) return ISC_ERR_INVALID_ARG;
  resolve_timers(h);
  memset(&h->stats, 0, sizeof(h->stats));
  return ISC_OK;
}

int isc_bsr_spmv_device(int32_t nrows, const int32_t* d_rowptr, const int32_t* d_col, const double* d_val,
                        const double* d_x, double* d_y, int32_t unit_diag, void* stream) {
  if (nrows < 0 || (nrows > 0 && (!d_rowptr || !d_col || !d_val || !d_x || !d_y))) return ISC_ERR_INVALID_ARG;
  if (nrows == 0) return ISC_OK;
  launch_spmv(nrows, d_rowptr, d_col, d_val, d_x, d_y, unit_diag, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? ISC_OK : ISC_ERR_CUDA;
}

int32_t isc_num_coupled_wells(const isc_handle* h) { return h ? h->nwc : 0; }

int isc_set_well_bhp(isc_handle* h, const double* bhp) {
  if (!h || (h->nwc && !bhp)) return ISC_ERR_INVALID_ARG;
  if (h->nwc) {
    CUDA_TRY(h, cudaMemcpyAsync(h->bhp, bhp, sizeof(double) * h->nwc, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  h->assembled = h->decoupled = h->prec_built = false;
  return ISC_OK;
}

int isc_get_well_bhp(isc_handle* h, double* bhp) {
  if (!h || (h->nwc && !bhp)) return ISC_ERR_INVALID_ARG;
  if (h->nwc) {
    CUDA_TRY(h, cudaMemcpyAsync(bhp, h->bhp, sizeof(double) * h->nwc, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return ISC_OK;
}

int isc_get_well_system(isc_handle* h, double* B, double* C, double* D, double* Fw) {
  if (!h) return ISC_ERR_INVALID_ARG;
  if (!h->assembled || h->decoupled) return set_err(h, ISC_ERR_STATE, "assemble first (and do not decouple)");
  if (h->nwc == 0) return ISC_OK;
  // the coupled wells' slots, in creation order
  std::vector<int> order;
  for (int q = 0; q < h->nslots; ++q)
    if (h->h_slots[q].wc >= 0) order.push_back(q);
  std::vector<double> bv((size_t)h->nslots * 8), cv((size_t)h->nslots * 8);
  CUDA_TRY(h, cudaMemcpyAsync(bv.data(), h->Bv, sizeof(double) * bv.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(cv.data(), h->Cv, sizeof(double) * cv.size(), cudaMemcpyDeviceToHost, h->stream));
  if (D) CUDA_TRY(h, cudaMemcpyAsync(D, h->Dw, sizeof(double) * h->nwc, cudaMemcpyDeviceToHost, h->stream));
  if (Fw)
    CUDA_TRY(h, cudaMemcpyAsync(Fw, h->R + (size_t)h->n * 8, sizeof(double) * h->nwc, cudaMemcpyDeviceToHost,
                                h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (size_t k = 0; k < order.size(); ++k) {
    if (B) memcpy(B + k * 8, bv.data() + (size_t)order[k] * 8, sizeof(double) * 8);
    if (C) memcpy(C + k * 8, cv.data() + (size_t)order[k] * 8, sizeof(double) * 8);
  }
  return ISC_OK;
}

int isc_set_parameters(isc_handle* h, const double* log_k, const double* Ea, const double* lnA) {
  if (!h) return ISC_ERR_INVALID_ARG;
  if (log_k) {
    for (int c = 0; c < h->n; ++c)
      if (!isfinite(log_k[c])) return set_err(h, ISC_ERR_INVALID_ARG, "non-finite ln k multiplier");
  }
  for (int r = 0; r < h->P.nr; ++r) {
    if (Ea && !isfinite(Ea[r])) return set_err(h, ISC_ERR_INVALID_ARG, "non-finite activation energy");
    if (lnA && !isfinite(lnA[r])) return set_err(h, ISC_ERR_INVALID_ARG, "non-finite ln A");
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (log_k) {
    h->h_lnk.assign(log_k, log_k + h->n);
    int st = refresh_parameters(h);
    if (st) return st;
  }
  for (int r = 0; r < h->P.nr; ++r) {
    if (Ea) {
      h->h_Ea[r] = Ea[r];
      h->P.EaR[r] = Ea[r] / R_GAS;
    }
    if (lnA) {
      h->h_lnA[r] = lnA[r];
      h->P.A[r] = exp(lnA[r]);
    }
  }
  h->assembled = h->decoupled = h->prec_built = false;
  h->adj.ready = false;  // the stored forward sweep belongs to the old parameters
  return ISC_OK;
}

int isc_get_parameters(isc_handle* h, double* log_k, double* Ea, double* lnA) {
  if (!h) return ISC_ERR_INVALID_ARG;
  if (log_k) memcpy(log_k, h->h_lnk.data(), sizeof(double) * h->n);
  for (int r = 0; r < h->P.nr; ++r) {
    if (Ea) Ea[r] = h->h_Ea[r];
    if (lnA) lnA[r] = h->h_lnA[r];
  }
  return ISC_OK;
}

int isc_adjoint(isc_handle* h, const isc_adjoint_spec* spec, double* loss, double* g_log_k, double* g_Ea,
                double* g_lnA, isc_adjoint_info* info) {
  if (!h || !spec) return ISC_ERR_INVALID_ARG;
  isc_adjoint_info loc{};
  if (!info) info = &loc;
  memset(info, 0, sizeof(*info));
  int st = adjoint_forward(h, spec, loss, info);
  if (st || !(g_log_k || g_Ea || g_lnA)) return st;
  return adjoint_backward(h, g_log_k, g_Ea, g_lnA, info);
}

int isc_adjoint_forward(isc_handle* h, const isc_adjoint_spec* spec, double* loss, isc_adjoint_info* info) {
  if (!h || !spec) return ISC_ERR_INVALID_ARG;
  isc_adjoint_info loc{};
  if (!info) info = &loc;
  memset(info, 0, sizeof(*info));
  return adjoint_forward(h, spec, loss, info);
}

int isc_adjoint_backward(isc_handle* h, double* g_log_k, double* g_Ea, double* g_lnA, isc_adjoint_info* info) {
  if (!h) return ISC_ERR_INVALID_ARG;
  isc_adjoint_info loc{};
  if (!info) info = &loc;
  memset(info, 0, sizeof(*info));
  return adjoint_backward(h, g_log_k, g_Ea, g_lnA, info);
}

}  // extern "C"
