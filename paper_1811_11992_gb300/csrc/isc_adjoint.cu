// Discrete adjoint of the implicit-Euler time loop (sensitivities of the
// cumulative produced oil mass). The paper computes no sensitivities; the
// kernels differentiate exactly the discrete equations of Sec. 3.1 that the
// assembly kernels evaluate.
//
// Per step n (reverse order), with lambda^n the multiplier of the residual
// F^n(u^n, u^{n-1}, C^{n-1}, theta) = 0 and C^n = Phi(u^n, C^{n-1}, theta)
// the per-cell coke solve:
//   ubar^n   += Phi_u^T Cbar^n + dt_n dP/du^n                   (k_adj_pre)
//   J_n^T lambda^n = ubar^n                                     (k_bsr_transpose + the Krylov solve)
//   gamma^n   = (dF^n/dC^n)^T lambda^n, kappa = Cbar^n - gamma  (k_adj_face, k_adj_local)
//   gbar     += -(dF^n/dtheta)^T lambda^n + Phi_theta^T kappa + dt_n dP/dtheta
//   ubar^{n-1} = (V/dt_n) (dacc/du^{n-1})^T lambda^n             (k_adj_old)
//   Cbar^{n-1} = (V/dt_n) (dacc/dC^{n-1})^T lambda^n + kappa / (dg/dC)
// theta = (ln k of every cell, through the harmonic transmissibilities and
// the well indices; E_a and ln A of every reaction).
#include <math.h>

#include "dual8.cuh"
#include "isc_internal.cuh"
#include "isc_props.cuh"

namespace isc {

namespace {

__device__ __forceinline__ int producer_slot(const int32_t* __restrict__ well_slot, const WellSlot* __restrict__ slots,
                                             int i, WellSlot* w) {
  int sl = well_slot[i];
  if (sl < 0) return 0;
  *w = slots[sl];
  return w->kind == ISC_WELL_BHP_PRODUCER;
}

// loss_cell[i] += dt * (oil mass rate produced in cell i) at the converged u^n
// (and, for a coupled producer's perforation, its converged bottom-hole pressure)
__global__ void __launch_bounds__(128) k_oil_rate(Params P, const double* __restrict__ u,
                                                  const double* __restrict__ phi_ref,
                                                  const int32_t* __restrict__ well_slot,
                                                  const WellSlot* __restrict__ slots, const double* __restrict__ bhp,
                                                  const double* __restrict__ depth, double dt,
                                                  double* __restrict__ loss_cell) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const int sl = well_slot[i];
  if (sl < 0) return;
  const WellSlot w = slots[sl];
  if (w.kind != ISC_WELL_BHP_PRODUCER && w.kind != ISC_WELL_COUPLED_PRODUCER) return;
  Base b;
  base_properties(P, u, i, phi_ref[i], b);
  if (w.kind == ISC_WELL_BHP_PRODUCER) {
    loss_cell[i] += dt * oil_production(P, b, w.WI, w.bhp).v;
  } else {
    D8 Q[3];
    double dQ[3];
    bool on[3];
    coupled_producer_rates(b, w.WI, bhp[w.wc], w.zref, depth[i], Q, dQ, on);
    loss_cell[i] += dt * oil_of_rates(P, b, Q).v;
  }
}

// ubar^n += Phi_u^T Cbar^n + dt dP/du;  glnk += dt P (the produced rate is linear in WI)
__global__ void __launch_bounds__(128) k_adj_pre(Params P, const double* __restrict__ u,
                                                 const double* __restrict__ coke_old,
                                                 const double* __restrict__ phi_ref,
                                                 const int32_t* __restrict__ well_slot,
                                                 const WellSlot* __restrict__ slots, const double* __restrict__ bhp,
                                                 const double* __restrict__ depth, const double* __restrict__ cbar,
                                                 double* __restrict__ ubar, double* __restrict__ glnk,
                                                 int* __restrict__ dstatus) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  Base b;
  base_properties(P, u, i, phi_ref[i], b);
  D8 kT[ISC_MAX_RXN];
  for (int r = 0; r < P.nr; ++r) kT[r] = P.A[r] * dexp(-P.EaR[r] * (1.0 / b.T));
  D8 C = solve_coke(P, b, kT, coke_old[i], dstatus);
  const double cb = cbar[i];
  double g[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) g[k] = cb * C.d[k];
  WellSlot w;
  if (producer_slot(well_slot, slots, i, &w)) {
    D8 q = oil_production(P, b, w.WI, w.bhp);
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] += P.dt * q.d[k];
    glnk[i] += P.dt * q.v;
  } else if (well_slot[i] >= 0 && w.kind == ISC_WELL_COUPLED_PRODUCER) {
    // the same with the converged bottom-hole pressure; its own derivative is k_adj_wells_pre's
    D8 Q[3];
    double dQ[3];
    bool on[3];
    coupled_producer_rates(b, w.WI, bhp[w.wc], w.zref, depth[i], Q, dQ, on);
    const D8 q = oil_of_rates(P, b, Q);
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] += P.dt * q.d[k];
    glnk[i] += P.dt * q.v;
  }
  double* ub = ubar + (size_t)i * 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) ub[k] += g[k];
}

// In-place block transpose of a BSR matrix with a symmetric pattern:
// block (i, j) <- block (j, i)^T. One warp per stored block; the warp of the
// block with j > i swaps it with its mirror, the diagonal warp transposes in
// place, the warps of blocks with j < i do nothing.
__global__ void __launch_bounds__(256) k_bsr_transpose(int n, const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ col, double* __restrict__ J) {
  const int warp = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);  // 32 nnzb may pass 2^32
  const int lane = threadIdx.x & 31;
  const int nnzb = rowptr[n];
  if (warp >= nnzb) return;
  // row of this block: rows hold at most 7 blocks, search from an estimate
  int lo = 0, hi = n;  // rowptr[lo] <= warp < rowptr[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (rowptr[mid] <= warp)
      lo = mid;
    else
      hi = mid;
  }
  const int i = lo;
  const int j = col[warp];
  double* A = J + (size_t)warp * BB;
  if (j == i) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int e = lane + 32 * h;
      int r = e >> 3, c = e & 7;
      if (r < c) {
        double a = A[r * 8 + c];
        double t = A[c * 8 + r];
        A[r * 8 + c] = t;
        A[c * 8 + r] = a;
      }
    }
    return;
  }
  if (j < i) return;
  int m = -1;
  for (int s = rowptr[j]; s < rowptr[j + 1]; ++s)
    if (col[s] == i) m = s;
  if (m < 0) return;  // pattern not symmetric: nothing to swap (cannot happen for the 7-point stencil)
  double* B = J + (size_t)m * BB;
  double a[2], t[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int e = lane + 32 * h;
    int r = e >> 3, c = e & 7;
    a[h] = A[r * 8 + c];
    t[h] = B[c * 8 + r];
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int e = lane + 32 * h;
    int r = e >> 3, c = e & 7;
    A[r * 8 + c] = t[h];
    B[c * 8 + r] = a[h];
  }
}

__device__ __forceinline__ double qv(const double* __restrict__ props, int n, int q, int cell) {
  return __ldg(props + (size_t)(q * 9) * n + cell);
}

// sum_r dl[r] * (advective flux of row r over face (lo, hi)), with the
// upstream decisions and arithmetic of the assembly's face flux.
__device__ double adv_flux_dot(const Params& P, int lo, int hi, double Tf, double dz, const double* __restrict__ u,
                               const double* __restrict__ props, const double* dl) {
  const int n = P.n;
  const double plo = __ldg(u + lo), phi_ = __ldg(u + hi);
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double glo = qv(props, n, Q_GAM + a, lo), ghi = qv(props, n, Q_GAM + a, hi);
    double gavg = __dmul_rn(0.5, __dadd_rn(glo, ghi));
    double dphi = __dsub_rn(__dsub_rn(plo, phi_), __dmul_rn(gavg, dz));
    int up = dphi >= 0.0 ? lo : hi;
    double c;
    if (a == 0) {
      c = dl[0] * qv(props, n, Q_LW, up) + dl[6] * qv(props, n, Q_LWH, up);
    } else if (a == 1) {
      c = dl[1] * qv(props, n, Q_LOX_LO, up) + dl[2] * qv(props, n, Q_LOX_HO, up) + dl[6] * qv(props, n, Q_LOH, up);
    } else {
      c = dl[6] * qv(props, n, Q_LGH, up);
#pragma unroll
      for (int k = 0; k < 6; ++k) c += dl[k] * qv(props, n, Q_LGY + k, up);
    }
    s += Tf * dphi * c;
  }
  return s;
}

// Face terms of cell i: glnk[i] -= sum_faces w_i (lambda_lo - lambda_hi) . F_adv
// (dT/d ln k_i = w_i T); scond[i] = sum_faces (lambda_E,lo - lambda_E,hi) G dKh/dK_T,i dT.
__global__ void __launch_bounds__(128) k_adj_face(Params P, const double* __restrict__ u,
                                                  const double* __restrict__ props, const double* __restrict__ tx,
                                                  const double* __restrict__ ty, const double* __restrict__ tz,
                                                  const double* __restrict__ wx, const double* __restrict__ wy,
                                                  const double* __restrict__ wz, const double* __restrict__ depth,
                                                  const double* __restrict__ lam, double* __restrict__ glnk,
                                                  double* __restrict__ scond) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const int n = P.n;
  const int nx = P.nx, ny = P.ny, nxy = P.nx * P.ny;
  const int ix = i % nx, iy = (i / nx) % ny, iz = i / nxy;
  const bool has[6] = {iz > 0, iy > 0, ix > 0, ix < nx - 1, iy < ny - 1, iz < P.nz - 1};
  const int nb[6] = {i - nxy, i - nx, i - 1, i + 1, i + nx, i + nxy};
  double gk = 0.0, sc = 0.0;
  const double Ki = qv(props, n, Q_KT, i);
  for (int f = 0; f < 6; ++f) {
    if (!has[f]) continue;
    const int j = nb[f];
    const int lo = min(i, j), hi = max(i, j);
    double Tf, Gf, wlo;
    if (f == 2 || f == 3) {
      Tf = tx[lo];
      wlo = wx[lo];
      Gf = P.gx;
    } else if (f == 1 || f == 4) {
      Tf = ty[lo];
      wlo = wy[lo];
      Gf = P.gy;
    } else {
      Tf = tz[lo];
      wlo = wz[lo];
      Gf = P.gz;
    }
    const double dz = depth[lo] - depth[hi];
    double dl[7];
#pragma unroll
    for (int r = 0; r < 7; ++r) dl[r] = lam[(size_t)lo * 8 + r] - lam[(size_t)hi * 8 + r];
    const double wi = (i == lo) ? wlo : 1.0 - wlo;
    gk -= wi * adv_flux_dot(P, lo, hi, Tf, dz, u, props, dl);
    // conduction: Kh = 2 K_lo K_hi / (K_lo + K_hi)
    const double Kj = qv(props, n, Q_KT, j);
    const double s = Ki + Kj;
    const double dKh = 2.0 * Kj * Kj / (s * s);
    const double dT = __ldg(u + (size_t)5 * n + lo) - __ldg(u + (size_t)5 * n + hi);
    sc += dl[6] * Gf * dKh * dT;
  }
  glnk[i] += gk;
  scond[i] = sc;
}

// Local terms at (u^n, C^n): gamma (dF/dC^T lambda), kappa = Cbar - gamma,
// the reaction-parameter gradients and the producer's ln k term.
__global__ void __launch_bounds__(128) k_adj_local(Params P, const double* __restrict__ u,
                                                   const double* __restrict__ coke_new,
                                                   const double* __restrict__ phi_ref,
                                                   const int32_t* __restrict__ well_slot,
                                                   const WellSlot* __restrict__ slots, const double* __restrict__ lam,
                                                   const double* __restrict__ cbar, const double* __restrict__ scond,
                                                   double* __restrict__ glnk, double* __restrict__ grx,
                                                   double* __restrict__ kd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const int n = P.n;
  Base b;
  base_properties(P, u, i, phi_ref[i], b);
  double l[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) l[r] = lam[(size_t)i * 8 + r];
  const double C = coke_new[i];
  const double Tv = b.T.v;
  // reactions at (u^n, C^n)
  double rt[ISC_MAX_RXN], drt[ISC_MAX_RXN];
  double dg = 1.0;
  for (int r = 0; r < P.nr; ++r) {
    double kT = P.A[r] * exp(-P.EaR[r] * (1.0 / Tv));
    rate_dC(P, r, b, kT, C, &rt[r], &drt[r]);
    dg -= P.dt * P.stoich[r][6] * drt[r];
  }
  // dF_r/dC of the cell's own rows (accumulation and reactions)
  const double gas = b.rho_g.v * b.Sg.v, oil = b.rho_o.v * b.So.v;
  double X[7];
  X[0] = b.rho_w.v * b.Sw.v + gas * b.y[0].v;
  X[1] = oil * b.xlo.v + gas * b.y[1].v;
  X[2] = oil * b.xho.v + gas * b.y[2].v;
  X[3] = gas * b.y[3].v;
  X[4] = gas * b.y[4].v;
  X[5] = gas * b.y[5].v;
  X[6] = b.rho_w.v * b.Sw.v * b.U[0].v + oil * b.U[1].v + gas * b.U[2].v;
  const double Vdt = P.V * P.inv_dt;
  double gam = 0.0;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double d = Vdt * (-X[c] / P.coke_rho);
    for (int r = 0; r < P.nr; ++r) d -= P.V * P.stoich[r][c] * drt[r];
    gam += l[c] * d;
  }
  {
    double d = Vdt * (-X[6] / P.coke_rho + b.Uc.v);
    for (int r = 0; r < P.nr; ++r) d -= P.V * P.dH[r] * drt[r];
    gam += l[6] * d;
  }
  // conduction through K_T(C)
  const double dKT = -(b.Sw.v * P.K_phase[0] + b.So.v * P.K_phase[1] + b.Sg.v * P.K_phase[2]) / P.coke_rho + P.coke_K;
  gam += scond[i] * dKT;
  const double kappa = cbar[i] - gam;
  const double kdi = kappa / dg;
  kd[i] = kdi;
  // d/d ln A_r (rates are linear in A); d/d E_a = -1/(R T) d/d ln A
  for (int r = 0; r < P.nr; ++r) {
    double s = P.dH[r] * l[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) s += P.stoich[r][c] * l[c];
    double a = P.V * rt[r] * s + kdi * P.dt * P.stoich[r][6] * rt[r];
    grx[(size_t)r * n + i] += a;
    grx[(size_t)(P.nr + r) * n + i] += -a / (R_GAS * Tv);
  }
  // producer: its residual terms are linear in WI = WI_0 exp(ln k)
  WellSlot w;
  if (producer_slot(well_slot, slots, i, &w)) {
    double dpw = w.bhp - b.p.v;
    if (dpw < 0.0) {
      double Qw = w.WI * b.lam[0].v * dpw, Qo = w.WI * b.lam[1].v * dpw, Qg = w.WI * b.lam[2].v * dpw;
      double t = l[0] * Qw + l[1] * Qo * b.xlo.v + l[2] * Qo * b.xho.v +
                 l[6] * (Qw * b.H[0].v + Qo * b.H[1].v + Qg * b.H[2].v);
#pragma unroll
      for (int c = 0; c < 6; ++c) t += l[c] * Qg * b.y[c].v;
      glnk[i] += t;  // -(dF/d ln k)^T lambda with dF = -Q x
    }
  }
}

// Rate injectors: the source of perforation j is share_j q_tot with
// share_j = WI_j / sum WI, so d src_i / d ln k_j = src_i (delta_ij - share_j).
// One thread per injector well, fixed summation order.
__global__ void k_adj_inj(int nw, const int32_t* __restrict__ first, const int32_t* __restrict__ count,
                          const WellSlot* __restrict__ slots, const double* __restrict__ lam,
                          double* __restrict__ glnk) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  const int f = first[w], m = count[w];
  double S = 0.0;
  for (int q = 0; q < m; ++q) {
    const WellSlot& sl = slots[f + q];
    const double* l = lam + (size_t)sl.cell * 8;
    double s = 0.0;
    for (int r = 0; r < 7; ++r) s += l[r] * sl.src[r];
    S += s;
  }
  for (int q = 0; q < m; ++q) {
    const WellSlot& sl = slots[f + q];
    const double* l = lam + (size_t)sl.cell * 8;
    double s = 0.0;
    for (int r = 0; r < 7; ++r) s += l[r] * sl.src[r];
    glnk[sl.cell] += s - sl.share * S;
  }
}

// Old-state terms: ubar^{n-1} = (V/dt)(dacc/du^{n-1})^T lambda,
// Cbar^{n-1} = (V/dt)(dacc/dC^{n-1})^T lambda + kappa/(dg/dC).
__global__ void __launch_bounds__(128) k_adj_old(Params P, const double* __restrict__ u_old,
                                                 const double* __restrict__ coke_old,
                                                 const double* __restrict__ phi_ref, const double* __restrict__ lam,
                                                 const double* __restrict__ kd, double* __restrict__ ubar,
                                                 double* __restrict__ cbar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  Base b;
  base_properties(P, u_old, i, phi_ref[i], b);
  const double C = coke_old[i];
  double l[7];
#pragma unroll
  for (int r = 0; r < 7; ++r) l[r] = lam[(size_t)i * 8 + r];
  D8 phif = b.phi - C / P.coke_rho;
  D8 gas = b.rho_g * b.Sg;
  D8 oil = b.rho_o * b.So;
  D8 X[7];
  X[0] = b.rho_w * b.Sw + gas * b.y[0];
  X[1] = oil * b.xlo + gas * b.y[1];
  X[2] = oil * b.xho + gas * b.y[2];
  X[3] = gas * b.y[3];
  X[4] = gas * b.y[4];
  X[5] = gas * b.y[5];
  X[6] = b.rho_w * b.Sw * b.U[0] + oil * b.U[1] + gas * b.U[2];
  const double Vdt = P.V * P.inv_dt;
  double g[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) g[k] = 0.0;
  double gc = 0.0;
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    D8 acc = phif * X[r];
    if (r == 6) acc = acc + (1.0 - b.phi) * b.Ur + C * b.Uc;
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] += l[r] * acc.d[k];
    gc += l[r] * (-X[r].v / P.coke_rho);
  }
  gc += l[6] * b.Uc.v;
  double* ub = ubar + (size_t)i * 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) ub[k] = Vdt * g[k];
  cbar[i] = Vdt * gc + kd[i];
}

// Coupled wells, before the transposed solve: the right-hand side of each
// well's row, ubar_w = dt dP/d bhp_w (the produced oil's bottom-hole-pressure
// derivative; zero for injectors). One thread per coupled well, its
// perforations in fixed order.
__global__ void k_adj_wells_pre(Params P, int nwc, const CoupledWell* __restrict__ cw,
                                const WellSlot* __restrict__ slots, const double* __restrict__ u,
                                const double* __restrict__ phi_ref, const double* __restrict__ bhp,
                                const double* __restrict__ depth, double* __restrict__ ubar_w) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwc) return;
  const CoupledWell c = cw[w];
  double s = 0.0;
  for (int q = c.first; q < c.first + c.count; ++q) {
    const WellSlot sl = slots[q];
    if (sl.kind != ISC_WELL_COUPLED_PRODUCER) continue;
    Base b;
    base_properties(P, u, sl.cell, phi_ref[sl.cell], b);
    D8 Q[3];
    double dQ[3];
    bool on[3];
    coupled_producer_rates(b, sl.WI, bhp[w], sl.zref, depth[sl.cell], Q, dQ, on);
    const double mo = P.M[1] * b.xlo.v + P.M[2] * b.xho.v;
    const double mg = P.M[1] * b.y[1].v + P.M[2] * b.y[2].v;
    s += -(dQ[1] * mo + dQ[2] * mg);
  }
  ubar_w[w] = P.dt * s;
}

// Coupled wells, after the transposed solve: the ln k terms of their
// perforations. A perforation's residual terms F_well and its part f_q of a
// rate-controlled well equation are linear in WI = WI_0 exp(ln k), so
// glnk[cell] += -(lambda_cell . F_well + mu_w f_q), mu_w the well row's
// multiplier. One thread per coupled well, perforations in fixed order.
__global__ void k_adj_wells_post(Params P, int nwc, const CoupledWell* __restrict__ cw,
                                 const WellSlot* __restrict__ slots, const double* __restrict__ u,
                                 const double* __restrict__ phi_ref, const double* __restrict__ bhp,
                                 const double* __restrict__ depth, const double* __restrict__ lam,
                                 double* __restrict__ glnk) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwc) return;
  const CoupledWell c = cw[w];
  const double mu = lam[(size_t)P.n * 8 + w];
  for (int q = c.first; q < c.first + c.count; ++q) {
    const WellSlot sl = slots[q];
    const int i = sl.cell;
    Base b;
    base_properties(P, u, i, phi_ref[i], b);
    const double* l = lam + (size_t)i * 8;
    double Fw[7] = {0, 0, 0, 0, 0, 0, 0};
    double fq = 0.0;
    if (sl.kind == ISC_WELL_COUPLED_PRODUCER) {
      D8 Q[3];
      double dQ[3];
      bool on[3];
      coupled_producer_rates(b, sl.WI, bhp[w], sl.zref, depth[i], Q, dQ, on);
      Fw[0] = -Q[0].v - Q[2].v * b.y[0].v;
      Fw[1] = -Q[1].v * b.xlo.v - Q[2].v * b.y[1].v;
      Fw[2] = -Q[1].v * b.xho.v - Q[2].v * b.y[2].v;
#pragma unroll
      for (int k = 3; k < 6; ++k) Fw[k] = -Q[2].v * b.y[k].v;
      Fw[6] = -(Q[0].v * b.H[0].v + Q[1].v * b.H[1].v + Q[2].v * b.H[2].v);
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (c.control & (1 << a)) fq -= Q[a].v;
    } else {
      bool flows;
      double dQ;
      const D8 Q = coupled_injector_rate(b, sl.WI, bhp[w], sl.zref, depth[i], sl.phase, &flows, &dQ);
      if (flows) {
#pragma unroll
        for (int r = 0; r < 7; ++r) Fw[r] = -Q.v * sl.src[r];
        if (c.control != ISC_CTRL_BHP) fq = Q.v;
      }
    }
    double t = mu * fq;
#pragma unroll
    for (int r = 0; r < 7; ++r) t += l[r] * Fw[r];
    glnk[i] -= t;
  }
}

// out[r] = sum_i x[r*len + i], one block per row, fixed order.
__global__ void __launch_bounds__(256) k_row_sums(int len, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double sh[256];
  const double* xr = x + (size_t)blockIdx.x * len;
  double s = 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) s += xr[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

}  // namespace

void launch_oil_rate(Handle& h, double dt, cudaStream_t s) {
  int tb = 128;
  k_oil_rate<<<(h.n + tb - 1) / tb, tb, 0, s>>>(h.P, h.u, h.phi_ref, h.well_slot, h.slots, h.bhp, h.depth, dt,
                                                h.adj.loss_cell);
}

void launch_adj_pre(Handle& h, double dt, cudaStream_t s) {
  int tb = 128;
  Params P = h.P;
  P.dt = dt;
  P.inv_dt = 1.0 / dt;
  k_adj_pre<<<(h.n + tb - 1) / tb, tb, 0, s>>>(P, h.u, h.coke_n, h.phi_ref, h.well_slot, h.slots, h.bhp, h.depth,
                                               h.adj.cbar, h.adj.ubar, h.adj.glnk, h.dstatus);
  if (h.nwc)
    k_adj_wells_pre<<<(h.nwc + 31) / 32, 32, 0, s>>>(P, h.nwc, h.cw, h.slots, h.u, h.phi_ref, h.bhp, h.depth,
                                                     h.adj.ubar + (size_t)h.n * 8);
}

void launch_bsr_transpose(Handle& h, cudaStream_t s) {
  int tb = 256;
  k_bsr_transpose<<<(int)(((size_t)h.nnzb * 32 + tb - 1) / tb), tb, 0, s>>>(h.n, h.rowptr, h.col, h.J);
}

void launch_adj_post(Handle& h, bool has_old, cudaStream_t s) {
  int tb = 128;
  int grid = (h.n + tb - 1) / tb;
  AdjointWork& a = h.adj;
  k_adj_face<<<grid, tb, 0, s>>>(h.P, h.u, h.props, h.tx, h.ty, h.tz, h.wx, h.wy, h.wz, h.depth, a.lam, a.glnk,
                                 a.scond);
  k_adj_local<<<grid, tb, 0, s>>>(h.P, h.u, h.coke, h.phi_ref, h.well_slot, h.slots, a.lam, a.cbar, a.scond, a.glnk,
                                  a.grx, a.kd);
  if (a.n_inj > 0)
    k_adj_inj<<<(a.n_inj + 31) / 32, 32, 0, s>>>(a.n_inj, a.inj_first, a.inj_count, h.slots, a.lam, a.glnk);
  if (h.nwc)
    k_adj_wells_post<<<(h.nwc + 31) / 32, 32, 0, s>>>(h.P, h.nwc, h.cw, h.slots, h.u, h.phi_ref, h.bhp, h.depth,
                                                      a.lam, a.glnk);
  if (has_old) k_adj_old<<<grid, tb, 0, s>>>(h.P, h.u_n, h.coke_n, h.phi_ref, a.lam, a.kd, a.ubar, a.cbar);
}

void launch_row_sums(int nrows, int len, const double* x, double* out, cudaStream_t s) {
  if (nrows <= 0) return;
  k_row_sums<<<nrows, 256, 0, s>>>(len, x, out);
}

}  // namespace isc
