// Residual and analytical Jacobian assembly of the ISC model (Sec. 2.2, 3.1).
//
// k_props   one thread per cell: properties with exact derivatives
//           (forward-mode, 8 tangents), local coke equation, accumulation,
//           reactions and wells -> residual, diagonal Jacobian block and the
//           staged face quantities (lambda_alpha * carried quantity, gamma,
//           K_T with their derivatives).
// k_flux    one thread per (direction, cell, equation row): the cell's face
//           towards +x, +y or +z, evaluated once in its (lo, hi) orientation:
//           upstream weighting per phase, harmonic transmissibility, the face
//           flux and its derivatives w.r.t. both cells; writes both cells'
//           off-diagonal blocks of the face and parks the flux for
// k_flux_gather, which adds each cell's residual and diagonal-block shares of
//           its six faces (the diagonal shares read back from those blocks).
#include <math.h>

#include "dual8.cuh"
#include "isc_internal.cuh"
#include "isc_props.cuh"

namespace isc {

namespace {

__device__ __forceinline__ void store_q(double* __restrict__ props, int n, int i, int q, const D8& x) {
  props[(size_t)(q * 9) * n + i] = x.v;
#pragma unroll
  for (int k = 0; k < 8; ++k) props[(size_t)(q * 9 + 1 + k) * n + i] = x.d[k];
}

__device__ __forceinline__ int diag_slot(const Params& P, int i) {
  int ix = i % P.nx, iy = (i / P.nx) % P.ny, iz = i / (P.nx * P.ny);
  return (iz > 0) + (iy > 0) + (ix > 0);
}

__global__ void __launch_bounds__(128) k_props(Params P, const double* __restrict__ u, const double* __restrict__ coke_n,
                                               const double* __restrict__ acc_n, const double* __restrict__ phi_ref,
                                               const int32_t* __restrict__ well_slot, const WellSlot* __restrict__ slots,
                                               const int32_t* __restrict__ rowptr, double* __restrict__ R,
                                               double* __restrict__ J, double* __restrict__ props,
                                               double* __restrict__ ntot, double* __restrict__ coke_out,
                                               int* __restrict__ dstatus, const double* __restrict__ depth,
                                               const double* __restrict__ bhp, double* __restrict__ Bv,
                                               double* __restrict__ Cv, double* __restrict__ Fq,
                                               double* __restrict__ Dq) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const int n = P.n;
  Base b;
  base_properties(P, u, i, phi_ref[i], b);
  D8 kT[ISC_MAX_RXN];
  for (int r = 0; r < P.nr; ++r) kT[r] = P.A[r] * dexp(-P.EaR[r] * (1.0 / b.T));
  D8 C = solve_coke(P, b, kT, coke_n[i], dstatus);
  D8 phif = b.phi - C / P.coke_rho;
  // accumulation (moles and energy per bulk volume)
  D8 gas = b.rho_g * b.Sg;
  D8 oil = b.rho_o * b.So;
  D8 acc[7];
  acc[0] = phif * (b.rho_w * b.Sw + gas * b.y[0]);
  acc[1] = phif * (oil * b.xlo + gas * b.y[1]);
  acc[2] = phif * (oil * b.xho + gas * b.y[2]);
  acc[3] = phif * (gas * b.y[3]);
  acc[4] = phif * (gas * b.y[4]);
  acc[5] = phif * (gas * b.y[5]);
  acc[6] = phif * (b.rho_w * b.Sw * b.U[0] + oil * b.U[1] + gas * b.U[2]) + (1.0 - b.phi) * b.Ur + C * b.Uc;
  double nt = 0.0;
  for (int c = 0; c < 6; ++c) nt += fabs(acc[c].v);
  ntot[i] = nt;
  const double Vdt = P.V * P.inv_dt;
  D8 Rl[8];
#pragma unroll
  for (int r = 0; r < 7; ++r) Rl[r] = Vdt * (acc[r] - acc_n[(size_t)r * n + i]);
  // reactions: q_c = sum_R s_cR r_R, Q = sum_R H_R r_R
  for (int r = 0; r < P.nr; ++r) {
    D8 rt = rate(P, r, b, kT[r], phif, C) * P.V;
#pragma unroll
    for (int c = 0; c < 6; ++c)
      if (P.stoich[r][c] != 0.0) Rl[c] = Rl[c] - P.stoich[r][c] * rt;
    Rl[6] = Rl[6] - P.dH[r] * rt;
  }
  // wells
  int sl = well_slot[i];
  if (sl >= 0) {
    WellSlot w = slots[sl];
    if (w.kind == ISC_WELL_RATE_INJECTOR) {
#pragma unroll
      for (int r = 0; r < 7; ++r) Rl[r] = Rl[r] - w.src[r];
    } else if (w.kind == ISC_WELL_COUPLED_PRODUCER) {
      // Peaceman rates with the bottom-hole pressure unknown and the hydrostatic
      // head between its reference depth and the perforation (Sec. 2.2):
      // Q_a = WI lambda_a (bhp - p - gamma_a (z_ref - z)), outflow only.
      // Also the border of the Newton system: dF/d bhp (B), and for a rate
      // control the perforation's part of the well equation, its u-gradient
      // (C) and its bhp-derivative.
      double bcol[8] = {0, 0, 0, 0, 0, 0, 0, 0}, crow[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      double fq = 0.0, dq = 0.0;
      D8 Qa[3];
      double dQa[3];
      bool on[3];
      coupled_producer_rates(b, w.WI, bhp[w.wc], w.zref, depth[i], Qa, dQa, on);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (!on[a]) continue;
        const D8 Q = Qa[a];
        const double dQ = dQa[a];
        if (a == 0) {
          Rl[0] = Rl[0] - Q;
          bcol[0] -= dQ;
        } else if (a == 1) {
          Rl[1] = Rl[1] - Q * b.xlo;
          Rl[2] = Rl[2] - Q * b.xho;
          bcol[1] -= dQ * b.xlo.v;
          bcol[2] -= dQ * b.xho.v;
        } else {
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            Rl[c] = Rl[c] - Q * b.y[c];
            bcol[c] -= dQ * b.y[c].v;
          }
        }
        Rl[6] = Rl[6] - Q * b.H[a];
        bcol[6] -= dQ * b.H[a].v;
        if (w.control & (1 << a)) {
          fq -= Q.v;
          dq -= dQ;
#pragma unroll
          for (int k = 0; k < 8; ++k) crow[k] -= Q.d[k];
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        Bv[(size_t)sl * 8 + k] = bcol[k];
        Cv[(size_t)sl * 8 + k] = (w.control == ISC_CTRL_BHP) ? 0.0 : crow[k];
      }
      Fq[sl] = fq;
      Dq[sl] = dq;
    } else if (w.kind == ISC_WELL_COUPLED_INJECTOR) {
      // The injected stream (mole fractions src[0..5], molar enthalpy src[6])
      // enters at Q = WI lambda_T (bhp - p - gamma (z_ref - z)) mol/s with the
      // cell's total molar mobility lambda_T and the injected phase's specific
      // weight gamma, inflow only (Sec. 2.2, Well Modeling, for injection).
      // Border: dF/d bhp = -dQ/d bhp times the stream; for a rate control the
      // perforation's Q, its u-gradient and its bhp-derivative.
      bool flows;
      double dQ;
      const D8 Q = coupled_injector_rate(b, w.WI, bhp[w.wc], w.zref, depth[i], w.phase, &flows, &dQ);
      if (flows) {
#pragma unroll
        for (int r = 0; r < 7; ++r) Rl[r] = Rl[r] - Q * w.src[r];
      }
      const bool rate = w.control != ISC_CTRL_BHP;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        Bv[(size_t)sl * 8 + k] = k < 7 ? -dQ * w.src[k] : 0.0;
        Cv[(size_t)sl * 8 + k] = (rate && flows) ? Q.d[k] : 0.0;
      }
      Fq[sl] = flows ? Q.v : 0.0;
      Dq[sl] = dQ;
    } else {
      D8 dpw = w.bhp - b.p;
      if (dpw.v < 0.0) {
        D8 Qw = (w.WI * b.lam[0]) * dpw;
        D8 Qo = (w.WI * b.lam[1]) * dpw;
        D8 Qg = (w.WI * b.lam[2]) * dpw;
        Rl[0] = Rl[0] - Qw;
        Rl[1] = Rl[1] - Qo * b.xlo;
        Rl[2] = Rl[2] - Qo * b.xho;
#pragma unroll
        for (int c = 0; c < 6; ++c) Rl[c] = Rl[c] - Qg * b.y[c];
        Rl[6] = Rl[6] - Qw * b.H[0] - Qo * b.H[1] - Qg * b.H[2];
      }
    }
  }
  // heat loss through the top and / or bottom face of a boundary-layer cell (Sec. 2.1 energy equation)
  if (P.hl_AK != 0.0) {
    const int iz = i / (P.nx * P.ny);
    const int nf = ((iz == 0 && (P.hl_faces & 1)) ? 1 : 0) + ((iz == P.nz - 1 && (P.hl_faces & 2)) ? 1 : 0);
    if (nf) Rl[6] = Rl[6] + (nf * P.hl_AK) * ((b.T - P.hl_Tini) * P.hl_inv_d - P.hl_rho);
  }
  D8 sy = b.y[0] + b.y[1] + b.y[2] + b.y[3] + b.y[4] + b.y[5];
  Rl[7] = sy - 1.0;
  // residual (block-major) and diagonal block
  double* Jd = J + (size_t)(rowptr[i] + diag_slot(P, i)) * BB;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    R[(size_t)i * 8 + r] = Rl[r].v;
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      double2 v = make_double2(Rl[r].d[k], Rl[r].d[k + 1]);
      *reinterpret_cast<double2*>(Jd + r * 8 + k) = v;
    }
  }
  coke_out[i] = C.v;
  // staged face quantities
  store_q(props, n, i, Q_LW, b.lam[0]);
  store_q(props, n, i, Q_LWH, b.lam[0] * b.H[0]);
  store_q(props, n, i, Q_LOX_LO, b.lam[1] * b.xlo);
  store_q(props, n, i, Q_LOX_HO, b.lam[1] * b.xho);
  store_q(props, n, i, Q_LOH, b.lam[1] * b.H[1]);
#pragma unroll
  for (int c = 0; c < 6; ++c) store_q(props, n, i, Q_LGY + c, b.lam[2] * b.y[c]);
  store_q(props, n, i, Q_LGH, b.lam[2] * b.H[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) store_q(props, n, i, Q_GAM + a, b.gam[a]);
  D8 KT = phif * (b.Sw * P.K_phase[0] + b.So * P.K_phase[1] + b.Sg * P.K_phase[2]) + (1.0 - b.phi) * P.K_rock +
          C * P.coke_K;
  store_q(props, n, i, Q_KT, KT);
  bool fin = isfinite(Rl[0].v) && isfinite(Rl[6].v) && isfinite(Rl[7].v);
  if (!fin) atomicOr(dstatus, DS_NONFINITE);
}

__global__ void __launch_bounds__(128) k_old_acc(Params P, const double* __restrict__ u, const double* __restrict__ coke,
                                                 const double* __restrict__ phi_ref, double* __restrict__ acc_n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const int n = P.n;
  Base b;
  base_properties(P, u, i, phi_ref[i], b);
  double C = coke[i];
  D8 phif = b.phi - C / P.coke_rho;
  D8 gas = b.rho_g * b.Sg;
  D8 oil = b.rho_o * b.So;
  acc_n[0 * (size_t)n + i] = (phif * (b.rho_w * b.Sw + gas * b.y[0])).v;
  acc_n[1 * (size_t)n + i] = (phif * (oil * b.xlo + gas * b.y[1])).v;
  acc_n[2 * (size_t)n + i] = (phif * (oil * b.xho + gas * b.y[2])).v;
  acc_n[3 * (size_t)n + i] = (phif * (gas * b.y[3])).v;
  acc_n[4 * (size_t)n + i] = (phif * (gas * b.y[4])).v;
  acc_n[5 * (size_t)n + i] = (phif * (gas * b.y[5])).v;
  acc_n[6 * (size_t)n + i] =
      (phif * (b.rho_w * b.Sw * b.U[0] + oil * b.U[1] + gas * b.U[2]) + (1.0 - b.phi) * b.Ur + C * b.Uc).v;
}

// ------------------------------------------------------------------ fluxes
struct Q9 {
  double v, d[8];
};

__device__ __forceinline__ Q9 load_q(const double* __restrict__ props, int n, int q, int cell) {
  Q9 x;
  x.v = __ldg(props + (size_t)(q * 9) * n + cell);
#pragma unroll
  for (int k = 0; k < 8; ++k) x.d[k] = __ldg(props + (size_t)(q * 9 + 1 + k) * n + cell);
  return x;
}

// phases carrying row r: (phase, staged quantity); count in *m
__device__ __forceinline__ int row_phases(int r, int* ph, int* q) {
  switch (r) {
    case 0: ph[0] = 0; q[0] = Q_LW; ph[1] = 2; q[1] = Q_LGY + 0; return 2;
    case 1: ph[0] = 1; q[0] = Q_LOX_LO; ph[1] = 2; q[1] = Q_LGY + 1; return 2;
    case 2: ph[0] = 1; q[0] = Q_LOX_HO; ph[1] = 2; q[1] = Q_LGY + 2; return 2;
    case 3: ph[0] = 2; q[0] = Q_LGY + 3; return 1;
    case 4: ph[0] = 2; q[0] = Q_LGY + 4; return 1;
    case 5: ph[0] = 2; q[0] = Q_LGY + 5; return 1;
    case 6: ph[0] = 0; q[0] = Q_LWH; ph[1] = 1; q[1] = Q_LOH; ph[2] = 2; q[2] = Q_LGH; return 3;
    default: return 0;
  }
}

// Flux of row r out of lo into hi over one face, with d/du_lo and d/du_hi.
__device__ __forceinline__ double face_flux(const Params& P, int r, int lo, int hi, double Tf, double Gf, double dz,
                                            const double* __restrict__ u, const double* __restrict__ props,
                                            double* dlo, double* dhi) {
  const int n = P.n;
  int ph[3], qq[3];
  int m = row_phases(r, ph, qq);
  double F = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) dlo[k] = dhi[k] = 0.0;
  double plo = __ldg(u + lo), phi_ = __ldg(u + hi);
  for (int a = 0; a < m; ++a) {
    Q9 glo = load_q(props, n, Q_GAM + ph[a], lo);
    Q9 ghi = load_q(props, n, Q_GAM + ph[a], hi);
    // potential difference: the decision quantity is formed without contraction
    double gavg = __dmul_rn(0.5, __dadd_rn(glo.v, ghi.v));
    double dphi = __dsub_rn(__dsub_rn(plo, phi_), __dmul_rn(gavg, dz));
    bool up_lo = dphi >= 0.0;
    Q9 q = load_q(props, n, qq[a], up_lo ? lo : hi);
    double tq = Tf * q.v;
    F += tq * dphi;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double e = (k == 0) ? 1.0 : 0.0;
      dlo[k] += tq * (e - 0.5 * dz * glo.d[k]);
      dhi[k] += tq * (-e - 0.5 * dz * ghi.d[k]);
    }
    if (up_lo) {
#pragma unroll
      for (int k = 0; k < 8; ++k) dlo[k] += Tf * q.d[k] * dphi;
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) dhi[k] += Tf * q.d[k] * dphi;
    }
  }
  if (r == 6) {
    Q9 Klo = load_q(props, n, Q_KT, lo);
    Q9 Khi = load_q(props, n, Q_KT, hi);
    double s = Klo.v + Khi.v;
    double Kh = 2.0 * Klo.v * Khi.v / s;
    double dKlo = 2.0 * Khi.v * Khi.v / (s * s);
    double dKhi = 2.0 * Klo.v * Klo.v / (s * s);
    double dT = __ldg(u + (size_t)5 * n + lo) - __ldg(u + (size_t)5 * n + hi);
    F += Gf * Kh * dT;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double e = (k == 5) ? 1.0 : 0.0;
      dlo[k] += Gf * (dKlo * Klo.d[k] * dT + Kh * e);
      dhi[k] += Gf * (dKhi * Khi.d[k] * dT - Kh * e);
    }
  }
  return F;
}

// Face pass: thread (direction d, cell i, row r) evaluates the flux F of row
// r over the face between i and its neighbour j towards +d, once per face
// (blockIdx.y is the direction: three threads per cell and row keep enough
// independent faces in flight). It writes both cells' off-diagonal block rows
// of the face, J(i, +d) = dF/du_j and J(j, -d) = -dF/du_i (no other thread
// writes them), and parks F in fbuf[(d * 7 + r) * N + i] for k_flux_gather:
// a cell's own row is shared by the faces of six threads, so it is not added
// to here. The diagonal-block shares are the negatives of those two
// off-diagonal rows (dF/du_i for i, -dF/du_j for j), which the gather reads
// back from J.
__global__ void __launch_bounds__(256, 3) k_flux(Params P, const double* __restrict__ u, const double* __restrict__ props,
                                              const double* __restrict__ tx, const double* __restrict__ ty,
                                              const double* __restrict__ tz, const double* __restrict__ depth,
                                              const int32_t* __restrict__ rowptr, double* __restrict__ J,
                                              double* __restrict__ fbuf) {
  const int r = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int dir = blockIdx.y;
  if (i >= P.n) return;
  const int n = P.n, nx = P.nx, ny = P.ny, nxy = P.nx * P.ny;
  const int ix = i % nx, iy = (i / nx) % ny, iz = i / nxy;
  const bool lz = iz > 0, ly = iy > 0, lx = ix > 0;
  const int base = rowptr[i];
  const int dslot = (int)lz + (int)ly + (int)lx;
  if (r == 7) {
    // the gas constraint has no flux: its off-diagonal rows are zero (the
    // buffer may hold the previous, decoupled system); one direction does it
    if (dir != 0) return;
    const int nblk = rowptr[i + 1] - base;
    for (int s = 0; s < nblk; ++s) {
      if (s == dslot) continue;
      double* Jb = J + (size_t)(base + s) * BB + 56;
#pragma unroll
      for (int k = 0; k < 8; k += 2) *reinterpret_cast<double2*>(Jb + k) = make_double2(0.0, 0.0);
    }
    return;
  }
  const bool has = dir == 0 ? ix < nx - 1 : dir == 1 ? iy < ny - 1 : iz < P.nz - 1;
  if (!has) return;
  const int j = i + (dir == 0 ? 1 : dir == 1 ? nx : nxy);
  const double Tf = dir == 0 ? tx[i] : dir == 1 ? ty[i] : tz[i];
  const double Gf = dir == 0 ? P.gx : dir == 1 ? P.gy : P.gz;
  double dlo[8], dhi[8];
  const double F = face_flux(P, r, i, j, Tf, Gf, depth[i] - depth[j], u, props, dlo, dhi);
  // cell i's +dir block (after the diagonal: +x, +y, +z, those present)
  const int si = dslot + 1 + (dir >= 1 ? (int)(ix < nx - 1) : 0) + (dir == 2 ? (int)(iy < ny - 1) : 0);
  double* Jb = J + (size_t)(base + si) * BB + r * 8;
#pragma unroll
  for (int k = 0; k < 8; k += 2) *reinterpret_cast<double2*>(Jb + k) = make_double2(dhi[k], dhi[k + 1]);
  // cell j's -dir block (its lower neighbours before it: -z, -y when dir is x; -z when dir is y)
  const int jy = iy + (dir == 1), jz = iz + (dir == 2);
  const int sj = dir == 0 ? (int)(jz > 0) + (int)(jy > 0) : dir == 1 ? (int)(jz > 0) : 0;
  double* Jn = J + (size_t)(rowptr[j] + sj) * BB + r * 8;
#pragma unroll
  for (int k = 0; k < 8; k += 2) *reinterpret_cast<double2*>(Jn + k) = make_double2(-dlo[k], -dlo[k + 1]);
  fbuf[(size_t)(dir * 7 + r) * n + i] = F;
}

// Gather pass: thread (cell i, row r < 7) adds cell i's shares of its six
// faces to its residual (+F over the faces towards +x, +y, +z, -F over those
// towards -x, -y, -z, F from fbuf) and to its diagonal block row: minus the
// face's off-diagonal row in the neighbour's row of J (the neighbour's -d
// block for a face towards +d, its +d block for a face towards -d).
__global__ void __launch_bounds__(256) k_flux_gather(Params P, const int32_t* __restrict__ rowptr,
                                                     const double* __restrict__ fbuf, double* __restrict__ R,
                                                     double* __restrict__ J) {
  const int r = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  if (i >= P.n || r == 7) return;
  const int n = P.n, nx = P.nx, ny = P.ny, nz = P.nz, nxy = P.nx * P.ny;
  const int ix = i % nx, iy = (i / nx) % ny, iz = i / nxy;
  double Rs = 0.0;
  double dd[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) dd[k] = 0.0;
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    const int e = dir == 0 ? 1 : dir == 1 ? nx : nxy;
    const int c = dir == 0 ? ix : dir == 1 ? iy : iz, cmax = dir == 0 ? nx : dir == 1 ? ny : nz;
    if (c < cmax - 1) {
      // face (i, j = i + e): the neighbour's -dir block holds -dF/du_i
      const int j = i + e;
      const int jy = iy + (dir == 1), jz = iz + (dir == 2);
      const int sj = dir == 0 ? (int)(jz > 0) + (int)(jy > 0) : dir == 1 ? (int)(jz > 0) : 0;
      Rs += fbuf[(size_t)(dir * 7 + r) * n + i];
      const double* b = J + (size_t)(rowptr[j] + sj) * BB + r * 8;
#pragma unroll
      for (int k = 0; k < 8; ++k) dd[k] -= b[k];
    }
    if (c > 0) {
      // face (j = i - e, i): the neighbour's +dir block holds dF/du_i
      const int j = i - e;
      const int jx = ix - (dir == 0), jy = iy - (dir == 1), jz = iz - (dir == 2);
      const int sj = (int)(jz > 0) + (int)(jy > 0) + (int)(jx > 0) + 1 + (dir >= 1 ? (int)(jx < nx - 1) : 0) +
                     (dir == 2 ? (int)(jy < ny - 1) : 0);
      Rs -= fbuf[(size_t)(dir * 7 + r) * n + j];
      const double* b = J + (size_t)(rowptr[j] + sj) * BB + r * 8;
#pragma unroll
      for (int k = 0; k < 8; ++k) dd[k] -= b[k];
    }
  }
  const int dslot = (int)(iz > 0) + (int)(iy > 0) + (int)(ix > 0);
  R[(size_t)i * 8 + r] += Rs;
  double* Jd = J + (size_t)(rowptr[i] + dslot) * BB + r * 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) Jd[k] += dd[k];
}

// Well equations of the coupled wells (Sec. 2.2): bhp - c, or the summed
// production rate of the controlled phases (producer) or the total injected
// rate (injector) minus c, the perforation terms coming from k_props; their
// bhp-derivatives;
// and max |F_w| / |c| into norm_out. One thread, fixed order (wells are few).
__global__ void k_well_eq(int nwc, const CoupledWell* __restrict__ cw, const double* __restrict__ Fq,
                          const double* __restrict__ Dq, const double* __restrict__ bhp, double* __restrict__ Rw,
                          double* __restrict__ Dw, double* __restrict__ norm_out) {
  if (blockIdx.x * blockDim.x + threadIdx.x != 0) return;
  double e = 0.0;
  for (int w = 0; w < nwc; ++w) {
    const CoupledWell c = cw[w];
    double F, D;
    if (c.control == ISC_CTRL_BHP) {
      F = bhp[w] - c.target;
      D = 1.0;
    } else {
      F = 0.0;
      D = 0.0;
      for (int q = c.first; q < c.first + c.count; ++q) {
        F += Fq[q];
        D += Dq[q];
      }
      F -= c.target;
    }
    Rw[w] = F;
    Dw[w] = D;
    e = fmax(e, fabs(F) / fmax(fabs(c.target), 1e-300));
    if (!isfinite(F)) e = INFINITY;
  }
  *norm_out = e;
}

// scaled max-norms: mass |F_c|/(V N_tot), energy |F_E|/(V cv), constraint |F_GS|
__global__ void k_norms(Params P, const double* __restrict__ R, const double* __restrict__ ntot,
                        unsigned long long* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double em = 0.0, ee = 0.0, eg = 0.0;
  if (i < P.n) {
    const double* Ri = R + (size_t)i * 8;
    double s = P.V * ntot[i];
    for (int c = 0; c < 6; ++c) em = fmax(em, fabs(Ri[c]) / s);
    ee = fabs(Ri[6]) / (P.V * P.cv_scale);
    eg = fabs(Ri[7]);
    if (!isfinite(Ri[0] + Ri[1] + Ri[2] + Ri[3] + Ri[4] + Ri[5] + Ri[6] + Ri[7])) em = ee = eg = INFINITY;
  }
  for (int o = 16; o > 0; o >>= 1) {
    em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
    ee = fmax(ee, __shfl_xor_sync(0xffffffffu, ee, o));
    eg = fmax(eg, __shfl_xor_sync(0xffffffffu, eg, o));
  }
  if ((threadIdx.x & 31) == 0) {
    // non-negative doubles order like their bit patterns
    atomicMax(out + 0, (unsigned long long)__double_as_longlong(em));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(ee));
    atomicMax(out + 2, (unsigned long long)__double_as_longlong(eg));
  }
}

__global__ void k_init_equilibrium(Params P, double p0, double T0, double Sw0, double So0, double xlo0, double r0,
                                   double r1, double r2, double* __restrict__ u, double* __restrict__ coke) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const int n = P.n;
  D8 p = dc(p0), T = dc(T0), Sw = dc(Sw0), So = dc(So0), xlo = dc(xlo0);
  D8 yW = per_f(P, Sw) * k_value(P, 0, p, T);
  D8 yLO = k_value(P, 1, p, T) * xlo;
  D8 yHO = per_f(P, So) * k_value(P, 2, p, T) * (1.0 - xlo);
  double rest = 1.0 - (yW.v + yLO.v + yHO.v);
  u[0 * (size_t)n + i] = p0;
  u[1 * (size_t)n + i] = xlo0;
  u[2 * (size_t)n + i] = r0 * rest;
  u[3 * (size_t)n + i] = r1 * rest;
  u[4 * (size_t)n + i] = r2 * rest;
  u[5 * (size_t)n + i] = T0;
  u[6 * (size_t)n + i] = Sw0;
  u[7 * (size_t)n + i] = 1.0 - Sw0 - So0;
  coke[i] = 0.0;
}

}  // namespace

void launch_props(Handle& h, cudaStream_t s) {
  int tb = 128;
  k_props<<<(h.n + tb - 1) / tb, tb, 0, s>>>(h.P, h.u, h.coke_n, h.acc_n, h.phi_ref, h.well_slot, h.slots, h.rowptr,
                                               h.R, h.J, h.props, h.ntot, h.coke, h.dstatus, h.depth, h.bhp, h.Bv,
                                               h.Cv, h.Fq, h.Dq);
}

void launch_flux(Handle& h, cudaStream_t s) {
  k_flux<<<dim3((h.n + 31) / 32, 3), 256, 0, s>>>(h.P, h.u, h.props, h.tx, h.ty, h.tz, h.depth, h.rowptr, h.J, h.fbuf);
  k_flux_gather<<<(h.n + 31) / 32, 256, 0, s>>>(h.P, h.rowptr, h.fbuf, h.R, h.J);
}

void launch_old_accumulation(Handle& h, cudaStream_t s) {
  int tb = 128;
  k_old_acc<<<(h.n + tb - 1) / tb, tb, 0, s>>>(h.P, h.u_n, h.coke_n, h.phi_ref, h.acc_n);
}

void launch_well_equations(Handle& h, cudaStream_t s) {
  if (h.nwc == 0) return;
  k_well_eq<<<1, 32, 0, s>>>(h.nwc, h.cw, h.Fq, h.Dq, h.bhp, h.R + (size_t)h.n * 8, h.Dw, h.scal + 3);
}

void launch_norms(Handle& h, cudaStream_t s) {
  cudaMemsetAsync(h.scal, 0, 3 * sizeof(double), s);
  int tb = 256;
  k_norms<<<(h.n + tb - 1) / tb, tb, 0, s>>>(h.P, h.R, h.ntot, reinterpret_cast<unsigned long long*>(h.scal));
}

void launch_init_equilibrium(Handle& h, double p0, double T0, double Sw0, double So0, double xlo0,
                             const double* y_rest, cudaStream_t s) {
  int tb = 128;
  k_init_equilibrium<<<(h.n + tb - 1) / tb, tb, 0, s>>>(h.P, p0, T0, Sw0, So0, xlo0, y_rest[0], y_rest[1], y_rest[2],
                                                         h.u, h.coke);
}

}  // namespace isc
