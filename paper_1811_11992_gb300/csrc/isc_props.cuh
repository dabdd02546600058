// Cell properties of the ISC model (Sec. 2.2) with exact derivatives with
// respect to the cell's 8 unknowns (forward mode, D8), the Arrhenius rates
// and the per-cell backward-Euler coke equation. Shared by the assembly and
// the adjoint kernels.
#pragma once

#include <math.h>

#include "dual8.cuh"
#include "isc_internal.cuh"

namespace isc {
namespace {

constexpr double OMEGA_A = 0.427480;
constexpr double OMEGA_B = 0.086640;

struct Base {
  D8 p, T, Sw, Sg, So, xlo, xho;
  D8 y[6];
  D8 rho_w, rho_o, rho_g;
  D8 lam[3];
  D8 H[3];
  D8 U[3];
  D8 phi, Ur, Uc;
  D8 gam[3];
};

__device__ __forceinline__ D8 clamp01(const D8& s) {
  if (s.v <= 0.0) return dc(0.0);
  if (s.v >= 1.0) return dc(1.0);
  return s;
}

// largest real root of z^3 - z^2 + a1 z + a0 (trigonometric / Cardano), 2 Newton polishes
__device__ double cubic_root(double a1, double a0) {
  const double a2 = -1.0;
  double pp = a1 - a2 * a2 / 3.0;
  double qq = 2.0 * a2 * a2 * a2 / 27.0 - a2 * a1 / 3.0 + a0;
  double disc = (qq * 0.5) * (qq * 0.5) + (pp / 3.0) * (pp / 3.0) * (pp / 3.0);
  double z;
  if (disc < 0.0) {
    double m = 2.0 * sqrt(-pp / 3.0);
    double arg = 3.0 * qq / (pp * m);
    arg = fmin(1.0, fmax(-1.0, arg));
    z = m * cos(acos(arg) / 3.0);
  } else {
    double sd = sqrt(disc);
    z = cbrt(-qq * 0.5 + sd) + cbrt(-qq * 0.5 - sd);
  }
  z -= a2 / 3.0;
  for (int it = 0; it < 2; ++it) {
    double f = ((z - 1.0) * z + a1) * z + a0;
    double df = (3.0 * z - 2.0) * z + a1;
    z -= f / df;
  }
  return z;
}

__device__ __forceinline__ D8 k_value(const Params& P, int c, const D8& p, const D8& T) {
  D8 pre = P.kv[c][0] / p + P.kv[c][1] * p + P.kv[c][2];
  D8 ex = dexp(P.kv[c][3] / (T - P.kv[c][4]));
  return pre * ex;
}

__device__ __forceinline__ D8 per_f(const Params& P, const D8& s) { return s / (s + P.per_eps); }

__device__ __forceinline__ D8 liquid_rho(const Params& P, int c, const D8& dp, const D8& dT) {
  D8 e = P.cp[c] * dp - P.ct1[c] * dT - (0.5 * P.ct2[c]) * (dT * dT) + P.cpt[c] * (dp * dT);
  return P.rho_ref[c] * dexp(e);
}

__device__ __forceinline__ D8 gas_enthalpy(const Params& P, int c, const D8& T) {
  double t = T.v, tr = P.T_ref;
  double h = 0.0, cp = 0.0, tk = t, trk = tr, tpow = 1.0;
  for (int k = 0; k < 4; ++k) {
    h += P.cpg[c][k] / (k + 1) * (tk - trk);
    cp += P.cpg[c][k] * tpow;
    tpow *= t;
    tk *= t;
    trk *= tr;
  }
  return dchain(T, h, cp);
}

__device__ __forceinline__ D8 vap_enthalpy(const Params& P, int c, const D8& T) {
  D8 d = P.Tc[c] - T;
  if (d.v > 0.0) return P.hvr[c] * dpow(d, P.ev[c]);
  return dc(0.0);
}

__device__ void base_properties(const Params& P, const double* __restrict__ u, int i, double phi_ref, Base& b) {
  const int n = P.n;
  b.p = dvar(u[0 * n + i], 0);
  b.xlo = dvar(u[1 * n + i], 1);
  D8 yo2 = dvar(u[2 * n + i], 2);
  D8 yn2 = dvar(u[3 * n + i], 3);
  D8 yco2 = dvar(u[4 * n + i], 4);
  b.T = dvar(u[5 * n + i], 5);
  b.Sw = dvar(u[6 * n + i], 6);
  b.Sg = dvar(u[7 * n + i], 7);
  b.So = 1.0 - b.Sw - b.Sg;
  b.xho = 1.0 - b.xlo;
  const D8& p = b.p;
  const D8& T = b.T;
  // gas mole fractions: Tab4.4 with the modified PER (eq. PER1/PER2)
  b.y[0] = per_f(P, b.Sw) * k_value(P, 0, p, T);
  b.y[1] = k_value(P, 1, p, T) * b.xlo;
  b.y[2] = per_f(P, b.So) * k_value(P, 2, p, T) * b.xho;
  b.y[3] = yo2;
  b.y[4] = yn2;
  b.y[5] = yco2;
  // Redlich-Kwong Z factor with the mixing rule: A = Oa p a^2 / T^2.5, B = Ob p b / T
  D8 am = dc(0.0), bm = dc(0.0), ym = dc(0.0), ysq = dc(0.0);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    am = am + b.y[c] * P.a_rk[c];
    bm = bm + b.y[c] * P.b_rk[c];
    ym = ym + b.y[c] * P.M[c];
    ysq = ysq + b.y[c] * P.sqM[c];
  }
  D8 T25 = dpow(T, 2.5);
  D8 A = OMEGA_A * p * (am * am) / T25;
  D8 B = OMEGA_B * p * bm / T;
  double a1 = A.v - B.v - B.v * B.v;
  double a0 = -A.v * B.v;
  double z = cubic_root(a1, a0);
  double fz = (3.0 * z - 2.0) * z + a1;
  D8 Z;
  Z.v = z;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    double da1 = A.d[k] - B.d[k] - 2.0 * B.v * B.d[k];
    double da0 = -(A.d[k] * B.v + A.v * B.d[k]);
    Z.d[k] = -(z * da1 + da0) / fz;
  }
  b.rho_g = p / (Z * (R_GAS * T));
  // liquid densities (exponential correlation) and harmonic oil mixing
  D8 dp = p - P.p_ref;
  D8 dT = T - P.T_ref;
  b.rho_w = liquid_rho(P, 0, dp, dT);
  D8 rho_lo = liquid_rho(P, 1, dp, dT);
  D8 rho_ho = liquid_rho(P, 2, dp, dT);
  b.rho_o = 1.0 / (b.xlo / rho_lo + b.xho / rho_ho);
  // viscosities: liquids avisc e^{bvisc/T}, oil log-mixing, gas sqrt(M)-weighted
  D8 invT = 1.0 / T;
  D8 mu_w = dexp(P.ln_avisc[0] + P.bvisc[0] * invT);
  D8 mu_o = dexp(b.xlo * (P.ln_avisc[1] + P.bvisc[1] * invT) + b.xho * (P.ln_avisc[2] + P.bvisc[2] * invT));
  D8 lnT = dlog(T);
  D8 num = dc(0.0);
#pragma unroll
  for (int c = 0; c < 6; ++c) num = num + (P.avg[c] * P.sqM[c]) * (dexp(P.bvg[c] * lnT) * b.y[c]);
  D8 mu_g = num / ysq;
  // relative permeabilities: Corey (exponent 2) and Stone II with k_rocw = 1
  D8 krw = clamp01((b.Sw - P.Swc) / (1.0 - P.Swc - P.Sorw));
  krw = krw * krw;
  D8 krow = clamp01((1.0 - b.Sw - P.Sorw) / (1.0 - P.Swc - P.Sorw));
  krow = krow * krow;
  D8 krg = clamp01((b.Sg - P.Sgc) / (1.0 - P.Swc - P.Sgc));
  krg = krg * krg;
  D8 krog = clamp01((1.0 - b.Sg - P.Swc - P.Sorg) / (1.0 - P.Swc - P.Sorg));
  krog = krog * krog;
  D8 kro = (krow + krw) * (krog + krg) - krw - krg;
  if (kro.v < 0.0) kro = dc(0.0);
  b.lam[0] = b.rho_w * krw / mu_w;
  b.lam[1] = b.rho_o * kro / mu_o;
  b.lam[2] = b.rho_g * krg / mu_g;
  // enthalpies and internal energies
  D8 Hg[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) Hg[c] = gas_enthalpy(P, c, T);
  b.H[0] = Hg[0] - vap_enthalpy(P, 0, T);
  b.H[1] = b.xlo * (Hg[1] - vap_enthalpy(P, 1, T)) + b.xho * (Hg[2] - vap_enthalpy(P, 2, T));
  D8 hg = dc(0.0);
#pragma unroll
  for (int c = 0; c < 6; ++c) hg = hg + b.y[c] * Hg[c];
  b.H[2] = hg;
  b.U[0] = b.H[0] - p / b.rho_w;
  b.U[1] = b.H[1] - p / b.rho_o;
  b.U[2] = b.H[2] - p / b.rho_g;
  // porosity and solid energies
  D8 dpr = p - P.rock_p_ref;
  D8 dTr = T - P.rock_T_ref;
  b.phi = phi_ref * (1.0 + P.cpor * dpr - P.ctpor * dTr + P.cptpor * (dpr * dTr));
  b.Ur = P.cv1 * dTr + (0.5 * P.cv2) * (T * T - P.rock_T_ref * P.rock_T_ref);
  b.Uc = P.coke_cp * (T - P.T_ref);
  // specific weights
  b.gam[0] = b.rho_w * (P.M[0] * P.gravity);
  b.gam[1] = b.rho_o * (b.xlo * P.M[1] + b.xho * P.M[2]) * P.gravity;
  b.gam[2] = b.rho_g * ym * P.gravity;
}

// Arrhenius rate of reaction r (value and u-derivatives) at coke C (dual).
__device__ __forceinline__ D8 rate(const Params& P, int r, const Base& b, const D8& kT, const D8& phif, const D8& C) {
  D8 pO2 = b.y[3] * b.p;
  int kind = P.kind[r];
  if (kind == ISC_RXN_OIL_OXIDATION) {
    const D8& x = (P.comp[r] == 1) ? b.xlo : b.xho;
    return kT * pO2 * (phif * b.So * b.rho_o * x);
  } else if (kind == ISC_RXN_CRACKING) {
    const D8& x = (P.comp[r] == 1) ? b.xlo : b.xho;
    D8 q = C / P.coke_max;
    D8 q2 = q * q;
    D8 lim = 1.0 - q2 * q2 * q;
    return kT * (phif * b.So * b.rho_o * x) * lim;
  }
  return kT * pO2 * C;
}

// Solve the per-cell backward-Euler coke equation g(C) = C - C^n - dt sum_R s_R r_R(C) = 0
// by Newton on values, then dC/du = -(dg/du)/(dg/dC) at the root.
__device__ D8 solve_coke(const Params& P, const Base& b, const D8* kT, double C_old, int* dstatus) {
  const double dt = P.dt;
  double C = C_old;
  double pO2 = b.y[3].v * b.p.v;
  double oil = b.So.v * b.rho_o.v;
  bool ok = false;
  double dg = 1.0;
  for (int it = 0; it < 60; ++it) {
    double phif = b.phi.v - C / P.coke_rho;
    double g = C - C_old;
    dg = 1.0;
    for (int r = 0; r < P.nr; ++r) {
      double s = P.stoich[r][6];
      if (s == 0.0) continue;
      double k = kT[r].v;
      int kind = P.kind[r];
      double x = (P.comp[r] == 1) ? b.xlo.v : b.xho.v;
      double rt, drt;
      if (kind == ISC_RXN_OIL_OXIDATION) {
        rt = k * pO2 * (phif * oil * x);
        drt = k * pO2 * (-1.0 / P.coke_rho) * oil * x;
      } else if (kind == ISC_RXN_CRACKING) {
        double q = C / P.coke_max;
        double q4 = q * q * q * q;
        double lim = 1.0 - q4 * q;
        double conc = phif * oil * x;
        rt = k * conc * lim;
        drt = k * ((-1.0 / P.coke_rho) * oil * x * lim + conc * (-5.0 * q4 / P.coke_max));
      } else {
        rt = k * pO2 * C;
        drt = k * pO2;
      }
      g -= dt * s * rt;
      dg -= dt * s * drt;
    }
    double step = g / dg;
    C -= step;
    if (fabs(step) <= 1e-14 * (fabs(C) + fabs(C_old) + 1e-300)) {
      ok = true;
      break;
    }
  }
  if (!ok || !isfinite(C)) atomicOr(dstatus, DS_COKE);
  // u-derivative of g at fixed C
  D8 Cc = dc(C);
  D8 phif = b.phi - C / P.coke_rho;
  D8 gd = dc(0.0);
  for (int r = 0; r < P.nr; ++r) {
    double s = P.stoich[r][6];
    if (s == 0.0) continue;
    gd = gd - (dt * s) * rate(P, r, b, kT[r], phif, Cc);
  }
  D8 out;
  out.v = C;
#pragma unroll
  for (int k = 0; k < 8; ++k) out.d[k] = -gd.d[k] / dg;
  return out;
}


// Rate of reaction r and its derivative with respect to the coke C at fixed
// cell unknowns (values; the same terms as dg/dC of the coke equation).
__device__ __forceinline__ void rate_dC(const Params& P, int r, const Base& b, double kT, double C, double* rt,
                                        double* drt) {
  const double pO2 = b.y[3].v * b.p.v;
  const double oil = b.So.v * b.rho_o.v;
  const double phif = b.phi.v - C / P.coke_rho;
  const double x = (P.comp[r] == 1) ? b.xlo.v : b.xho.v;
  const int kind = P.kind[r];
  if (kind == ISC_RXN_OIL_OXIDATION) {
    *rt = kT * pO2 * (phif * oil * x);
    *drt = kT * pO2 * (-1.0 / P.coke_rho) * oil * x;
  } else if (kind == ISC_RXN_CRACKING) {
    double q = C / P.coke_max;
    double q4 = q * q * q * q;
    double lim = 1.0 - q4 * q;
    double conc = phif * oil * x;
    *rt = kT * conc * lim;
    *drt = kT * ((-1.0 / P.coke_rho) * oil * x * lim + conc * (-5.0 * q4 / P.coke_max));
  } else {
    *rt = kT * pO2 * C;
    *drt = kT * pO2;
  }
}

// Oil mass (LO + HO, any phase) leaving through a BHP producer perforation
// per second, Peaceman rates (Sec. 2.2 Well Modeling), outflow only.
// Phase rates of a coupled producer's perforation (Sec. 2.2, Well Modeling):
// Q_a = WI lambda_a (bhp - p - gamma_a (zref - z)) where that is negative
// (outflow, on[a]), else zero; dQ[a] = dQ_a / d bhp.
__device__ __forceinline__ void coupled_producer_rates(const Base& b, double WI, double bhp, double zref, double zi,
                                                       D8 (&Q)[3], double (&dQ)[3], bool (&on)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const D8 dphi = bhp - b.p - b.gam[a] * (zref - zi);
    on[a] = dphi.v < 0.0;
    if (on[a]) {
      Q[a] = (WI * b.lam[a]) * dphi;
      dQ[a] = WI * b.lam[a].v;
    } else {
      Q[a] = dc(0.0);
      dQ[a] = 0.0;
    }
  }
}

// Molar rate of the injected stream at a coupled injector's perforation:
// Q = WI lambda_T (bhp - p - gamma (zref - z)) where that is positive (inflow),
// lambda_T the cell's total molar mobility and gamma the injected phase's
// specific weight; *flows and *dQ = dQ / d bhp (zero when not flowing).
__device__ __forceinline__ D8 coupled_injector_rate(const Base& b, double WI, double bhp, double zref, double zi,
                                                    int phase, bool* flows, double* dQ) {
  const D8 lamT = b.lam[0] + b.lam[1] + b.lam[2];
  const D8 dphi = bhp - b.p - b.gam[phase] * (zref - zi);
  *flows = dphi.v > 0.0;
  *dQ = *flows ? WI * lamT.v : 0.0;
  return (WI * lamT) * dphi;
}

// Oil mass rate (LO + HO carried by the oil and gas phases, kg/s, positive
// when produced) of a perforation's phase rates Q (negative = outflow).
__device__ __forceinline__ D8 oil_of_rates(const Params& P, const Base& b, const D8 (&Q)[3]) {
  D8 mo = P.M[1] * b.xlo + P.M[2] * b.xho;
  D8 mg = P.M[1] * b.y[1] + P.M[2] * b.y[2];
  return -(Q[1] * mo + Q[2] * mg);
}

__device__ __forceinline__ D8 oil_production(const Params& P, const Base& b, double WI, double bhp) {
  D8 dpw = bhp - b.p;
  if (!(dpw.v < 0.0)) return dc(0.0);
  D8 Qo = (WI * b.lam[1]) * dpw;
  D8 Qg = (WI * b.lam[2]) * dpw;
  D8 mo = P.M[1] * b.xlo + P.M[2] * b.xho;
  D8 mg = P.M[1] * b.y[1] + P.M[2] * b.y[2];
  return -(Qo * mo + Qg * mg);
}

}  // namespace
}  // namespace isc
