/*
 * isc.h -- C ABI of the GB300 in-situ-combustion Newton step library (libisc).
 *
 * The library implements the Newton linearise-and-solve step of the fully
 * implicit FDM in-situ-combustion model of He, Yang, Liu and Chen,
 * "A New In-Situ Combustion Simulator for Parallel Computers" (arXiv 1811.11992):
 *   property evaluation (Sec. 2.2), residual and analytical Jacobian on the
 *   7-point stencil (Sec. 3.1), Gauss-Jordan decoupling (Sec. 3.2) and the
 *   preconditioned Krylov solve of the resulting block-sparse system.
 *
 * Conventions
 *   - All reals are double, SI units (Pa, K, m, s, mol, J, kg/mol, Pa*s).
 *   - All indices are int32_t. Cell id = i + nx*(j + ny*k).
 *   - Components: 0 W, 1 LO, 2 HO, 3 O2, 4 N2, 5 CO2; coke is species 6 in
 *     stoichiometry rows.
 *   - Primary unknowns per cell (natural variables of Tab:nco&ncg with x_HO
 *     and C_c eliminated locally): u = (p, x_LO, y_O2, y_N2, y_CO2, T, S_w, S_g).
 *   - Equation rows per cell: mass W, LO, HO, O2, N2, CO2, energy, gas
 *     constraint sum(y) - 1.
 *   - "SoA state" means u[k*N + cell], k = 0..7.
 *   - "block-major vector" means v[cell*8 + k].
 *   - BSR: rowptr[N+1], col[nnzb] sorted per row, val[nnzb*64] with block b
 *     stored row-major: val[b*64 + r*8 + c] = dF_r(row cell)/du_c(col cell).
 *   - Host pointers are read during the call and not retained: arrays passed
 *     to isc_create are copied; the handle owns all device memory it uses.
 *   - Every function returns ISC_OK (0) or a negative ISC_ERR_* code; no C++
 *     exception crosses the ABI. After an error the handle stays valid and
 *     isc_last_error() describes it.
 *   - All GPU work of a handle is issued on the stream given in isc_options
 *     (NULL = the legacy default stream); calls that return host data
 *     synchronise that stream before returning.
 */
#ifndef ISC_H
#define ISC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The opaque simulator handle (owns every device allocation; see isc_create). */
struct isc_handle;

#define ISC_NC 6          /* fluid components */
#define ISC_NU 8          /* unknowns (and equations) per cell */
#define ISC_MAX_RXN 8

enum isc_status {
  ISC_OK = 0,
  ISC_ERR_INVALID_ARG = -1,
  ISC_ERR_CUDA = -2,
  ISC_ERR_NOMEM = -3,
  ISC_ERR_SINGULAR_BLOCK = -4,  /* zero pivot in Gauss-Jordan or ILU(0) */
  ISC_ERR_KRYLOV_NOCONV = -5,
  ISC_ERR_NEWTON_NOCONV = -6,
  ISC_ERR_NONFINITE = -7,
  ISC_ERR_COKE = -8,            /* per-cell coke equation did not converge */
  ISC_ERR_TIMEOUT = -9,         /* a bounded device-side wait gave up */
  ISC_ERR_UNIMPLEMENTED = -10,
  ISC_ERR_STATE = -11           /* call order violated (e.g. solve before assemble) */
};

enum isc_krylov { ISC_KRYLOV_GMRES = 0, ISC_KRYLOV_BICGSTAB = 1 };
/* ISC_PREC_CPR is the two-stage CPR-PF preconditioner of Sec. 4 (Example 2):
 * on the decoupled system, one V-cycle of an aggregation multigrid on the
 * pressure matrix (the (0,0) entry of every block: 2x2 x-y aggregates with
 * Galerkin coarse operators, red-black z-line Gauss-Seidel, one pre- and one
 * post-smoothing sweep), then block ILU(0) on the remaining residual; the
 * ILU(0) stage follows options.precision. It expects options.decouple = 1. */
enum isc_prec { ISC_PREC_NONE = 0, ISC_PREC_BJACOBI = 1, ISC_PREC_BILU0 = 2, ISC_PREC_CPR = 3 };
/* Precision of the linear solve.
 * ISC_PRECISION_FP64: FP64 throughout.
 * ISC_PRECISION_MIXED: the block ILU(0) factors are computed, stored and applied
 *   in FP32 (from an FP32 copy of the decoupled blocks; under CPR-PF the pressure
 *   multigrid too) inside the FP64 GMRES (residual, SpMV, orthogonalisation and
 *   update stay FP64).
 * ISC_PRECISION_MIXED_FGMRES: the FP64 GMRES is flexible and its preconditioner
 *   is options.inner_its iterations of an FP32 GMRES on the FP32 copy of the
 *   decoupled matrix (FP32 SpMV, FP32 Gram-Schmidt, FP32 block ILU(0), or
 *   CPR-PF with the FP32 pressure multigrid); the outer residual, SpMV,
 *   orthogonalisation and update stay FP64. Requires krylov = GMRES and
 *   prec = BILU0 or CPR. */
enum isc_precision { ISC_PRECISION_FP64 = 0, ISC_PRECISION_MIXED = 1, ISC_PRECISION_MIXED_FGMRES = 2 };
/* Orthogonalisation of the FP64 GMRES basis (the paper leaves it open).
 * ISC_ORTH_CGS2: classical Gram-Schmidt applied twice (three passes over the
 *   basis per iteration; orthogonal to working precision).
 * ISC_ORTH_CGS1: classical Gram-Schmidt once (two passes; half the FP64 work
 *   of CGS2, which on GB300's narrow FP64 pipe is the bound). The basis may
 *   lose orthogonality on ill-conditioned Krylov spaces; the solver still
 *   recomputes the true residual before it reports convergence. */
enum isc_orth { ISC_ORTH_CGS2 = 0, ISC_ORTH_CGS1 = 1 };
enum isc_rxn_kind {
  ISC_RXN_OIL_OXIDATION = 0,   /* r = A e^{-Ea/RT} (y_O2 p)(phi_f S_o rho_o x_i)           */
  ISC_RXN_CRACKING = 1,        /* r = A e^{-Ea/RT} (phi_f S_o rho_o x_i)(1-(C_c/C_max)^5)  */
  ISC_RXN_COKE_OXIDATION = 2   /* r = A e^{-Ea/RT} (y_O2 p) C_c                            */
};
enum isc_well_kind {
  ISC_WELL_RATE_INJECTOR = 0, ISC_WELL_BHP_PRODUCER = 1, ISC_WELL_COUPLED_PRODUCER = 2, ISC_WELL_COUPLED_INJECTOR = 3
};
/* Controls of a coupled producer: ISC_CTRL_BHP fixes the bottom-hole pressure
 * (target in Pa); otherwise the bits select the phases (1 water, 2 oil, 4 gas)
 * whose summed molar production rate (mol/s, positive out of the reservoir)
 * is fixed at target. A coupled injector takes ISC_CTRL_BHP or
 * ISC_CTRL_TOTAL_RATE (the injected molar rate, mol/s, positive into the
 * reservoir); other controls are ISC_ERR_INVALID_ARG. */
enum isc_well_control {
  ISC_CTRL_BHP = 0, ISC_CTRL_WATER_RATE = 1, ISC_CTRL_OIL_RATE = 2, ISC_CTRL_LIQUID_RATE = 3,
  ISC_CTRL_GAS_RATE = 4, ISC_CTRL_TOTAL_RATE = 7
};

/* Cartesian grid (Sec. 3.1). depth: N cell-centre depths in m (increasing
 * downwards), or NULL for depth = (k + 0.5) dz. */
typedef struct isc_grid {
  int32_t nx, ny, nz;
  double dx, dy, dz;
  const double* depth;
} isc_grid;

/* Rock (Sec. 2.2 Porosity, Non-isothermal Description). phi_ref: N values.
 * perm: 3N values, k_x of all cells, then k_y, then k_z (m^2).
 * phi = phi_ref (1 + cpor (p-p_ref) - ctpor (T-T_ref) + cptpor (p-p_ref)(T-T_ref)),
 * U_r = cv1 (T-T_ref) + cv2/2 (T^2 - T_ref^2) in J/m^3, K_rock in W/m/K. */
typedef struct isc_rock {
  const double* phi_ref;
  const double* perm;
  double cpor, ctpor, cptpor, p_ref, T_ref, cv1, cv2, K_rock;
} isc_rock;

/* Fluid data (Sec. 2.2), SI, T absolute. Arrays [6] are per component,
 * arrays [3] are per liquid-capable component (W, LO, HO).
 *   K-values: K = (kv1/p + kv2 p + kv3) exp(kv4/(T-kv5)), kv[c] = {kv1..kv5}
 *   liquid density: rho = rho_ref exp(cp dp - ct1 dT - ct2/2 dT^2 + cpt dp dT),
 *                   dp = p - p_ref, dT = T - T_ref
 *   gas enthalpy: H_g,c = int_{T_ref}^T sum_k cpg[c][k] t^k dt
 *   vaporisation: H_v,c = hvr (Tc - T)^ev for T < Tc (Tc from Tc[c]), else 0
 *   viscosities: mu_c = avisc exp(bvisc/T) (liquids), mu_g,c = avg T^bvg
 *   Corey endpoints Swc, Sorw, Sgc, Sorg (exponent 2), PER epsilon per_eps. */
typedef struct isc_fluid {
  double M[6], pc[6], Tc[6];
  double rho_ref[3], cp[3], ct1[3], ct2[3], cpt[3];
  double p_ref, T_ref;
  double cpg[6][4];
  double hvr[3], ev[3];
  double avg[6], bvg[6], avisc[3], bvisc[3];
  double kv[3][5];
  double K_phase[3];            /* thermal conductivity of water, oil, gas phases */
  double coke_rho, coke_cp, coke_K, coke_M;
  double Swc, Sorw, Sgc, Sorg;
  double per_eps, gravity;
} isc_fluid;

/* Reactions (Sec. 2.1 Chemical Reaction, Sec. 2.2 Reaction Model).
 * stoich[r][0..6]: coefficients of W, LO, HO, O2, N2, CO2, coke (products
 * positive). comp[r]: the oil component (1 LO or 2 HO) of oxidation/cracking
 * rates. Validated: |sum_c stoich[r][c] M_c| <= 1e-12 sum_c |stoich[r][c]| M_c
 * (the paper's N M = 0 check), else ISC_ERR_INVALID_ARG. */
typedef struct isc_reactions {
  int32_t nr;
  int32_t kind[ISC_MAX_RXN];
  int32_t comp[ISC_MAX_RXN];
  double stoich[ISC_MAX_RXN][7];
  double A[ISC_MAX_RXN], Ea[ISC_MAX_RXN], dH[ISC_MAX_RXN];
  double coke_max;
} isc_reactions;

/* Wells (Sec. 2.2 Well Modeling). A BHP producer perforation at cell i takes
 * Q_alpha = WI rho_alpha k_r,alpha/mu_alpha (bhp - p_i) when p_i > bhp (no
 * cross-flow). A rate injector puts target mol/s of composition inj_y at
 * T_inj, split over its perforations in proportion to WI; inj_phase 2 carries
 * gas enthalpy, inj_phase 0 liquid-water enthalpy. A coupled producer has
 * its bottom-hole pressure bhp, defined at depth ref_depth, as an unknown and
 * one well equation (control, target; see isc_well_control); its perforation
 * at cell i takes Q_alpha = WI lambda_alpha (bhp - p_i - gamma_alpha (ref_depth
 * - z_i)) per phase when that is negative (gamma_alpha the phase's specific
 * weight in the cell), and bhp starts at bhp_init. A coupled injector has the
 * same unknown and equation; its perforation at cell i takes the stream inj_y
 * (molar enthalpy at inj_T as for a rate injector) at Q = WI lambda_T (bhp -
 * p_i - gamma (ref_depth - z_i)) mol/s when that is positive (lambda_T the
 * cell's total molar mobility, gamma the specific weight of the injected
 * phase: gas, or water for inj_phase 0); at a Newton iterate where no
 * perforation flows, a rate-controlled injector's well row is zero and the
 * linear solve returns ISC_ERR_NONFINITE (the preconditioner's well row
 * divides by D_w = 0). A cell
 * may be perforated by at most one well. */
typedef struct isc_well {
  int32_t kind;
  int32_t n_perf;
  const int32_t* cells;
  const double* WI;
  double target;
  double inj_y[6];
  double inj_T;
  int32_t inj_phase;
  int32_t control;    /* coupled well: isc_well_control */
  double ref_depth;   /* coupled well: depth of the bottom-hole pressure (m) */
  double bhp_init;    /* coupled well: initial bottom-hole pressure (Pa) */
} isc_well;

typedef struct isc_wells {
  int32_t nw;
  const isc_well* wells;
} isc_wells;

/* Solver and Newton options. stream is a cudaStream_t (NULL = default). */
typedef struct isc_options {
  int32_t krylov;               /* isc_krylov */
  int32_t restart;              /* GMRES restart length, 1..64 */
  int32_t prec;                 /* isc_prec */
  int32_t decouple;             /* 1: Gauss-Jordan decoupling before the solve */
  double tol_lin;               /* relative residual of the (decoupled) system */
  int32_t maxit_lin;
  double tol_newton;            /* scaled residual norm */
  int32_t maxit_newton;
  double max_dp_frac;           /* |dp| <= max_dp_frac p (0.2) */
  double max_dT;                /* |dT| <= max_dT (50 K) */
  int32_t profile;              /* 1: record per-kernel CUDA-event times */
  int32_t precision;            /* isc_precision (applies to ISC_PREC_BILU0; MIXED also to CPR) */
  void* stream;
  int32_t inner_its;            /* ISC_PRECISION_MIXED_FGMRES: FP32 GMRES iterations per outer one, 1..32 (10) */
  int32_t orth;                 /* isc_orth of the FP64 GMRES (default CGS2) */
} isc_options;

typedef struct isc_newton_info {
  int32_t status;
  int32_t converged;            /* 1 if the residual was already below tol (no solve done) */
  double norm;                  /* scaled residual norm before the step */
  double norm_mass, norm_energy, norm_gs;
  int32_t krylov_iterations;
  double krylov_rel_residual;
} isc_newton_info;

typedef struct isc_step_info {
  int32_t status;
  int32_t newton_iterations;
  int32_t krylov_iterations;
  double final_norm;
} isc_step_info;

/* Per-kernel-class timing (milliseconds, CUDA events on the handle's stream,
 * accumulated while options.profile = 1) and launch counts. */
enum isc_kernel_class {
  ISC_K_PROPS = 0, ISC_K_FLUX = 1, ISC_K_NORM = 2, ISC_K_GJ = 3, ISC_K_ILU_FACTOR = 4,
  ISC_K_SPMV = 5, ISC_K_PREC_APPLY = 6, ISC_K_BLAS1 = 7, ISC_K_UPDATE = 8, ISC_K_ADJOINT = 9,
  ISC_K_CPR = 10,   /* CPR pressure stage: extraction and coarsening, V-cycle, second-stage residual */
  ISC_K_SPMV32 = 11, /* FP32 SpMV of the inner solve (ISC_PRECISION_MIXED_FGMRES) */
  ISC_K_COUNT = 12
};
typedef struct isc_stats {
  double ms[ISC_K_COUNT];
  int64_t launches[ISC_K_COUNT];
  int64_t calls[ISC_K_COUNT];   /* timed regions (one region may hold several launches) */
} isc_stats;

/* ---------------------------------------------------------------- lifecycle */

/* Create a handle: validates the input, precomputes face transmissibilities
 * (harmonic average of A k/h, Sec. 3.1) and the BSR pattern of the 7-point
 * stencil (fixed, Sec. 3.1 end), allocates device memory. opts may be NULL
 * for defaults (GMRES(30), block ILU(0), decoupling on, tol_lin 1e-6,
 * tol_newton 1e-6). *out receives the handle or NULL on error. */
int isc_create(const isc_grid* grid, const isc_rock* rock, const isc_fluid* fluid,
               const isc_reactions* reactions, const isc_wells* wells,
               const isc_options* opts, struct isc_handle** out);
void isc_destroy(struct isc_handle* h);
int isc_set_options(struct isc_handle* h, const isc_options* opts);
void isc_default_options(isc_options* opts);
const char* isc_status_string(int status);
const char* isc_last_error(const struct isc_handle* h);
int32_t isc_num_cells(const struct isc_handle* h);
int32_t isc_nnzb(const struct isc_handle* h);

/* Heat loss to the overburden and underburden (Sec. 2.1, the last term of the
 * energy equation, Q_loss = A K_ob ((T(ob) - T_ini)/d - rho); it enters the
 * discrete energy residual of Sec. 3.1 as an outflow). Reading: every cell of
 * the top layer (k = 0, faces bit 1) and / or of the bottom layer (k = nz - 1,
 * faces bit 2) loses A K_ob ((T - T_ini)/d - rho) watts through its horizontal
 * face (A = dx dy) by conduction into a confining layer of thickness d (m,
 * > 0) and conductivity K_ob (W/m/K, >= 0) whose far side stays at T_ini (K);
 * T(ob), the interface temperature, is the cell's temperature and rho (K/m)
 * the paper's fitted offset. faces = 0 (the default at isc_create) switches
 * it off. Takes effect at the next assembly. ISC_ERR_INVALID_ARG on
 * non-finite or out-of-range values. */
int isc_set_heat_loss(struct isc_handle* h, double K_ob, double d, double T_ini, double rho, int32_t faces);

/* ---------------------------------------------------------------- state */

/* Initial-state recipe: uniform p0, T0, S_w0, S_o0 (S_g = 1 - S_w0 - S_o0),
 * x_LO0; gas y_W = f(S_w)K_W, y_LO = K_LO x_LO, y_HO = f(S_o)K_HO x_HO
 * (Tab4.4 with eq. PER1/PER2) and the remainder split over O2, N2, CO2 in the
 * ratios y_rest[3]; n_ignited cells start at T_ignite; C_c = 0. Also makes
 * this the accepted state of the time step (see isc_begin_step). */
int isc_init_equilibrium(struct isc_handle* h, double p0, double T0, double Sw0, double So0,
                         double x_LO0, const double y_rest[3], int32_t n_ignited,
                         const int32_t* ignited, double T_ignite);
/* Copy in / out the Newton iterate u (host, SoA 8N) and coke C_c (host, N;
 * may be NULL on get). set_state does not touch the accepted state. */
int isc_set_state(struct isc_handle* h, const double* u, const double* coke);
int isc_get_state(struct isc_handle* h, double* u, double* coke);
/* Device-pointer variants (SoA 8N and N doubles in device memory), ordered on
 * the handle's stream, no synchronisation. */
int isc_set_state_device(struct isc_handle* h, const double* d_u, const double* d_coke);
int isc_get_state_device(struct isc_handle* h, double* d_u, double* d_coke);
/* Make the current iterate (u, C_c) the accepted state of time level n: stores
 * C_c^n and the accumulation N^n, E^n used by the next residuals (and the
 * coupled wells' bottom-hole pressures). */
int isc_begin_step(struct isc_handle* h);
/* Coupled wells (ISC_WELL_COUPLED_PRODUCER, ISC_WELL_COUPLED_INJECTOR), in the
 * order of the wells given at creation. With nwc > 0 the Newton system is bordered: unknowns
 * (u, bhp), equations (F, F_w); Krylov vectors, isc_spmv and
 * isc_precond_apply then have length 8N + nwc (the well entries last), and
 * the preconditioner is block lower-triangular (the cells' preconditioner,
 * then z_w = (r_w - C z) / D_w). Bottom-hole pressures in and out (host, nwc
 * doubles); set_well_bhp does not touch the accepted state. */
int32_t isc_num_coupled_wells(const struct isc_handle* h);
int isc_set_well_bhp(struct isc_handle* h, const double* bhp);
int isc_get_well_bhp(struct isc_handle* h, double* bhp);
/* After isc_assemble (before decoupling): the border of the Newton system,
 * for the coupled wells' perforations in creation order,
 * B[q*8 + r] = dF_r(cell of q)/d bhp, C[q*8 + k] = dF_w/du_k(cell of q), and
 * per coupled well D[w] = dF_w/d bhp_w and Fw[w] the well equation (host
 * arrays; any may be NULL). */
int isc_get_well_system(struct isc_handle* h, double* B, double* C, double* D, double* Fw);

/* ---------------------------------------------------------------- hot path */

/* Assemble the residual F (Sec. 3.1 discrete equations, outflow positive) and
 * its analytical Jacobian dF/du at the current iterate for step size dt. */
int isc_assemble(struct isc_handle* h, double dt);
/* Gauss-Jordan decoupling with partial pivoting of the assembled system
 * (Sec. 3.2): J <- C_L J, F <- C_L F with C_L = blockdiag(J_ii)^-1, done by
 * elementary row operations on each block row; the diagonal blocks become I.
 * ISC_ERR_SINGULAR_BLOCK on a zero pivot. */
int isc_decouple(struct isc_handle* h);
/* Solve J du = -F on the assembled (decoupled, if done) system with the
 * handle's Krylov method and preconditioner; du stays on the device. */
int isc_solve(struct isc_handle* h, isc_newton_info* info);
/* u <- u + du with the safeguards (|dp| <= max_dp_frac p, |dT| <= max_dT,
 * saturations and mole fractions that would turn negative are halved: the
 * 0.5 S rule of Sec. 2.2 Phase Equilibrium). */
int isc_update(struct isc_handle* h);
/* One Newton linearise-and-solve step: assemble, convergence test (returns
 * with info->converged = 1 if the scaled norm is below tol_newton), decouple,
 * precondition, Krylov solve, safeguarded update. */
int isc_newton_step(struct isc_handle* h, double dt, isc_newton_info* info);
/* One implicit-Euler time step: Newton until converged (at most
 * maxit_newton solves); on failure the accepted state is restored and
 * ISC_ERR_NEWTON_NOCONV (or the failing status) is returned; on success the
 * converged state becomes the accepted state. */
int isc_timestep(struct isc_handle* h, double dt, isc_step_info* info);

/* Result of isc_run. */
typedef struct isc_run_info {
  int32_t status;
  int32_t steps;                /* accepted time steps */
  int32_t cuts;                 /* step halvings after failed attempts */
  int32_t newton_iterations;    /* Newton solves, failed attempts included */
  int64_t krylov_iterations;    /* Krylov iterations, failed attempts included */
  double t;                     /* time reached, from 0 at the call's start (s) */
  double dt_next;               /* the controller's next step after the last one (s) */
} isc_run_info;

/* Time loop of the implicit-Euler scheme (Sec. 3.1) from the accepted state
 * (isc_init_equilibrium or the last accepted step; the handle keeps no clock,
 * so time runs from 0 to t_end here). Each step tries dt = min(dt, t_end - t)
 * with isc_timestep; when that fails with ISC_ERR_NEWTON_NOCONV,
 * ISC_ERR_KRYLOV_NOCONV, ISC_ERR_NONFINITE, ISC_ERR_COKE or
 * ISC_ERR_SINGULAR_BLOCK the accepted state is restored and dt halves, at most
 * max_cuts times in a row (then that status is returned, with info->t the time
 * reached); any other error returns at once. After an accepted step of length
 * dt with largest changes dT = max |T_new - T_old| and
 * dS = max(|S_w,new - S_w,old|, |S_g,new - S_g,old|) over the cells, the next
 * step is min(dt * clamp(min(dT_target / dT, dS_target / dS), 0.5, 2), dt_max)
 * (dT and dS taken as at least 1e-12; the paper fixes no step controller:
 * the oracle's loop uses 20 K and 0.2). Stops at t_end or after
 * max_steps accepted steps. dt_history (may be NULL) receives the accepted
 * step lengths, room for max_steps doubles. Allocates 3N + 2 doubles of
 * device memory on its first call. Synchronous. ISC_ERR_INVALID_ARG for
 * t_end < 0, dt0, dt_max or a target not positive, max_cuts < 0 or
 * max_steps < 1; ISC_ERR_STATE before any accepted state. */
int isc_run(struct isc_handle* h, double t_end, double dt0, double dt_max, double dT_target, double dS_target,
            int32_t max_cuts, int32_t max_steps, double* dt_history, isc_run_info* info);

/* Replace the assembled system by a caller's one (the method's linear step of
 * Sec. 3.2 on given data): val, the nnzb*64 BSR blocks on the handle's 7-point
 * pattern (the rowptr and col that isc_get_jacobian_bsr returns), and F, the
 * block-major residual (8N); isc_solve then solves J du = -F. decoupled = 1
 * declares val already decoupled: every diagonal block must be exactly the
 * identity (checked; ISC_ERR_INVALID_ARG otherwise) and isc_decouple does
 * nothing; 0 gives an assembled system that isc_decouple will scale. Host
 * arrays, copied; the preconditioner must be rebuilt; the state is untouched.
 * Handles with coupled wells return ISC_ERR_UNIMPLEMENTED. Synchronous. */
int isc_set_system(struct isc_handle* h, const double* val, const double* F, int32_t decoupled);
/* Solve A x = b for a caller's BSR matrix with the handle's linear solver
 * (Gauss-Jordan decoupling of Sec. 3.2 if options.decouple, then the
 * preconditioned Krylov method and tolerance of the options). A is rowptr
 * (N+1), col (nnzb), val (nnzb*64) and must have the handle's 7-point pattern
 * (else ISC_ERR_INVALID_ARG: the preconditioner kernels depend on it); b and x
 * are block-major 8N host arrays. info (may be NULL) receives the Krylov
 * iterations and the achieved relative residual of the (decoupled) system. It
 * overwrites the handle's assembled system (isc_set_system with F = -b);
 * the state is untouched. Synchronous. */
int isc_solve_external(struct isc_handle* h, const int32_t* rowptr, const int32_t* col, const double* val,
                       const double* b, double* x, isc_newton_info* info);

/* ---------------------------------------------------------------- exports */

/* Residual F of the last assembly (host, block-major 8N), after decoupling
 * if isc_decouple ran. */
int isc_get_residual(struct isc_handle* h, double* F);
/* BSR Jacobian of the last assembly (after decoupling if it ran). rowptr
 * (N+1), col (nnzb), val (nnzb*64); any may be NULL. */
int isc_get_jacobian_bsr(struct isc_handle* h, int32_t* rowptr, int32_t* col, double* val);
/* Newton update du of the last isc_solve (host, block-major 8N). */
int isc_get_update(struct isc_handle* h, double* du);
/* Coke C_c solved during the last assembly (host, N). */
int isc_get_coke(struct isc_handle* h, double* coke);
/* y = A x with the handle's current BSR matrix (host, block-major 8N). */
int isc_spmv(struct isc_handle* h, const double* x, double* y);
/* z = M^-1 r with the preconditioner built by the last isc_solve or
 * isc_build_preconditioner (host, block-major 8N). */
int isc_build_preconditioner(struct isc_handle* h);
int isc_precond_apply(struct isc_handle* h, const double* r, double* z);
/* The inverted diagonal blocks D_i^-1 of the block ILU(0) factors built by the
 * last isc_build_preconditioner (or isc_solve), D-ILU form: D_i = A_ii -
 * sum_{k<i} A_ik D_k^-1 A_ki over the 7-point neighbours in natural order;
 * N*64 host doubles, row-major blocks (the FP32 factors of the mixed modes
 * converted exactly). ISC_ERR_STATE unless options.prec is BILU0 or CPR and
 * the preconditioner is built. */
int isc_get_ilu_diag(struct isc_handle* h, double* dinv);
int isc_get_stats(struct isc_handle* h, isc_stats* stats);
int isc_reset_stats(struct isc_handle* h);
/* Bytes of device memory the handle holds now: the arrays allocated by
 * isc_create (Jacobian blocks, state, staged face quantities, ILU factors,
 * the GMRES basis of options.restart + 1 vectors) and the workspaces
 * allocated on first use (FP32 preconditioner copies and inner FP32 GMRES
 * basis of the mixed modes, CPR multigrid levels, adjoint checkpoints), as
 * requested from cudaMalloc (the allocator's rounding not included). Excludes
 * the CUDA context, module code and pinned host memory. Host-only: launches
 * nothing. ISC_ERR_INVALID_ARG on a null pointer. */
int isc_get_device_bytes(struct isc_handle* h, uint64_t* bytes);

/* ---------------------------------------------------------------- kernels */

/* y = A x for a BSR matrix with 8x8 FP64 blocks, all pointers in device
 * memory (x, y block-major), ordered on stream. unit_diag = 1 asserts the
 * diagonal blocks are the identity (as after decoupling) and skips them. */
int isc_bsr_spmv_device(int32_t nrows, const int32_t* d_rowptr, const int32_t* d_col,
                        const double* d_val, const double* d_x, double* d_y,
                        int32_t unit_diag, void* stream);

/* Allocation-free block ILU(0) apply, for callers that cannot allocate GPU
 * memory themselves (code running inside another framework's memory pool,
 * restricted hosts): z = (L U)^-1 r with the D-ILU factors of the 7-point
 * pattern on an nx*ny*nz grid. It is a variant of the preconditioner apply of
 * isc_precond_apply; the paper has no counterpart (its preconditioners come
 * from a CPU platform). Inputs and outputs are caller-owned device memory:
 * d_rowptr (N+1) and d_A (nnzb*64) in the BSR layout above, d_Dinv (N*64,
 * the inverted ILU(0) diagonal blocks, row-major), d_r and d_z (block-major 8N).
 * The call allocates nothing: its scratch (the forward-sweep vector and the
 * sweep counters) is a static device array sized for at most
 * ISC_NOALLOC_MAX_CELLS cells (about 4 MB, held by every GPU that loads the
 * library until the process exits). Larger grids return ISC_ERR_INVALID_ARG.
 * Every call resolves that array's device address with the caller's device
 * current. All calls share the one array, which keeps the previous call's
 * contents (the call clears what must start at zero), so calls that overlap on
 * the GPU (different streams or threads) race and must be serialised by the
 * caller. The call synchronises stream before it returns: ISC_ERR_TIMEOUT if a
 * device-side wait gave up, ISC_ERR_CUDA if a launch or copy failed. */
#define ISC_NOALLOC_MAX_CELLS 65536
int isc_bilu0_apply_noalloc(int32_t nx, int32_t ny, int32_t nz, const int32_t* d_rowptr, const double* d_A,
                            const double* d_Dinv, const double* d_r, double* d_z, void* stream);

/* Numerics self-check of the device reciprocal used for the pivots of the
 * Gauss-Jordan decoupling and of the block ILU(0) / block-Jacobi inverses
 * (Newton-Raphson from the hardware approximation): for n host doubles x,
 * y[i] = that reciprocal and z[i] = the device's 1.0 / x[i]. Host buffers,
 * allocated and freed inside (a diagnostic, not a hot-path call); synchronous
 * on the default stream. n < 0 or NULL pointers: ISC_ERR_INVALID_ARG. */
int isc_check_reciprocal(int32_t n, const double* x, double* y, double* z);

/* Roofline denominators measured on the current device (a diagnostic, not a
 * hot-path call): the FMA throughput of a register-resident loop of
 * independent FMA chains over every SM, best of five CUDA-event-timed runs,
 * returned in GFLOP/s (2 flops per FMA) for FP64 and FP32. The paper reports no
 * per-kernel throughput; these give the ALU roof of the FP64 kernels (on GB300
 * the FP64 pipe, not HBM, bounds a kernel above ~0.18 flop per byte). Either
 * pointer may be NULL to skip that precision. Allocates and frees a small
 * output buffer; default stream; synchronous (about 30 ms). */
int isc_measure_fma_rates(double* fp64_gflops, double* fp32_gflops);

/* Failure-detection self-test (no GPU fault): runs the ILU(0) forward sweep on a
 * 4x4x1 grid with its pencil counter started past pencil 0, so the neighbour
 * value pencil 1 waits for never arrives and the wait ends by its iteration
 * limit (a few seconds). Returns ISC_ERR_TIMEOUT when the kernel gave up and
 * reported it in its status word (the expected outcome; the CUDA context stays
 * usable), ISC_OK if the wait ended otherwise, ISC_ERR_NOMEM / ISC_ERR_CUDA on
 * allocation or copy failures. Allocates and frees its own buffers; default
 * stream; synchronous. */
int isc_check_bounded_wait(void);

/* Self-check of the index arithmetic of the ILU(0) sweeps and factorisation
 * (a diagnostic, not a hot-path call): those kernels compute the start of
 * each cell's BSR row of the 7-point pattern (columns sorted, one block per
 * existing neighbour and the diagonal) in closed form instead of loading it.
 * Given the nx x ny x nz grid and that pattern's rowptr (host, N + 1 int32,
 * copied), a kernel compares both closed forms with it for every cell, and the
 * total block count with rowptr[N]; *mismatches receives the number of cells
 * that differ and *first_cell the smallest of them (-1 if none). Synchronous,
 * allocates N + 1 ints of device memory for the call. ISC_ERR_INVALID_ARG for
 * an empty grid, a null pointer or a grid beyond the handle's limits. */
int isc_check_row_starts(int32_t nx, int32_t ny, int32_t nz, const int32_t* rowptr, int64_t* mismatches,
                         int32_t* first_cell);

/* ------------------------------------------------------------ sensitivities */

/* Parameters theta of the sensitivity analysis. The paper computes no
 * sensitivities; these calls differentiate its discrete equations (Sec. 3.1)
 * exactly.
 *   log_k  N host doubles: per-cell ln k multipliers m_i. The permeabilities
 *          become k_d,i = k_d,i(create) exp(m_i) for d = x, y, z, so the
 *          harmonic face transmissibilities change, and so does the well index
 *          of a perforation in cell i, WI_i(create) exp(m_i) (Peaceman WI is
 *          linear in k). A rate injector's perforation shares WI_i / sum WI
 *          follow. All zero at creation.
 *   Ea     nr host doubles: activation energies E_a (J/mol) of the reactions.
 *   lnA    nr host doubles: ln of the pre-exponential factors A.
 * A NULL pointer leaves that group unchanged. The arrays are copied; the call
 * synchronises the handle's stream. Non-finite values: ISC_ERR_INVALID_ARG. */
int isc_set_parameters(struct isc_handle* h, const double* log_k, const double* Ea, const double* lnA);
/* The current parameters (NULL skips a group). */
int isc_get_parameters(struct isc_handle* h, double* log_k, double* Ea, double* lnA);

typedef struct isc_adjoint_spec {
  int32_t n_steps;           /* implicit-Euler steps of the time loop, >= 1 */
  const double* dt;          /* host [n_steps] step sizes (s); the sequence is frozen (no step cutting) */
  int32_t checkpoint_every;  /* states kept on the device every this many steps; the reverse sweep
                                recomputes each segment from its checkpoint (>= 1) */
  double tol_adjoint;        /* relative residual of every transposed linear solve (0: options.tol_lin) */
} isc_adjoint_spec;

typedef struct isc_adjoint_info {
  int32_t status;
  int32_t newton_iterations;          /* forward and recomputed steps */
  int32_t krylov_iterations_forward;  /* Krylov iterations of those Newton solves */
  int32_t krylov_iterations_adjoint;  /* Krylov iterations of the transposed solves */
  int32_t recomputed_steps;
  double loss;
  double adjoint_rel_residual;        /* largest final relative residual of a transposed solve */
} isc_adjoint_info;

/* Discrete adjoint of the time loop. From the handle's accepted state (after
 * isc_init_equilibrium or a converged isc_timestep) the call runs the
 * spec->n_steps implicit-Euler steps with Newton as isc_timestep does (the
 * handle's options), and evaluates the loss
 *     L = sum_n dt_n sum_{producer perforations} (M_LO (Q_o x_LO + Q_g y_LO)
 *                                                 + M_HO (Q_o x_HO + Q_g y_HO))
 * the cumulative LO + HO mass (kg) produced in any phase at the converged
 * states (Peaceman rates of Sec. 2.2, outflow only; fixed-BHP producers and
 * coupled producers, the latter at their converged bottom-hole pressures). If
 * any gradient pointer is non-NULL it then sweeps the steps backwards: per
 * step one transposed linear solve J_n^T lambda_n = ubar_n with the
 * preconditioned Krylov method of the options (the transposed blocks are
 * decoupled and factored like J; with coupled wells the transposed bordered
 * system, whose well rows carry dL/d bhp and whose multipliers weight the well
 * equations' ln k terms), the coke equation entering through the
 * implicit-function theorem, and accumulates
 *   g_log_k  N host doubles  dL/d log_k (as set by isc_set_parameters),
 *   g_Ea     nr host doubles dL/dE_a (per J/mol),
 *   g_lnA    nr host doubles dL/d ln A.
 * Each may be NULL. States are kept every spec->checkpoint_every steps
 * ((ceil(n_steps/K) + K + 2) x (9N + nwc) doubles of device memory, allocated
 * on first use and kept with the handle) and recomputed bit-exactly during the reverse
 * sweep. loss (may be NULL) and info->loss receive L. On success the handle is
 * at the final state of the loop. A step that does not converge returns
 * ISC_ERR_NEWTON_NOCONV (the handle keeps its last accepted state); a
 * transposed solve that misses tol_adjoint returns ISC_ERR_KRYLOV_NOCONV. */
int isc_adjoint(struct isc_handle* h, const isc_adjoint_spec* spec, double* loss, double* g_log_k,
                double* g_Ea, double* g_lnA, isc_adjoint_info* info);

/* The two halves of isc_adjoint, for callers that want the loss now and its
 * gradient later (the backward pass of an automatic-differentiation framework).
 * isc_adjoint_forward runs the time loop exactly as isc_adjoint does, returns
 * L and keeps the checkpoints on the device; it computes no gradient.
 * isc_adjoint_backward then runs the reverse sweep over those checkpoints
 * (recomputing each segment), writes the gradients like isc_adjoint (any
 * pointer may be NULL) and leaves the handle at the loop's final state; it
 * may be repeated. ISC_ERR_STATE if no forward sweep is stored, or if
 * isc_set_parameters, isc_set_options or isc_set_heat_loss changed the model
 * since (a forward sweep must then be run again). The step sizes, checkpoint
 * interval and tol_adjoint of the forward's spec are kept with the store. */
int isc_adjoint_forward(struct isc_handle* h, const isc_adjoint_spec* spec, double* loss, isc_adjoint_info* info);
int isc_adjoint_backward(struct isc_handle* h, double* g_log_k, double* g_Ea, double* g_lnA, isc_adjoint_info* info);

#ifdef __cplusplus
}
#endif

#endif /* ISC_H */
