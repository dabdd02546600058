// Internal declarations of libisc (GB300, sm_103a). Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "isc.h"

namespace isc {

constexpr int NU = 8;
constexpr int NC = 6;
constexpr int BS = 8;
constexpr int BB = 64;          // doubles per 8x8 block
// 1/x by Newton-Raphson iteration (r <- r + r (1 - x r), each step squaring the
// relative error) from the hardware approximation rcp.approx.ftz.f64 (about 20
// correct bits): two steps reach full double precision (within 1 ulp of the
// correctly rounded quotient; isc_check_reciprocal compares it with 1.0 / x).
// Subnormal, zero, infinite and NaN x, and |x| >= 2^1022 (whose reciprocal is
// subnormal, which the approximation flushes to zero) take the ordinary division. A pivot
// reciprocal costs 4 DFMA this way instead of the division's longer sequence,
// which matters on GB300's narrow FP64 pipe inside the factorisation wavefront.
#ifdef __CUDACC__
__device__ __forceinline__ double recip_nr(double x) {
  const unsigned long long e = (unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull;
  if (e == 0ull || e >= 0x7fd0000000000000ull) return 1.0 / x;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double t = fma(-x, r, 1.0);
  r = fma(r, t, r);
  t = fma(-x, r, 1.0);
  return fma(r, t, r);
}
__device__ __forceinline__ float recip_nr(float x) { return 1.0f / x; }
#endif
constexpr int NQ = 16;          // staged face quantities per cell
constexpr int NQD = NQ * 9;     // doubles per cell in the staged buffer (value + 8 tangents)
constexpr double R_GAS = 8.314462618;

// staged face quantities (value and d/du of each, per cell)
enum FaceQ {
  Q_LW = 0,        // lambda_w                (water carried by the water phase)
  Q_LWH = 1,       // lambda_w H_w
  Q_LOX_LO = 2,    // lambda_o x_LO
  Q_LOX_HO = 3,    // lambda_o x_HO
  Q_LOH = 4,       // lambda_o H_o
  Q_LGY = 5,       // lambda_g y_c, c = 0..5  -> 5..10
  Q_LGH = 11,      // lambda_g H_g
  Q_GAM = 12,      // gamma_w, gamma_o, gamma_g -> 12..14
  Q_KT = 15        // bulk thermal conductivity
};

// Parameters of the discrete model, passed to kernels by value (constant bank).
struct Params {
  int nx, ny, nz, n;
  double V;                   // cell volume
  double dt, inv_dt;
  double gx, gy, gz;          // (A/h) of x, y, z faces (conduction)
  // fluid
  double M[6], a_rk[6], b_rk[6], sqM[6];
  double rho_ref[3], cp[3], ct1[3], ct2[3], cpt[3];
  double p_ref, T_ref;
  double cpg[6][4];
  double hvr[3], ev[3], Tc[3];
  double avg[6], bvg[6], ln_avisc[3], bvisc[3];
  double kv[3][5];
  double K_phase[3];
  double coke_rho, coke_cp, coke_K;
  double Swc, Sorw, Sgc, Sorg;
  double per_eps, gravity;
  // rock
  double cpor, ctpor, cptpor, rock_p_ref, rock_T_ref, cv1, cv2, K_rock;
  // reactions
  int nr;
  int kind[ISC_MAX_RXN];
  int comp[ISC_MAX_RXN];
  double stoich[ISC_MAX_RXN][7];
  double A[ISC_MAX_RXN], EaR[ISC_MAX_RXN], dH[ISC_MAX_RXN];
  double coke_max;
  // heat loss to the overburden / underburden: per boundary face A K_ob ((T - T_ini)/d - rho)
  double hl_AK;               // dx dy K_ob (0: no heat loss)
  double hl_inv_d, hl_Tini, hl_rho;
  int hl_faces;               // 1: top layer (k = 0), 2: bottom layer (k = nz - 1)
  // convergence scaling
  double cv_scale;            // rock volumetric heat capacity for the energy norm
};

// One well perforation slot (a cell holds at most one).
struct WellSlot {
  int kind;                   // ISC_WELL_*
  int cell;                   // perforated cell
  double WI;
  double bhp;                 // producer
  double share;               // injector: WI / sum of the well's WI
  double src[7];              // rate injector: mol/s per component and J/s; coupled injector: the
                              // stream's mole fractions and molar enthalpy (J/mol)
  int wc;                     // coupled well: its index among the coupled wells, else -1
  int control;                // coupled well: ISC_CTRL_*
  double zref;                // coupled well: depth of the bottom-hole pressure
  int phase;                  // coupled injector: phase whose specific weight sets the head (0 water, 2 gas)
};

// One coupled well (bottom-hole pressure unknown) on the device.
struct CoupledWell {
  int control;
  int first, count;           // slot range
  double target;
};

// Host record of one well (the slots of a well are contiguous).
struct WellInfo {
  int kind;
  int first, count;           // slot range
  double target;
  double inj_y[6];
  double Hinj;                // molar enthalpy of the injected stream
};

// Workspace of the discrete adjoint (allocated on first use).
struct AdjointWork {
  int cap_states = 0;         // states (9N doubles: u SoA 8N, then coke N) the store holds
  double* store = nullptr;
  double* ubar = nullptr;     // adjoint of u^n, block-major 8N
  double* cbar = nullptr;     // adjoint of the coke C^n (N)
  double* lam = nullptr;      // multiplier of the step's residual, block-major 8N
  double* glnk = nullptr;     // dL/d ln k per cell (N)
  double* grx = nullptr;      // per-cell parts of dL/d ln A_r (rows 0..nr-1) and dL/d Ea_r (rows nr..2nr-1)
  double* scond = nullptr;    // conduction sensitivity per cell (N)
  double* kd = nullptr;       // (C-bar - gamma) / (dg/dC) per cell (N)
  double* loss_cell = nullptr;// per-cell cumulative produced oil mass (N)
  double* sums = nullptr;     // reduced loss and reaction gradients
  // the last forward sweep (isc_adjoint_forward) that a reverse sweep can follow
  bool ready = false;
  bool traj_used = false;     // the trajectory slots no longer hold the forward sweep's last segment
  std::vector<double> dts;
  int K = 1;
  double tol_adjoint = 0.0, loss = 0.0;
  int32_t* inj_first = nullptr;  // injector wells: first slot and slot count
  int32_t* inj_count = nullptr;
  int n_inj = 0;
};

// One level of the CPR pressure multigrid: a 7-point stencil on nx*ny*nz
// cells (coefficients SoA c[d*n + i], d = -z, -y, -x, diagonal, +x, +y, +z,
// cell index x + nx (y + ny z)), iterate, right-hand side and the factors of
// every column's z-tridiagonal system (e = 1/pivot, f = upper / pivot).
// T is double, or float when the preconditioner runs in mixed precision.
template <typename T>
struct MGLevel {
  int nx, ny, nz, n;
  T *c, *x, *b, *e, *f;
};
constexpr int MG_AGG = 2;             // x-y aggregation factor (MG_AGG x MG_AGG fine columns per coarse column)
constexpr int MG_BLOCK_CELLS = 2048;  // levels this small run inside one thread block

// Workspace of the CPR-PF preconditioner (allocated on first use, for one precision).
struct CprWork {
  std::vector<MGLevel<double>> h64;   // level tables (the one of the current precision is set)
  std::vector<MGLevel<float>> h32;
  void* d_levels = nullptr;           // device copy of the current table
  void* pool = nullptr;               // every level's arrays
  double* col0 = nullptr;             // unknown-0 column of every block, nnzb x 8
  double* r1 = nullptr;               // right-hand side of the second stage, block-major 8N
  int nlev = 0, ngrid = 0;            // levels; levels done by grid-wide kernels
  bool fp32 = false;                  // precision of the level arrays
  size_t bytes = 0;                   // device bytes of pool, d_levels, col0 and r1
};

// device status word bits
enum DevStatus { DS_SINGULAR = 1, DS_COKE = 2, DS_NONFINITE = 4, DS_TIMEOUT = 8 };

struct KTimer {
  cudaEvent_t a = nullptr, b = nullptr;
};

struct Handle {
  // sizes
  int nx = 0, ny = 0, nz = 0, n = 0, nnzb = 0, nlevels = 0;
  std::unordered_map<void*, size_t> dev_sizes;  // bytes of every live allocation made through dalloc
  Params P{};
  isc_options opt{};
  cudaStream_t stream = nullptr;
  std::string last_error;
  // host copies
  std::vector<int32_t> h_rowptr, h_col, h_level_ptr;
  // device: static
  int32_t *rowptr = nullptr, *col = nullptr, *level_cells = nullptr;
  double *phi_ref = nullptr, *depth = nullptr, *tx = nullptr, *ty = nullptr, *tz = nullptr;
  int32_t* well_slot = nullptr;
  WellSlot* slots = nullptr;
  int nslots = 0;
  double *wx = nullptr, *wy = nullptr, *wz = nullptr;  // face weights d ln T / d ln k_lo, indexed by lo
  // coupled producers: count, vector length of the bordered system (8N + nwc)
  int nwc = 0;
  int vlen = 0;                                   // logical length of a Krylov vector
  int vstride = 0;                                // its storage stride (vlen rounded up to 8 doubles)
  CoupledWell* cw = nullptr;                      // nwc
  double *bhp = nullptr, *bhp_n = nullptr;        // iterate and accepted bottom-hole pressures (nwc)
  double *Bv = nullptr, *Cv = nullptr;            // border per slot (nslots x 8)
  double *Fq = nullptr, *Dq = nullptr;            // per-slot parts of F_w and D_w (nslots)
  double* Dw = nullptr;                           // dF_w/d bhp_w (nwc)
  std::vector<double> h_bhp_init;
  // sensitivity parameters: creation-time permeabilities and well indices, the
  // per-cell ln k multipliers and the host copies they generate
  std::vector<double> h_perm0, h_WI0, h_lnk;
  std::vector<WellSlot> h_slots;
  std::vector<WellInfo> h_wells;
  double face_area[3] = {0, 0, 0};                 // A/h of x, y, z faces
  double area_xy = 0.0;                            // dx dy: a cell's top / bottom face
  double h_Ea[ISC_MAX_RXN] = {}, h_lnA[ISC_MAX_RXN] = {};  // current reaction parameters
  AdjointWork adj;
  CprWork cpr;
  // device: state
  double *u = nullptr, *coke = nullptr;          // iterate (SoA 8N), solved coke (N)
  double *u_n = nullptr, *coke_n = nullptr;       // accepted state
  double* acc_n = nullptr;                        // accumulation of the accepted state (7N SoA)
  // device: assembly
  double* props = nullptr;                        // staged face quantities (NQD * N)
  double* fbuf = nullptr;                         // face pass: each face's flux per row, parked for the
                                                  // gather (3 directions * 7 rows * N)
  double* R = nullptr;                            // residual, block-major 8N
  double* J = nullptr;                            // BSR values nnzb*64
  double* ntot = nullptr;                         // per-cell total moles (norm scaling)
  double* du = nullptr;                           // Newton update, block-major 8N
  double* rhs = nullptr;                          // -F, right-hand side of the solve
  double* dinv = nullptr;                         // preconditioner diagonal inverses N*64
  double* uhat = nullptr;                         // ILU(0): pre-scaled upper blocks D_i^-1 A_{i,up}, 3 per cell (+x, +y, +z)
  float* J32 = nullptr;                           // mixed precision: FP32 copy of the decoupled blocks
  float* dinv32 = nullptr;                        // mixed precision: FP32 D^-1
  float* uhat32 = nullptr;                        // mixed precision: FP32 pre-scaled upper blocks
  float* vec32 = nullptr;                         // mixed precision: 2 x 8N FP32 sweep vectors
  // Krylov workspace
  double* V = nullptr;                            // (restart+1) vectors of 8N
  double* Z = nullptr;                            // restart preconditioned vectors
  double* w = nullptr;
  double* tmp = nullptr;
  double* partial = nullptr;                      // reduction partials
  double* scal = nullptr;                         // device scalars
  double* h_scal = nullptr;                       // pinned host mirror
  int* dstatus = nullptr;
  int* h_status = nullptr;                        // pinned
  int* pipe = nullptr;                            // sweep counter, abort flag
  unsigned* red_counter = nullptr;                // last-block counter of the fused reductions
  double* gmres = nullptr;                        // GMRES Hessenberg, rotations, g and status (device)
  // inner FP32 GMRES of ISC_PRECISION_MIXED_FGMRES
  float* V32 = nullptr;                           // (inner_alloc + 1) x 8N basis
  float* Z32 = nullptr;                           // inner_alloc x 8N preconditioned basis
  float* w32 = nullptr;                           // 8N
  double* gm_in = nullptr;                        // GMRES_STATE
  double* scal_in = nullptr;                      // 256: h0, h1, ||w||^2, y
  int inner_alloc = 0;
  // step controller of isc_run (allocated on its first call)
  double* u_prev = nullptr;                       // T, S_w, S_g of the accepted state before the step (3N)
  unsigned long long* run_max = nullptr;          // max |dT| and max |dS| over the cells, as bit patterns
  double* h_ring = nullptr;                       // pinned: two slots of GMRES status (rel, 1/h, h)
  cudaEvent_t gm_ev[2] = {nullptr, nullptr};      // completion of those copies
  int restart_alloc = 0;
  int red_blocks = 0;
  // flags
  bool assembled = false, decoupled = false, prec_built = false, have_acc = false;
  double last_dt = 0.0;
  // timing
  isc_stats stats{};
  KTimer timers[ISC_K_COUNT];
};

// --------------------------------------------------------------- launchers
// assembly (isc_assembly.cu)
void launch_props(Handle& h, cudaStream_t s);
void launch_flux(Handle& h, cudaStream_t s);
void launch_old_accumulation(Handle& h, cudaStream_t s);
void launch_norms(Handle& h, cudaStream_t s);
void launch_well_equations(Handle& h, cudaStream_t s);
// bordered-system pieces of the coupled producers (isc_linalg.cu)
void launch_well_border_spmv(Handle& h, const double* x, double* y, cudaStream_t s);
void launch_well_prec(Handle& h, const double* r, double* z, cudaStream_t s);
void launch_well_update(Handle& h, cudaStream_t s);
void launch_init_equilibrium(Handle& h, double p0, double T0, double Sw0, double So0, double xlo0,
                             const double* y_rest, cudaStream_t s);
// linear algebra (isc_linalg.cu)
void launch_gj(Handle& h, cudaStream_t s);
void launch_spmv(int nrows, const int32_t* rowptr, const int32_t* col, const double* val, const double* x,
                 double* y, int unit_diag, cudaStream_t s);
void launch_ilu_factor(Handle& h, cudaStream_t s);
void launch_bjacobi_factor(Handle& h, cudaStream_t s);
void launch_prec_apply(Handle& h, const double* r, double* z, cudaStream_t s);
// pencil-pipelined ILU(0) sweeps (isc_ilu_pipe.cu)
void launch_ilu_apply_pipe(Handle& h, const double* r, double* z, cudaStream_t s);
void launch_ilu_factor_pipe(Handle& h, cudaStream_t s);
void launch_update(Handle& h, cudaStream_t s);
// CPR-PF preconditioner (isc_cpr.cu)
int cpr_setup_levels(Handle& h);
void launch_cpr_setup(Handle& h, cudaStream_t s);
void launch_cpr_pressure(Handle& h, const double* r, cudaStream_t s);
void launch_cpr_finish(Handle& h, double* z, cudaStream_t s);
// FP32 vectors (inner solve of ISC_PRECISION_MIXED_FGMRES): p and r1 = r - A E p into r1; z += E p
void launch_cpr_pressure32(Handle& h, const float* r, float* r1, cudaStream_t s);
void launch_cpr_finish32(Handle& h, float* z, cudaStream_t s);
int cpr_pressure_launches(const Handle& h);
void cpr_free(Handle& h);
// discrete adjoint (isc_adjoint.cu)
void launch_oil_rate(Handle& h, double dt, cudaStream_t s);
void launch_adj_pre(Handle& h, double dt, cudaStream_t s);
void launch_bsr_transpose(Handle& h, cudaStream_t s);
void launch_adj_post(Handle& h, bool has_old, cudaStream_t s);
void launch_row_sums(int nrows, int len, const double* x, double* out, cudaStream_t s);
void launch_to_f32(size_t n, const double* x, float* y, cudaStream_t s);
void launch_max_change(int n, const double* a, const double* b, unsigned long long* out, cudaStream_t s);
// GMRES bookkeeping on the device (isc_linalg.cu); the buffer Handle::gmres holds
// GMRES_STATE doubles
constexpr int GMRES_STATE = 64 * 67 + 64 + 8;
void launch_gmres_givens(Handle& h, int j, int m, double bnorm, int off_h0, int off_h1, int off_nrm, cudaStream_t s);
void launch_gmres_start(Handle& h, int m, double beta, cudaStream_t s);
void launch_gmres_backsub(Handle& h, int jdone, int m, int off_y, cudaStream_t s);
void launch_scale_dev(Handle& h, const double* x, double* y, cudaStream_t s);
const double* gmres_status(const Handle& h);
// inner FP32 GMRES of the mixed-precision scheme (precision = ISC_PRECISION_MIXED_FGMRES);
// G is a GMRES_STATE-sized device state, vectors are FP32 of length len stored vs apart
void launch_f32_nrm(Handle& h, int len, const double* x, float* y, double* out, cudaStream_t s);
void launch_gmres_start_dev(double* G, int m, const double* nrm2, cudaStream_t s);
void launch_gmres_givens_at(double* G, int j, int m, const double* h0, const double* h1, const double* nrm, cudaStream_t s);
void launch_gmres_backsub_at(double* G, int jdone, int m, double* y, cudaStream_t s);
void launch_scale_dev32(double* G, int len, const float* x, float* y, cudaStream_t s);
void launch_spmv32(int nrows, const int32_t* rowptr, const int32_t* col, const float* val, const float* x, float* y,
                   int unit_diag, cudaStream_t s);
void launch_mdot32(Handle& h, int len, size_t vs, const float* V, int nvec, const float* w, double* out, cudaStream_t s);
void launch_maxpy_mdot32(Handle& h, int len, size_t vs, float* w, const float* V, int nvec, const double* coef,
                         double* out, cudaStream_t s);
void launch_maxpy_norm32(Handle& h, int len, size_t vs, float* w, const float* V, int nvec, const double* coef,
                         double* out, cudaStream_t s);
void launch_comb_out32(int len, const float* V, size_t vs, int nvec, const double* coef, double* out, cudaStream_t s);
void launch_recip_check(int n, const double* x, double* y, double* z, cudaStream_t s);
// FP32 ILU(0) apply on FP32 vectors (the factors of the mixed-precision modes)
void launch_ilu_apply_f32(Handle& h, const float* r, float* z, cudaStream_t s);
// BLAS-1 with fixed-order two-stage reductions; results land in h.scal[off..]
void launch_mdot(Handle& h, const double* V, int nvec, const double* w, int off, cudaStream_t s);
void launch_maxpy(Handle& h, double* w, const double* V, int nvec, int coef_off, double sign, cudaStream_t s);
void launch_maxpy_norm(Handle& h, double* w, const double* V, int nvec, int coef_off, int out_off, cudaStream_t s);
// w <- w - V scal[coef_off..], then scal[out_off..] = V^T w (one read of V)
void launch_maxpy_mdot(Handle& h, double* w, const double* V, int nvec, int coef_off, int out_off, cudaStream_t s);
void launch_axpby(int n, double a, const double* x, double b, double* y, cudaStream_t s);
void launch_scale_copy(int n, double a, const double* x, double* y, cudaStream_t s);
void launch_axpy_dev(int n, const double* coef, double sign, const double* x, double* y, cudaStream_t s);

}  // namespace isc
