// Pencil-pipelined block ILU(0): the factorisation and the two triangular
// sweeps of the preconditioner.
//
// For the 7-point pattern in natural order, ILU(0) keeps the off-diagonal
// blocks of A and changes only the diagonal (D-ILU form):
//   D_i       = A_ii - sum_{k in {i-1, i-nx, i-nxy}} A_ik D_k^-1 A_ki
//   forward   y_i = D_i^-1 (r_i - A_{i,i-1} y_{i-1} - A_{i,i-nx} y_{i-nx} - A_{i,i-nxy} y_{i-nxy})
//   backward  z_i = y_i - D_i^-1 (A_{i,i+1} z_{i+1} + A_{i,i+nx} z_{i+nx} + A_{i,i+nxy} z_{i+nxy})
// Cell i depends on its x-predecessor (same pencil) and on the pencils
// (j-1,k) and (j,k-1) at the same x. A pencil's x-recurrence stays in the
// registers of the warp (or half-warp) that owns it; pencils are taken from a
// counter in dependency order, so a warp only ever waits on pencils already
// held by running warps. The cross-pencil hand-off is the data itself: the
// output vector is filled with a NaN sentinel before a sweep and a consumer
// polls the neighbour's 64-byte block vector until the sentinel is gone,
// requesting it one cell before use. The matrix operands of upcoming cells
// are streamed into a per-warp shared-memory ring with cp.async. Row starts
// are computed, not loaded. Every wait is bounded: on timeout the kernel raises
// DS_TIMEOUT and a global abort flag that makes every other waiter return.
//
// The sweep time is the FP64 pipe (FP64) or HBM (FP32) in steady state plus
// the wavefront's fill and drain: a hand-off between pencils costs about one
// cell time plus an L2 round trip, over the ny + nz - 2 pencil diagonals.
#include <vector>

#include "isc_internal.cuh"

namespace isc {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SPIN_LIMIT = 1 << 22;

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// morally strong store paired with the relaxed polling loads of other warps
__device__ __forceinline__ void st_relaxed(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ double2 ld_nc2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }

// Start of the BSR row of cell i for the 7-point pattern with sorted columns,
// computed instead of loaded: 7 i minus the neighbours missing at the
// boundaries among the cells before i (a dependent rowptr load per cell would
// put a memory round trip into every step of the sweep recurrences).
__device__ __forceinline__ int rowptr_of(int nx, int ny, int nz, int i) {
  const int nxy = nx * ny;
  const int x = i % nx, rr = i / nx;
  const int y = rr % ny, z = rr / ny;
  const int miss = rr + (x > 0)                       // -x
                   + rr                               // +x
                   + z * nx + (y > 0 ? nx : x)        // -y
                   + z * nx + (y == ny - 1 ? x : 0)   // +y
                   + (z > 0 ? nxy : i)                // -z
                   + (z == nz - 1 ? i - z * nxy : 0); // +z
  return 7 * i - miss;
}

// Row starts along one x-pencil: base(x) = base(0) + x L + max(2x - 1, 0) with
// L the pencil's neighbour count outside x (no division per cell).
struct Pen {
  int base_jk, base0, L;
};

__device__ __forceinline__ Pen make_pen(int nx, int ny, int nz, int j, int k, int base_jk) {
  Pen P;
  P.base_jk = base_jk;
  P.base0 = rowptr_of(nx, ny, nz, base_jk);
  P.L = 1 + (k > 0) + (j > 0) + (j < ny - 1) + (k < nz - 1);
  return P;
}

__device__ __forceinline__ int row_start(const Pen& P, int x) { return P.base0 + x * P.L + (x > 0 ? 2 * x - 1 : 0); }

// |v| as an unsigned integer whose order is the numeric order of |v| (IEEE 754)
template <typename T> struct MagBits;
template <> struct MagBits<double> {
  using U = unsigned long long;
  static constexpr U INF = 0x7ff0000000000000ull;
  static __device__ __forceinline__ U get(double v) { return (U)__double_as_longlong(v) & 0x7fffffffffffffffull; }
};
template <> struct MagBits<float> {
  using U = unsigned;
  static constexpr U INF = 0x7f800000u;
  static __device__ __forceinline__ U get(float v) { return (U)__float_as_int(v) & 0x7fffffffu; }
};

// Vector element types of the sweeps: FP64 (all-FP64 solve) or FP32 (factors,
// off-diagonal blocks and the hand-off vector of the mixed-precision solve).
template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };

__device__ __forceinline__ void ld_relaxed_v2(const double* p, double& a, double& b) {
  asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2(const float* p, float& a, float& b) {
  asm volatile("ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2];" : "=f"(a), "=f"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
  asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ float2 ld_nc2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

// The hand-off sentinel is the all-ones bit pattern the vector is filled with
// before a sweep (a NaN no arithmetic produces). It is tested with an integer
// compare: on GB300 the FP64 pipe is the sweep's scarcest resource, and a
// floating-point NaN test would spend it on every poll of a waiting warp.
__device__ __forceinline__ bool arrived(double a) { return __double_as_longlong(a) != -1LL; }
__device__ __forceinline__ bool arrived(float a) { return __float_as_int(a) != -1; }

// Poll the block vector v[8] of a neighbouring pencil until every entry has
// arrived: each store is single-copy atomic, so an entry that is not the
// sentinel is final. The data itself is the hand-off (one L2 round trip, no
// flags or fences). Returns false if the sweep was aborted (timeout here or
// elsewhere).
template <typename T>
__device__ __forceinline__ bool poll_vec(const T* v, int c, typename V2<T>::t& out, int* abortf, int* dstatus) {
  const T* p = v + c;
  for (int spins = 0;; ++spins) {
    T a, b;
    ld_relaxed_v2(p, a, b);
    const bool ok = arrived(a) && arrived(b);
    if (__all_sync(FULL, ok)) {
      out.x = a;
      out.y = b;
      return true;
    }
    if ((spins & 63) == 63 && __any_sync(FULL, ld_relaxed(abortf) != 0)) return false;
    if (spins > SPIN_LIMIT) {
      if ((threadIdx.x & 31) == 0) {
        atomicOr(dstatus, DS_TIMEOUT);
        atomicExch(abortf, 1);
      }
      return false;
    }
    __nanosleep(20);
  }
}

// ------------------------------------------------- sweep kernels
// Two x-pencils per warp, one per half-warp: a pencil's 8x8 block is spread
// over 16 lanes, lane h holding row r = h/2 and four columns (two pairs), so a
// block-vector product is four FMAs per lane and a row sum is ONE shuffle and
// one add over the lane pair. On GB300 the FP64 pipe is the sweep's scarcest
// unit; against one pencil per 32-lane warp (quad sums: two adds per row) this
// halves the reduction adds, and the two pencils of a warp share every
// shuffle, address and staging instruction. The pair of a warp lies on one
// anti-diagonal j + k = d of the (y, z) pencil grid, so the two are independent
// (each waits only on pencils of diagonal d - 1, claimed earlier from the same
// counter) and share one of their neighbours.
//
// Forward sweep  y_i = D_i^-1 (r_i - A_z y_z - A_y y_y - A_x y_{i-1});
// backward sweep z_i = y_i - Dhat_z z_z - Dhat_y z_y - Dhat_x z_{i+1} with the
// pre-scaled upper blocks Dhat = D_i^-1 A_{i,up}, which the factorisation
// computes anyway (they are its D_k^-1 A_ki products) and stores, so the
// backward sweep reads no D^-1 and does no second product. A row sum starts
// from r_i (or y_i) and subtracts the products with negated FMA operands, so no
// separate subtraction or negation reaches the FP64 pipe.

// the lane's four columns of a block row: (e0, e0 + 1) and (e2, e2 + 1). FP64
// lanes 4-7 and 12-15 of a half take the two pairs in the other order, so that
// each 16-byte shared-memory load of a quarter-warp touches 32 distinct banks
struct LaneCols {
  int hl, h, r, q, e0, e2, s0, s2;
};

template <typename TM>
__device__ __forceinline__ LaneCols lane_cols() {
  LaneCols L;
  const int lane = threadIdx.x & 31;
  L.hl = lane >> 4;
  L.h = lane & 15;
  L.r = L.h >> 1;
  L.q = L.h & 1;
  const int sw = sizeof(TM) == 8 ? ((L.h >> 2) & 1) : 0;
  L.e0 = 4 * L.q + 2 * sw;
  L.e2 = 4 * L.q + 2 * (1 - sw);
  // lanes holding the row sums of those columns (both lanes of a row pair hold it)
  L.s0 = (L.hl << 4) + 2 * L.e0;
  L.s2 = (L.hl << 4) + 2 * L.e2;
  return L;
}

// four entries of block row r (columns e0, e0+1, e2, e2+1) from shared memory
__device__ __forceinline__ void ld4s(const double* b, const LaneCols& L, double (&x)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(b + L.r * 8 + L.e0);
  const double2 c = *reinterpret_cast<const double2*>(b + L.r * 8 + L.e2);
  x[0] = a.x, x[1] = a.y, x[2] = c.x, x[3] = c.y;
}
__device__ __forceinline__ void ld4s(const float* b, const LaneCols& L, float (&x)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(b + L.r * 8 + L.e0);  // e2 = e0 + 2 in FP32
  x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w;
}

// the same four entries of a neighbour's 8-vector, relaxed gpu-scope loads (hand-off polling)
__device__ __forceinline__ void ld4r(const double* v, const LaneCols& L, double (&x)[4]) {
  ld_relaxed_v2(v + L.e0, x[0], x[1]);
  ld_relaxed_v2(v + L.e2, x[2], x[3]);
}
__device__ __forceinline__ void ld4r(const float* v, const LaneCols& L, float (&x)[4]) {
  asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3])
               : "l"(v + L.e0)
               : "memory");
}

// lanes 0 and 1 of a half hold the whole 8-vector after the broadcast: columns 0-3 and 4-7
__device__ __forceinline__ void st4r(double* v, const LaneCols& L, const double (&x)[4]) {
  asm volatile("st.relaxed.gpu.global.v2.f64 [%0], {%1, %2};" ::"l"(v + L.e0), "d"(x[0]), "d"(x[1]) : "memory");
  asm volatile("st.relaxed.gpu.global.v2.f64 [%0], {%1, %2};" ::"l"(v + L.e2), "d"(x[2]), "d"(x[3]) : "memory");
}
__device__ __forceinline__ void st4r(float* v, const LaneCols& L, const float (&x)[4]) {
  asm volatile("st.relaxed.gpu.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(v + L.e0), "f"(x[0]), "f"(x[1]),
               "f"(x[2]), "f"(x[3])
               : "memory");
}

template <typename TM>
__device__ __forceinline__ bool arrived4(const TM (&x)[4]) {
  return arrived(x[0]) && arrived(x[1]) && arrived(x[2]) && arrived(x[3]);
}

template <typename TM>
__device__ __forceinline__ void zero4(TM (&x)[4]) {
  x[0] = x[1] = x[2] = x[3] = TM(0);
}

// Wait until the neighbour values a half needs (z and/or y neighbour pencil,
// four entries each per lane) are all numbers, across the whole warp. The
// values were requested one cell ahead; entries still holding the sentinel are
// re-read. Returns false on abort (a timeout here or elsewhere).
template <typename TM>
__device__ __forceinline__ bool await_nbrs(const TM* pz, bool hz, TM (&vz)[4], const TM* py, bool hy, TM (&vy)[4],
                                           const LaneCols& L, int* abortf, int* dstatus) {
  for (int spins = 0;; ++spins) {
    const bool okz = !hz || arrived4<TM>(vz), oky = !hy || arrived4<TM>(vy);
    if (__all_sync(FULL, okz && oky)) return true;
    if ((spins & 63) == 63 && __any_sync(FULL, ld_relaxed(abortf) != 0)) return false;
    if (spins > SPIN_LIMIT) {
      if ((threadIdx.x & 31) == 0) {
        atomicOr(dstatus, DS_TIMEOUT);
        atomicExch(abortf, 1);
      }
      return false;
    }
    __nanosleep(20);
    if (!okz) ld4r(pz, L, vz);
    if (!oky) ld4r(py, L, vy);
  }
}

// ------------------------------------------------- shared-memory operand pipeline
// A cell's operands (its up-to-three off-diagonal blocks of the sweep
// direction, D^-1 where the sweep needs it, and the right-hand side) do not
// depend on the sweep. Each warp streams them into its own ring of R slots with
// 16-byte cp.async copies, R-1 cells ahead of use, so the per-cell chain does
// not wait on DRAM. Every iteration commits exactly one group (possibly empty)
// and waits until the group of the current cell has landed (a hardware wait).
__device__ __forceinline__ void cp16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename TM, typename RT>
struct alignas(16) Slot2 {
  TM blk[2][4][64];  // per half: blocks in fixed positions (direction slots 0..2, D^-1 at 3)
  RT rhs[2][8];
};

// one block (64 entries) copied by the 16 lanes of a half
template <typename TM>
__device__ __forceinline__ void stage_blk(TM* dst, const TM* src, int h) {
  constexpr int PER = 64 / 16;             // entries per lane
  constexpr int CH = 16 / sizeof(TM);      // entries per 16-byte copy
#pragma unroll
  for (int c = 0; c < PER; c += CH) cp16(dst + h * PER + c, src + h * PER + c);
}

// an 8-vector (the right-hand side, or the forward result in the backward sweep)
template <typename RT>
__device__ __forceinline__ void stage_vec(RT* dst, const RT* src, int h) {
  constexpr int CH = 16 / sizeof(RT);
  if (h < 8 / CH) cp16(dst + h * CH, src + h * CH);
}

// Anti-diagonal task map of the (y, z) pencil grid: diagonal d holds pencils
// (j, d - j) for j in [jlo, jlo + len), taken two per task in order of j.
struct Diag {
  int d, t0, jlo, len;
};

__device__ __forceinline__ void diag_set(Diag& D, int d, int ny, int nz) {
  D.d = d;
  D.jlo = d - (nz - 1) > 0 ? d - (nz - 1) : 0;
  const int jhi = d < ny - 1 ? d : ny - 1;
  D.len = jhi - D.jlo + 1;
}

// move forward to the diagonal holding task t (a warp's tasks only increase);
// false past the last diagonal
__device__ __forceinline__ bool diag_seek(Diag& D, int t, int ny, int nz) {
  while (t >= D.t0 + ((D.len + 1) >> 1)) {
    D.t0 += (D.len + 1) >> 1;
    if (D.d >= ny + nz - 2) return false;
    diag_set(D, D.d + 1, ny, nz);
  }
  return true;
}

// pencil (j, k) of a half for task t on diagonal D; act = the half has a pencil
__device__ __forceinline__ void task_pencil(const Diag& D, int t, int hl, int& j, int& k, bool& act) {
  const int j0 = D.jlo + 2 * (t - D.t0);
  act = hl == 0 || j0 + 1 < D.jlo + D.len;
  j = act ? j0 + hl : j0;
  k = D.d - j;
}

constexpr int AWARPS = 4;  // warps per block of the sweeps

template <typename TM, int R, typename RT>
__global__ void __launch_bounds__(AWARPS * 32) k_sweep_fwd(int nx, int ny, int nz, const TM* __restrict__ A,
                                                           const TM* __restrict__ Dinv, const RT* __restrict__ rhs,
                                                           TM* __restrict__ y, int* __restrict__ pipe,
                                                           int* __restrict__ dstatus) {
  using SL = Slot2<TM, RT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SL* ring = reinterpret_cast<SL*>(smem_raw) + (threadIdx.x >> 5) * R;
  const LaneCols L = lane_cols<TM>();
  const int nxy = nx * ny;
  int* counter = pipe;
  int* abortf = pipe + 1;
  Diag D;
  diag_set(D, 0, ny, nz);
  D.t0 = 0;
  for (;;) {
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(FULL, t, 0);
    if (!diag_seek(D, t, ny, nz)) return;
    int j, k;
    bool act;
    task_pencil(D, t, L.hl, j, k, act);
    const bool hy = act && j > 0, hz = act && k > 0;
    const int base_jk = nx * (j + ny * k);
    const Pen PEN = make_pen(nx, ny, nz, j, k, base_jk);
    auto stage = [&](int x) {
      SL* sl = ring + x % R;
      if (act) {
        const int base = row_start(PEN, x);  // BSR row of cell (x, j, k): -z, -y, -x, diag, ...
        if (hz) stage_blk<TM>(sl->blk[L.hl][0], A + (size_t)base * BB, L.h);
        if (hy) stage_blk<TM>(sl->blk[L.hl][1], A + (size_t)(base + hz) * BB, L.h);
        if (x > 0) stage_blk<TM>(sl->blk[L.hl][2], A + (size_t)(base + hz + hy) * BB, L.h);
        stage_blk<TM>(sl->blk[L.hl][3], Dinv + (size_t)(base_jk + x) * BB, L.h);
        stage_vec<RT>(sl->rhs[L.hl], rhs + (size_t)(base_jk + x) * 8, L.h);
      }
    };
#pragma unroll 1
    for (int x = 0; x < R - 1; ++x) {
      if (x < nx) stage(x);
      cp_async_commit();
    }
    TM vz[4], vy[4], yp[4];
    zero4(vz), zero4(vy), zero4(yp);
    if (hz) ld4r(y + (size_t)(base_jk - nxy) * 8, L, vz);
    if (hy) ld4r(y + (size_t)(base_jk - nx) * 8, L, vy);
    for (int x = 0; x < nx; ++x) {
      const int i = base_jk + x;
      if (x + R - 1 < nx) stage(x + R - 1);
      cp_async_commit();
      cp_async_wait<R - 1>();
      __syncwarp();
      const SL* sl = ring + x % R;
      TM az[4], ay[4], ax[4], d[4];
      zero4(az), zero4(ay), zero4(ax), zero4(d);
      TM acc = TM(0);
      if (act) {
        if (hz) ld4s(sl->blk[L.hl][0], L, az);
        if (hy) ld4s(sl->blk[L.hl][1], L, ay);
        if (x > 0) ld4s(sl->blk[L.hl][2], L, ax);
        ld4s(sl->blk[L.hl][3], L, d);
        if (L.q == 0) acc = (TM)sl->rhs[L.hl][L.r];
      }
      // (the addresses are formed only when the neighbour exists)
      if (!await_nbrs<TM>(hz ? y + (size_t)(i - nxy) * 8 : y, hz, vz, hy ? y + (size_t)(i - nx) * 8 : y, hy, vy, L,
                          abortf, dstatus)) {
        cp_async_wait<0>();  // no copy of this warp is left in flight when it leaves
        return;
      }
      // row sums of r - A v: the neighbours' terms, then the x-recurrence term last
      // (the minus signs are FMA operand modifiers, not instructions)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(-az[c], vz[c], acc);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(-ay[c], vy[c], acc);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(-ax[c], yp[c], acc);
      const TM s = acc + __shfl_xor_sync(FULL, acc, 1);  // t_r, t = r - A v
      const TM n0 = __shfl_sync(FULL, s, L.s0), n1 = __shfl_sync(FULL, s, L.s0 + 2);
      const TM n2 = __shfl_sync(FULL, s, L.s2), n3 = __shfl_sync(FULL, s, L.s2 + 2);
      TM yr = fma(d[0], n0, fma(d[1], n1, fma(d[2], n2, d[3] * n3)));  // (D^-1 t)_r, partial
      yr += __shfl_xor_sync(FULL, yr, 1);
      yp[0] = __shfl_sync(FULL, yr, L.s0);
      yp[1] = __shfl_sync(FULL, yr, L.s0 + 2);
      yp[2] = __shfl_sync(FULL, yr, L.s2);
      yp[3] = __shfl_sync(FULL, yr, L.s2 + 2);
      if (act && L.h < 2) st4r(y + (size_t)i * 8, L, yp);
      if (x + 1 < nx) {
        if (hz) ld4r(y + (size_t)(i + 1 - nxy) * 8, L, vz);
        if (hy) ld4r(y + (size_t)(i + 1 - nx) * 8, L, vy);
      }
      __syncwarp();  // every lane is done with this slot before it is refilled
    }
    cp_async_wait<0>();
    __syncwarp();
  }
}

// PRE: the upper blocks are the pre-scaled D^-1 A_{i,up} (array uhat, three
// per cell in the order +x, +y, +z); otherwise the BSR upper blocks and D^-1.
template <typename TM, int R, bool PRE>
__global__ void __launch_bounds__(AWARPS * 32) k_sweep_bwd(int nx, int ny, int nz, const TM* __restrict__ A,
                                                           const TM* __restrict__ Dinv, const TM* __restrict__ uhat,
                                                           const TM* __restrict__ yin, TM* __restrict__ zs,
                                                           double* __restrict__ z64, int* __restrict__ pipe,
                                                           int* __restrict__ dstatus) {
  using SL = Slot2<TM, TM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SL* ring = reinterpret_cast<SL*>(smem_raw) + (threadIdx.x >> 5) * R;
  const LaneCols L = lane_cols<TM>();
  const int nxy = nx * ny;
  int* counter = pipe;
  int* abortf = pipe + 1;
  Diag D;
  diag_set(D, 0, ny, nz);
  D.t0 = 0;
  for (;;) {
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(FULL, t, 0);
    if (!diag_seek(D, t, ny, nz)) return;
    int jm, km;
    bool act;
    task_pencil(D, t, L.hl, jm, km, act);
    // the backward sweep runs the mirrored grid: its dependencies point to +y and +z
    const int j = ny - 1 - jm, k = nz - 1 - km;
    const bool hy = act && j < ny - 1, hz = act && k < nz - 1;
    const int nlow = (k > 0) + (j > 0);
    const int base_jk = nx * (j + ny * k);
    const Pen PEN = make_pen(nx, ny, nz, j, k, base_jk);
    auto stage = [&](int step) {
      const int x = nx - 1 - step;
      SL* sl = ring + step % R;
      if (act) {
        const int i = base_jk + x;
        const bool hx = x < nx - 1;
        if (PRE) {
          const TM* u = uhat + (size_t)3 * i * BB;
          if (hx) stage_blk<TM>(sl->blk[L.hl][0], u, L.h);
          if (hy) stage_blk<TM>(sl->blk[L.hl][1], u + BB, L.h);
          if (hz) stage_blk<TM>(sl->blk[L.hl][2], u + 2 * BB, L.h);
        } else {
          const int up = row_start(PEN, x) + nlow + (x > 0) + 1;  // first block after the diagonal
          if (hx) stage_blk<TM>(sl->blk[L.hl][0], A + (size_t)up * BB, L.h);
          if (hy) stage_blk<TM>(sl->blk[L.hl][1], A + (size_t)(up + hx) * BB, L.h);
          if (hz) stage_blk<TM>(sl->blk[L.hl][2], A + (size_t)(up + hx + hy) * BB, L.h);
          stage_blk<TM>(sl->blk[L.hl][3], Dinv + (size_t)i * BB, L.h);
        }
        stage_vec<TM>(sl->rhs[L.hl], yin + (size_t)i * 8, L.h);  // the forward result
      }
    };
#pragma unroll 1
    for (int step = 0; step < R - 1; ++step) {
      if (step < nx) stage(step);
      cp_async_commit();
    }
    TM vz[4], vy[4], zp[4];  // zp: the previous cell's z
    zero4(vz), zero4(vy), zero4(zp);
    if (hz) ld4r(zs + (size_t)(base_jk + nx - 1 + nxy) * 8, L, vz);
    if (hy) ld4r(zs + (size_t)(base_jk + nx - 1 + nx) * 8, L, vy);
    for (int step = 0; step < nx; ++step) {
      const int x = nx - 1 - step;
      const int i = base_jk + x;
      if (step + R - 1 < nx) stage(step + R - 1);
      cp_async_commit();
      cp_async_wait<R - 1>();
      __syncwarp();
      const SL* sl = ring + step % R;
      TM ux[4], uy[4], uz[4], d[4];
      zero4(ux), zero4(uy), zero4(uz), zero4(d);
      TM yi = TM(0);
      if (act) {
        if (x < nx - 1) ld4s(sl->blk[L.hl][0], L, ux);
        if (hy) ld4s(sl->blk[L.hl][1], L, uy);
        if (hz) ld4s(sl->blk[L.hl][2], L, uz);
        if (!PRE) ld4s(sl->blk[L.hl][3], L, d);
        if (L.q == 0) yi = sl->rhs[L.hl][L.r];
      }
      if (!await_nbrs<TM>(hz ? zs + (size_t)(i + nxy) * 8 : zs, hz, vz, hy ? zs + (size_t)(i + nx) * 8 : zs, hy, vy,
                          L, abortf, dstatus)) {
        cp_async_wait<0>();  // no copy of this warp is left in flight when it leaves
        return;
      }
      // PRE: y - Dhat z directly; otherwise U z, then y - D^-1 (U z)
      TM acc = PRE ? yi : TM(0);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(PRE ? -uz[c] : uz[c], vz[c], acc);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(PRE ? -uy[c] : uy[c], vy[c], acc);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(PRE ? -ux[c] : ux[c], zp[c], acc);
      TM sr = acc + __shfl_xor_sync(FULL, acc, 1);  // PRE: z_r; else (U z)_r
      if (!PRE) {
        const TM t0 = __shfl_sync(FULL, sr, L.s0), t1 = __shfl_sync(FULL, sr, L.s0 + 2);
        const TM t2 = __shfl_sync(FULL, sr, L.s2), t3 = __shfl_sync(FULL, sr, L.s2 + 2);
        const TM zr = fma(-d[0], t0, fma(-d[1], t1, fma(-d[2], t2, fma(-d[3], t3, yi))));  // y - D^-1 U z, partial
        sr = zr + __shfl_xor_sync(FULL, zr, 1);
      }
      zp[0] = __shfl_sync(FULL, sr, L.s0);
      zp[1] = __shfl_sync(FULL, sr, L.s0 + 2);
      zp[2] = __shfl_sync(FULL, sr, L.s2);
      zp[3] = __shfl_sync(FULL, sr, L.s2 + 2);
      if (act && L.h < 2) {
        st4r(zs + (size_t)i * 8, L, zp);
        if (z64) {
          z64[(size_t)i * 8 + L.e0] = (double)zp[0];
          z64[(size_t)i * 8 + L.e0 + 1] = (double)zp[1];
          z64[(size_t)i * 8 + L.e2] = (double)zp[2];
          z64[(size_t)i * 8 + L.e2 + 1] = (double)zp[3];
        }
      }
      if (step + 1 < nx) {
        if (hz) ld4r(zs + (size_t)(i - 1 + nxy) * 8, L, vz);
        if (hy) ld4r(zs + (size_t)(i - 1 + nx) * 8, L, vy);
      }
      __syncwarp();
    }
    cp_async_wait<0>();
    __syncwarp();
  }
}

// ------------------------------------------------- one pencil per warp (small grids)
// On grids with few pencils the wavefront's latency, not the FP64 pipe's
// throughput, sets the sweep time, and a lone pencil's cell costs fewer FP64
// warp instructions when all 32 lanes serve it: lane l holds row r = l/4,
// columns c = 2(l%4), c+1 of each 8x8 block (two FMAs per block and lane; row
// sums over the lane quad). Pencils are claimed in natural (j, then k) order;
// the backward sweep uses the unscaled upper blocks and D^-1.
template <typename T>
__device__ __forceinline__ typename V2<T>::t zero2() {
  typename V2<T>::t z;
  z.x = T(0);
  z.y = T(0);
  return z;
}

template <typename T>
__device__ __forceinline__ T quad_sum(T v) {
  v += __shfl_xor_sync(FULL, v, 1);
  v += __shfl_xor_sync(FULL, v, 2);
  return v;
}

// wait until the lane pair of the neighbour's vector, requested one cell ahead, is final in the whole warp
template <typename T>
__device__ __forceinline__ bool settle(const T* p, typename V2<T>::t& v, int* abortf, int* dstatus) {
  if (__all_sync(FULL, arrived(v.x) && arrived(v.y))) return true;
  return poll_vec<T>(p, 0, v, abortf, dstatus);
}

template <int BYTES>
__device__ __forceinline__ void cp_async_n(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gsrc), "n"(BYTES) : "memory");
}

template <typename TM>
struct Slot1 {
  TM blk[4][64];  // up to 3 off-diagonal blocks of the sweep direction, packed in row order, and D^-1 (index 3)
  double rhs[8];
};

// the copies of one cell into a slot: the blocks at row slots first_slot.. that mask marks
template <typename TM, typename RT>
__device__ __forceinline__ void stage_cell1(Slot1<TM>* sl, int i, int first_slot, int mask, const Pen& P,
                                            const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                            const RT* __restrict__ rhs, int lane) {
  const int base = row_start(P, i - P.base_jk);
  int s = first_slot, dst = 0;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (mask & (1 << b)) {
      cp_async_n<2 * sizeof(TM)>(&sl->blk[dst][2 * lane], A + (size_t)(base + s) * BB + 2 * lane);
      ++s;
      ++dst;
    }
  }
  cp_async_n<2 * sizeof(TM)>(&sl->blk[3][2 * lane], Dinv + (size_t)i * BB + 2 * lane);
  if (lane < 8) cp_async_n<sizeof(RT)>(reinterpret_cast<RT*>(sl->rhs) + lane, rhs + (size_t)i * 8 + lane);
}

template <typename TM>
__device__ __forceinline__ typename V2<TM>::t sl_pair(const Slot1<TM>* sl, int b, int lane) {
  return *reinterpret_cast<const typename V2<TM>::t*>(&sl->blk[b][2 * lane]);
}

template <typename TM, int R, typename RT>
__global__ void __launch_bounds__(AWARPS * 32) k_sweep1_fwd(int nx, int ny, int nz, const TM* __restrict__ A,
                                                            const TM* __restrict__ Dinv, const RT* __restrict__ rhs,
                                                            TM* __restrict__ y, int* __restrict__ pipe,
                                                            int* __restrict__ dstatus) {
  using T2 = typename V2<TM>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Slot1<TM>* ring = reinterpret_cast<Slot1<TM>*>(smem_raw) + (threadIdx.x >> 5) * R;
  const int lane = threadIdx.x & 31;
  const int r = lane >> 2, c = (lane & 3) * 2;
  const int npen = ny * nz, nxy = nx * ny;
  int* counter = pipe;
  int* abortf = pipe + 1;
  for (;;) {
    int p = 0;
    if (lane == 0) p = atomicAdd(counter, 1);
    p = __shfl_sync(FULL, p, 0);
    if (p >= npen) return;
    const int j = p % ny, k = p / ny;
    const bool hy = j > 0, hz = k > 0;
    const int base_jk = nx * (j + ny * k);
    const Pen PEN = make_pen(nx, ny, nz, j, k, base_jk);
    // blocks of row (j, k, x) in order -z, -y, -x
    auto mask_of = [&](int x) { return (hz ? 1 : 0) | (hy ? 2 : 0) | (x > 0 ? 4 : 0); };
#pragma unroll 1
    for (int q = 0; q < R - 1; ++q) {
      if (q < nx) stage_cell1<TM, RT>(ring + q, base_jk + q, 0, mask_of(q), PEN, A, Dinv, rhs, lane);
      cp_async_commit();
    }
    T2 rz = zero2<TM>(), ry = zero2<TM>();
    if (hz) ld_relaxed_v2(y + (size_t)(base_jk - nxy) * 8 + c, rz.x, rz.y);
    if (hy) ld_relaxed_v2(y + (size_t)(base_jk - nx) * 8 + c, ry.x, ry.y);
    TM yp0 = TM(0), yp1 = TM(0);
    for (int x = 0; x < nx; ++x) {
      const int i = base_jk + x;
      if (x + R - 1 < nx)
        stage_cell1<TM, RT>(ring + (x + R - 1) % R, base_jk + x + R - 1, 0, mask_of(x + R - 1), PEN, A, Dinv, rhs,
                            lane);
      cp_async_commit();
      cp_async_wait<R - 1>();
      __syncwarp();
      const Slot1<TM>* sl = ring + x % R;
      const int m = mask_of(x);
      int b = 0;
      T2 az = zero2<TM>(), ay = zero2<TM>(), ax = zero2<TM>();
      if (m & 1) az = sl_pair<TM>(sl, b++, lane);
      if (m & 2) ay = sl_pair<TM>(sl, b++, lane);
      if (m & 4) ax = sl_pair<TM>(sl, b, lane);
      const T2 d = sl_pair<TM>(sl, 3, lane);
      // the row sum starts from r_i / 4 on each lane of the quad and subtracts with negated FMA operands
      TM acc = (TM)reinterpret_cast<const RT*>(sl->rhs)[r] * TM(0.25);
      acc = fma(-ax.x, yp0, fma(-ax.y, yp1, acc));
      if (hz) {
        if (!settle<TM>(y + (size_t)(i - nxy) * 8 + c, rz, abortf, dstatus)) {
          cp_async_wait<0>();  // no copy of this warp is left in flight when it leaves
          return;
        }
        acc = fma(-az.x, rz.x, fma(-az.y, rz.y, acc));
      }
      if (hy) {
        if (!settle<TM>(y + (size_t)(i - nx) * 8 + c, ry, abortf, dstatus)) {
          cp_async_wait<0>();
          return;
        }
        acc = fma(-ay.x, ry.x, fma(-ay.y, ry.y, acc));
      }
      const TM t = quad_sum(acc);  // t_r = r - A v
      const TM t0 = __shfl_sync(FULL, t, 4 * c), t1 = __shfl_sync(FULL, t, 4 * c + 4);
      const TM yr = quad_sum(fma(d.x, t0, d.y * t1));
      if ((lane & 3) == 0) st_relaxed(y + (size_t)i * 8 + r, yr);
      yp0 = __shfl_sync(FULL, yr, 4 * c);
      yp1 = __shfl_sync(FULL, yr, 4 * c + 4);
      if (x + 1 < nx) {
        if (hz) ld_relaxed_v2(y + (size_t)(i + 1 - nxy) * 8 + c, rz.x, rz.y);
        if (hy) ld_relaxed_v2(y + (size_t)(i + 1 - nx) * 8 + c, ry.x, ry.y);
      }
      __syncwarp();  // every lane is done with this slot before it is refilled
    }
    cp_async_wait<0>();
    __syncwarp();
  }
}

template <typename TM, int R>
__global__ void __launch_bounds__(AWARPS * 32) k_sweep1_bwd(int nx, int ny, int nz, const TM* __restrict__ A,
                                                            const TM* __restrict__ Dinv, const TM* __restrict__ yin,
                                                            TM* __restrict__ zs, double* __restrict__ z64,
                                                            int* __restrict__ pipe, int* __restrict__ dstatus) {
  using T2 = typename V2<TM>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Slot1<TM>* ring = reinterpret_cast<Slot1<TM>*>(smem_raw) + (threadIdx.x >> 5) * R;
  const int lane = threadIdx.x & 31;
  const int r = lane >> 2, c = (lane & 3) * 2;
  const int npen = ny * nz, nxy = nx * ny;
  int* counter = pipe;
  int* abortf = pipe + 1;
  for (;;) {
    int g = 0;
    if (lane == 0) g = atomicAdd(counter, 1);
    g = __shfl_sync(FULL, g, 0);
    if (g >= npen) return;
    const int p = npen - 1 - g;
    const int j = p % ny, k = p / ny;
    const bool hy = j < ny - 1, hz = k < nz - 1;
    const int nlow_jk = (k > 0) + (j > 0);
    const int base_jk = nx * (j + ny * k);
    const Pen PEN = make_pen(nx, ny, nz, j, k, base_jk);
    // blocks of row (j, k, x) after the diagonal in order +x, +y, +z
    auto mask_of = [&](int x) { return (x < nx - 1 ? 1 : 0) | (hy ? 2 : 0) | (hz ? 4 : 0); };
    auto first_of = [&](int x) { return nlow_jk + (x > 0) + 1; };
#pragma unroll 1
    for (int q = 0; q < R - 1; ++q) {
      if (q < nx) {
        const int x = nx - 1 - q;
        stage_cell1<TM, TM>(ring + q, base_jk + x, first_of(x), mask_of(x), PEN, A, Dinv, yin, lane);
      }
      cp_async_commit();
    }
    T2 rz = zero2<TM>(), ry = zero2<TM>();
    if (hz) ld_relaxed_v2(zs + (size_t)(base_jk + nx - 1 + nxy) * 8 + c, rz.x, rz.y);
    if (hy) ld_relaxed_v2(zs + (size_t)(base_jk + nx - 1 + nx) * 8 + c, ry.x, ry.y);
    TM zp0 = TM(0), zp1 = TM(0);
    for (int step = 0; step < nx; ++step) {
      const int x = nx - 1 - step;
      const int i = base_jk + x;
      const int ss = step + R - 1;
      if (ss < nx)
        stage_cell1<TM, TM>(ring + ss % R, base_jk + (nx - 1 - ss), first_of(nx - 1 - ss), mask_of(nx - 1 - ss), PEN,
                            A, Dinv, yin, lane);
      cp_async_commit();
      cp_async_wait<R - 1>();
      __syncwarp();
      const Slot1<TM>* sl = ring + step % R;
      const int m = mask_of(x);
      int b = 0;
      T2 ax = zero2<TM>(), ay = zero2<TM>(), az = zero2<TM>();
      if (m & 1) ax = sl_pair<TM>(sl, b++, lane);
      if (m & 2) ay = sl_pair<TM>(sl, b++, lane);
      if (m & 4) az = sl_pair<TM>(sl, b, lane);
      const T2 d = sl_pair<TM>(sl, 3, lane);
      const TM yi = reinterpret_cast<const TM*>(sl->rhs)[r];  // the forward result, staged with the blocks
      TM acc = fma(ax.x, zp0, ax.y * zp1);
      if (hz) {
        if (!settle<TM>(zs + (size_t)(i + nxy) * 8 + c, rz, abortf, dstatus)) {
          cp_async_wait<0>();
          return;
        }
        acc = fma(az.x, rz.x, fma(az.y, rz.y, acc));
      }
      if (hy) {
        if (!settle<TM>(zs + (size_t)(i + nx) * 8 + c, ry, abortf, dstatus)) {
          cp_async_wait<0>();
          return;
        }
        acc = fma(ay.x, ry.x, fma(ay.y, ry.y, acc));
      }
      const TM sr = quad_sum(acc);  // (U z)_r
      const TM s0 = __shfl_sync(FULL, sr, 4 * c), s1 = __shfl_sync(FULL, sr, 4 * c + 4);
      // z_r = y_r - (D^-1 U z)_r: the quad sum starts from y_r / 4 on each lane
      const TM zr = quad_sum(fma(-d.x, s0, fma(-d.y, s1, yi * TM(0.25))));
      if ((lane & 3) == 0) {
        st_relaxed(zs + (size_t)i * 8 + r, zr);
        if (z64) z64[(size_t)i * 8 + r] = (double)zr;
      }
      zp0 = __shfl_sync(FULL, zr, 4 * c);
      zp1 = __shfl_sync(FULL, zr, 4 * c + 4);
      if (step + 1 < nx) {
        if (hz) ld_relaxed_v2(zs + (size_t)(i - 1 + nxy) * 8 + c, rz.x, rz.y);
        if (hy) ld_relaxed_v2(zs + (size_t)(i - 1 + nx) * 8 + c, ry.x, ry.y);
      }
      __syncwarp();
    }
    cp_async_wait<0>();
    __syncwarp();
  }
}

// slot of neighbour direction d (0 -z, 1 -y, 2 -x, 3 diag, 4 +x, 5 +y, 6 +z) in the sorted BSR row of cell c
__device__ __forceinline__ int slot_of(int nx, int ny, int nz, int c, int d) {
  const int ix = c % nx, iy = (c / nx) % ny, iz = c / (nx * ny);
  const bool has[7] = {iz > 0, iy > 0, ix > 0, true, ix < nx - 1, iy < ny - 1, iz < nz - 1};
  int s = 0;
#pragma unroll
  for (int e = 0; e < 7; ++e)
    if (e < d) s += has[e];
  return s;
}

// Factorisation D_i = A_ii - sum_{k lower} A_ik D_k^-1 A_ki and D_i^-1 (Gauss-Jordan with partial
// pivoting), same pencil pipeline; the hand-off is the neighbour's D^-1 block (NaN-filled before).
constexpr int FWARPS = 4;

template <typename T>
__global__ void __launch_bounds__(FWARPS * 32) k_ilu_factor_pipe(int nx, int ny, int nz,
                                                                 const int32_t* __restrict__ rowptr,
                                                                 const T* __restrict__ A, T* __restrict__ Dinv,
                                                                 T* __restrict__ uhat, int* __restrict__ pipe,
                                                                 int* __restrict__ dstatus) {
  using T2 = typename V2<T>::t;
  __shared__ T sm[FWARPS][6][64];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  T* sD = sm[wid][0];
  T* sI = sm[wid][1];
  T* sL = sm[wid][2];
  T* sU = sm[wid][3];
  T* sK = sm[wid][4];
  T* sP = sm[wid][5];  // D^-1 of the previous cell of this pencil
  const int r = lane >> 2, c = (lane & 3) * 2;
  const int npen = ny * nz, nxy = nx * ny;
  int* counter = pipe;
  int* abortf = pipe + 1;
  for (;;) {
    int p = 0;
    if (lane == 0) p = atomicAdd(counter, 1);
    p = __shfl_sync(FULL, p, 0);
    if (p >= npen) return;
    const int j = p % ny, k = p / ny;
    const int base_jk = nx * (j + ny * k);
    const Pen PEN = make_pen(nx, ny, nz, j, k, base_jk);
    for (int x = 0; x < nx; ++x) {
      const int i = base_jk + x;
      const int base = rowptr_of(nx, ny, nz, i);
      const int nlow = (k > 0) + (j > 0) + (x > 0);
      T2 d = ld_nc2(A + (size_t)(base + nlow) * BB + 2 * lane);
      // lower neighbours in pattern order -z, -y, -x
#pragma unroll
      for (int dl = 0; dl < 3; ++dl) {
        const bool ex = (dl == 0) ? (k > 0) : (dl == 1) ? (j > 0) : (x > 0);
        if (!ex) continue;
        const int kk = (dl == 0) ? i - nxy : (dl == 1) ? i - nx : i - 1;
        const int sl = slot_of(nx, ny, nz, i, dl);
        const int su = slot_of(nx, ny, nz, kk, 6 - dl);
        const T2 aik = ld_nc2(A + (size_t)(base + sl) * BB + 2 * lane);
        const T2 aki = ld_nc2(A + (size_t)(rowptr_of(nx, ny, nz, kk) + su) * BB + 2 * lane);
        T2 dk;
        if (dl < 2) {
          if (!poll_vec<T>(Dinv + (size_t)kk * BB, 2 * lane, dk, abortf, dstatus)) return;
        } else {
          dk.x = sP[2 * lane];
          dk.y = sP[2 * lane + 1];
        }
        __syncwarp();
        sL[2 * lane] = aik.x;
        sL[2 * lane + 1] = aik.y;
        sU[2 * lane] = aki.x;
        sU[2 * lane + 1] = aki.y;
        sK[2 * lane] = dk.x;
        sK[2 * lane + 1] = dk.y;
        __syncwarp();
        // M = D_k^-1 A_ki (entries (r, c), (r, c+1))
        T m0 = T(0), m1 = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          m0 = fma(sK[r * 8 + q], sU[q * 8 + c], m0);
          m1 = fma(sK[r * 8 + q], sU[q * 8 + c + 1], m1);
        }
        __syncwarp();
        sU[r * 8 + c] = m0;  // reuse sU for M
        sU[r * 8 + c + 1] = m1;
        // M = D_k^-1 A_ki is the pre-scaled upper block of row k towards i (+z, +y, +x for
        // dl = 0, 1, 2), which the backward sweep applies without D^-1
        if (uhat) {
          T* u = uhat + ((size_t)3 * kk + (2 - dl)) * BB + r * 8 + c;
          u[0] = m0;
          u[1] = m1;
        }
        __syncwarp();
        T s0 = T(0), s1 = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          s0 = fma(sL[r * 8 + q], sU[q * 8 + c], s0);
          s1 = fma(sL[r * 8 + q], sU[q * 8 + c + 1], s1);
        }
        d.x -= s0;
        d.y -= s1;
        __syncwarp();
      }
      // invert D by Gauss-Jordan with partial pivoting
      sD[2 * lane] = d.x;
      sD[2 * lane + 1] = d.y;
      sI[2 * lane] = (r == c) ? T(1) : T(0);
      sI[2 * lane + 1] = (r == c + 1) ? T(1) : T(0);
      __syncwarp();
      bool bad = false;
      for (int kp = 0; kp < 8; ++kp) {
        // pivot search on the integer bit patterns of |D| (same choice as a float compare;
        // keeps the FP64 pipe out of the wavefront's dependent chain)
        int piv = kp;
        typename MagBits<T>::U best = 0;
        for (int q = kp; q < 8; ++q) {
          const typename MagBits<T>::U v = MagBits<T>::get(sD[q * 8 + kp]);
          if (q == kp || v > best) {
            best = v;
            piv = q;
          }
        }
        if (best == 0 || best >= MagBits<T>::INF) {  // zero column, or inf / NaN
          bad = true;
          break;
        }
        if (piv != kp && r == kp) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            T t1 = sD[kp * 8 + c + e];
            sD[kp * 8 + c + e] = sD[piv * 8 + c + e];
            sD[piv * 8 + c + e] = t1;
            t1 = sI[kp * 8 + c + e];
            sI[kp * 8 + c + e] = sI[piv * 8 + c + e];
            sI[piv * 8 + c + e] = t1;
          }
        }
        __syncwarp();
        // one FMA per entry for every row: the pivot row becomes p (1 + (inv - 1)) = p inv,
        // row r != kp becomes a_r - (a_r,kp inv) p; the multiplier costs one FP64 op per lane
        const T inv = recip_nr(sD[kp * 8 + kp]);
        const T g = (r == kp) ? inv - T(1) : -sD[r * 8 + kp] * inv;
        const T p0 = sD[kp * 8 + c], p1 = sD[kp * 8 + c + 1];
        const T q0 = sI[kp * 8 + c], q1 = sI[kp * 8 + c + 1];
        __syncwarp();
        sD[r * 8 + c] = fma(g, p0, sD[r * 8 + c]);
        sD[r * 8 + c + 1] = fma(g, p1, sD[r * 8 + c + 1]);
        sI[r * 8 + c] = fma(g, q0, sI[r * 8 + c]);
        sI[r * 8 + c + 1] = fma(g, q1, sI[r * 8 + c + 1]);
        __syncwarp();
      }
      if (bad) {
        if (lane == 0) {
          atomicOr(dstatus, DS_SINGULAR);
          atomicExch(abortf, 1);
        }
        return;
      }
      const T o0 = sI[2 * lane], o1 = sI[2 * lane + 1];
      st_relaxed(Dinv + (size_t)i * BB + 2 * lane, o0);
      st_relaxed(Dinv + (size_t)i * BB + 2 * lane + 1, o1);
      sP[2 * lane] = o0;
      sP[2 * lane + 1] = o1;
      __syncwarp();
    }
  }
}


}  // namespace

// Factor the decoupled blocks: FP64 into dinv (and the pre-scaled upper blocks
// into uhat), or under mixed precision FP32 from the FP32 copy of the blocks
// (J32, written first) into dinv32 and uhat32.
void launch_ilu_factor_pipe(Handle& h, cudaStream_t s) {
  const int npen = h.ny * h.nz;
  // up to 32 warps per SM (38 registers, 12 KB of shared memory per 4-warp block):
  // more pencils in flight on the larger grids
  const int warps = npen < 152 * 32 ? npen : 152 * 32;
  const int blocks = (warps + FWARPS - 1) / FWARPS;
  cudaMemsetAsync(h.pipe, 0, 2 * sizeof(int), s);
  if (h.opt.precision != ISC_PRECISION_FP64) {
    launch_to_f32((size_t)h.nnzb * BB, h.J, h.J32, s);
    cudaMemsetAsync(h.dinv32, 0xff, sizeof(float) * (size_t)h.n * BB, s);  // NaN sentinel
    k_ilu_factor_pipe<float><<<blocks, FWARPS * 32, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J32, h.dinv32, h.uhat32,
                                                            h.pipe, h.dstatus);
    return;
  }
  cudaMemsetAsync(h.dinv, 0xff, sizeof(double) * (size_t)h.n * BB, s);  // NaN sentinel
  k_ilu_factor_pipe<double><<<blocks, FWARPS * 32, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J, h.dinv, h.uhat, h.pipe,
                                                           h.dstatus);
}

namespace {

// cells staged in each warp's shared-memory ring, per precision
constexpr int SWEEP_R64 = 4;
constexpr int SWEEP_R32 = 4;
template <typename TM>
constexpr int sweep_r() {
  return sizeof(TM) == 8 ? SWEEP_R64 : SWEEP_R32;
}

template <typename TM, typename RT>
size_t sweep_smem() {
  return sizeof(Slot2<TM, RT>) * sweep_r<TM>() * AWARPS;
}

// tasks of the anti-diagonal map: ceil(len/2) per diagonal of the ny x nz pencil grid
int sweep_tasks(int ny, int nz) {
  int t = 0;
  for (int d = 0; d <= ny + nz - 2; ++d) {
    const int jlo = d - (nz - 1) > 0 ? d - (nz - 1) : 0;
    const int jhi = d < ny - 1 ? d : ny - 1;
    t += (jhi - jlo + 2) / 2;
  }
  return t;
}

// Persistent grid: no more warps than tasks, and no more blocks than fit on
// the device at once (resident blocks from the occupancy calculator).
template <typename K>
int sweep_blocks(K kernel, size_t smem, int tasks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, AWARPS * 32, smem);
  if (per_sm < 1) per_sm = 1;
  const int need = (tasks + AWARPS - 1) / AWARPS;
  return need < per_sm * sms ? need : per_sm * sms;
}

// Grids with at most this many x-pencils run the one-pencil-per-warp sweeps
// (latency-bound wavefront); larger grids the pencil pairs (FP64-pipe- or
// HBM-bound). Measured per apply, one pencil / pairs: 1,200 pencils (60x60x20)
// 0.331 / 0.393 ms FP64, 0.230 / 0.249 ms FP32; 3,000 (100x100x30) 0.739 /
// 0.759 and 0.423 / 0.441; 3,600 (120x120x30) 0.990 / 0.900 and 0.512 / 0.532;
// 10,000 (200x200x50) FP32 1.53 / 1.16.
constexpr int SWEEP1_MAX_PENCILS64 = 3000;
constexpr int SWEEP1_MAX_PENCILS32 = 3600;
template <typename TM>
constexpr int sweep1_max() {
  return sizeof(TM) == 8 ? SWEEP1_MAX_PENCILS64 : SWEEP1_MAX_PENCILS32;
}

template <typename TM, typename RT>
cudaError_t launch_fwd(int nx, int ny, int nz, const TM* A, const TM* Dinv, const RT* r, TM* y, int* pipe,
                       int* dstatus, cudaStream_t s) {
  if (ny * nz <= sweep1_max<TM>()) {
    auto kern = k_sweep1_fwd<TM, sweep_r<TM>(), RT>;
    const size_t smem = sizeof(Slot1<TM>) * sweep_r<TM>() * AWARPS;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(pipe, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(y, 0xff, sizeof(TM) * (size_t)nx * ny * nz * 8, s);  // NaN sentinel
    if (e != cudaSuccess) return e;
    kern<<<sweep_blocks(kern, smem, ny * nz), AWARPS * 32, smem, s>>>(nx, ny, nz, A, Dinv, r, y, pipe, dstatus);
    return cudaGetLastError();
  }
  auto kern = k_sweep_fwd<TM, sweep_r<TM>(), RT>;
  const size_t smem = sweep_smem<TM, RT>();
  // idempotent; the rings need more than the default 48 KB of dynamic shared memory
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(pipe, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(y, 0xff, sizeof(TM) * (size_t)nx * ny * nz * 8, s);  // NaN sentinel
  if (e != cudaSuccess) return e;
  kern<<<sweep_blocks(kern, smem, sweep_tasks(ny, nz)), AWARPS * 32, smem, s>>>(nx, ny, nz, A, Dinv, r, y, pipe,
                                                                                  dstatus);
  return cudaGetLastError();
}

template <typename TM, bool PRE>
cudaError_t launch_bwd(int nx, int ny, int nz, const TM* A, const TM* Dinv, const TM* uhat, const TM* y, TM* z,
                       double* z64, int* pipe, int* dstatus, cudaStream_t s) {
  if (ny * nz <= sweep1_max<TM>()) {  // (the one-pencil sweep applies D^-1 to the unscaled upper blocks)
    auto kern = k_sweep1_bwd<TM, sweep_r<TM>()>;
    const size_t smem = sizeof(Slot1<TM>) * sweep_r<TM>() * AWARPS;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(pipe, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(z, 0xff, sizeof(TM) * (size_t)nx * ny * nz * 8, s);  // NaN sentinel
    if (e != cudaSuccess) return e;
    kern<<<sweep_blocks(kern, smem, ny * nz), AWARPS * 32, smem, s>>>(nx, ny, nz, A, Dinv, y, z, z64, pipe, dstatus);
    return cudaGetLastError();
  }
  auto kern = k_sweep_bwd<TM, sweep_r<TM>(), PRE>;
  const size_t smem = sweep_smem<TM, TM>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(pipe, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(z, 0xff, sizeof(TM) * (size_t)nx * ny * nz * 8, s);  // NaN sentinel
  if (e != cudaSuccess) return e;
  kern<<<sweep_blocks(kern, smem, sweep_tasks(ny, nz)), AWARPS * 32, smem, s>>>(nx, ny, nz, A, Dinv, uhat, y, z,
                                                                                  z64, pipe, dstatus);
  return cudaGetLastError();
}

}  // namespace

// FP32 in, FP32 out (inner solve of ISC_PRECISION_MIXED_FGMRES): y in vec32, z written as the hand-off vector
void launch_ilu_apply_f32(Handle& h, const float* r, float* z, cudaStream_t s) {
  launch_fwd<float, float>(h.nx, h.ny, h.nz, h.J32, h.dinv32, r, h.vec32, h.pipe, h.dstatus, s);
  launch_bwd<float, true>(h.nx, h.ny, h.nz, h.J32, h.dinv32, h.uhat32, h.vec32, z, nullptr, h.pipe, h.dstatus, s);
}

void launch_ilu_apply_pipe(Handle& h, const double* r, double* z, cudaStream_t s) {
  if (h.opt.precision != ISC_PRECISION_FP64) {
    // FP64 right-hand side in, FP32 sweeps, FP64 result out
    const size_t n8 = (size_t)h.n * 8;
    launch_fwd<float, double>(h.nx, h.ny, h.nz, h.J32, h.dinv32, r, h.vec32, h.pipe, h.dstatus, s);
    launch_bwd<float, true>(h.nx, h.ny, h.nz, h.J32, h.dinv32, h.uhat32, h.vec32, h.vec32 + n8, z, h.pipe, h.dstatus,
                            s);
    return;
  }
  launch_fwd<double, double>(h.nx, h.ny, h.nz, h.J, h.dinv, r, h.tmp, h.pipe, h.dstatus, s);
  launch_bwd<double, true>(h.nx, h.ny, h.nz, h.J, h.dinv, h.uhat, h.tmp, z, nullptr, h.pipe, h.dstatus, s);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the ILU(0) apply for callers that cannot call
// cudaMalloc (for example code running inside another framework's memory
// pool, or a host that has no allocation rights). Its scratch -- the
// intermediate vector of the forward sweep, the sweep counter, the abort flag
// and a status word -- lives in this file-scope device array, which every GPU
// that loads the library holds until the process exits.
namespace {

constexpr size_t NOALLOC_INTS = 64;  // counter, abort flag, status word, padding to 256 bytes
static __device__ __align__(256) double g_noalloc_scratch[(size_t)ISC_NOALLOC_MAX_CELLS * 8 + NOALLOC_INTS / 2];

// Host code may not use g_noalloc_scratch as an address: its device address is
// resolved on every call, with the caller's device current (cheap next to the
// synchronising sweeps, and never stale after a context is re-created).
int noalloc_scratch(double** out) {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return ISC_ERR_CUDA;
  *out = static_cast<double*>(ptr);
  return ISC_OK;
}

}  // namespace

namespace {

// Both closed forms of the BSR row starts that the sweeps and the factorisation
// compute instead of loading rowptr (rowptr_of per cell, row_start along a
// pencil) against rowptr itself: one thread per cell, mismatches counted, the
// first mismatching cell kept (atomicMin).
__global__ void k_check_row_starts(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                   unsigned long long* __restrict__ count, int* __restrict__ first) {
  const long long n = (long long)nx * ny * nz;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c <= n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)c;
    bool ok;
    if (c == n) {
      ok = 7 * i - (2 * ny * nz + 2 * nx * nz + 2 * nx * ny) == rowptr[n];  // the total block count
    } else {
      const int x = i % nx, j = (i / nx) % ny, k = i / (nx * ny);
      const Pen P = make_pen(nx, ny, nz, j, k, i - x);
      ok = rowptr_of(nx, ny, nz, i) == rowptr[i] && row_start(P, x) == rowptr[i];
    }
    if (!ok) {
      atomicAdd(count, 1ull);
      atomicMin(first, i);
    }
  }
}

}  // namespace

}  // namespace isc

extern "C" int isc_check_row_starts(int32_t nx, int32_t ny, int32_t nz, const int32_t* rowptr, int64_t* mismatches,
                                    int32_t* first_cell) {
  using namespace isc;
  if (nx < 1 || ny < 1 || nz < 1 || !rowptr || !mismatches || !first_cell) return ISC_ERR_INVALID_ARG;
  const long long n = (long long)nx * ny * nz;
  if (n * 7 > (long long)INT32_MAX || n > (1LL << 28)) return ISC_ERR_INVALID_ARG;
  int32_t* d_rp = nullptr;
  unsigned long long* d_count = nullptr;
  int* d_first = nullptr;
  int st = ISC_OK;
  if (cudaMalloc(&d_rp, sizeof(int32_t) * (size_t)(n + 1)) != cudaSuccess ||
      cudaMalloc(&d_count, sizeof(unsigned long long)) != cudaSuccess || cudaMalloc(&d_first, sizeof(int)) != cudaSuccess)
    st = ISC_ERR_NOMEM;
  if (st == ISC_OK) {
    const int big = INT32_MAX;
    bool ok = cudaMemcpy(d_rp, rowptr, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(d_count, 0, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMemcpy(d_first, &big, sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
      k_check_row_starts<<<152 * 8, 256>>>(nx, ny, nz, d_rp, d_count, d_first);
      ok = cudaGetLastError() == cudaSuccess;
    }
    unsigned long long cnt = 0;
    int first = big;
    if (!ok || cudaMemcpy(&cnt, d_count, sizeof(cnt), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&first, d_first, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = ISC_ERR_CUDA;
    } else {
      *mismatches = (int64_t)cnt;
      *first_cell = cnt ? first : -1;
    }
  }
  cudaFree(d_rp);
  cudaFree(d_count);
  cudaFree(d_first);
  return st;
}

// Failure-detection self-test: a forward sweep on a 4x4x1 grid whose pencil
// counter starts at 1, so pencil 0 is never processed and pencil 1's wait on it
// can only end by its iteration limit. Returns ISC_ERR_TIMEOUT when the bounded
// wait gave up and reported it (the expected outcome), ISC_OK if it did not.
extern "C" int isc_check_bounded_wait(void) {
  using namespace isc;
  const int nx = 4, ny = 4, nz = 1, n = nx * ny * nz;
  std::vector<int32_t> rp(n + 1, 0);
  int nnzb = 0;
  for (int j = 0; j < ny; ++j)
    for (int x = 0; x < nx; ++x) {
      nnzb += 1 + (x > 0) + (x < nx - 1) + (j > 0) + (j < ny - 1);
      rp[x + nx * j + 1] = nnzb;
    }
  std::vector<double> dinv((size_t)n * BB, 0.0);
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 8; ++a) dinv[(size_t)i * BB + a * 9] = 1.0;
  int32_t* d_rp = nullptr;
  double *d_A = nullptr, *d_D = nullptr, *d_r = nullptr, *d_y = nullptr;
  int* d_ints = nullptr;
  int st = ISC_OK;
  if (cudaMalloc(&d_rp, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
      cudaMalloc(&d_A, sizeof(double) * (size_t)nnzb * BB) != cudaSuccess ||
      cudaMalloc(&d_D, sizeof(double) * (size_t)n * BB) != cudaSuccess ||
      cudaMalloc(&d_r, sizeof(double) * (size_t)n * 8) != cudaSuccess ||
      cudaMalloc(&d_y, sizeof(double) * (size_t)n * 8) != cudaSuccess ||
      cudaMalloc(&d_ints, sizeof(int) * 4) != cudaSuccess)
    st = ISC_ERR_NOMEM;
  if (st == ISC_OK) {
    const int h_ints[4] = {1, 0, 0, 0};  // counter = 1 (pencil 0 skipped), abort, status
    bool ok = cudaMemcpy(d_rp, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(d_A, 0, sizeof(double) * (size_t)nnzb * BB) == cudaSuccess &&
              cudaMemcpy(d_D, dinv.data(), sizeof(double) * (size_t)n * BB, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(d_r, 0, sizeof(double) * (size_t)n * 8) == cudaSuccess &&
              cudaMemcpy(d_ints, h_ints, sizeof(h_ints), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
      // the forward sweep, its counter then moved past task 0 (pencil 0 of the 4x4x1 grid):
      // pencil 1 waits for values that never arrive
      auto kern = k_sweep_fwd<double, sweep_r<double>(), double>;
      const size_t smem = sweep_smem<double, double>();
      ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
           cudaMemset(d_y, 0xff, sizeof(double) * (size_t)n * 8) == cudaSuccess;  // NaN sentinel
      if (ok) {
        kern<<<1, AWARPS * 32, smem>>>(nx, ny, nz, d_A, d_D, d_r, d_y, d_ints, d_ints + 2);
        ok = cudaGetLastError() == cudaSuccess;
      }
    }
    int h_status = 0;
    // a set-up or launch failure is ISC_ERR_CUDA, never the "no timeout" answer
    if (!ok || cudaMemcpy(&h_status, d_ints + 2, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = ISC_ERR_CUDA;
    else
      st = (h_status & DS_TIMEOUT) ? ISC_ERR_TIMEOUT : ISC_OK;
  }
  cudaFree(d_rp);
  cudaFree(d_A);
  cudaFree(d_D);
  cudaFree(d_r);
  cudaFree(d_y);
  cudaFree(d_ints);
  return st;
}

extern "C" int isc_bilu0_apply_noalloc(int32_t nx, int32_t ny, int32_t nz, const int32_t* d_rowptr,
                                       const double* d_A, const double* d_Dinv, const double* d_r, double* d_z,
                                       void* stream) {
  using namespace isc;
  if (nx < 1 || ny < 1 || nz < 1) return ISC_ERR_INVALID_ARG;
  const long long n = (long long)nx * ny * nz;
  if (n > ISC_NOALLOC_MAX_CELLS) return ISC_ERR_INVALID_ARG;  // beyond the static scratch
  if (!d_rowptr || !d_A || !d_Dinv || !d_r || !d_z) return ISC_ERR_INVALID_ARG;
  double* scratch = nullptr;
  int st = noalloc_scratch(&scratch);
  if (st != ISC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* y = scratch;                                                  // 8n doubles
  int* ints = reinterpret_cast<int*>(scratch + (size_t)ISC_NOALLOC_MAX_CELLS * 8);
  int* pipe = ints;                                                     // counter, abort flag
  int* status = ints + 2;
  // everything that must start at zero (or NaN) is cleared inside: the array
  // keeps the previous call's contents
  if (cudaMemsetAsync(ints, 0, NOALLOC_INTS * sizeof(int), s) != cudaSuccess) return ISC_ERR_CUDA;
  // the caller gives D^-1 and the BSR blocks only: the backward sweep applies D^-1 itself
  if (launch_fwd<double, double>(nx, ny, nz, d_A, d_Dinv, d_r, y, pipe, status, s) != cudaSuccess ||
      launch_bwd<double, false>(nx, ny, nz, d_A, d_Dinv, nullptr, y, d_z, nullptr, pipe, status, s) != cudaSuccess)
    return ISC_ERR_CUDA;
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ISC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ISC_ERR_CUDA;
  if (h_status & DS_TIMEOUT) return ISC_ERR_TIMEOUT;
  return ISC_OK;
}
