// Pencil-pipelined triangular sweeps of the block ILU(0) preconditioner.
//
// For the 7-point pattern in natural order, ILU(0) keeps the off-diagonal
// blocks of A and changes only the diagonal (D-ILU form):
//   forward   y_i = D_i^-1 (r_i - A_{i,i-1} y_{i-1} - A_{i,i-nx} y_{i-nx} - A_{i,i-nxy} y_{i-nxy})
//   backward  z_i = y_i - D_i^-1 (A_{i,i+1} z_{i+1} + A_{i,i+nx} z_{i+nx} + A_{i,i+nxy} z_{i+nxy})
// Cell i depends on its x-predecessor (same pencil) and on the pencils
// (j-1,k) and (j,k-1) at the same x. One warp owns a whole x-pencil, so the
// x-recurrence stays in registers; pencils are taken from a counter in
// dependency order (so a warp only ever waits on pencils already held by
// running warps). The cross-pencil hand-off is the data itself: the output
// vector is filled with a NaN sentinel before a sweep and a consumer polls the
// neighbour's 64-byte block vector until the sentinel is gone; these values
// are requested LA cells before use. The matrix operands of upcoming cells are streamed into a
// per-warp shared-memory ring with cp.async. Row starts are computed, not
// loaded. Every wait is bounded: on timeout the kernel raises DS_TIMEOUT and a
// global abort flag that makes every other waiter return.
//
// Measured on the 60x60x20 field step, a lone pencil costs ~0.3 us (FP32) to
// ~0.6 us (FP64) per cell of sequential recurrence, and each pencil-to-pencil
// hand-off adds about one cell time plus ~0.5 us; the sweep time is that
// per-cell chain times the nx + ny + nz - 2 cells of the wavefront, not memory
// bandwidth.
//
// Lane layout per 8x8 block (row-major, 64 doubles): lane l holds the double2
// at offset 2l, i.e. row r = l/4, columns c = 2(l%4), c+1; a row sum is a
// reduction over the 4 lanes of a quad.
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

// Remote look-ahead: the neighbour-pencil values a cell needs are requested LA
// cells before they are used; entries still NaN on use are re-polled. A request
// only finds the value if the consumer trails its producer by about LA cells,
// so every pencil-to-pencil hand-off adds that lag to the wavefront: one cell
// ahead is the best measured (sweep pair 347 / 387 / 388 us for LA = 1 / 2 / 4
// in FP64 at 60x60x20, 241 / 283 / 279 us in FP32).
constexpr int LA = 1;

template <typename TM>
__device__ __forceinline__ typename V2<TM>::t ld_remote(const TM* p) {
  typename V2<TM>::t v;
  ld_relaxed_v2(p, v.x, v.y);
  return v;
}

template <typename TM>
__device__ __forceinline__ bool ready2(const typename V2<TM>::t& v) {
  return arrived(v.x) && arrived(v.y);
}

// re-poll until the lane pair is a number everywhere in the warp
template <typename TM>
__device__ __forceinline__ bool settle(const TM* p, typename V2<TM>::t& v, int* abortf, int* dstatus) {
  if (__all_sync(FULL, ready2<TM>(v))) return true;
  return poll_vec<TM>(p, 0, v, abortf, dstatus);
}

// ------------------------------------------------- shared-memory operand pipeline
// The operands of a cell (its up-to-three off-diagonal blocks of the sweep
// direction, D^-1 and the right-hand side) do not depend on the sweep. Each
// warp streams them into its own ring of R cell slots in shared memory with
// cp.async, R-1 cells ahead of use, so the per-cell chain no longer waits on
// DRAM. Every iteration commits exactly one group (possibly empty) and waits
// until the group of the current cell has landed (a hardware wait).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gsrc), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename TM>
struct Slot {
  TM blk[4][64];   // up to 3 off-diagonal blocks and D^-1 (index 3)
  double rhs[8];
};

// issue the copies of one cell into a slot: blocks at row slots first_slot.. (mask says which exist)
template <typename TM, typename RT = double>
__device__ __forceinline__ void stage_cell(Slot<TM>* sl, int i, int first_slot, int mask, const Pen& P,
                                           const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                           const RT* __restrict__ rhs, int lane) {
  const int base = row_start(P, i - P.base_jk);
  int s = first_slot, dst = 0;  // present blocks are packed into blk[0..] in row order
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (mask & (1 << b)) {
      cp_async<2 * sizeof(TM)>(&sl->blk[dst][2 * lane], A + (size_t)(base + s) * BB + 2 * lane);
      ++s;
      ++dst;
    }
  }
  cp_async<2 * sizeof(TM)>(&sl->blk[3][2 * lane], Dinv + (size_t)i * BB + 2 * lane);
  // the right-hand side is FP64, or FP32 in the inner solve of the mixed-precision scheme
  if (rhs && lane < 8) cp_async<sizeof(RT)>(reinterpret_cast<RT*>(sl->rhs) + lane, rhs + (size_t)i * 8 + lane);
}

template <typename TM>
__device__ __forceinline__ typename V2<TM>::t sl_pair(const Slot<TM>* sl, int b, int lane) {
  return *reinterpret_cast<const typename V2<TM>::t*>(&sl->blk[b][2 * lane]);
}

// warps per block of the sweeps: 4 (six FP64 blocks per SM) ran the 100x100x30 sweep pair in
// 0.74-0.76 ms against 0.82 ms with 8 (three blocks per SM); equal at 60x60x20
constexpr int AWARPS = 4;

template <typename TM, int R, typename RT = double>
__global__ void __launch_bounds__(AWARPS * 32) k_ilu_fwd_async(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                                               const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                                               const RT* __restrict__ rhs, TM* __restrict__ y,
                                                               int* __restrict__ pipe, int* __restrict__ dstatus) {
  using T2 = typename V2<TM>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Slot<TM>* ring = reinterpret_cast<Slot<TM>*>(smem_raw) + (threadIdx.x >> 5) * R;
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
    // blocks of row (j,k,x) in order -z, -y, -x
    auto mask_of = [&](int x) { return (hz ? 1 : 0) | (hy ? 2 : 0) | (x > 0 ? 4 : 0); };
#pragma unroll 1
    for (int q = 0; q < R - 1; ++q) {
      if (q < nx) stage_cell<TM, RT>(ring + q, base_jk + q, 0, mask_of(q), PEN, A, Dinv, rhs, lane);
      cp_async_commit();
    }
    T2 rz[LA], ry[LA];
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      if (q < nx) {
        if (hz) rz[q] = ld_remote<TM>(y + (size_t)(base_jk + q - nxy) * 8 + c);
        if (hy) ry[q] = ld_remote<TM>(y + (size_t)(base_jk + q - nx) * 8 + c);
      }
    }
    TM yp0 = TM(0), yp1 = TM(0);
    for (int x0 = 0; x0 < nx; x0 += LA) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int x = x0 + q;
        if (x >= nx) break;
        const int i = base_jk + x;
        const int xs = x + R - 1;
        if (xs < nx) stage_cell<TM, RT>(ring + xs % R, base_jk + xs, 0, mask_of(xs), PEN, A, Dinv, rhs, lane);
        cp_async_commit();
        cp_async_wait<R - 1>();
        __syncwarp();
        const Slot<TM>* sl = ring + x % R;
        const int m = mask_of(x);
        int b = 0;
        T2 az = zero2<TM>(), ay = zero2<TM>(), ax = zero2<TM>();
        if (m & 1) az = sl_pair<TM>(sl, b++, lane);
        if (m & 2) ay = sl_pair<TM>(sl, b++, lane);
        if (m & 4) ax = sl_pair<TM>(sl, b, lane);
        const T2 d = sl_pair<TM>(sl, 3, lane);
        const TM ri = (TM)reinterpret_cast<const RT*>(sl->rhs)[r];
        TM acc = fma(ax.x, yp0, ax.y * yp1);
        if (hz) {
          if (!settle<TM>(y + (size_t)(i - nxy) * 8 + c, rz[q], abortf, dstatus)) {
            cp_async_wait<0>();  // no copy of this warp is left in flight when it leaves
            return;
          }
          acc = fma(az.x, rz[q].x, fma(az.y, rz[q].y, acc));
        }
        if (hy) {
          if (!settle<TM>(y + (size_t)(i - nx) * 8 + c, ry[q], abortf, dstatus)) {
            cp_async_wait<0>();  // no copy of this warp is left in flight when it leaves
            return;
          }
          acc = fma(ay.x, ry[q].x, fma(ay.y, ry[q].y, acc));
        }
        const TM t = ri - quad_sum(acc);
        const TM t0 = __shfl_sync(FULL, t, 4 * c), t1 = __shfl_sync(FULL, t, 4 * c + 4);
        const TM yr = quad_sum(fma(d.x, t0, d.y * t1));
        if ((lane & 3) == 0) st_relaxed(y + (size_t)i * 8 + r, yr);
        yp0 = __shfl_sync(FULL, yr, 4 * c);
        yp1 = __shfl_sync(FULL, yr, 4 * c + 4);
        if (x + LA < nx) {
          if (hz) rz[q] = ld_remote<TM>(y + (size_t)(i + LA - nxy) * 8 + c);
          if (hy) ry[q] = ld_remote<TM>(y + (size_t)(i + LA - nx) * 8 + c);
        }
        __syncwarp();  // every lane is done with this slot before it is refilled
      }
    }
    cp_async_wait<0>();
    __syncwarp();
  }
}

template <typename TM, int R>
__global__ void __launch_bounds__(AWARPS * 32) k_ilu_bwd_async(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                                               const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                                               const TM* __restrict__ yin, TM* __restrict__ zs,
                                                               double* __restrict__ z64, int* __restrict__ pipe,
                                                               int* __restrict__ dstatus) {
  using T2 = typename V2<TM>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Slot<TM>* ring = reinterpret_cast<Slot<TM>*>(smem_raw) + (threadIdx.x >> 5) * R;
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
    // blocks of row (j,k,x) after the diagonal in order +x, +y, +z; slot index of b is its bit
    auto mask_of = [&](int x) { return (x < nx - 1 ? 1 : 0) | (hy ? 2 : 0) | (hz ? 4 : 0); };
    auto first_of = [&](int x) { return nlow_jk + (x > 0) + 1; };
#pragma unroll 1
    for (int q = 0; q < R - 1; ++q) {
      if (q < nx) {
        const int x = nx - 1 - q;
        stage_cell<TM, TM>(ring + q, base_jk + x, first_of(x), mask_of(x), PEN, A, Dinv, yin, lane);
      }
      cp_async_commit();
    }
    T2 rz[LA], ry[LA];
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      if (q < nx) {
        const int x = nx - 1 - q;
        if (hz) rz[q] = ld_remote<TM>(zs + (size_t)(base_jk + x + nxy) * 8 + c);
        if (hy) ry[q] = ld_remote<TM>(zs + (size_t)(base_jk + x + nx) * 8 + c);
      }
    }
    TM zp0 = TM(0), zp1 = TM(0);
    for (int s0 = 0; s0 < nx; s0 += LA) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int step = s0 + q;
        if (step >= nx) break;
        const int x = nx - 1 - step;
        const int i = base_jk + x;
        const int ss = step + R - 1;
        if (ss < nx)
          stage_cell<TM, TM>(ring + ss % R, base_jk + (nx - 1 - ss), first_of(nx - 1 - ss), mask_of(nx - 1 - ss), PEN,
                             A, Dinv, yin, lane);
        cp_async_commit();
        cp_async_wait<R - 1>();
        __syncwarp();
        const Slot<TM>* sl = ring + step % R;
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
          if (!settle<TM>(zs + (size_t)(i + nxy) * 8 + c, rz[q], abortf, dstatus)) {
            cp_async_wait<0>();  // no copy of this warp is left in flight when it leaves
            return;
          }
          acc = fma(az.x, rz[q].x, fma(az.y, rz[q].y, acc));
        }
        if (hy) {
          if (!settle<TM>(zs + (size_t)(i + nx) * 8 + c, ry[q], abortf, dstatus)) {
            cp_async_wait<0>();  // no copy of this warp is left in flight when it leaves
            return;
          }
          acc = fma(ay.x, ry[q].x, fma(ay.y, ry[q].y, acc));
        }
        const TM sr = quad_sum(acc);
        const TM s_0 = __shfl_sync(FULL, sr, 4 * c), s_1 = __shfl_sync(FULL, sr, 4 * c + 4);
        const TM zr = yi - quad_sum(fma(d.x, s_0, d.y * s_1));
        if ((lane & 3) == 0) {
          st_relaxed(zs + (size_t)i * 8 + r, zr);
          if (z64) z64[(size_t)i * 8 + r] = (double)zr;
        }
        zp0 = __shfl_sync(FULL, zr, 4 * c);
        zp1 = __shfl_sync(FULL, zr, 4 * c + 4);
        if (step + LA < nx) {
          if (hz) rz[q] = ld_remote<TM>(zs + (size_t)(i - LA + nxy) * 8 + c);
          if (hy) ry[q] = ld_remote<TM>(zs + (size_t)(i - LA + nx) * 8 + c);
        }
        __syncwarp();
      }
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
                                                                 int* __restrict__ pipe, int* __restrict__ dstatus) {
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
        const T inv = recip_nr(sD[kp * 8 + kp]);
        const T f = sD[r * 8 + kp];
        __syncwarp();
        if (r == kp) {
          sD[kp * 8 + c] *= inv;
          sD[kp * 8 + c + 1] *= inv;
          sI[kp * 8 + c] *= inv;
          sI[kp * 8 + c + 1] *= inv;
        }
        __syncwarp();
        if (r != kp) {
          sD[r * 8 + c] -= f * sD[kp * 8 + c];
          sD[r * 8 + c + 1] -= f * sD[kp * 8 + c + 1];
          sI[r * 8 + c] -= f * sI[kp * 8 + c];
          sI[r * 8 + c + 1] -= f * sI[kp * 8 + c + 1];
        }
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

// Factor the decoupled blocks: FP64 into dinv, or under mixed precision FP32
// from the FP32 copy of the blocks (J32, written first) into dinv32.
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
    k_ilu_factor_pipe<float><<<blocks, FWARPS * 32, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J32, h.dinv32, h.pipe,
                                                            h.dstatus);
    return;
  }
  cudaMemsetAsync(h.dinv, 0xff, sizeof(double) * (size_t)h.n * BB, s);  // NaN sentinel
  k_ilu_factor_pipe<double><<<blocks, FWARPS * 32, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J, h.dinv, h.pipe,
                                                           h.dstatus);
}

// cells staged in each warp's shared-memory ring: 4 keeps an FP64 warp at 8.4 KB, so 24
// warps fit on an SM; with 8 an 8-warp block took 135 KB, one per SM, and 3,000 pencils
// (100x100x30) ran in two rounds (sweep pair 1.13 against 0.89 ms; equal at 60x60x20)
constexpr int SWEEP_R = 4;

// resident warps per SM: 24 for the FP64 sweeps (registers and the 68 KB rings), 32 for
// the FP32 ones (35 KB rings, fewer registers)
template <typename TM>
int sweep_blocks(int npen) {
  constexpr int per_sm = sizeof(TM) == 8 ? 24 : 32;
  const int warps = npen < 152 * per_sm ? npen : 152 * per_sm;
  return (warps + AWARPS - 1) / AWARPS;
}

template <typename TM>
size_t sweep_smem() {
  return sizeof(Slot<TM>) * SWEEP_R * AWARPS;
}

template <typename TM>
cudaError_t sweep_attributes() {
  // idempotent; the rings need more than the default 48 KB of dynamic shared memory
  cudaError_t e = cudaFuncSetAttribute(k_ilu_fwd_async<TM, SWEEP_R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sweep_smem<TM>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ilu_fwd_async<TM, SWEEP_R, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep_smem<TM>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ilu_bwd_async<TM, SWEEP_R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep_smem<TM>());
  return e;
}

// Forward and backward sweep on the stream; returns the first error of the
// attribute calls, the clears or the launches (cudaSuccess if all were issued).
template <typename TM>
cudaError_t sweep_pair(int nx, int ny, int nz, const int32_t* rowptr, const TM* A, const TM* Dinv, const double* r,
                       TM* y, TM* zs, double* z64, int* pipe, int* dstatus, cudaStream_t s) {
  const size_t n8 = (size_t)nx * ny * nz * 8;
  const int blocks = sweep_blocks<TM>(ny * nz);
  const size_t smem = sweep_smem<TM>();
  cudaError_t e = sweep_attributes<TM>();
  if (e == cudaSuccess) e = cudaMemsetAsync(pipe, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(y, 0xff, sizeof(TM) * n8, s);  // NaN sentinel
  if (e != cudaSuccess) return e;
  k_ilu_fwd_async<TM, SWEEP_R><<<blocks, AWARPS * 32, smem, s>>>(nx, ny, nz, rowptr, A, Dinv, r, y, pipe, dstatus);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(pipe, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(zs, 0xff, sizeof(TM) * n8, s);
  if (e != cudaSuccess) return e;
  k_ilu_bwd_async<TM, SWEEP_R><<<blocks, AWARPS * 32, smem, s>>>(nx, ny, nz, rowptr, A, Dinv, y, zs, z64, pipe,
                                                                 dstatus);
  return cudaGetLastError();
}

// FP32 in, FP32 out (inner solve of ISC_PRECISION_MIXED_FGMRES): y in vec32, z written as the hand-off vector
void launch_ilu_apply_f32(Handle& h, const float* r, float* z, cudaStream_t s) {
  const size_t n8 = (size_t)h.n * 8;
  const int blocks = sweep_blocks<float>(h.ny * h.nz);
  const size_t smem = sweep_smem<float>();
  sweep_attributes<float>();
  cudaMemsetAsync(h.pipe, 0, 2 * sizeof(int), s);
  cudaMemsetAsync(h.vec32, 0xff, sizeof(float) * n8, s);  // NaN sentinel
  k_ilu_fwd_async<float, SWEEP_R, float><<<blocks, AWARPS * 32, smem, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J32, h.dinv32,
                                                                           r, h.vec32, h.pipe, h.dstatus);
  cudaMemsetAsync(h.pipe, 0, 2 * sizeof(int), s);
  cudaMemsetAsync(z, 0xff, sizeof(float) * n8, s);
  k_ilu_bwd_async<float, SWEEP_R><<<blocks, AWARPS * 32, smem, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J32, h.dinv32, h.vec32,
                                                                    z, nullptr, h.pipe, h.dstatus);
}

void launch_ilu_apply_pipe(Handle& h, const double* r, double* z, cudaStream_t s) {
  if (h.opt.precision != ISC_PRECISION_FP64) {
    const size_t n8 = (size_t)h.n * 8;
    sweep_pair<float>(h.nx, h.ny, h.nz, h.rowptr, h.J32, h.dinv32, r, h.vec32, h.vec32 + n8, z, h.pipe, h.dstatus, s);
    return;
  }
  sweep_pair<double>(h.nx, h.ny, h.nz, h.rowptr, h.J, h.dinv, r, h.tmp, z, nullptr, h.pipe, h.dstatus, s);
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

}  // namespace isc

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
              // NaN sentinel: nothing arrives from pencil 0
              cudaMemset(d_y, 0xff, sizeof(double) * (size_t)n * 8) == cudaSuccess &&
              cudaMemcpy(d_ints, h_ints, sizeof(h_ints), cudaMemcpyHostToDevice) == cudaSuccess &&
              sweep_attributes<double>() == cudaSuccess;
    if (ok) {
      const size_t smem = sweep_smem<double>();
      k_ilu_fwd_async<double, SWEEP_R><<<1, AWARPS * 32, smem>>>(nx, ny, nz, d_rp, d_A, d_D, d_r, d_y, d_ints,
                                                                  d_ints + 2);
      ok = cudaGetLastError() == cudaSuccess;
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
  if (sweep_pair<double>(nx, ny, nz, d_rowptr, d_A, d_Dinv, d_r, y, d_z, nullptr, pipe, status, s) != cudaSuccess)
    return ISC_ERR_CUDA;
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ISC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ISC_ERR_CUDA;
  if (h_status & DS_TIMEOUT) return ISC_ERR_TIMEOUT;
  return ISC_OK;
}
