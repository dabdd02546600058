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
// vector is NaN-filled before a sweep and a consumer polls the neighbour's
// 64-byte block vector until it holds numbers. Matrix operands are
// prefetched PF cells ahead into a register ring. Every wait is bounded: on
// timeout the kernel raises DS_TIMEOUT and a global abort flag that makes
// every other waiter return.
//
// Lane layout per 8x8 block (row-major, 64 doubles): lane l holds the double2
// at offset 2l, i.e. row r = l/4, columns c = 2(l%4), c+1; a row sum is a
// reduction over the 4 lanes of a quad.
#include <mutex>

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

// Poll the block vector v[8] of a neighbouring pencil until every entry is a
// number: the vector is filled with NaN before the sweep and each store is
// single-copy atomic, so a non-NaN entry is final. The data itself is the
// hand-off (one L2 round trip, no flags or fences). Returns false if the
// sweep was aborted (timeout here or elsewhere).
template <typename T>
__device__ __forceinline__ bool poll_vec(const T* v, int c, typename V2<T>::t& out, int* abortf, int* dstatus) {
  const T* p = v + c;
  for (int spins = 0;; ++spins) {
    T a, b;
    ld_relaxed_v2(p, a, b);
    const bool ok = !isnan(a) && !isnan(b);
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
__device__ __forceinline__ T quad_sum(T v) {
  v += __shfl_xor_sync(FULL, v, 1);
  v += __shfl_xor_sync(FULL, v, 2);
  return v;
}

// operands of one cell that do not depend on the sweep
template <typename T>
struct Ops {
  typename V2<T>::t a0, a1, a2, d;  // up to three off-diagonal blocks (lane's pair) and D^-1
  T ri;
};

constexpr int PF = 4;  // prefetch distance in cells (register ring)

template <typename T>
__device__ __forceinline__ typename V2<T>::t zero2() {
  typename V2<T>::t z;
  z.x = T(0);
  z.y = T(0);
  return z;
}

template <typename TM, typename TR>
__device__ __forceinline__ Ops<TM> load_fwd(int x, int base_jk, bool hy, bool hz, const int32_t* __restrict__ rowptr,
                                            const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                            const TR* __restrict__ rhs, int lane, int r) {
  Ops<TM> o;
  const int i = base_jk + x;
  const int base = __ldg(rowptr + i);
  int s = 0;
  o.a0 = hz ? ld_nc2(A + (size_t)(base + s++) * BB + 2 * lane) : zero2<TM>();    // -z
  o.a1 = hy ? ld_nc2(A + (size_t)(base + s++) * BB + 2 * lane) : zero2<TM>();    // -y
  o.a2 = (x > 0) ? ld_nc2(A + (size_t)(base + s) * BB + 2 * lane) : zero2<TM>();  // -x
  o.d = ld_nc2(Dinv + (size_t)i * BB + 2 * lane);
  o.ri = (TM)__ldg(rhs + (size_t)i * 8 + r);
  return o;
}

template <typename TM>
__device__ __forceinline__ Ops<TM> load_bwd(int x, int nx, int base_jk, int nlow_jk, bool hy, bool hz,
                                            const int32_t* __restrict__ rowptr, const TM* __restrict__ A,
                                            const TM* __restrict__ Dinv, const TM* __restrict__ yin, int lane, int r) {
  Ops<TM> o;
  const int i = base_jk + x;
  const int base = __ldg(rowptr + i);
  int s = nlow_jk + (x > 0) + 1;  // first slot after the diagonal
  o.a2 = (x < nx - 1) ? ld_nc2(A + (size_t)(base + s++) * BB + 2 * lane) : zero2<TM>();  // +x
  o.a1 = hy ? ld_nc2(A + (size_t)(base + s++) * BB + 2 * lane) : zero2<TM>();            // +y
  o.a0 = hz ? ld_nc2(A + (size_t)(base + s) * BB + 2 * lane) : zero2<TM>();              // +z
  o.d = ld_nc2(Dinv + (size_t)i * BB + 2 * lane);
  o.ri = __ldg(yin + (size_t)i * 8 + r);
  return o;
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Pull the operands of a cell that is PD cells ahead into L2 (one request per
// 128-byte line): the lower (forward) or upper (backward) blocks of its row and
// its D^-1 block.
template <typename TM>
__device__ __forceinline__ void prefetch_cell(int i, int first_slot, int nblk, const int32_t* __restrict__ rowptr,
                                              const TM* __restrict__ A, const TM* __restrict__ Dinv, int lane) {
  constexpr int LANES_PER_LINE = 128 / (2 * sizeof(TM));
  if (lane % LANES_PER_LINE != 0) return;
  const int base = __ldg(rowptr + i);
  for (int b = 0; b < nblk; ++b) prefetch_l2(A + (size_t)(base + first_slot + b) * BB + 2 * lane);
  prefetch_l2(Dinv + (size_t)i * BB + 2 * lane);
}

// forward sweep: TM = matrix/vector precision, rhs always FP64
template <typename TM, int PD>
__global__ void __launch_bounds__(256) k_ilu_fwd_pipe(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                                      const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                                      const double* __restrict__ rhs, TM* __restrict__ y,
                                                      int* __restrict__ pipe, int* __restrict__ dstatus) {
  using T2 = typename V2<TM>::t;
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
    Ops<TM> ring[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q)
      if (q < nx) ring[q] = load_fwd<TM, double>(q, base_jk, hy, hz, rowptr, A, Dinv, rhs, lane, r);
    TM yp0 = TM(0), yp1 = TM(0);
    for (int x0 = 0; x0 < nx; x0 += PF) {
#pragma unroll
      for (int q = 0; q < PF; ++q) {
        const int x = x0 + q;
        if (x >= nx) break;
        const Ops<TM> o = ring[q];
        if (x + PF < nx) ring[q] = load_fwd<TM, double>(x + PF, base_jk, hy, hz, rowptr, A, Dinv, rhs, lane, r);
        if (PD > 0 && x + PD < nx) prefetch_cell<TM>(base_jk + x + PD, 0, (int)hz + (int)hy + 1, rowptr, A, Dinv, lane);
        const int i = base_jk + x;
        TM acc = fma(o.a2.x, yp0, o.a2.y * yp1);
        if (hz) {
          T2 v;
          if (!poll_vec<TM>(y + (size_t)(i - nxy) * 8, c, v, abortf, dstatus)) return;
          acc = fma(o.a0.x, v.x, fma(o.a0.y, v.y, acc));
        }
        if (hy) {
          T2 v;
          if (!poll_vec<TM>(y + (size_t)(i - nx) * 8, c, v, abortf, dstatus)) return;
          acc = fma(o.a1.x, v.x, fma(o.a1.y, v.y, acc));
        }
        const TM t = o.ri - quad_sum(acc);
        const TM t0 = __shfl_sync(FULL, t, 4 * c), t1 = __shfl_sync(FULL, t, 4 * c + 4);
        const TM yr = quad_sum(fma(o.d.x, t0, o.d.y * t1));
        if ((lane & 3) == 0) st_relaxed(y + (size_t)i * 8 + r, yr);
        yp0 = __shfl_sync(FULL, yr, 4 * c);
        yp1 = __shfl_sync(FULL, yr, 4 * c + 4);
      }
    }
  }
}

// backward sweep: hand-off through zs (precision TM); z64, if given, receives the FP64 result
template <typename TM, int PD>
__global__ void __launch_bounds__(256) k_ilu_bwd_pipe(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                                      const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                                      const TM* __restrict__ yin, TM* __restrict__ zs,
                                                      double* __restrict__ z64, int* __restrict__ pipe,
                                                      int* __restrict__ dstatus) {
  using T2 = typename V2<TM>::t;
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
    Ops<TM> ring[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q)
      if (q < nx) ring[q] = load_bwd<TM>(nx - 1 - q, nx, base_jk, nlow_jk, hy, hz, rowptr, A, Dinv, yin, lane, r);
    TM zp0 = TM(0), zp1 = TM(0);
    for (int x0 = 0; x0 < nx; x0 += PF) {
#pragma unroll
      for (int q = 0; q < PF; ++q) {
        const int step = x0 + q;
        if (step >= nx) break;
        const int x = nx - 1 - step;
        const Ops<TM> o = ring[q];
        if (step + PF < nx)
          ring[q] = load_bwd<TM>(x - PF, nx, base_jk, nlow_jk, hy, hz, rowptr, A, Dinv, yin, lane, r);
        if (PD > 0 && step + PD < nx)
          prefetch_cell<TM>(base_jk + x - PD, nlow_jk + (x - PD > 0) + 1, (int)hz + (int)hy + 1, rowptr, A, Dinv, lane);
        const int i = base_jk + x;
        TM acc = fma(o.a2.x, zp0, o.a2.y * zp1);
        if (hz) {
          T2 v;
          if (!poll_vec<TM>(zs + (size_t)(i + nxy) * 8, c, v, abortf, dstatus)) return;
          acc = fma(o.a0.x, v.x, fma(o.a0.y, v.y, acc));
        }
        if (hy) {
          T2 v;
          if (!poll_vec<TM>(zs + (size_t)(i + nx) * 8, c, v, abortf, dstatus)) return;
          acc = fma(o.a1.x, v.x, fma(o.a1.y, v.y, acc));
        }
        const TM sr = quad_sum(acc);
        const TM s0 = __shfl_sync(FULL, sr, 4 * c), s1 = __shfl_sync(FULL, sr, 4 * c + 4);
        const TM zr = o.ri - quad_sum(fma(o.d.x, s0, o.d.y * s1));
        if ((lane & 3) == 0) {
          st_relaxed(zs + (size_t)i * 8 + r, zr);
          if (z64) z64[(size_t)i * 8 + r] = (double)zr;
        }
        zp0 = __shfl_sync(FULL, zr, 4 * c);
        zp1 = __shfl_sync(FULL, zr, 4 * c + 4);
      }
    }
  }
}

// ------------------------------------------------------------------ tiled sweeps
// A CTA of TW warps owns TW consecutive pencils (j0..j0+TW-1) of one k-plane.
// Each warp keeps its whole pencil result in shared memory (NaN-filled), so
// the j-neighbour hand-off inside the CTA is a shared-memory poll; only the
// first (forward) / last (backward) warp of a tile and every k-neighbour go
// through global memory. Tiles are taken from a counter in dependency order.
// A warp that meets an abort stops its pencil but still reaches the CTA
// barriers; the CTA then leaves together.
constexpr int TW = 8;
#ifndef SWEEP_PD
#define SWEEP_PD 16  // L2 prefetch distance of the sweeps, in cells
#endif
constexpr int TILE_MAX_NX = 256;

__device__ __forceinline__ double ld_shared_volatile(const double* p) { return *(const volatile double*)p; }
__device__ __forceinline__ float ld_shared_volatile(const float* p) { return *(const volatile float*)p; }

template <typename T>
__device__ __forceinline__ bool poll_smem(const T* v, int c, typename V2<T>::t& out, int* abortf, int* dstatus) {
  for (int spins = 0;; ++spins) {
    const T a = ld_shared_volatile(v + c), b = ld_shared_volatile(v + c + 1);
    const bool ok = !isnan(a) && !isnan(b);
    if (__all_sync(FULL, ok)) {
      out.x = a;
      out.y = b;
      return true;
    }
    if ((spins & 255) == 255 && __any_sync(FULL, ld_relaxed(abortf) != 0)) return false;
    if (spins > SPIN_LIMIT) {
      if ((threadIdx.x & 31) == 0) {
        atomicOr(dstatus, DS_TIMEOUT);
        atomicExch(abortf, 1);
      }
      return false;
    }
  }
}

template <typename T>
__device__ __forceinline__ void st_shared_volatile(T* p, T v) {
  *(volatile T*)p = v;
}

template <typename TM, int PD>
__global__ void __launch_bounds__(TW * 32) k_ilu_fwd_tile(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                                          const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                                          const double* __restrict__ rhs, TM* __restrict__ y,
                                                          int* __restrict__ pipe, int* __restrict__ dstatus) {
  using T2 = typename V2<TM>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TM* sy = reinterpret_cast<TM*>(smem_raw);
  __shared__ int s_tile, s_abort;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = lane >> 2, c = (lane & 3) * 2;
  const int nxy = nx * ny, ntj = (ny + TW - 1) / TW, ntiles = ntj * nz;
  int* counter = pipe;
  int* abortf = pipe + 1;
  TM* mine = sy + (size_t)w * nx * 8;
  const TM* prev = (w > 0) ? sy + (size_t)(w - 1) * nx * 8 : nullptr;
  const TM nanv = TM(NAN);
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(counter, 1);
      s_abort = 0;
    }
    for (int e = lane; e < nx * 8; e += 32) mine[e] = nanv;
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) return;
    const int jt = t % ntj, k = t / ntj;
    const int j = jt * TW + w;
    bool ok = true;
    if (j < ny) {
      const bool hy = j > 0, hz = k > 0;
      const int base_jk = nx * (j + ny * k);
      Ops<TM> ring[PF];
#pragma unroll
      for (int q = 0; q < PF; ++q)
        if (q < nx) ring[q] = load_fwd<TM, double>(q, base_jk, hy, hz, rowptr, A, Dinv, rhs, lane, r);
      TM yp0 = TM(0), yp1 = TM(0);
      for (int x0 = 0; x0 < nx && ok; x0 += PF) {
#pragma unroll
        for (int q = 0; q < PF; ++q) {
          const int x = x0 + q;
          if (x >= nx || !ok) break;
          const Ops<TM> o = ring[q];
          if (x + PF < nx) ring[q] = load_fwd<TM, double>(x + PF, base_jk, hy, hz, rowptr, A, Dinv, rhs, lane, r);
          if (PD > 0 && x + PD < nx)
            prefetch_cell<TM>(base_jk + x + PD, 0, (int)hz + (int)hy + 1, rowptr, A, Dinv, lane);
          const int i = base_jk + x;
          TM acc = fma(o.a2.x, yp0, o.a2.y * yp1);
          if (hz) {
            T2 v;
            ok = poll_vec<TM>(y + (size_t)(i - nxy) * 8, c, v, abortf, dstatus);
            if (!ok) break;
            acc = fma(o.a0.x, v.x, fma(o.a0.y, v.y, acc));
          }
          if (hy) {
            T2 v;
            ok = (w > 0) ? poll_smem<TM>(prev + x * 8, c, v, abortf, dstatus)
                         : poll_vec<TM>(y + (size_t)(i - nx) * 8, c, v, abortf, dstatus);
            if (!ok) break;
            acc = fma(o.a1.x, v.x, fma(o.a1.y, v.y, acc));
          }
          const TM tt = o.ri - quad_sum(acc);
          const TM t0 = __shfl_sync(FULL, tt, 4 * c), t1 = __shfl_sync(FULL, tt, 4 * c + 4);
          const TM yr = quad_sum(fma(o.d.x, t0, o.d.y * t1));
          if ((lane & 3) == 0) {
            st_relaxed(y + (size_t)i * 8 + r, yr);
            st_shared_volatile(mine + x * 8 + r, yr);
          }
          yp0 = __shfl_sync(FULL, yr, 4 * c);
          yp1 = __shfl_sync(FULL, yr, 4 * c + 4);
        }
      }
    }
    if (!ok && lane == 0) s_abort = 1;
    __syncthreads();
    if (s_abort) return;
  }
}

template <typename TM, int PD>
__global__ void __launch_bounds__(TW * 32) k_ilu_bwd_tile(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                                          const TM* __restrict__ A, const TM* __restrict__ Dinv,
                                                          const TM* __restrict__ yin, TM* __restrict__ zs,
                                                          double* __restrict__ z64, int* __restrict__ pipe,
                                                          int* __restrict__ dstatus) {
  using T2 = typename V2<TM>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TM* sz = reinterpret_cast<TM*>(smem_raw);
  __shared__ int s_tile, s_abort;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = lane >> 2, c = (lane & 3) * 2;
  const int nxy = nx * ny, ntj = (ny + TW - 1) / TW, ntiles = ntj * nz;
  int* counter = pipe;
  int* abortf = pipe + 1;
  TM* mine = sz + (size_t)w * nx * 8;
  const TM* next = (w < TW - 1) ? sz + (size_t)(w + 1) * nx * 8 : nullptr;
  const TM nanv = TM(NAN);
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(counter, 1);
      s_abort = 0;
    }
    for (int e = lane; e < nx * 8; e += 32) mine[e] = nanv;
    __syncthreads();
    const int g = s_tile;
    if (g >= ntiles) return;
    const int t = ntiles - 1 - g;
    const int jt = t % ntj, k = t / ntj;
    const int j = jt * TW + w;
    bool ok = true;
    if (j < ny) {
      const bool hy = j < ny - 1, hz = k < nz - 1;
      const bool hy_local = hy && (w < TW - 1);
      const int nlow_jk = (k > 0) + (j > 0);
      const int base_jk = nx * (j + ny * k);
      Ops<TM> ring[PF];
#pragma unroll
      for (int q = 0; q < PF; ++q)
        if (q < nx) ring[q] = load_bwd<TM>(nx - 1 - q, nx, base_jk, nlow_jk, hy, hz, rowptr, A, Dinv, yin, lane, r);
      TM zp0 = TM(0), zp1 = TM(0);
      for (int x0 = 0; x0 < nx && ok; x0 += PF) {
#pragma unroll
        for (int q = 0; q < PF; ++q) {
          const int step = x0 + q;
          if (step >= nx || !ok) break;
          const int x = nx - 1 - step;
          const Ops<TM> o = ring[q];
          if (step + PF < nx)
            ring[q] = load_bwd<TM>(x - PF, nx, base_jk, nlow_jk, hy, hz, rowptr, A, Dinv, yin, lane, r);
          if (PD > 0 && step + PD < nx)
            prefetch_cell<TM>(base_jk + x - PD, nlow_jk + (x - PD > 0) + 1, (int)hz + (int)hy + 1, rowptr, A, Dinv, lane);
          const int i = base_jk + x;
          TM acc = fma(o.a2.x, zp0, o.a2.y * zp1);
          if (hz) {
            T2 v;
            ok = poll_vec<TM>(zs + (size_t)(i + nxy) * 8, c, v, abortf, dstatus);
            if (!ok) break;
            acc = fma(o.a0.x, v.x, fma(o.a0.y, v.y, acc));
          }
          if (hy) {
            T2 v;
            ok = hy_local ? poll_smem<TM>(next + x * 8, c, v, abortf, dstatus)
                          : poll_vec<TM>(zs + (size_t)(i + nx) * 8, c, v, abortf, dstatus);
            if (!ok) break;
            acc = fma(o.a1.x, v.x, fma(o.a1.y, v.y, acc));
          }
          const TM sr = quad_sum(acc);
          const TM s0 = __shfl_sync(FULL, sr, 4 * c), s1 = __shfl_sync(FULL, sr, 4 * c + 4);
          const TM zr = o.ri - quad_sum(fma(o.d.x, s0, o.d.y * s1));
          if ((lane & 3) == 0) {
            st_relaxed(zs + (size_t)i * 8 + r, zr);
            st_shared_volatile(mine + x * 8 + r, zr);
            if (z64) z64[(size_t)i * 8 + r] = (double)zr;
          }
          zp0 = __shfl_sync(FULL, zr, 4 * c);
          zp1 = __shfl_sync(FULL, zr, 4 * c + 4);
        }
      }
    }
    if (!ok && lane == 0) s_abort = 1;
    __syncthreads();
    if (s_abort) return;
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

__global__ void __launch_bounds__(FWARPS * 32) k_ilu_factor_pipe(int nx, int ny, int nz,
                                                                 const int32_t* __restrict__ rowptr,
                                                                 const double* __restrict__ A, double* __restrict__ Dinv,
                                                                 int* __restrict__ pipe, int* __restrict__ dstatus) {
  __shared__ double sm[FWARPS][6][64];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  double* sD = sm[wid][0];
  double* sI = sm[wid][1];
  double* sL = sm[wid][2];
  double* sU = sm[wid][3];
  double* sK = sm[wid][4];
  double* sP = sm[wid][5];  // D^-1 of the previous cell of this pencil
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
    for (int x = 0; x < nx; ++x) {
      const int i = base_jk + x;
      const int base = __ldg(rowptr + i);
      const int nlow = (k > 0) + (j > 0) + (x > 0);
      double2 d = ld_nc2(A + (size_t)(base + nlow) * BB + 2 * lane);
      // lower neighbours in pattern order -z, -y, -x
#pragma unroll
      for (int dl = 0; dl < 3; ++dl) {
        const bool ex = (dl == 0) ? (k > 0) : (dl == 1) ? (j > 0) : (x > 0);
        if (!ex) continue;
        const int kk = (dl == 0) ? i - nxy : (dl == 1) ? i - nx : i - 1;
        const int sl = slot_of(nx, ny, nz, i, dl);
        const int su = slot_of(nx, ny, nz, kk, 6 - dl);
        const double2 aik = ld_nc2(A + (size_t)(base + sl) * BB + 2 * lane);
        const double2 aki = ld_nc2(A + (size_t)(__ldg(rowptr + kk) + su) * BB + 2 * lane);
        double2 dk;
        if (dl < 2) {
          if (!poll_vec<double>(Dinv + (size_t)kk * BB, 2 * lane, dk, abortf, dstatus)) return;
        } else {
          dk = make_double2(sP[2 * lane], sP[2 * lane + 1]);
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
        double m0 = 0.0, m1 = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          m0 = fma(sK[r * 8 + q], sU[q * 8 + c], m0);
          m1 = fma(sK[r * 8 + q], sU[q * 8 + c + 1], m1);
        }
        __syncwarp();
        sU[r * 8 + c] = m0;  // reuse sU for M
        sU[r * 8 + c + 1] = m1;
        __syncwarp();
        double s0 = 0.0, s1 = 0.0;
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
      sI[2 * lane] = (r == c) ? 1.0 : 0.0;
      sI[2 * lane + 1] = (r == c + 1) ? 1.0 : 0.0;
      __syncwarp();
      bool bad = false;
      for (int kp = 0; kp < 8; ++kp) {
        int piv = kp;
        double best = -1.0;
        for (int q = kp; q < 8; ++q) {
          const double v = fabs(sD[q * 8 + kp]);
          if (v > best) {
            best = v;
            piv = q;
          }
        }
        if (!(best > 0.0) || !isfinite(best)) {
          bad = true;
          break;
        }
        if (piv != kp && r == kp) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            double t1 = sD[kp * 8 + c + e];
            sD[kp * 8 + c + e] = sD[piv * 8 + c + e];
            sD[piv * 8 + c + e] = t1;
            t1 = sI[kp * 8 + c + e];
            sI[kp * 8 + c + e] = sI[piv * 8 + c + e];
            sI[piv * 8 + c + e] = t1;
          }
        }
        __syncwarp();
        const double inv = 1.0 / sD[kp * 8 + kp];
        const double f = sD[r * 8 + kp];
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
      const double o0 = sI[2 * lane], o1 = sI[2 * lane + 1];
      st_relaxed(Dinv + (size_t)i * BB + 2 * lane, o0);
      st_relaxed(Dinv + (size_t)i * BB + 2 * lane + 1, o1);
      sP[2 * lane] = o0;
      sP[2 * lane + 1] = o1;
      __syncwarp();
    }
  }
}

int pipe_blocks(int npen) {
  int warps = npen < 152 * 16 ? npen : 152 * 16;
  return (warps + 7) / 8;
}

}  // namespace

void launch_ilu_factor_pipe(Handle& h, cudaStream_t s) {
  const int npen = h.ny * h.nz;
  cudaMemsetAsync(h.pipe, 0, 2 * sizeof(int), s);
  cudaMemsetAsync(h.dinv, 0xff, sizeof(double) * (size_t)h.n * BB, s);  // NaN sentinel
  const int warps = npen < 152 * 8 ? npen : 152 * 8;
  k_ilu_factor_pipe<<<(warps + FWARPS - 1) / FWARPS, FWARPS * 32, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J, h.dinv,
                                                                          h.pipe, h.dstatus);
}

template <typename TM>
void sweep_pair(Handle& h, const TM* A, const TM* Dinv, const double* r, TM* y, TM* zs, double* z64, cudaStream_t s) {
  const int npen = h.ny * h.nz;
  const size_t n8 = (size_t)h.n * 8;
  cudaMemsetAsync(h.pipe, 0, 2 * sizeof(int), s);
  cudaMemsetAsync(y, 0xff, sizeof(TM) * n8, s);  // NaN sentinel
  if (h.nx <= TILE_MAX_NX) {
    const int ntiles = ((h.ny + TW - 1) / TW) * h.nz;
    const int blocks = ntiles < 152 ? ntiles : 152;
    const size_t smem = sizeof(TM) * (size_t)TW * h.nx * 8;
    if (smem > 48 * 1024) {
      cudaFuncSetAttribute(k_ilu_fwd_tile<TM, SWEEP_PD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_ilu_bwd_tile<TM, SWEEP_PD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    k_ilu_fwd_tile<TM, SWEEP_PD><<<blocks, TW * 32, smem, s>>>(h.nx, h.ny, h.nz, h.rowptr, A, Dinv, r, y, h.pipe, h.dstatus);
    cudaMemsetAsync(h.pipe, 0, 2 * sizeof(int), s);
    cudaMemsetAsync(zs, 0xff, sizeof(TM) * n8, s);
    k_ilu_bwd_tile<TM, SWEEP_PD><<<blocks, TW * 32, smem, s>>>(h.nx, h.ny, h.nz, h.rowptr, A, Dinv, y, zs, z64, h.pipe,
                                                     h.dstatus);
    return;
  }
  k_ilu_fwd_pipe<TM, SWEEP_PD><<<pipe_blocks(npen), 256, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, A, Dinv, r, y, h.pipe, h.dstatus);
  cudaMemsetAsync(h.pipe, 0, 2 * sizeof(int), s);
  cudaMemsetAsync(zs, 0xff, sizeof(TM) * n8, s);
  k_ilu_bwd_pipe<TM, SWEEP_PD><<<pipe_blocks(npen), 256, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, A, Dinv, y, zs, z64, h.pipe,
                                                        h.dstatus);
}

void launch_ilu_apply_pipe(Handle& h, const double* r, double* z, cudaStream_t s) {
  if (h.opt.precision == ISC_PRECISION_MIXED) {
    const size_t n8 = (size_t)h.n * 8;
    sweep_pair<float>(h, h.J32, h.dinv32, r, h.vec32, h.vec32 + n8, z, s);
    return;
  }
  sweep_pair<double>(h, h.J, h.dinv, r, h.tmp, z, nullptr, s);
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

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[MAX_DEVICES] = {};

// Host code may not use g_noalloc_scratch as an address: resolve the device
// address once per device, with that device current.
int noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return ISC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return ISC_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return ISC_OK;
}

}  // namespace

}  // namespace isc

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
  const int npen = ny * nz;
  const size_t vbytes = sizeof(double) * (size_t)n * 8;
  // everything that must start at zero (or NaN) is cleared here: the array
  // keeps the previous call's contents
  if (cudaMemsetAsync(ints, 0, NOALLOC_INTS * sizeof(int), s) != cudaSuccess) return ISC_ERR_CUDA;
  cudaMemsetAsync(y, 0xff, vbytes, s);
  k_ilu_fwd_pipe<double, 0><<<pipe_blocks(npen), 256, 0, s>>>(nx, ny, nz, d_rowptr, d_A, d_Dinv, d_r, y, pipe, status);
  cudaMemsetAsync(pipe, 0, 2 * sizeof(int), s);
  cudaMemsetAsync(d_z, 0xff, vbytes, s);
  k_ilu_bwd_pipe<double, 0><<<pipe_blocks(npen), 256, 0, s>>>(nx, ny, nz, d_rowptr, d_A, d_Dinv, y, d_z, nullptr, pipe,
                                                            status);
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ISC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ISC_ERR_CUDA;
  if (h_status & DS_TIMEOUT) return ISC_ERR_TIMEOUT;
  return ISC_OK;
}
