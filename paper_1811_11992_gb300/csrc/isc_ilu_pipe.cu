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
// running warps), and the cross-pencil hand-off is a per-pencil progress
// counter written with release and read with acquire semantics. Every wait
// is bounded: on timeout the kernel raises DS_TIMEOUT and a global abort flag
// that makes every other waiter return.
//
// Lane layout per 8x8 block (row-major, 64 doubles): lane l holds the double2
// at offset 2l, i.e. row r = l/4, columns c = 2(l%4), c+1; a row sum is a
// reduction over the 4 lanes of a quad.
#include "isc_internal.cuh"

namespace isc {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SPIN_LIMIT = 1 << 22;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double2 ld_cg2(const double* p) { return __ldcg(reinterpret_cast<const double2*>(p)); }

__device__ __forceinline__ double2 ld_nc2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }

// Wait (lane 0 polls) until prog[q] >= need. Returns false if the sweep was aborted.
__device__ __forceinline__ bool wait_for(const int* prog_q, int need, int& known, int* abortf, int* dstatus,
                                         int lane) {
  if (known >= need) return true;
  int ok = 1, v = 0;
  if (lane == 0) {
    v = ld_acquire(prog_q);
    int spins = 0;
    while (v < need) {
      if (ld_relaxed(abortf)) {
        ok = 0;
        break;
      }
      if (++spins > SPIN_LIMIT) {
        atomicOr(dstatus, DS_TIMEOUT);
        atomicExch(abortf, 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
      v = ld_acquire(prog_q);
    }
  }
  ok = __shfl_sync(FULL, ok, 0);
  known = __shfl_sync(FULL, v, 0);
  __syncwarp();
  return ok != 0;
}

__device__ __forceinline__ double quad_sum(double v) {
  v += __shfl_xor_sync(FULL, v, 1);
  v += __shfl_xor_sync(FULL, v, 2);
  return v;
}

__global__ void __launch_bounds__(256) k_ilu_fwd_pipe(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                                      const double* __restrict__ A, const double* __restrict__ Dinv,
                                                      const double* __restrict__ rhs, double* __restrict__ y,
                                                      int* __restrict__ pipe, int* __restrict__ dstatus) {
  const int lane = threadIdx.x & 31;
  const int r = lane >> 2, c = (lane & 3) * 2;
  const int npen = ny * nz, nxy = nx * ny;
  int* counter = pipe;
  int* abortf = pipe + 1;
  int* prog = pipe + 2;
  for (;;) {
    int p = 0;
    if (lane == 0) p = atomicAdd(counter, 1);
    p = __shfl_sync(FULL, p, 0);
    if (p >= npen) return;
    const int j = p % ny, k = p / ny;
    const bool hy = j > 0, hz = k > 0;
    int known_y = 0, known_z = 0;
    double yp0 = 0.0, yp1 = 0.0;
    for (int x = 0; x < nx; ++x) {
      const int i = x + nx * (j + ny * k);
      const int base = __ldg(rowptr + i);
      // operands that do not depend on the sweep are loaded before any wait
      int s = 0;
      double2 az = make_double2(0.0, 0.0), ay = az, ax = az;
      if (hz) az = ld_nc2(A + (size_t)(base + s++) * BB + 2 * lane);
      if (hy) ay = ld_nc2(A + (size_t)(base + s++) * BB + 2 * lane);
      if (x > 0) ax = ld_nc2(A + (size_t)(base + s) * BB + 2 * lane);
      const double2 d = ld_nc2(Dinv + (size_t)i * BB + 2 * lane);
      const double ri = __ldg(rhs + (size_t)i * 8 + r);
      double acc = 0.0;
      if (x > 0) acc = fma(ax.x, yp0, fma(ax.y, yp1, acc));
      if (hz) {
        if (!wait_for(prog + p - ny, x + 1, known_z, abortf, dstatus, lane)) return;
        const double2 v = ld_cg2(y + (size_t)(i - nxy) * 8 + c);
        acc = fma(az.x, v.x, fma(az.y, v.y, acc));
      }
      if (hy) {
        if (!wait_for(prog + p - 1, x + 1, known_y, abortf, dstatus, lane)) return;
        const double2 v = ld_cg2(y + (size_t)(i - nx) * 8 + c);
        acc = fma(ay.x, v.x, fma(ay.y, v.y, acc));
      }
      const double t = ri - quad_sum(acc);
      const double t0 = __shfl_sync(FULL, t, 4 * c), t1 = __shfl_sync(FULL, t, 4 * c + 4);
      const double yr = quad_sum(fma(d.x, t0, d.y * t1));
      if ((lane & 3) == 0) y[(size_t)i * 8 + r] = yr;
      yp0 = __shfl_sync(FULL, yr, 4 * c);
      yp1 = __shfl_sync(FULL, yr, 4 * c + 4);
      __syncwarp();
      if (lane == 0) st_release(prog + p, x + 1);
    }
  }
}

__global__ void __launch_bounds__(256) k_ilu_bwd_pipe(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                                                      const double* __restrict__ A, const double* __restrict__ Dinv,
                                                      const double* __restrict__ yin, double* __restrict__ z,
                                                      int* __restrict__ pipe, int* __restrict__ dstatus) {
  const int lane = threadIdx.x & 31;
  const int r = lane >> 2, c = (lane & 3) * 2;
  const int npen = ny * nz, nxy = nx * ny;
  int* counter = pipe;
  int* abortf = pipe + 1;
  int* prog = pipe + 2;
  for (;;) {
    int g = 0;
    if (lane == 0) g = atomicAdd(counter, 1);
    g = __shfl_sync(FULL, g, 0);
    if (g >= npen) return;
    const int p = npen - 1 - g;
    const int j = p % ny, k = p / ny;
    const bool hy = j < ny - 1, hz = k < nz - 1;
    const int nlow_jk = (k > 0) + (j > 0);
    int known_y = 0, known_z = 0;
    double zp0 = 0.0, zp1 = 0.0;
    for (int x = nx - 1; x >= 0; --x) {
      const int i = x + nx * (j + ny * k);
      const int base = __ldg(rowptr + i);
      int s = nlow_jk + (x > 0) + 1;  // first slot after the diagonal
      double2 ax = make_double2(0.0, 0.0), ay = ax, az = ax;
      if (x < nx - 1) ax = ld_nc2(A + (size_t)(base + s++) * BB + 2 * lane);
      if (hy) ay = ld_nc2(A + (size_t)(base + s++) * BB + 2 * lane);
      if (hz) az = ld_nc2(A + (size_t)(base + s) * BB + 2 * lane);
      const double2 d = ld_nc2(Dinv + (size_t)i * BB + 2 * lane);
      const double yi = __ldg(yin + (size_t)i * 8 + r);
      const int done = nx - x;
      double acc = 0.0;
      if (x < nx - 1) acc = fma(ax.x, zp0, fma(ax.y, zp1, acc));
      if (hz) {
        if (!wait_for(prog + p + ny, done, known_z, abortf, dstatus, lane)) return;
        const double2 v = ld_cg2(z + (size_t)(i + nxy) * 8 + c);
        acc = fma(az.x, v.x, fma(az.y, v.y, acc));
      }
      if (hy) {
        if (!wait_for(prog + p + 1, done, known_y, abortf, dstatus, lane)) return;
        const double2 v = ld_cg2(z + (size_t)(i + nx) * 8 + c);
        acc = fma(ay.x, v.x, fma(ay.y, v.y, acc));
      }
      const double sr = quad_sum(acc);
      const double s0 = __shfl_sync(FULL, sr, 4 * c), s1 = __shfl_sync(FULL, sr, 4 * c + 4);
      const double zr = yi - quad_sum(fma(d.x, s0, d.y * s1));
      if ((lane & 3) == 0) z[(size_t)i * 8 + r] = zr;
      zp0 = __shfl_sync(FULL, zr, 4 * c);
      zp1 = __shfl_sync(FULL, zr, 4 * c + 4);
      __syncwarp();
      if (lane == 0) st_release(prog + p, done);
    }
  }
}

int pipe_blocks(int npen) {
  int warps = npen < 152 * 16 ? npen : 152 * 16;
  return (warps + 7) / 8;
}

}  // namespace

void launch_ilu_apply_pipe(Handle& h, const double* r, double* z, cudaStream_t s) {
  const int npen = h.ny * h.nz;
  const size_t bytes = sizeof(int) * (size_t)(npen + 2);
  cudaMemsetAsync(h.pipe, 0, bytes, s);
  k_ilu_fwd_pipe<<<pipe_blocks(npen), 256, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J, h.dinv, r, h.tmp, h.pipe,
                                                    h.dstatus);
  cudaMemsetAsync(h.pipe, 0, bytes, s);
  k_ilu_bwd_pipe<<<pipe_blocks(npen), 256, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J, h.dinv, h.tmp, z, h.pipe,
                                                    h.dstatus);
}

}  // namespace isc
