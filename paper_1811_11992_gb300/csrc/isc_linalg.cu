// Linear algebra of the Newton step on the 8x8 block-sparse system.
//
// k_gj          Gauss-Jordan decoupling (Sec. 3.2): one half-warp per block row,
//               lanes own columns of the augmented row [J_i,* | F_i], partial
//               pivoting with warp shuffles; the diagonal block becomes I.
// k_spmv8       FP64 y = A x, eight lanes per block row, each lane a whole block row;
// k_spmv        FP32 y = A x, one warp per block row, each lane streams one pair
//               per 8x8 block (512 contiguous bytes per warp and block).
// k_ilu_factor  block ILU(0) diagonal recurrence D_i = A_ii - sum_k A_ik D_k^-1 A_ki
//               over the lower neighbours (the 7-point pattern has no other
//               fill), hyperplane wavefront i+j+k = level, 64 threads per cell.
// (the two triangular sweeps live in isc_ilu_pipe.cu)
// BLAS-1        dot products with fixed-order two-stage reductions.
// k_update      safeguarded Newton update (Sec. 2.2 saturation treatment).
#include <math.h>

#include "isc_internal.cuh"

namespace isc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// slot of neighbour direction d (0 -z, 1 -y, 2 -x, 3 diag, 4 +x, 5 +y, 6 +z) in the sorted BSR row
__device__ __forceinline__ int nbr_slot(int nx, int ny, int nz, int c, int d) {
  int ix = c % nx, iy = (c / nx) % ny, iz = c / (nx * ny);
  bool has[7] = {iz > 0, iy > 0, ix > 0, true, ix < nx - 1, iy < ny - 1, iz < nz - 1};
  int s = 0;
  for (int e = 0; e < d; ++e) s += has[e];
  return s;
}

__device__ __forceinline__ bool nbr_exists(int nx, int ny, int nz, int c, int d, int* j) {
  int ix = c % nx, iy = (c / nx) % ny, iz = c / (nx * ny);
  switch (d) {
    case 0: *j = c - nx * ny; return iz > 0;
    case 1: *j = c - nx; return iy > 0;
    case 2: *j = c - 1; return ix > 0;
    case 4: *j = c + 1; return ix < nx - 1;
    case 5: *j = c + nx; return iy < ny - 1;
    case 6: *j = c + nx * ny; return iz < nz - 1;
    default: *j = c; return true;
  }
}

// Gauss-Jordan decoupling, two block rows per warp (one per half-warp). Lane h
// of a half owns the columns h, h+16, h+32, h+48 of the augmented row
// [J_i,* | F_i (| B_i)] (at most 7*8 + 2 = 58 of 64 columns), all 8 rows of
// each, in registers. Per pivot step the FP64 work of a lane is the pivot
// reciprocal, one multiplier and 4 x 8 updates, shared by the half's 16 lanes:
// the multipliers -a_rk / a_kk are computed one per lane (lane h for row h % 8)
// and gathered by shuffles, so the narrow FP64 pipe spends almost all of its
// issue slots on the elimination itself. The pivot search and the pivot test
// run on the integer bit patterns of |a| (IEEE order is numeric order for
// non-negative values), with the exact floating-point test of the singularity
// threshold only when the exponents leave it undecided.
__global__ void __launch_bounds__(256) k_gj(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                            double* __restrict__ J, double* __restrict__ R, int* __restrict__ dstatus,
                                            const int32_t* __restrict__ well_slot, const WellSlot* __restrict__ slots,
                                            double* __restrict__ Bv) {
  const int lane = threadIdx.x & 31;
  const int h = lane & 15, hb = lane & 16;
  const int row = ((blockIdx.x * blockDim.x + threadIdx.x) >> 4);
  const bool live = row < n;
  const int i = live ? row : n - 1;  // a spare half repeats the last row and stores nothing
  const int b0 = rowptr[i];
  const int nb = rowptr[i + 1] - b0;
  int d = 0;
  for (int s = 0; s < nb; ++s)
    if (col[b0 + s] == i) d = s;
  const int nc = nb * 8;
  // a perforation of a coupled producer carries its border column dF/d bhp as
  // one more column of the augmented row
  int bs = -1;
  if (Bv) {
    const int sl = well_slot[i];
    if (sl >= 0 && slots[sl].wc >= 0) bs = sl;
  }
  double a[4][8];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int cc = h + 16 * m;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      double v = 0.0;
      if (cc < nc)
        v = J[(size_t)(b0 + cc / 8) * BB + r * 8 + (cc & 7)];
      else if (cc == nc)
        v = R[(size_t)i * 8 + r];
      else if (cc == nc + 1 && bs >= 0)
        v = Bv[(size_t)bs * 8 + r];
      a[m][r] = v;
    }
  }
  auto mag = [](double v) { return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull; };
  const int rr = h & 7;  // the row whose multiplier this lane computes
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int pc = d * 8 + k;
    const int pl = pc & 15, pm = pc >> 4;
    // the pivot column as seen by its owner lane
    double pcol[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) pcol[r] = pm == 0 ? a[0][r] : pm == 1 ? a[1][r] : pm == 2 ? a[2][r] : a[3][r];
    int piv = k;
    if (h == pl) {
      unsigned long long best = 0ull;
#pragma unroll
      for (int r = k; r < 8; ++r) {
        const unsigned long long v = mag(pcol[r]);
        if (r == k || v > best) {
          best = v;
          piv = r;
        }
      }
    }
    piv = __shfl_sync(FULL, piv, hb + pl);
    // largest |a| of row piv inside the diagonal block (columns d*8 .. d*8+7)
    unsigned long long rmb = 0ull;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int cc = h + 16 * m;
      if (cc >= d * 8 && cc < d * 8 + 8) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
          if (r == piv) rmb = max(rmb, mag(a[m][r]));
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) rmb = max(rmb, (unsigned long long)__shfl_xor_sync(FULL, rmb, o));
    // swap rows k and piv
#pragma unroll
    for (int m = 0; m < 4; ++m) {
#pragma unroll
      for (int r = k + 1; r < 8; ++r) {
        if (r == piv) {
          const double t = a[m][r];
          a[m][r] = a[m][k];
          a[m][k] = t;
        }
      }
    }
    // the pivot column after the swap, from its owner lane
    double colk[8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
      colk[r] = __shfl_sync(FULL, pm == 0 ? a[0][r] : pm == 1 ? a[1][r] : pm == 2 ? a[2][r] : a[3][r], hb + pl);
    const double pv = colk[k];
    // |pv| > 1e-300 max(|row max|, 1e-300): decided on the exponents when pv is a finite
    // normal number at most 900 binades below the row maximum (then the product side is
    // below 2^(e - 994) <= |pv|); otherwise in floating point
    const unsigned long long pb = mag(pv);
    const int epv = (int)(pb >> 52), erm = (int)(rmb >> 52);
    bool ok;
    if (epv > 0 && epv < 0x7ff && epv + 900 >= erm) {
      ok = true;
    } else {
      const double rm = __longlong_as_double((long long)rmb);
      ok = fabs(pv) > 1e-300 * fmax(rm, 1e-300);
    }
    // a singular half keeps stepping (its lanes take part in every shuffle of the
    // warp) with a zero reciprocal and stores nothing
    bad = bad || !ok;
    const double inv = ok ? recip_nr(pv) : 0.0;
    // this lane's multiplier -a_rk / a_kk for row rr (0 for the pivot row), gathered by the half
    double own = 0.0;
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (r == rr) own = colk[r];
    own = rr == k ? 0.0 : -own * inv;
    double coef[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) coef[r] = __shfl_sync(FULL, own, hb + r);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r != k) a[m][r] = fma(coef[r], a[m][k], a[m][r]);
      a[m][k] = a[m][k] * inv;
    }
  }
  if (bad) {
    if (live && h == 0) atomicOr(dstatus, DS_SINGULAR);
    return;
  }
  if (!live) return;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int cc = h + 16 * m;
    if (cc < nc) {
      const int s = cc / 8, c = cc & 7;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const double v = (s == d) ? (r == c ? 1.0 : 0.0) : a[m][r];
        J[(size_t)(b0 + s) * BB + r * 8 + c] = v;
      }
    } else if (cc == nc) {
#pragma unroll
      for (int r = 0; r < 8; ++r) R[(size_t)i * 8 + r] = a[m][r];
    } else if (cc == nc + 1 && bs >= 0) {
#pragma unroll
      for (int r = 0; r < 8; ++r) Bv[(size_t)bs * 8 + r] = a[m][r];
    }
  }
}

// ----------------------------------------------------- coupled producers
// Border of the Newton system: y_c(cell of q) += B_q x_w(well of q)
__global__ void k_well_border_cells(int nslots, const WellSlot* __restrict__ slots, const double* __restrict__ Bv,
                                    const double* __restrict__ x, double* __restrict__ y, size_t n8) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nslots * 8) return;
  const int q = e >> 3, r = e & 7;
  const int wc = slots[q].wc;
  if (wc < 0) return;
  y[(size_t)slots[q].cell * 8 + r] += Bv[(size_t)q * 8 + r] * x[n8 + wc];
}

// well rows: y_w = sum_q C_q . x_c(cell of q) + D_w x_w (one thread per well)
__global__ void k_well_border_rows(int nwc, const CoupledWell* __restrict__ cw, const WellSlot* __restrict__ slots,
                                   const double* __restrict__ Cv, const double* __restrict__ Dw,
                                   const double* __restrict__ x, double* __restrict__ y, size_t n8) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwc) return;
  const CoupledWell c = cw[w];
  double s = Dw[w] * x[n8 + w];
  for (int q = c.first; q < c.first + c.count; ++q) {
    const double* xc = x + (size_t)slots[q].cell * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += Cv[(size_t)q * 8 + k] * xc[k];
  }
  y[n8 + w] = s;
}

// block lower-triangular preconditioner, well part: z_w = (r_w - sum_q C_q . z_c) / D_w
__global__ void k_well_prec(int nwc, const CoupledWell* __restrict__ cw, const WellSlot* __restrict__ slots,
                            const double* __restrict__ Cv, const double* __restrict__ Dw, const double* __restrict__ r,
                            double* __restrict__ z, size_t n8) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwc) return;
  const CoupledWell c = cw[w];
  double s = r[n8 + w];
  for (int q = c.first; q < c.first + c.count; ++q) {
    const double* zc = z + (size_t)slots[q].cell * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) s -= Cv[(size_t)q * 8 + k] * zc[k];
  }
  z[n8 + w] = s / Dw[w];
}

// bhp_w += du_w with the pressure safeguard |d bhp| <= max_dp_frac bhp
__global__ void k_well_update(int nwc, const double* __restrict__ du, size_t n8, double max_dp_frac,
                              double* __restrict__ bhp) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwc) return;
  const double b = bhp[w];
  bhp[w] = b + fmin(fmax(du[n8 + w], -max_dp_frac * b), max_dp_frac * b);
}

template <typename TV> struct Pair;
template <> struct Pair<double> { using t = double2; };
template <> struct Pair<float> { using t = float2; };

// y = A x for a BSR matrix with 8x8 blocks: one warp per block row, lane (r, c)
// holds columns 2c, 2c+1 of row r of every block (FP64, or FP32 for the inner
// solve of the mixed-precision scheme); unit_diag: the diagonal block is I
template <typename TV>
__global__ void __launch_bounds__(256) k_spmv(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                              const TV* __restrict__ val, const TV* __restrict__ x,
                                              TV* __restrict__ y, int unit_diag) {
  using T2 = typename Pair<TV>::t;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const int b0 = __ldg(rowptr + row), b1 = __ldg(rowptr + row + 1);
  const int r = lane >> 2, c = (lane & 3) * 2;
  TV acc = TV(0);
#pragma unroll 7
  for (int b = b0; b < b1; ++b) {
    int j = __ldg(col + b);
    if (unit_diag && j == row) continue;
    T2 v = __ldcs(reinterpret_cast<const T2*>(val + (size_t)b * BB) + lane);  // streamed once: evict first
    T2 xv = __ldg(reinterpret_cast<const T2*>(x + (size_t)j * 8 + c));
    acc = fma(v.x, xv.x, acc);
    acc = fma(v.y, xv.y, acc);
  }
  acc += __shfl_xor_sync(FULL, acc, 1);
  acc += __shfl_xor_sync(FULL, acc, 2);
  if ((lane & 3) == 0) y[(size_t)row * 8 + r] = acc + (unit_diag ? x[(size_t)row * 8 + r] : TV(0));
}

// FP64 y = A x with eight lanes per block row (four rows per warp): lane (g, r)
// accumulates row r of block row 4w + g over every block, eight FMAs per block
// with the block row's 64 contiguous bytes and the neighbour's 8-vector (loaded
// by all eight lanes of the group, one broadcast transaction). No cross-lane sum
// is needed, so every FP64 instruction of the warp is a useful FMA: 12 per block
// row against 15 with one warp per block row (quad sums and the diagonal add),
// which matters because the FP64 SpMV is bound by GB300's narrow FP64 pipe.
// The unit diagonal enters as the accumulator's starting value.
__global__ void __launch_bounds__(256) k_spmv8(int n, const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col, const double* __restrict__ val,
                                               const double* __restrict__ x, double* __restrict__ y, int unit_diag) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t >> 3, r = t & 7;
  if (row >= n) return;
  const int b0 = __ldg(rowptr + row), b1 = __ldg(rowptr + row + 1);
  double acc = unit_diag ? __ldg(x + (size_t)row * 8 + r) : 0.0;
#pragma unroll 7
  for (int b = b0; b < b1; ++b) {
    const int j = __ldg(col + b);
    if (unit_diag && j == row) continue;
    const double2* a = reinterpret_cast<const double2*>(val + (size_t)b * BB + r * 8);
    const double2* xv = reinterpret_cast<const double2*>(x + (size_t)j * 8);
    const double2 a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2), a3 = __ldg(a + 3);
    const double2 x0 = __ldg(xv), x1 = __ldg(xv + 1), x2 = __ldg(xv + 2), x3 = __ldg(xv + 3);
    acc = fma(a0.x, x0.x, acc);
    acc = fma(a0.y, x0.y, acc);
    acc = fma(a1.x, x1.x, acc);
    acc = fma(a1.y, x1.y, acc);
    acc = fma(a2.x, x2.x, acc);
    acc = fma(a2.y, x2.y, acc);
    acc = fma(a3.x, x3.x, acc);
    acc = fma(a3.y, x3.y, acc);
  }
  y[(size_t)row * 8 + r] = acc;
}

// ---------------------------------------------------------- block ILU(0)
constexpr int FCELLS = 4;  // cells per 256-thread block in the factorisation

__global__ void __launch_bounds__(256) k_ilu_factor(int nx, int ny, int nz, const int32_t* __restrict__ cells, int count,
                                                    int use_lower, const int32_t* __restrict__ rowptr,
                                                    const double* __restrict__ A, double* __restrict__ Dinv,
                                                    int* __restrict__ dstatus) {
  __shared__ double sD[FCELLS][64], sI[FCELLS][64], sL[FCELLS][64], sU[FCELLS][64], sM[FCELLS][64];
  __shared__ int spiv[FCELLS];
  __shared__ int sbad[FCELLS];
  const int g = threadIdx.x >> 6;
  const int t = threadIdx.x & 63;
  const int r = t >> 3, c = t & 7;
  const int ci = blockIdx.x * FCELLS + g;
  const bool active = ci < count;
  const int i = active ? cells[ci] : 0;
  if (active) {
    sD[g][t] = A[(size_t)(rowptr[i] + nbr_slot(nx, ny, nz, i, 3)) * BB + t];
    sI[g][t] = (r == c) ? 1.0 : 0.0;
  }
  if (t == 0) sbad[g] = 0;
  __syncthreads();
  if (use_lower) {
    for (int dlow = 0; dlow < 3; ++dlow) {
      int k = 0;
      bool ex = active && nbr_exists(nx, ny, nz, i, dlow, &k);
      if (ex) {
        sL[g][t] = A[(size_t)(rowptr[i] + nbr_slot(nx, ny, nz, i, dlow)) * BB + t];
        sU[g][t] = A[(size_t)(rowptr[k] + nbr_slot(nx, ny, nz, k, 6 - dlow)) * BB + t];
        sM[g][t] = Dinv[(size_t)k * BB + t];
      }
      __syncthreads();
      double m = 0.0;
      if (ex) {
#pragma unroll
        for (int q = 0; q < 8; ++q) m = fma(sM[g][r * 8 + q], sU[g][q * 8 + c], m);
      }
      __syncthreads();
      if (ex) sM[g][t] = m;  // M = D_k^-1 A_ki
      __syncthreads();
      if (ex) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) s = fma(sL[g][r * 8 + q], sM[g][q * 8 + c], s);
        sD[g][t] -= s;
      }
      __syncthreads();
    }
  }
  // invert D by Gauss-Jordan with partial pivoting
  for (int k = 0; k < 8; ++k) {
    if (t == 0 && active) {
      // pivot search on the integer bit patterns of |D| (the same choice as a float compare)
      int piv = k;
      unsigned long long best = 0ull;
      for (int q = k; q < 8; ++q) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(sD[g][q * 8 + k]) & 0x7fffffffffffffffull;
        if (q == k || v > best) {
          best = v;
          piv = q;
        }
      }
      spiv[g] = piv;
      if (best == 0ull || best >= 0x7ff0000000000000ull) sbad[g] = 1;  // zero column, or inf / NaN
    }
    __syncthreads();
    const int piv = spiv[g];
    if (active && r == k && piv != k) {
      double t1 = sD[g][k * 8 + c];
      sD[g][k * 8 + c] = sD[g][piv * 8 + c];
      sD[g][piv * 8 + c] = t1;
      t1 = sI[g][k * 8 + c];
      sI[g][k * 8 + c] = sI[g][piv * 8 + c];
      sI[g][piv * 8 + c] = t1;
    }
    __syncthreads();
    double pv = sD[g][k * 8 + k];
    double f = sD[g][r * 8 + k];
    __syncthreads();
    if (active && r == k && !sbad[g]) {
      const double inv = recip_nr(pv);
      sD[g][k * 8 + c] *= inv;
      sI[g][k * 8 + c] *= inv;
    }
    __syncthreads();
    if (active && r != k && !sbad[g]) {
      sD[g][r * 8 + c] -= f * sD[g][k * 8 + c];
      sI[g][r * 8 + c] -= f * sI[g][k * 8 + c];
    }
    __syncthreads();
  }
  if (active) {
    if (sbad[g]) {
      if (t == 0) atomicOr(dstatus, DS_SINGULAR);
    } else {
      Dinv[(size_t)i * BB + t] = sI[g][t];
    }
  }
}

__global__ void k_bjacobi_apply(int n, const double* __restrict__ Dinv, const double* __restrict__ rhs,
                                double* __restrict__ z) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = tid >> 3, r = threadIdx.x & 7;
  double v = (i < n) ? rhs[(size_t)i * 8 + r] : 0.0;
  double out = 0.0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    double vm = __shfl_sync(FULL, v, m, 8);
    if (i < n) out = fma(Dinv[(size_t)i * BB + r * 8 + m], vm, out);
  }
  if (i < n) z[(size_t)i * 8 + r] = out;
}

// ------------------------------------------------------------------ BLAS-1
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double s, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  s = (threadIdx.x < RED_THREADS / 32) ? sh[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  }
  return s;  // valid in thread 0
}

// The last block to finish sums the per-block partials of every result in a
// fixed order (deterministic), writes out[c] and re-arms the counter.
__device__ __forceinline__ void last_block_finish(int nres, int nblk_x, const double* __restrict__ partial,
                                                  unsigned* counter, double* __restrict__ out) {
  __shared__ bool last;
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < nres; c += RED_THREADS / 32) {
    double s = 0.0;
    for (int b = lane; b < nblk_x; b += 32) s += __ldcg(partial + (size_t)c * nblk_x + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) out[c] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

constexpr int DOT_G = 8;  // vectors per block row of the grid (register accumulators)
constexpr int MAX_VEC = 72;

// out[c] = V_c . w for c < nvec; blockIdx.y takes vectors DOT_G*y .. DOT_G*y+DOT_G-1
__global__ void __launch_bounds__(RED_THREADS) k_mdot(int len, const double* __restrict__ V, size_t vstride, int nvec,
                                                      const double* __restrict__ w, double* __restrict__ partial,
                                                      unsigned* counter, double* __restrict__ out) {
  __shared__ double sh[DOT_G][RED_THREADS / 32];
  const int c0 = blockIdx.y * DOT_G;
  const int stride = gridDim.x * blockDim.x;
  double acc[DOT_G];
#pragma unroll
  for (int g = 0; g < DOT_G; ++g) acc[g] = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    const double we = w[e];
#pragma unroll
    for (int g = 0; g < DOT_G; ++g)
      if (c0 + g < nvec) acc[g] = fma(V[(size_t)(c0 + g) * vstride + e], we, acc[g]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < DOT_G; ++g) {
    double v = acc[g];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0) sh[g][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < DOT_G && c0 + (int)threadIdx.x < nvec) {
    double v = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) v += sh[threadIdx.x][q];
    partial[(size_t)(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
  }
  last_block_finish(nvec, gridDim.x, partial, counter, out);
}

// Sum of eight per-lane values over the warp, transposed: each butterfly step
// exchanges half of the remaining values, so the eight sums cost 9 FP64 adds
// per lane instead of 40 (the FP64 pipe is GB300's scarcest unit). Lane l with
// (l & 3) == 0 returns the sum of value red8_index(l).
__device__ __forceinline__ double warp_reduce8(const double (&a)[8], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  double b[4], c2[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) b[i] = (h16 ? a[i + 4] : a[i]) + __shfl_xor_sync(FULL, h16 ? a[i] : a[i + 4], 16);
#pragma unroll
  for (int i = 0; i < 2; ++i) c2[i] = (h8 ? b[i + 2] : b[i]) + __shfl_xor_sync(FULL, h8 ? b[i] : b[i + 2], 8);
  double d = (h4 ? c2[1] : c2[0]) + __shfl_xor_sync(FULL, h4 ? c2[0] : c2[1], 4);
  d += __shfl_xor_sync(FULL, d, 2);
  d += __shfl_xor_sync(FULL, d, 1);
  return d;
}
__device__ __forceinline__ int red8_index(int lane) { return ((lane >> 2) & 1) * 1 + ((lane >> 3) & 1) * 2 + ((lane >> 4) & 1) * 4; }

// out[c] = V_c . w for all c < nvec <= 8 NG in one pass: w is read once and each
// thread keeps 8 NG accumulators; UE elements per iteration for more loads in flight
template <typename TV, int NG, int UE>
__global__ void __launch_bounds__(RED_THREADS) k_mdot_t(int len, const TV* __restrict__ V, size_t vstride, int nvec,
                                                        const TV* __restrict__ w, double* __restrict__ partial,
                                                        unsigned* counter, double* __restrict__ out) {
  __shared__ double sh[NG * 8][RED_THREADS / 32];
  TV acc[NG][8];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[g][i] = TV(0);
  const int stride = gridDim.x * blockDim.x;
  for (int e0 = blockIdx.x * blockDim.x + threadIdx.x; e0 < len; e0 += UE * stride) {
    TV we[UE];
#pragma unroll
    for (int u = 0; u < UE; ++u) we[u] = (e0 + u * stride < len) ? w[e0 + u * stride] : TV(0);
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (g * 8 + i < nvec) {
#pragma unroll
          for (int u = 0; u < UE; ++u)
            if (e0 + u * stride < len)
              acc[g][i] = fma(V[(size_t)(g * 8 + i) * vstride + e0 + u * stride], we[u], acc[g][i]);
        }
      }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    double a8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a8[i] = (double)acc[g][i];
    const double v = warp_reduce8(a8, lane);
    if ((lane & 3) == 0) sh[g * 8 + red8_index(lane)][warp] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nvec; c += blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < RED_THREADS / 32; ++q) v += sh[c][q];
    partial[(size_t)c * gridDim.x + blockIdx.x] = v;
  }
  last_block_finish(nvec, gridDim.x, partial, counter, out);
}

// The middle of classical Gram-Schmidt applied twice, fused: w <- w - V coef,
// then out = V^T w, with each V_c[e] loaded once for both (nvec <= 8 NG)
template <typename TV, int NG>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy_mdot(int len, TV* __restrict__ w, const TV* __restrict__ V,
                                                            size_t vstride, int nvec, const double* __restrict__ coef,
                                                            double* __restrict__ partial, unsigned* counter,
                                                            double* __restrict__ out) {
  __shared__ double sh[NG * 8][RED_THREADS / 32];
  __shared__ TV sc[NG * 8];
  for (int c = threadIdx.x; c < NG * 8; c += blockDim.x) sc[c] = c < nvec ? (TV)coef[c] : TV(0);
  __syncthreads();
  TV acc[NG][8];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[g][i] = TV(0);
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    TV v[NG][8];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i) v[g][i] = (g * 8 + i < nvec) ? V[(size_t)(g * 8 + i) * vstride + e] : TV(0);
    TV t = TV(0);
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (g * 8 + i < nvec) t = fma(sc[g * 8 + i], v[g][i], t);
    const TV we = w[e] - t;
    w[e] = we;
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (g * 8 + i < nvec) acc[g][i] = fma(v[g][i], we, acc[g][i]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    double a8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a8[i] = (double)acc[g][i];
    const double r = warp_reduce8(a8, lane);
    if ((lane & 3) == 0) sh[g * 8 + red8_index(lane)][warp] = r;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nvec; c += blockDim.x) {
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < RED_THREADS / 32; ++q) r += sh[c][q];
    partial[(size_t)c * gridDim.x + blockIdx.x] = r;
  }
  last_block_finish(nvec, gridDim.x, partial, counter, out);
}

// s = sum_c coef[c] V_c[e] with DOT_G independent loads in flight per element
template <typename TV, typename TS>
__device__ __forceinline__ TV comb(const TV* __restrict__ V, size_t vstride, int nvec, const TS* sc, int e) {
  TV s = TV(0);
  for (int c0 = 0; c0 < nvec; c0 += DOT_G) {
    TV v[DOT_G];
#pragma unroll
    for (int g = 0; g < DOT_G; ++g) v[g] = (c0 + g < nvec) ? V[(size_t)(c0 + g) * vstride + e] : TV(0);
#pragma unroll
    for (int g = 0; g < DOT_G; ++g)
      if (c0 + g < nvec) s = fma((TV)sc[c0 + g], v[g], s);
  }
  return s;
}

// w -= sum_c coef[c] V_c and out[0] = ||w||^2 of the result
template <typename TV>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy_norm(int len, TV* __restrict__ w, const TV* __restrict__ V,
                                                            size_t vstride, int nvec, const double* __restrict__ coef,
                                                            double* __restrict__ partial, unsigned* counter,
                                                            double* __restrict__ out) {
  __shared__ double sh[RED_THREADS / 32];
  __shared__ TV sc[MAX_VEC];
  for (int c = threadIdx.x; c < nvec; c += blockDim.x) sc[c] = (TV)coef[c];
  __syncthreads();
  const int stride = gridDim.x * blockDim.x;
  double nrm = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    const TV we = w[e] - comb<TV, TV>(V, vstride, nvec, sc, e);
    w[e] = we;
    nrm = fma((double)we, (double)we, nrm);
  }
  nrm = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = nrm;
  last_block_finish(1, gridDim.x, partial, counter, out);
}

// w += sign * sum_c coef[c] V_c
__global__ void k_maxpy(int len, double* __restrict__ w, const double* __restrict__ V, size_t vstride, int nvec,
                        const double* __restrict__ coef, double sign) {
  __shared__ double sc[MAX_VEC];
  for (int c = threadIdx.x; c < nvec; c += blockDim.x) sc[c] = coef[c];
  __syncthreads();
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride)
    w[e] = fma(sign, comb<double, double>(V, vstride, nvec, sc, e), w[e]);
}

__global__ void k_axpby(int len, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) y[e] = a * x[e] + b * y[e];
}

__global__ void k_scale_copy(int len, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) y[e] = a * x[e];
}

// y += sign * (*coef) * x with the coefficient read on the device
__global__ void k_axpy_dev(int len, const double* __restrict__ coef, double sign, const double* __restrict__ x,
                           double* __restrict__ y) {
  const double a = sign * coef[0];
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) y[e] = fma(a, x[e], y[e]);
}

// ------------------------------------------------------------ GMRES control
// The Arnoldi bookkeeping of GMRES(m) on the device, one thread: column j of
// the Hessenberg matrix from the two Gram-Schmidt passes (h0 + h1) and ||w||,
// the previous Givens rotations, the new one, the rotated right-hand side g;
// st[0] = |g[j+1]| / bnorm, st[1] = 1 / h_{j+1,j} (0 on breakdown), st[2] =
// h_{j+1,j}. No host round trip is needed per iteration.
constexpr int GM_MAX = 64;

__global__ void k_gmres_givens(int j, int m, double bnorm, const double* __restrict__ h0,
                               const double* __restrict__ h1, const double* __restrict__ nrm2,
                               double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                               double* __restrict__ g, double* __restrict__ st) {
  // one warp: the column and the previous rotations are loaded in parallel (two
  // entries per lane, j <= GM_MAX - 1 < 64), then lane 0 runs the dependent chain of
  // rotations with the operands fetched by shuffles instead of global loads
  const int lane = threadIdx.x & 31;
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  double c0 = 0.0, c1 = 0.0, s0 = 0.0, s1 = 0.0, v0 = 0.0, v1 = 0.0;
  if (lane <= j) v0 = h0[lane] + h1[lane];
  if (lane + 32 <= j) v1 = h0[lane + 32] + h1[lane + 32];
  if (lane < j) {
    c0 = cs[lane];
    s0 = sn[lane];
  }
  if (lane + 32 < j) {
    c1 = cs[lane + 32];
    s1 = sn[lane + 32];
  }
  const double hn = sqrt(fmax(*nrm2, 0.0));
  // rotated column: entry i is final once rotation i has been applied
  double out0 = 0.0, out1 = 0.0;
  double cur = __shfl_sync(FULL, v0, 0);  // running entry i (after rotations < i)
  for (int i = 0; i < j; ++i) {
    const double ci = __shfl_sync(FULL, i < 32 ? c0 : c1, i & 31);
    const double si = __shfl_sync(FULL, i < 32 ? s0 : s1, i & 31);
    const double nxt = __shfl_sync(FULL, (i + 1) < 32 ? v0 : v1, (i + 1) & 31);
    const double fin = ci * cur + si * nxt;  // final entry i
    cur = -si * cur + ci * nxt;              // entry i + 1 after rotation i
    if (lane == (i & 31)) {
      if (i < 32) out0 = fin;
      else out1 = fin;
    }
  }
  // the new rotation on (entry j, hn)
  const double a = cur, c = hn;
  const double den = hypot(a, c);
  const double cj = den > 0.0 ? a / den : 1.0, sj = den > 0.0 ? c / den : 0.0;
  const double dj = den > 0.0 ? den : a;
  if (lane == (j & 31)) {
    if (j < 32) out0 = dj;
    else out1 = dj;
  }
  if (lane <= j) H[(size_t)lane * m + j] = out0;
  if (lane + 32 <= j) H[(size_t)(lane + 32) * m + j] = out1;
  if (lane == 0) {
    cs[j] = cj;
    sn[j] = sj;
    const double gj = g[j];
    g[j + 1] = -sj * gj;
    g[j] = cj * gj;
    st[0] = fabs(g[j + 1]) / bnorm;
    st[1] = (hn > 0.0 && isfinite(hn)) ? 1.0 / hn : 0.0;
    st[2] = hn;
  }
}

__global__ void k_gmres_start(int m, double beta, double* __restrict__ g) {
  const int i = threadIdx.x;
  if (i <= m) g[i] = (i == 0) ? beta : 0.0;
}

// y = R^-1 g over the first jdone columns (back substitution), into y: one warp
// copies R and g into shared memory in parallel, then solves bottom-up with the
// row products split over the lanes
__global__ void k_gmres_backsub(int jdone, int m, const double* __restrict__ H, const double* __restrict__ g,
                                double* __restrict__ y) {
  __shared__ double sR[GM_MAX * GM_MAX];
  __shared__ double sy[GM_MAX];
  const int lane = threadIdx.x & 31;
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  for (int e = lane; e < jdone * jdone; e += 32) {
    const int i = e / jdone, k = e % jdone;
    sR[i * GM_MAX + k] = H[(size_t)i * m + k];
  }
  for (int i = lane; i < jdone; i += 32) sy[i] = g[i];
  __syncwarp();
  for (int i = jdone - 1; i >= 0; --i) {
    double part = 0.0;
    for (int k = i + 1 + lane; k < jdone; k += 32) part += sR[i * GM_MAX + k] * sy[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
    if (lane == 0) {
      const double d = sR[i * GM_MAX + i];
      const double acc = sy[i] - part;
      sy[i] = d != 0.0 ? acc / d : 0.0;  // a zero pivot only follows an exact (lucky) breakdown
    }
    __syncwarp();
  }
  for (int i = lane; i < jdone; i += 32) y[i] = sy[i];
}

// y = (*coef) x with the coefficient read on the device
template <typename TV>
__global__ void k_scale_dev(int len, const double* __restrict__ coef, const TV* __restrict__ x, TV* __restrict__ y) {
  const TV a = (TV)coef[0];
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) y[e] = a * x[e];
}

// ------------------------------------------------ inner FP32 GMRES (mixed precision)
// y32 = (float) x and out = ||y32||^2
__global__ void __launch_bounds__(RED_THREADS) k_f32_nrm(int len, const double* __restrict__ x, float* __restrict__ y,
                                                         double* __restrict__ partial, unsigned* counter,
                                                         double* __restrict__ out) {
  __shared__ double sh[RED_THREADS / 32];
  const int stride = gridDim.x * blockDim.x;
  double nrm = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    const float v = (float)x[e];
    y[e] = v;
    nrm = fma((double)v, (double)v, nrm);
  }
  nrm = block_sum(nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = nrm;
  last_block_finish(1, gridDim.x, partial, counter, out);
}

// g = (beta, 0, ..., 0) with beta = sqrt(*nrm2) read on the device; inv = 1 / beta (0 for a zero vector)
__global__ void k_gmres_start_dev(int m, const double* __restrict__ nrm2, double* __restrict__ g,
                                  double* __restrict__ inv) {
  const int i = threadIdx.x;
  const double beta = sqrt(fmax(*nrm2, 0.0));
  if (i <= m) g[i] = (i == 0) ? beta : 0.0;
  if (i == 0) *inv = (beta > 0.0 && isfinite(beta)) ? 1.0 / beta : 0.0;
}

// out = sum_c coef[c] V_c (FP32 basis, FP64 result)
template <typename TV>
__global__ void k_comb_out(int len, const TV* __restrict__ V, size_t vstride, int nvec, const double* __restrict__ coef,
                           double* __restrict__ out) {
  __shared__ TV sc[MAX_VEC];
  for (int c = threadIdx.x; c < nvec; c += blockDim.x) sc[c] = (TV)coef[c];
  __syncthreads();
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride)
    out[e] = (double)comb<TV, TV>(V, vstride, nvec, sc, e);
}

// y = recip_nr(x) and z = 1.0 / x, for the reciprocal self-check
__global__ void k_recip_check(int n, const double* __restrict__ x, double* __restrict__ y, double* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = recip_nr(x[i]);
  z[i] = 1.0 / x[i];
}

// ------------------------------------------------------------ Newton update
__global__ void k_update(int n, double* __restrict__ u, const double* __restrict__ du, double max_dp_frac,
                         double max_dT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double uo[8], d[8], un[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uo[k] = u[(size_t)k * n + i];
    d[k] = du[(size_t)i * 8 + k];
  }
  const double p = uo[0];
  un[0] = p + fmin(fmax(d[0], -max_dp_frac * p), max_dp_frac * p);
  un[5] = uo[5] + fmin(fmax(d[5], -max_dT), max_dT);
  // values taken in the halving branches are formed without contraction, so the
  // update is bit-identical to a plain evaluation of the same formulas
  double x = uo[1] + d[1];
  if (x < 0.0) x = 0.5 * uo[1];
  if (x > 1.0) x = __dsub_rn(1.0, __dmul_rn(0.5, __dsub_rn(1.0, uo[1])));
  un[1] = x;
  const int ks[5] = {2, 3, 4, 6, 7};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    int k = ks[q];
    double v = uo[k] + d[k];
    un[k] = (v < 0.0) ? 0.5 * uo[k] : v;
  }
  const double so_old = 1.0 - uo[6] - uo[7];
  const double so_new = 1.0 - un[6] - un[7];
  if (so_new < 0.0) {
    double target = __dsub_rn(1.0, __dmul_rn(0.5, so_old));
    double s = un[6] + un[7];
    un[6] *= target / s;
    un[7] *= target / s;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) u[(size_t)k * n + i] = un[k];
}

__global__ void k_to_f32(size_t n, const double* __restrict__ x, float* __restrict__ y) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += stride) y[e] = (float)x[e];
}

// The step controller's state changes: max |a - b| over the first n entries
// (temperature) into out[0] and over the next 2n (S_w, S_g) into out[1], as the
// bit patterns of non-negative doubles (IEEE order is numeric order there, so
// the integer maximum is the floating-point one and the result does not depend
// on the order of the blocks). out must be zero on entry.
__global__ void __launch_bounds__(256) k_max_change(int n, const double* __restrict__ a,
                                                    const double* __restrict__ b, unsigned long long* out) {
  unsigned long long mT = 0ull, mS = 0ull;
  const size_t len = (size_t)3 * n, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += stride) {
    const unsigned long long d = (unsigned long long)__double_as_longlong(fabs(a[e] - b[e]));
    if (e < (size_t)n)
      mT = max(mT, d);
    else
      mS = max(mS, d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mT = max(mT, (unsigned long long)__shfl_xor_sync(FULL, mT, o));
    mS = max(mS, (unsigned long long)__shfl_xor_sync(FULL, mS, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, mT);
    atomicMax(out + 1, mS);
  }
}

int grid_for(size_t work, int tb) {
  size_t b = (work + tb - 1) / tb;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_gj(Handle& h, cudaStream_t s) {
  int tb = 256;
  k_gj<<<(h.n * 16 + tb - 1) / tb, tb, 0, s>>>(h.n, h.rowptr, h.col, h.J, h.R, h.dstatus, h.well_slot, h.slots,
                                               h.nwc > 0 ? h.Bv : nullptr);
}

void launch_well_border_spmv(Handle& h, const double* x, double* y, cudaStream_t s) {
  if (h.nwc == 0) return;
  const size_t n8 = (size_t)h.n * 8;
  k_well_border_cells<<<(h.nslots * 8 + 127) / 128, 128, 0, s>>>(h.nslots, h.slots, h.Bv, x, y, n8);
  k_well_border_rows<<<(h.nwc + 31) / 32, 32, 0, s>>>(h.nwc, h.cw, h.slots, h.Cv, h.Dw, x, y, n8);
}

void launch_well_prec(Handle& h, const double* r, double* z, cudaStream_t s) {
  if (h.nwc == 0) return;
  k_well_prec<<<(h.nwc + 31) / 32, 32, 0, s>>>(h.nwc, h.cw, h.slots, h.Cv, h.Dw, r, z, (size_t)h.n * 8);
}

void launch_well_update(Handle& h, cudaStream_t s) {
  if (h.nwc == 0) return;
  k_well_update<<<(h.nwc + 31) / 32, 32, 0, s>>>(h.nwc, h.du, (size_t)h.n * 8, h.opt.max_dp_frac, h.bhp);
}

void launch_spmv(int nrows, const int32_t* rowptr, const int32_t* col, const double* val, const double* x, double* y,
                 int unit_diag, cudaStream_t s) {
  int tb = 256;
  k_spmv8<<<(int)(((size_t)nrows * 8 + tb - 1) / tb), tb, 0, s>>>(nrows, rowptr, col, val, x, y, unit_diag);
}

void launch_ilu_factor(Handle& h, cudaStream_t s) { launch_ilu_factor_pipe(h, s); }

void launch_bjacobi_factor(Handle& h, cudaStream_t s) {
  // all cells at once, no lower-neighbour terms; level_cells holds every cell
  k_ilu_factor<<<(h.n + FCELLS - 1) / FCELLS, 256, 0, s>>>(h.nx, h.ny, h.nz, h.level_cells, h.n, 0, h.rowptr, h.J,
                                                           h.dinv, h.dstatus);
}

void launch_prec_apply(Handle& h, const double* r, double* z, cudaStream_t s) {
  const int len = h.n * 8;
  if (h.opt.prec == ISC_PREC_NONE) {
    cudaMemcpyAsync(z, r, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    return;
  }
  if (h.opt.prec == ISC_PREC_BJACOBI) {
    k_bjacobi_apply<<<(h.n * 8 + 255) / 256, 256, 0, s>>>(h.n, h.dinv, r, z);
    return;
  }
  launch_ilu_apply_pipe(h, r, z, s);
}

void launch_gmres_givens(Handle& h, int j, int m, double bnorm, int off_h0, int off_h1, int off_nrm,
                         cudaStream_t s) {
  double* G = h.gmres;
  k_gmres_givens<<<1, 32, 0, s>>>(j, m, bnorm, h.scal + off_h0, h.scal + off_h1, h.scal + off_nrm, G,
                                  G + GM_MAX * (GM_MAX + 1), G + GM_MAX * (GM_MAX + 2), G + GM_MAX * (GM_MAX + 3),
                                  G + GM_MAX * (GM_MAX + 3) + GM_MAX + 1);
}

void launch_gmres_start(Handle& h, int m, double beta, cudaStream_t s) {
  k_gmres_start<<<1, GM_MAX + 1, 0, s>>>(m, beta, h.gmres + GM_MAX * (GM_MAX + 3));
}

void launch_gmres_backsub(Handle& h, int jdone, int m, int off_y, cudaStream_t s) {
  k_gmres_backsub<<<1, 32, 0, s>>>(jdone, m, h.gmres, h.gmres + GM_MAX * (GM_MAX + 3), h.scal + off_y);
}

void launch_scale_dev(Handle& h, const double* x, double* y, cudaStream_t s) {
  // coefficient: 1 / h_{j+1,j} from the last k_gmres_givens
  k_scale_dev<double><<<grid_for(h.vlen, 256), 256, 0, s>>>(h.vlen, h.gmres + GM_MAX * (GM_MAX + 3) + GM_MAX + 2, x, y);
}

const double* gmres_status(const Handle& h) { return h.gmres + GM_MAX * (GM_MAX + 3) + GM_MAX + 1; }

void launch_max_change(int n, const double* a, const double* b, unsigned long long* out, cudaStream_t s) {
  k_max_change<<<grid_for((size_t)3 * n, 256), 256, 0, s>>>(n, a, b, out);
}

void launch_to_f32(size_t n, const double* x, float* y, cudaStream_t s) {
  k_to_f32<<<grid_for(n, 256), 256, 0, s>>>(n, x, y);
}

void launch_update(Handle& h, cudaStream_t s) {
  k_update<<<(h.n + 127) / 128, 128, 0, s>>>(h.n, h.u, h.du, h.opt.max_dp_frac, h.opt.max_dT);
}

// FP32 Gram-Schmidt passes of the inner solve with 16-byte loads (four elements
// per lane and load). An FP32 vector carries half the bytes of an FP64 one per
// element, so with scalar loads too few bytes were in flight per SM to cover
// the HBM latency; the norm is accumulated in FP32 per lane (about 100 elements
// each) so that no per-element work reaches the narrow FP64 pipe. Lengths are
// multiples of 4 (8 per cell) and the vectors 16-byte aligned.
template <int NG>
__global__ void __launch_bounds__(RED_THREADS) k_mdot4(int len4, const float4* __restrict__ V, size_t vs4, int nvec,
                                                       const float4* __restrict__ w, double* __restrict__ partial,
                                                       unsigned* counter, double* __restrict__ out) {
  __shared__ double sh[NG * 8][RED_THREADS / 32];
  float acc[NG][8];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[g][i] = 0.f;
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len4; e += stride) {
    const float4 we = w[e];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (g * 8 + i < nvec) {
          const float4 v = V[(size_t)(g * 8 + i) * vs4 + e];
          acc[g][i] = fmaf(v.x, we.x, fmaf(v.y, we.y, fmaf(v.z, we.z, fmaf(v.w, we.w, acc[g][i]))));
        }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    double a8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a8[i] = (double)acc[g][i];
    const double v = warp_reduce8(a8, lane);
    if ((lane & 3) == 0) sh[g * 8 + red8_index(lane)][warp] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nvec; c += blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < RED_THREADS / 32; ++q) v += sh[c][q];
    partial[(size_t)c * gridDim.x + blockIdx.x] = v;
  }
  last_block_finish(nvec, gridDim.x, partial, counter, out);
}

// w <- w - V coef, then out = V^T w (each V_c loaded once for both)
template <int NG>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy_mdot4(int len4, float4* __restrict__ w,
                                                             const float4* __restrict__ V, size_t vs4, int nvec,
                                                             const double* __restrict__ coef,
                                                             double* __restrict__ partial, unsigned* counter,
                                                             double* __restrict__ out) {
  __shared__ double sh[NG * 8][RED_THREADS / 32];
  __shared__ float sc[NG * 8];
  for (int c = threadIdx.x; c < NG * 8; c += blockDim.x) sc[c] = c < nvec ? (float)coef[c] : 0.f;
  __syncthreads();
  float acc[NG][8];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[g][i] = 0.f;
  const int stride = gridDim.x * blockDim.x;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len4; e += stride) {
    float4 v[NG][8];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        v[g][i] = (g * 8 + i < nvec) ? V[(size_t)(g * 8 + i) * vs4 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 we = w[e];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (g * 8 + i < nvec) {
          const float c = sc[g * 8 + i];
          we.x = fmaf(-c, v[g][i].x, we.x);
          we.y = fmaf(-c, v[g][i].y, we.y);
          we.z = fmaf(-c, v[g][i].z, we.z);
          we.w = fmaf(-c, v[g][i].w, we.w);
        }
    w[e] = we;
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (g * 8 + i < nvec)
          acc[g][i] = fmaf(v[g][i].x, we.x, fmaf(v[g][i].y, we.y, fmaf(v[g][i].z, we.z, fmaf(v[g][i].w, we.w, acc[g][i]))));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    double a8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a8[i] = (double)acc[g][i];
    const double r = warp_reduce8(a8, lane);
    if ((lane & 3) == 0) sh[g * 8 + red8_index(lane)][warp] = r;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nvec; c += blockDim.x) {
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < RED_THREADS / 32; ++q) r += sh[c][q];
    partial[(size_t)c * gridDim.x + blockIdx.x] = r;
  }
  last_block_finish(nvec, gridDim.x, partial, counter, out);
}

// w <- w - V coef, then out = ||w||^2
__global__ void __launch_bounds__(RED_THREADS) k_maxpy_norm4(int len4, float4* __restrict__ w,
                                                             const float4* __restrict__ V, size_t vs4, int nvec,
                                                             const double* __restrict__ coef,
                                                             double* __restrict__ partial, unsigned* counter,
                                                             double* __restrict__ out) {
  __shared__ double sh[RED_THREADS / 32];
  __shared__ float sc[MAX_VEC];
  for (int c = threadIdx.x; c < nvec; c += blockDim.x) sc[c] = (float)coef[c];
  __syncthreads();
  const int stride = gridDim.x * blockDim.x;
  float nrm = 0.f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len4; e += stride) {
    float4 we = w[e];
    for (int c0 = 0; c0 < nvec; c0 += DOT_G) {
      float4 v[DOT_G];
#pragma unroll
      for (int g = 0; g < DOT_G; ++g)
        v[g] = (c0 + g < nvec) ? V[(size_t)(c0 + g) * vs4 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int g = 0; g < DOT_G; ++g) {
        const float c = (c0 + g < nvec) ? sc[c0 + g] : 0.f;
        we.x = fmaf(-c, v[g].x, we.x);
        we.y = fmaf(-c, v[g].y, we.y);
        we.z = fmaf(-c, v[g].z, we.z);
        we.w = fmaf(-c, v[g].w, we.w);
      }
    }
    w[e] = we;
    nrm = fmaf(we.x, we.x, fmaf(we.y, we.y, fmaf(we.z, we.z, fmaf(we.w, we.w, nrm))));
  }
  const double b = block_sum((double)nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
  last_block_finish(1, gridDim.x, partial, counter, out);
}

// Gram-Schmidt passes over vectors of length len stored vs apart (FP64 for the
// outer Krylov solve, FP32 for the inner one of the mixed-precision scheme);
// results (FP64) go to out; reductions use the handle's partial/counter buffers
template <typename TV>
bool mdot_t(Handle& h, int len, size_t vs, const TV* V, int nvec, const TV* w, double* out, cudaStream_t s) {
  // one pass over w for up to 32 vectors; grid and unrolling as measured best on GB300
  // (576,000-element FP64 vectors: 22 / 43 / 53 / 70 us for 8 / 16 / 24 / 30 vectors
  // against 49 / 57 / 70 / 100 us with the vectors split over blockIdx.y)
  switch ((nvec + 7) / 8) {
    case 1: k_mdot_t<TV, 1, 1><<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len, V, vs, nvec, w, h.partial, h.red_counter, out); return true;
    case 2: k_mdot_t<TV, 2, 2><<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len, V, vs, nvec, w, h.partial, h.red_counter, out); return true;
    case 3: k_mdot_t<TV, 3, 1><<<h.red_blocks, RED_THREADS, 0, s>>>(len, V, vs, nvec, w, h.partial, h.red_counter, out); return true;
    case 4: k_mdot_t<TV, 4, 1><<<h.red_blocks, RED_THREADS, 0, s>>>(len, V, vs, nvec, w, h.partial, h.red_counter, out); return true;
    default: return false;
  }
}

template <typename TV>
bool maxpy_mdot_t(Handle& h, int len, size_t vs, TV* w, const TV* V, int nvec, const double* coef, double* out,
                  cudaStream_t s) {
  switch ((nvec + 7) / 8) {
    case 1: k_maxpy_mdot<TV, 1><<<h.red_blocks, RED_THREADS, 0, s>>>(len, w, V, vs, nvec, coef, h.partial, h.red_counter, out); return true;
    case 2: k_maxpy_mdot<TV, 2><<<h.red_blocks, RED_THREADS, 0, s>>>(len, w, V, vs, nvec, coef, h.partial, h.red_counter, out); return true;
    case 3: k_maxpy_mdot<TV, 3><<<h.red_blocks, RED_THREADS, 0, s>>>(len, w, V, vs, nvec, coef, h.partial, h.red_counter, out); return true;
    case 4: k_maxpy_mdot<TV, 4><<<h.red_blocks, RED_THREADS, 0, s>>>(len, w, V, vs, nvec, coef, h.partial, h.red_counter, out); return true;
    default: return false;
  }
}

template <typename TV>
void maxpy_norm_t(Handle& h, int len, size_t vs, TV* w, const TV* V, int nvec, const double* coef, double* out,
                  cudaStream_t s) {
  // 608 blocks: 20.7 / 28 / 40 / 46 us for 8 / 16 / 24 / 30 FP64 vectors against 23 / 36 / 51 / 60 with 304
  k_maxpy_norm<TV><<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len, w, V, vs, nvec, coef, h.partial, h.red_counter, out);
}

void launch_mdot(Handle& h, const double* V, int nvec, const double* w, int off, cudaStream_t s) {
  if (mdot_t<double>(h, h.vlen, (size_t)h.vstride, V, nvec, w, h.scal + off, s)) return;
  dim3 grid(h.red_blocks, (nvec + DOT_G - 1) / DOT_G);
  k_mdot<<<grid, RED_THREADS, 0, s>>>(h.vlen, V, (size_t)h.vstride, nvec, w, h.partial, h.red_counter, h.scal + off);
}

void launch_maxpy_mdot(Handle& h, double* w, const double* V, int nvec, int coef_off, int out_off, cudaStream_t s) {
  if (maxpy_mdot_t<double>(h, h.vlen, (size_t)h.vstride, w, V, nvec, h.scal + coef_off, h.scal + out_off, s)) return;
  launch_maxpy(h, w, V, nvec, coef_off, -1.0, s);
  launch_mdot(h, V, nvec, w, out_off, s);
}

void launch_maxpy_norm(Handle& h, double* w, const double* V, int nvec, int coef_off, int out_off, cudaStream_t s) {
  maxpy_norm_t<double>(h, h.vlen, (size_t)h.vstride, w, V, nvec, h.scal + coef_off, h.scal + out_off, s);
}

void launch_maxpy(Handle& h, double* w, const double* V, int nvec, int coef_off, double sign, cudaStream_t s) {
  const int len = h.vlen;
  k_maxpy<<<grid_for(len, 256), 256, 0, s>>>(len, w, V, (size_t)h.vstride, nvec, h.scal + coef_off, sign);
}

void launch_axpby(int n, double a, const double* x, double b, double* y, cudaStream_t s) {
  k_axpby<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, b, y);
}

void launch_scale_copy(int n, double a, const double* x, double* y, cudaStream_t s) {
  k_scale_copy<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, y);
}

void launch_axpy_dev(int n, const double* coef, double sign, const double* x, double* y, cudaStream_t s) {
  k_axpy_dev<<<grid_for(n, 256), 256, 0, s>>>(n, coef, sign, x, y);
}

// ---- inner FP32 GMRES of the mixed-precision scheme (state G: GMRES_STATE doubles)
void launch_f32_nrm(Handle& h, int len, const double* x, float* y, double* out, cudaStream_t s) {
  k_f32_nrm<<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len, x, y, h.partial, h.red_counter, out);
}
void launch_gmres_start_dev(double* G, int m, const double* nrm2, cudaStream_t s) {
  k_gmres_start_dev<<<1, GM_MAX + 1, 0, s>>>(m, nrm2, G + GM_MAX * (GM_MAX + 3), G + GM_MAX * (GM_MAX + 3) + GM_MAX + 2);
}
void launch_gmres_givens_at(double* G, int j, int m, const double* h0, const double* h1, const double* nrm, cudaStream_t s) {
  k_gmres_givens<<<1, 32, 0, s>>>(j, m, 1.0, h0, h1, nrm, G, G + GM_MAX * (GM_MAX + 1), G + GM_MAX * (GM_MAX + 2),
                                  G + GM_MAX * (GM_MAX + 3), G + GM_MAX * (GM_MAX + 3) + GM_MAX + 1);
}
void launch_gmres_backsub_at(double* G, int jdone, int m, double* y, cudaStream_t s) {
  k_gmres_backsub<<<1, 32, 0, s>>>(jdone, m, G, G + GM_MAX * (GM_MAX + 3), y);
}
void launch_scale_dev32(double* G, int len, const float* x, float* y, cudaStream_t s) {
  // coefficient at the status slot used by k_gmres_givens (1 / h_{j+1,j}) and k_gmres_start_dev (1 / beta)
  k_scale_dev<float><<<grid_for(len, 256), 256, 0, s>>>(len, G + GM_MAX * (GM_MAX + 3) + GM_MAX + 2, x, y);
}
void launch_spmv32(int nrows, const int32_t* rowptr, const int32_t* col, const float* val, const float* x, float* y,
                   int unit_diag, cudaStream_t s) {
  const int tb = 256;
  k_spmv<float><<<(int)(((size_t)nrows * 32 + tb - 1) / tb), tb, 0, s>>>(nrows, rowptr, col, val, x, y, unit_diag);
}
// the inner solve's vectors are 8N floats stored 8N apart: 16-byte loads unless
// a caller passes a length or stride that is not a multiple of 4
static bool vec4_ok(int len, size_t vs, const void* a, const void* b) {
  return len % 4 == 0 && vs % 4 == 0 && ((uintptr_t)a & 15) == 0 && ((uintptr_t)b & 15) == 0;
}
void launch_mdot32(Handle& h, int len, size_t vs, const float* V, int nvec, const float* w, double* out, cudaStream_t s) {
  if (vec4_ok(len, vs, V, w) && nvec <= 16) {
    const float4 *V4 = reinterpret_cast<const float4*>(V), *w4 = reinterpret_cast<const float4*>(w);
    if (nvec <= 8)
      k_mdot4<1><<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len / 4, V4, vs / 4, nvec, w4, h.partial, h.red_counter, out);
    else
      k_mdot4<2><<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len / 4, V4, vs / 4, nvec, w4, h.partial, h.red_counter, out);
    return;
  }
  mdot_t<float>(h, len, vs, V, nvec, w, out, s);
}
void launch_maxpy_mdot32(Handle& h, int len, size_t vs, float* w, const float* V, int nvec, const double* coef,
                         double* out, cudaStream_t s) {
  if (vec4_ok(len, vs, V, w) && nvec <= 16) {
    float4* w4 = reinterpret_cast<float4*>(w);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    if (nvec <= 8)
      k_maxpy_mdot4<1><<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len / 4, w4, V4, vs / 4, nvec, coef, h.partial,
                                                                h.red_counter, out);
    else
      k_maxpy_mdot4<2><<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len / 4, w4, V4, vs / 4, nvec, coef, h.partial,
                                                                h.red_counter, out);
    return;
  }
  maxpy_mdot_t<float>(h, len, vs, w, V, nvec, coef, out, s);
}
void launch_maxpy_norm32(Handle& h, int len, size_t vs, float* w, const float* V, int nvec, const double* coef,
                         double* out, cudaStream_t s) {
  if (vec4_ok(len, vs, V, w)) {
    k_maxpy_norm4<<<2 * h.red_blocks, RED_THREADS, 0, s>>>(len / 4, reinterpret_cast<float4*>(w),
                                                           reinterpret_cast<const float4*>(V), vs / 4, nvec, coef,
                                                           h.partial, h.red_counter, out);
    return;
  }
  maxpy_norm_t<float>(h, len, vs, w, V, nvec, coef, out, s);
}
void launch_comb_out32(int len, const float* V, size_t vs, int nvec, const double* coef, double* out, cudaStream_t s) {
  k_comb_out<float><<<grid_for(len, 256), 256, 0, s>>>(len, V, vs, nvec, coef, out);
}

void launch_recip_check(int n, const double* x, double* y, double* z, cudaStream_t s) {
  k_recip_check<<<(n + 255) / 256, 256, 0, s>>>(n, x, y, z);
}

}  // namespace isc
