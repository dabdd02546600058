// CPR-PF two-stage preconditioner (Sec. 4, Example 2: the solver's
// preconditioner changes from RAS to CPR-PF). On the Gauss-Jordan-decoupled
// system (unit diagonal blocks, Sec. 3.2) row 0 of a block row is the equation
// paired with the cell's pressure; the pressure matrix A_p is the (0,0) entry
// of every block. One application:
//   p  = one V-cycle of A_p p = r_p (r_p the pressure rows of r, zero guess)
//   r1 = r - A E p            (E injects p into unknown 0 of every cell)
//   z  = ILU(0)^-1 r1 + E p
// Pressure multigrid: MG_AGG x MG_AGG x-y aggregates (piecewise-constant
// prolongation, Galerkin coarse operators, which keep the 7-point structure),
// z not coarsened, down to a single column; red-black z-line Gauss-Seidel
// (columns coloured by (x + y) mod 2, colour 0 first, each column's
// tridiagonal system solved exactly); one pre- and one post-smoothing sweep;
// exact column solve on the coarsest level.
//
// The tridiagonal factors of every column (1/pivot and upper/pivot of the
// Thomas elimination) are computed once per setup, so an application does no
// division: on GB300 a warp-wide FP64 division costs tens of FP64 issue
// slots. The level arrays are FP64, or FP32 when the preconditioner runs in
// mixed precision (the second-stage residual stays FP64).
//
// Kernels: k_cpr_extract (A_p stencil and the unknown-0 column of every
// block), k_mg_coarsen (Galerkin sums over an aggregate), k_mg_factor (column
// factors), k_zline (one thread per column of a colour), k_mg_restrict,
// k_mg_prolong, k_mg_coarse (the levels of at most MG_BLOCK_CELLS cells in
// one thread block with barriers), k_cpr_gather, k_cpr_residual, k_cpr_add.
#include "isc_internal.cuh"

namespace isc {

namespace {

// stencil directions: 0 -z, 1 -y, 2 -x, 3 diagonal, 4 +x, 5 +y, 6 +z
template <typename T>
__device__ __forceinline__ int nb_index(const MGLevel<T>& L, int i, int d) {
  const int nxy = L.nx * L.ny;
  switch (d) {
    case 0: return i - nxy;
    case 1: return i - L.nx;
    case 2: return i - 1;
    case 4: return i + 1;
    case 5: return i + L.nx;
    case 6: return i + nxy;
    default: return i;
  }
}

// A_p stencil and the unknown-0 column of every block, from the decoupled J
template <typename T>
__global__ void k_cpr_extract(int nx, int ny, int nz, const int32_t* __restrict__ rowptr,
                              const double* __restrict__ J, T* __restrict__ c, double* __restrict__ col0) {
  const int n = nx * ny * nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nxy = nx * ny;
  double cd[7] = {0, 0, 0, 0, 0, 0, 0};
  // the row holds the existing neighbours in the order -z, -y, -x, diagonal, +x, +y, +z
  const int x = i % nx, y = (i / nx) % ny, z = i / nxy;
  const bool has[7] = {z > 0, y > 0, x > 0, true, x < nx - 1, y < ny - 1, z < nz - 1};
  int b = rowptr[i];
  for (int d = 0; d < 7; ++d) {
    if (!has[d]) continue;
    const double* B = J + (size_t)b * BB;
    cd[d] = B[0];
#pragma unroll
    for (int r = 0; r < 8; ++r) col0[(size_t)b * 8 + r] = B[r * 8];
    ++b;
  }
#pragma unroll
  for (int d = 0; d < 7; ++d) c[(size_t)d * n + i] = (T)cd[d];
}

// Galerkin coarse operator of the x-y aggregation: sums of the fine entries
template <typename T>
__device__ __forceinline__ void coarsen_cell(const MGLevel<T>& F, const MGLevel<T>& C, int I) {
  const int X = I % C.nx, Y = (I / C.nx) % C.ny, k = I / (C.nx * C.ny);
  const int x0 = MG_AGG * X, y0 = MG_AGG * Y;
  T cd[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int fy = y0; fy < y0 + MG_AGG && fy < F.ny; ++fy) {
    for (int fx = x0; fx < x0 + MG_AGG && fx < F.nx; ++fx) {
      const int f = fx + F.nx * (fy + F.ny * k);
      cd[0] += F.c[(size_t)0 * F.n + f];
      cd[6] += F.c[(size_t)6 * F.n + f];
      cd[3] += F.c[(size_t)3 * F.n + f];
      // x and y couplings stay inside the aggregate (diagonal) or cross to a neighbour aggregate
      cd[(fx - 1 >= x0) ? 3 : 2] += F.c[(size_t)2 * F.n + f];
      cd[(fx + 1 < x0 + MG_AGG) ? 3 : 4] += F.c[(size_t)4 * F.n + f];
      cd[(fy - 1 >= y0) ? 3 : 1] += F.c[(size_t)1 * F.n + f];
      cd[(fy + 1 < y0 + MG_AGG) ? 3 : 5] += F.c[(size_t)5 * F.n + f];
    }
  }
#pragma unroll
  for (int d = 0; d < 7; ++d) C.c[(size_t)d * C.n + I] = cd[d];
}

// z-levels staged per chunk: a column's loads of one chunk are independent and
// in flight together; only the recurrences run in order, from registers
template <typename T> struct ZChunk;
template <> struct ZChunk<double> { static constexpr int v = 16; };
template <> struct ZChunk<float> { static constexpr int v = 32; };

// Thomas factors of column (cx, cy): e_k = 1 / (b_k - a_k f_{k-1}), f_k = c_k e_k
template <typename T>
__device__ __forceinline__ void factor_column(const MGLevel<T>& L, int cx, int cy) {
  constexpr int ZC = ZChunk<T>::v;
  const int nxy = L.nx * L.ny, n = L.n, i0 = cx + L.nx * cy;
  T lo[ZC], dg[ZC], up[ZC];
  T fp = 0;
  for (int k0 = 0; k0 < L.nz; k0 += ZC) {
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
      const int k = k0 + q, i = i0 + nxy * k;
      if (k < L.nz) {
        lo[q] = (k > 0) ? L.c[(size_t)0 * n + i] : T(0);
        dg[q] = L.c[(size_t)3 * n + i];
        up[q] = (k < L.nz - 1) ? L.c[(size_t)6 * n + i] : T(0);
      }
    }
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
      const int k = k0 + q, i = i0 + nxy * k;
      if (k < L.nz) {
        const T e = T(1) / (dg[q] - lo[q] * fp);
        fp = up[q] * e;
        L.e[i] = e;
        L.f[i] = fp;
      }
    }
  }
}

// Solve column (cx, cy)'s z-tridiagonal system with the other columns' current
// values (zero_guess: the other columns are zero). Forward y_k = e_k rhs_k -
// e_k a_k y_{k-1}, backward x_k = y_k - f_k x_{k+1}.
template <typename T>
__device__ __forceinline__ void zline_column(const MGLevel<T>& L, int cx, int cy, bool zero_guess) {
  constexpr int ZC = ZChunk<T>::v;
  const int nxy = L.nx * L.ny, n = L.n, i0 = cx + L.nx * cy;
  const T* __restrict__ c = L.c;
  T* __restrict__ x = L.x;
  T g[ZC], a[ZC];
  T bp = 0;
  for (int k0 = 0; k0 < L.nz; k0 += ZC) {
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
      const int k = k0 + q, i = i0 + nxy * k;
      if (k < L.nz) {
        T rhs = L.b[i];
        if (!zero_guess) {
          if (cy > 0) rhs -= c[(size_t)1 * n + i] * x[i - L.nx];
          if (cx > 0) rhs -= c[(size_t)2 * n + i] * x[i - 1];
          if (cx < L.nx - 1) rhs -= c[(size_t)4 * n + i] * x[i + 1];
          if (cy < L.ny - 1) rhs -= c[(size_t)5 * n + i] * x[i + L.nx];
        }
        const T e = L.e[i];
        g[q] = e * rhs;
        a[q] = (k > 0) ? -c[(size_t)0 * n + i] * e : T(0);
      }
    }
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
      const int k = k0 + q;
      if (k < L.nz) {
        bp = fma(a[q], bp, g[q]);
        x[i0 + nxy * k] = bp;
      }
    }
  }
  T xn = 0;
  for (int k1 = L.nz; k1 > 0; k1 -= ZC) {
    const int k0 = k1 - ZC;
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
      const int k = k0 + q;
      if (k >= 0) {
        g[q] = x[i0 + nxy * k];
        a[q] = L.f[i0 + nxy * k];
      }
    }
#pragma unroll
    for (int q = ZC - 1; q >= 0; --q) {
      const int k = k0 + q;
      if (k >= 0) {
        xn = g[q] - a[q] * xn;
        x[i0 + nxy * k] = xn;
      }
    }
  }
}

// The same column solve by one warp (columns of at most 64 z-levels): lane l
// holds levels 2l and 2l+1. With the factors precomputed both recurrences
// are first-order linear, y_k = g_k + a_k y_{k-1} and x_k = y_k + b_k x_{k+1}
// (b = -f), so each runs as a Kogge-Stone scan of affine maps across the
// lanes: one round of independent loads and ten shuffle steps instead of a
// chain of nz dependent steps. Levels at or beyond nz are identity maps.
template <typename T>
__device__ __forceinline__ void zline_column_warp(const MGLevel<T>& L, int cx, int cy, bool zero_guess) {
  const unsigned FULLM = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nxy = L.nx * L.ny, n = L.n, i0 = cx + L.nx * cy;
  const T* __restrict__ c = L.c;
  T* __restrict__ x = L.x;
  T g[2], a[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = 2 * lane + h, i = i0 + nxy * k;
    g[h] = T(0);
    a[h] = T(0);
    if (k < L.nz) {
      T rhs = L.b[i];
      if (!zero_guess) {
        if (cy > 0) rhs -= c[(size_t)1 * n + i] * x[i - L.nx];
        if (cx > 0) rhs -= c[(size_t)2 * n + i] * x[i - 1];
        if (cx < L.nx - 1) rhs -= c[(size_t)4 * n + i] * x[i + 1];
        if (cy < L.ny - 1) rhs -= c[(size_t)5 * n + i] * x[i + L.nx];
      }
      const T e = L.e[i];
      g[h] = e * rhs;
      a[h] = (k > 0) ? -c[(size_t)0 * n + i] * e : T(0);
    }
  }
  // forward: the lane's map y_{2l-1} -> y_{2l+1}, then the inclusive scan over lanes
  T A = a[1] * a[0], G = fma(a[1], g[0], g[1]);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T Ad = __shfl_up_sync(FULLM, A, d), Gd = __shfl_up_sync(FULLM, G, d);
    if (lane >= d) {
      G = fma(A, Gd, G);
      A = A * Ad;
    }
  }
  T yprev = __shfl_up_sync(FULLM, G, 1);  // y_{2l-1}
  if (lane == 0) yprev = T(0);
  const T y0 = fma(a[0], yprev, g[0]);
  const T y1 = G;
  // backward: x_k = y_k + b_k x_{k+1}; the lane's map x_{2l+2} -> x_{2l}
  T bq[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = 2 * lane + h;
    bq[h] = (k < L.nz) ? -L.f[i0 + nxy * k] : T(0);
  }
  T B = bq[0] * bq[1], X = fma(bq[0], y1, y0);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T Bd = __shfl_down_sync(FULLM, B, d), Xd = __shfl_down_sync(FULLM, X, d);
    if (lane + d < 32) {
      X = fma(B, Xd, X);
      B = B * Bd;
    }
  }
  T xnext = __shfl_down_sync(FULLM, X, 1);  // x_{2l+2}
  if (lane == 31) xnext = T(0);
  const T x0 = X;
  const T x1 = fma(bq[1], xnext, y1);
  if (2 * lane < L.nz) x[i0 + nxy * (2 * lane)] = x0;
  if (2 * lane + 1 < L.nz) x[i0 + nxy * (2 * lane + 1)] = x1;
}

// b_C = sum over the aggregate of (b_F - A_F x_F)
template <typename T>
__device__ __forceinline__ void restrict_cell(const MGLevel<T>& F, const MGLevel<T>& C, int I) {
  const int X = I % C.nx, Y = (I / C.nx) % C.ny, k = I / (C.nx * C.ny);
  const int x0 = MG_AGG * X, y0 = MG_AGG * Y;
  T s = 0;
  for (int fy = y0; fy < y0 + MG_AGG && fy < F.ny; ++fy) {
    for (int fx = x0; fx < x0 + MG_AGG && fx < F.nx; ++fx) {
      const int f = fx + F.nx * (fy + F.ny * k);
      T r = F.b[f];
      const bool has[7] = {k > 0, fy > 0, fx > 0, true, fx < F.nx - 1, fy < F.ny - 1, k < F.nz - 1};
#pragma unroll
      for (int d = 0; d < 7; ++d)
        if (has[d]) r -= F.c[(size_t)d * F.n + f] * F.x[nb_index(F, f, d)];
      s += r;
    }
  }
  C.b[I] = s;
}

template <typename T>
__device__ __forceinline__ void prolong_cell(const MGLevel<T>& C, const MGLevel<T>& F, int f) {
  const int fx = f % F.nx, fy = (f / F.nx) % F.ny, k = f / (F.nx * F.ny);
  F.x[f] += C.x[(fx / MG_AGG) + C.nx * ((fy / MG_AGG) + C.ny * k)];
}

// column q of colour `colour` (columns with (cx + cy) % 2 == colour, row-major): its (cx, cy)
__device__ __forceinline__ bool colour_column(int nx, int ny, int colour, int q, int* cx, int* cy) {
  const int per_row0 = (nx + 1) / 2, per_row1 = nx / 2;  // colour-(row parity) columns in a row
  // rows alternate which parity comes first; count row by row
  const int pair = per_row0 + per_row1;                    // columns of one colour in two rows
  const int r2 = q / pair, rem = q % pair;
  int row, idx;
  const int first = (colour == 0) ? per_row0 : per_row1;   // this colour's count in an even row
  if (rem < first) {
    row = 2 * r2;
    idx = rem;
  } else {
    row = 2 * r2 + 1;
    idx = rem - first;
  }
  if (row >= ny) return false;
  // in row `row` the columns of this colour have x parity (colour + row) & 1
  const int x = 2 * idx + ((colour + row) & 1);
  if (x >= nx) return false;
  *cx = x;
  *cy = row;
  return true;
}

__host__ __device__ __forceinline__ int colour_count(int nx, int ny, int colour) {
  // columns (x, y) with (x + y) % 2 == colour
  const int even = ((nx * ny) + 1) / 2;
  return colour == 0 ? even : nx * ny - even;
}

template <typename T>
__global__ void k_mg_coarsen(const MGLevel<T>* __restrict__ lv, int l) {
  const MGLevel<T> F = lv[l], C = lv[l + 1];
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < C.n) coarsen_cell(F, C, I);
}

template <typename T>
__global__ void k_mg_factor(const MGLevel<T>* __restrict__ lv, int l) {
  const MGLevel<T> L = lv[l];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < L.nx * L.ny) factor_column(L, t % L.nx, t / L.nx);
}

constexpr int ZWARP_MAX = 64;  // columns this short are solved by one warp (two levels per lane)

// one warp per column of the colour (WARP: nz <= ZWARP_MAX), else one thread per column
template <typename T, bool WARP>
__global__ void k_zline(const MGLevel<T>* __restrict__ lv, int l, int colour, int zero_guess) {
  const MGLevel<T> L = lv[l];
  int cx, cy;
  if (WARP) {
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // the same in every lane
    if (colour_column(L.nx, L.ny, colour, q, &cx, &cy)) zline_column_warp(L, cx, cy, zero_guess != 0);
    return;
  }
  if (colour_column(L.nx, L.ny, colour, blockIdx.x * blockDim.x + threadIdx.x, &cx, &cy))
    zline_column(L, cx, cy, zero_guess != 0);
}

template <typename T>
__global__ void k_mg_restrict(const MGLevel<T>* __restrict__ lv, int l) {
  const MGLevel<T> F = lv[l], C = lv[l + 1];
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < C.n) restrict_cell(F, C, I);
}

template <typename T>
__global__ void k_mg_prolong(const MGLevel<T>* __restrict__ lv, int l) {
  const MGLevel<T> C = lv[l + 1], F = lv[l];
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < F.n) prolong_cell(C, F, f);
}

// all columns of one level (warps over columns when WARP)
template <typename T, bool WARP>
__device__ __forceinline__ void block_columns(const MGLevel<T>& L, int colour, bool zero_guess) {
  const int cnt = colour < 0 ? L.nx * L.ny : colour_count(L.nx, L.ny, colour);
  if (WARP) {
    for (int q = threadIdx.x >> 5; q < cnt; q += blockDim.x >> 5) {
      int cx = q % L.nx, cy = q / L.nx;
      if (colour < 0 || colour_column(L.nx, L.ny, colour, q, &cx, &cy)) zline_column_warp(L, cx, cy, zero_guess);
    }
  } else {
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      int cx = q % L.nx, cy = q / L.nx;
      if (colour < 0 || colour_column(L.nx, L.ny, colour, q, &cx, &cy)) zline_column(L, cx, cy, zero_guess);
    }
  }
  __syncthreads();
}

template <typename T, bool WARP>
__device__ __forceinline__ void block_smooth(const MGLevel<T>& L, bool zero_guess) {
  block_columns<T, WARP>(L, 0, zero_guess);
  block_columns<T, WARP>(L, 1, false);
}

// Levels l0 .. nlev-1 of the V-cycle in one thread block (b of level l0 is set).
template <typename T, bool WARP>
__global__ void __launch_bounds__(512) k_mg_coarse(const MGLevel<T>* __restrict__ lv, int l0, int nlev) {
  const int t = threadIdx.x, TT = blockDim.x;
  for (int l = l0; l < nlev - 1; ++l) {
    const MGLevel<T> L = lv[l], C = lv[l + 1];
    block_smooth<T, WARP>(L, true);
    for (int I = t; I < C.n; I += TT) restrict_cell(L, C, I);
    __syncthreads();
  }
  block_columns<T, WARP>(lv[nlev - 1], -1, true);  // the single-column level: exact solve
  for (int l = nlev - 2; l >= l0; --l) {
    const MGLevel<T> L = lv[l], C = lv[l + 1];
    for (int f = t; f < L.n; f += TT) prolong_cell(C, L, f);
    __syncthreads();
    block_smooth<T, WARP>(L, false);
  }
}

// RV: the type of the vectors the preconditioner is applied to (FP64 inside the
// FP64 GMRES, FP32 inside the inner solve of ISC_PRECISION_MIXED_FGMRES)
template <typename T, typename RV>
__global__ void k_cpr_gather(int n, const RV* __restrict__ r, T* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)r[(size_t)i * 8];
}

// r1 = r - A E p: thread (i, row) sums the unknown-0 column entries of row i's blocks
template <typename T, typename RV>
__global__ void k_cpr_residual(int n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ col0, const RV* __restrict__ r, const T* __restrict__ p,
                               RV* __restrict__ r1) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * 8) return;
  const int i = (int)(e >> 3), row = (int)(e & 7);
  double s = (double)r[e];
  for (int b = rowptr[i]; b < rowptr[i + 1]; ++b) s -= col0[(size_t)b * 8 + row] * (double)p[col[b]];
  r1[e] = (RV)s;
}

template <typename T, typename RV>
__global__ void k_cpr_add(int n, const T* __restrict__ p, RV* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[(size_t)i * 8] += (RV)p[i];
}

inline int nblk(long long n, int tb) { return (int)((n + tb - 1) / tb); }

template <typename T>
std::vector<MGLevel<T>>& table(CprWork& W);
template <>
std::vector<MGLevel<double>>& table<double>(CprWork& W) {
  return W.h64;
}
template <>
std::vector<MGLevel<float>>& table<float>(CprWork& W) {
  return W.h32;
}

template <typename T>
int setup_levels_t(Handle& h) {
  CprWork& W = h.cpr;
  std::vector<MGLevel<T>> lv;
  int nx = h.nx, ny = h.ny, nz = h.nz;
  for (;;) {
    MGLevel<T> L{};
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.n = nx * ny * nz;
    lv.push_back(L);
    if (nx == 1 && ny == 1) break;
    nx = (nx + MG_AGG - 1) / MG_AGG;
    ny = (ny + MG_AGG - 1) / MG_AGG;
  }
  size_t total = 0;
  for (auto& L : lv) total += (size_t)L.n * 11;
  if (cudaMalloc(&W.pool, sizeof(T) * total) != cudaSuccess) return ISC_ERR_NOMEM;
  W.bytes += sizeof(T) * total;
  T* q = static_cast<T*>(W.pool);
  for (auto& L : lv) {
    L.c = q;
    q += (size_t)7 * L.n;
    L.x = q;
    q += L.n;
    L.b = q;
    q += L.n;
    L.e = q;
    q += L.n;
    L.f = q;
    q += L.n;
  }
  if (cudaMalloc(&W.d_levels, sizeof(MGLevel<T>) * lv.size()) != cudaSuccess) return ISC_ERR_NOMEM;
  W.bytes += sizeof(MGLevel<T>) * lv.size();
  if (cudaMemcpy(W.d_levels, lv.data(), sizeof(MGLevel<T>) * lv.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return ISC_ERR_CUDA;
  W.nlev = (int)lv.size();
  W.ngrid = 0;
  while (W.ngrid < W.nlev - 1 && lv[W.ngrid].n > MG_BLOCK_CELLS) ++W.ngrid;
  table<T>(W) = lv;
  return ISC_OK;
}

template <typename T>
void setup_t(Handle& h, cudaStream_t s) {
  CprWork& W = h.cpr;
  const auto& lv = table<T>(W);
  const MGLevel<T>* d = static_cast<const MGLevel<T>*>(W.d_levels);
  const int tb = 128;
  k_cpr_extract<T><<<nblk(h.n, tb), tb, 0, s>>>(h.nx, h.ny, h.nz, h.rowptr, h.J, lv[0].c, W.col0);
  for (int l = 0; l + 1 < W.nlev; ++l) k_mg_coarsen<T><<<nblk(lv[l + 1].n, tb), tb, 0, s>>>(d, l);
  for (int l = 0; l < W.nlev; ++l) k_mg_factor<T><<<nblk(lv[l].nx * lv[l].ny, tb), tb, 0, s>>>(d, l);
}

template <typename T, typename RV>
void pressure_t(Handle& h, const RV* r, RV* r1, cudaStream_t s) {
  CprWork& W = h.cpr;
  const auto& lv = table<T>(W);
  const MGLevel<T>* d = static_cast<const MGLevel<T>*>(W.d_levels);
  const int tb = 128;
  k_cpr_gather<T, RV><<<nblk(h.n, tb), tb, 0, s>>>(h.n, r, lv[0].b);
  // threads of a z-line pass: a warp per column (nz <= ZWARP_MAX) or a thread per column
  const bool warp = h.nz <= ZWARP_MAX;
  auto zline = [&](int l, int colour, int zero) {
    const long long cnt = colour_count(lv[l].nx, lv[l].ny, colour);
    if (warp)
      k_zline<T, true><<<nblk(32 * cnt, tb), tb, 0, s>>>(d, l, colour, zero);
    else
      k_zline<T, false><<<nblk(cnt, tb), tb, 0, s>>>(d, l, colour, zero);
  };
  for (int l = 0; l < W.ngrid; ++l) {
    zline(l, 0, 1);
    zline(l, 1, 0);
    k_mg_restrict<T><<<nblk(lv[l + 1].n, tb), tb, 0, s>>>(d, l);
  }
  if (warp)
    k_mg_coarse<T, true><<<1, 512, 0, s>>>(d, W.ngrid, W.nlev);
  else
    k_mg_coarse<T, false><<<1, 512, 0, s>>>(d, W.ngrid, W.nlev);
  for (int l = W.ngrid - 1; l >= 0; --l) {
    k_mg_prolong<T><<<nblk(lv[l].n, tb), tb, 0, s>>>(d, l);
    zline(l, 0, 0);
    zline(l, 1, 0);
  }
  k_cpr_residual<T, RV><<<nblk((long long)h.n * 8, 256), 256, 0, s>>>(h.n, h.rowptr, h.col, W.col0, r, lv[0].x, r1);
}

}  // namespace

int cpr_setup_levels(Handle& h) {
  CprWork& W = h.cpr;
  const bool fp32 = h.opt.precision != ISC_PRECISION_FP64;
  if (W.nlev > 0 && W.fp32 == fp32) return ISC_OK;
  cpr_free(h);
  W.fp32 = fp32;
  if (cudaMalloc((void**)&W.col0, sizeof(double) * (size_t)h.nnzb * 8) != cudaSuccess) return ISC_ERR_NOMEM;
  if (cudaMalloc((void**)&W.r1, sizeof(double) * (size_t)h.n * 8) != cudaSuccess) return ISC_ERR_NOMEM;
  W.bytes = sizeof(double) * ((size_t)h.nnzb * 8 + (size_t)h.n * 8);
  return fp32 ? setup_levels_t<float>(h) : setup_levels_t<double>(h);
}

void launch_cpr_setup(Handle& h, cudaStream_t s) {
  if (h.cpr.fp32)
    setup_t<float>(h, s);
  else
    setup_t<double>(h, s);
}

// first stage and the second stage's right-hand side: p (level 0's x) and r1 = r - A E p
void launch_cpr_pressure(Handle& h, const double* r, cudaStream_t s) {
  if (h.cpr.fp32)
    pressure_t<float, double>(h, r, h.cpr.r1, s);
  else
    pressure_t<double, double>(h, r, h.cpr.r1, s);
}

// z += E p after the second stage wrote z = ILU^-1 r1
void launch_cpr_finish(Handle& h, double* z, cudaStream_t s) {
  const int tb = 128;
  if (h.cpr.fp32)
    k_cpr_add<float, double><<<nblk(h.n, tb), tb, 0, s>>>(h.n, h.cpr.h32[0].x, z);
  else
    k_cpr_add<double, double><<<nblk(h.n, tb), tb, 0, s>>>(h.n, h.cpr.h64[0].x, z);
}

// the same on FP32 vectors (inner solve of ISC_PRECISION_MIXED_FGMRES; FP32 multigrid)
void launch_cpr_pressure32(Handle& h, const float* r, float* r1, cudaStream_t s) {
  pressure_t<float, float>(h, r, r1, s);
}
void launch_cpr_finish32(Handle& h, float* z, cudaStream_t s) {
  const int tb = 128;
  k_cpr_add<float, float><<<nblk(h.n, tb), tb, 0, s>>>(h.n, h.cpr.h32[0].x, z);
}

int cpr_pressure_launches(const Handle& h) { return 1 + 6 * h.cpr.ngrid + 1 + 1; }

void cpr_free(Handle& h) {
  CprWork& W = h.cpr;
  if (W.pool) cudaFree(W.pool);
  if (W.d_levels) cudaFree(W.d_levels);
  if (W.col0) cudaFree(W.col0);
  if (W.r1) cudaFree(W.r1);
  W = CprWork{};
}

}  // namespace isc
