// Geometric multigrid V-cycle on the low-order refined matrix of a structured mesh.
//
// The paper solves A_LOR with a structured geometric multigrid V-cycle (Sec. 5.2).  On a
// structured N^3 mesh of Q_p elements the LOR DoFs form a logical (pN+1)^3 grid, numbered
// lexicographically, and A_LOR couples each node with its 26 logical neighbours.  The grid is
// coarsened vertex-centred (every other node) while every dimension is odd and >= 5.
// Interpolation P is trilinear in the logical indices; its rows at Dirichlet fine nodes and
// its columns at Dirichlet coarse nodes are zero.  Coarse operators are Galerkin products
// P^T A P, stored as 27-point stencils ([27][n], neighbour k = (dz+1) 9 + (dy+1) 3 + (dx+1)),
// with identity rows at Dirichlet coarse nodes; the fine LOR matrix is copied into the same
// structure-of-arrays form, so every smoother pass reads coalesced.  Smoothing: Chebyshev-Jacobi polynomials
// (the paper uses ordered ILU, a sequential method); the same polynomial before and after the
// coarse correction keeps the cycle a symmetric linear operator, as CG needs.
#include <cuda_runtime.h>

#include "hx_internal.h"

namespace {

constexpr int kT = 256;

unsigned grid_of(long long n) {
  long long b = (n + kT - 1) / kT;
  const long long cap = 148LL * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

#define MG_STRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// grids hold fewer than 2^31 nodes (the element vectors are int32-indexed): 32-bit index math
__device__ __forceinline__ void coords(const HxGrid& g, long long i, int& x, int& y, int& z) {
  const unsigned u = (unsigned)i, mx = (unsigned)g.mx, my = (unsigned)g.my;
  const unsigned r = u / mx;
  x = (int)(u - r * mx);
  z = (int)(r / my);
  y = (int)(r - (unsigned)z * my);
}

__device__ __forceinline__ bool inside(const HxGrid& g, int x, int y, int z) {
  return x >= 0 && y >= 0 && z >= 0 && x < g.mx && y < g.my && z < g.mz;
}

__device__ __forceinline__ long long index(const HxGrid& g, int x, int y, int z) {
  return (long long)x + (long long)g.mx * ((long long)y + (long long)g.my * z);
}

// The assembled LOR matrix in CSR (read once per assembly, into the fine stencil).
struct CsrRows {
  const long long* off;
  const int* col;
  const double* val;
  __device__ __forceinline__ double dot(long long i, const double* __restrict__ x) const {
    double s = 0.0;
    for (long long o = off[i]; o < off[i + 1]; ++o) s += __ldg(val + o) * __ldg(x + __ldg(col + o));
    return s;
  }
  template <typename F>
  __device__ __forceinline__ void each(long long i, F&& f) const {
    for (long long o = off[i]; o < off[i + 1]; ++o) f((long long)col[o], val[o]);
  }
};

// Every level: 27-point stencils on the logical grid.
struct StencilRows {
  HxGrid g;
  const double* val;  // [27][n]
  __device__ __forceinline__ double dot(long long i, const double* __restrict__ x) const {
    int ix, iy, iz;
    coords(g, i, ix, iy, iz);
    const long long sy = g.mx, sz = (long long)g.mx * g.my;
    double s = 0.0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      if (iz + dz < 0 || iz + dz >= g.mz) continue;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        if (iy + dy < 0 || iy + dy >= g.my) continue;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          if (ix + dx < 0 || ix + dx >= g.mx) continue;
          const int k = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
          s += __ldg(val + (long long)k * g.n + i) * __ldg(x + i + dx + dy * sy + dz * sz);
        }
      }
    }
    return s;
  }
  template <typename F>
  __device__ __forceinline__ void each(long long i, F&& f) const {
    int ix, iy, iz;
    coords(g, i, ix, iy, iz);
    for (int k = 0; k < 27; ++k) {
      const int jx = ix + k % 3 - 1, jy = iy + (k / 3) % 3 - 1, jz = iz + k / 9 - 1;
      if (inside(g, jx, jy, jz)) f(index(g, jx, jy, jz), val[(long long)k * g.n + i]);
    }
  }
};

// ---- Chebyshev-Jacobi on one level (the recurrence of hx_lor.cu, accumulating into x) ----
__global__ void __launch_bounds__(kT) mg_cheb_first_kernel(long long n, const double* __restrict__ dinv,
                                                           const double* __restrict__ b, double* __restrict__ res,
                                                           double* __restrict__ d, double* __restrict__ x,
                                                           const double* __restrict__ coef, int accumulate,
                                                           const int* done) {
  if (done && *(volatile const int*)done) return;
  const double c0 = coef[0];
  MG_STRIDE(i, n) {
    const double s = dinv[i] * b[i];
    res[i] = s;
    d[i] = c0 * s;
    x[i] = accumulate ? x[i] + c0 * s : c0 * s;
  }
}

template <typename Rows>
__global__ void __launch_bounds__(kT) mg_cheb_step_kernel(Rows A, long long n, const double* __restrict__ dinv,
                                                          const double* __restrict__ din, double* __restrict__ dout,
                                                          double* __restrict__ res, double* __restrict__ x,
                                                          const double* __restrict__ coef, int j, const int* done) {
  if (done && *(volatile const int*)done) return;
  const double c1 = coef[2 * j], c2 = coef[2 * j + 1];
  MG_STRIDE(i, n) {
    const double rs = res[i] - dinv[i] * A.dot(i, din);
    res[i] = rs;
    const double dn = c1 * din[i] + c2 * rs;
    dout[i] = dn;
    x[i] += dn;
  }
}

template <typename Rows>
__global__ void __launch_bounds__(kT) mg_residual_kernel(Rows A, long long n, const double* __restrict__ b,
                                                         const double* __restrict__ x, double* __restrict__ r,
                                                         const int* done) {
  if (done && *(volatile const int*)done) return;
  MG_STRIDE(i, n) { r[i] = b[i] - A.dot(i, x); }
}

// b_c = P^T r_f
__global__ void __launch_bounds__(kT) mg_restrict_kernel(HxGrid fg, const unsigned char* __restrict__ fdir,
                                                         const double* __restrict__ rf, HxGrid cg,
                                                         const unsigned char* __restrict__ cdir,
                                                         double* __restrict__ bc, const int* done) {
  if (done && *(volatile const int*)done) return;
  MG_STRIDE(I, cg.n) {
    double s = 0.0;
    if (!cdir[I]) {
      int X, Y, Z;
      coords(cg, I, X, Y, Z);
      for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        const int ix = 2 * X + dx, iy = 2 * Y + dy, iz = 2 * Z + dz;
        if (!inside(fg, ix, iy, iz)) continue;
        const long long i = index(fg, ix, iy, iz);
        if (fdir[i]) continue;
        const double w = (dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0);
        s += w * rf[i];
      }
    }
    bc[I] = s;
  }
}

// x_f += P x_c
__global__ void __launch_bounds__(kT) mg_prolong_kernel(HxGrid cg, const unsigned char* __restrict__ cdir,
                                                        const double* __restrict__ xc, HxGrid fg,
                                                        const unsigned char* __restrict__ fdir,
                                                        double* __restrict__ xf, const int* done) {
  if (done && *(volatile const int*)done) return;
  MG_STRIDE(i, fg.n) {
    if (fdir[i]) continue;
    int ix, iy, iz;
    coords(fg, i, ix, iy, iz);
    double s = 0.0;
    for (int oz = 0; oz < 2; ++oz) {
      if ((iz & 1) == 0 && oz) break;
      const int Z = (iz & 1) ? (iz - 1) / 2 + oz : iz / 2;
      const double wz = (iz & 1) ? 0.5 : 1.0;
      for (int oy = 0; oy < 2; ++oy) {
        if ((iy & 1) == 0 && oy) break;
        const int Y = (iy & 1) ? (iy - 1) / 2 + oy : iy / 2;
        const double wy = (iy & 1) ? 0.5 : 1.0;
        for (int ox = 0; ox < 2; ++ox) {
          if ((ix & 1) == 0 && ox) break;
          const int X = (ix & 1) ? (ix - 1) / 2 + ox : ix / 2;
          const double wx = (ix & 1) ? 0.5 : 1.0;
          const long long J = index(cg, X, Y, Z);
          if (!cdir[J]) s += wx * wy * wz * xc[J];
        }
      }
    }
    xf[i] += s;
  }
}

__global__ void __launch_bounds__(kT) mg_coarse_dir_kernel(HxGrid fg, const unsigned char* __restrict__ fdir, HxGrid cg,
                                                           unsigned char* __restrict__ cdir) {
  MG_STRIDE(I, cg.n) {
    int X, Y, Z;
    coords(cg, I, X, Y, Z);
    cdir[I] = fdir[index(fg, 2 * X, 2 * Y, 2 * Z)];
  }
}

// A_c = P^T A_f P, row by row of the coarse grid (no atomics: fixed order).
template <typename Rows>
__global__ void __launch_bounds__(kT) mg_galerkin_kernel(Rows A, HxGrid fg, const unsigned char* __restrict__ fdir,
                                                         HxGrid cg, const unsigned char* __restrict__ cdir,
                                                         double* __restrict__ vc) {
  MG_STRIDE(I, cg.n) {
    double acc[27];
    for (int k = 0; k < 27; ++k) acc[k] = 0.0;
    if (cdir[I]) {
      acc[13] = 1.0;
    } else {
      int X, Y, Z;
      coords(cg, I, X, Y, Z);
      for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        const int ix = 2 * X + dx, iy = 2 * Y + dy, iz = 2 * Z + dz;
        if (!inside(fg, ix, iy, iz)) continue;
        const long long i = index(fg, ix, iy, iz);
        if (fdir[i]) continue;
        const double wi = (dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0);
        A.each(i, [&](long long j, double a) {
          if (fdir[j]) return;
          int jx, jy, jz;
          coords(fg, j, jx, jy, jz);
          for (int oz = 0; oz < 2; ++oz) {
            if ((jz & 1) == 0 && oz) break;
            const int JZ = (jz & 1) ? (jz - 1) / 2 + oz : jz / 2;
            for (int oy = 0; oy < 2; ++oy) {
              if ((jy & 1) == 0 && oy) break;
              const int JY = (jy & 1) ? (jy - 1) / 2 + oy : jy / 2;
              for (int ox = 0; ox < 2; ++ox) {
                if ((jx & 1) == 0 && ox) break;
                const int JX = (jx & 1) ? (jx - 1) / 2 + ox : jx / 2;
                const int DX = JX - X, DY = JY - Y, DZ = JZ - Z;
                if (DX < -1 || DX > 1 || DY < -1 || DY > 1 || DZ < -1 || DZ > 1) continue;
                if (cdir[index(cg, JX, JY, JZ)]) continue;
                const double wj = ((jx & 1) ? 0.5 : 1.0) * ((jy & 1) ? 0.5 : 1.0) * ((jz & 1) ? 0.5 : 1.0);
                acc[(DZ + 1) * 9 + (DY + 1) * 3 + (DX + 1)] += wi * a * wj;
              }
            }
          }
        });
      }
    }
    for (int k = 0; k < 27; ++k) vc[(long long)k * cg.n + I] = acc[k];
  }
}

// The fine LOR matrix (CSR, rows of the logical grid) as a 27-point stencil [27][n]: the
// structure-of-arrays form the smoothers read with coalesced loads.
__global__ void __launch_bounds__(kT) mg_csr_to_stencil_kernel(CsrRows A, HxGrid g, double* __restrict__ v27) {
  MG_STRIDE(i, g.n) {
    for (int k = 0; k < 27; ++k) v27[(long long)k * g.n + i] = 0.0;
    int ix, iy, iz;
    coords(g, i, ix, iy, iz);
    A.each(i, [&](long long j, double a) {
      int jx, jy, jz;
      coords(g, j, jx, jy, jz);
      const int dx = jx - ix, dy = jy - iy, dz = jz - iz;
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1)
        v27[(long long)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)) * g.n + i] = a;
    });
  }
}

// dinv and the Gershgorin bound of D^-1 A of a stencil level
__global__ void __launch_bounds__(kT) mg_diag_kernel(StencilRows A, double* __restrict__ dinv,
                                                     unsigned long long* bound) {
  double mx = 0.0;
  MG_STRIDE(i, A.g.n) {
    double s = 0.0;
    A.each(i, [&](long long, double a) { s += fabs(a); });
    const double d = A.val[13 * A.g.n + i];
    dinv[i] = 1.0 / d;
    mx = fmax(mx, s / d);
  }
  for (int w = 16; w > 0; w >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, w));
  if ((threadIdx.x & 31) == 0) atomicMax(bound, (unsigned long long)__double_as_longlong(mx));
}

// Chebyshev coefficients on [b / ratio, b] (the recurrence of hx_lor.cu)
__global__ void mg_coef_kernel(const unsigned long long* bound, int k, double ratio, double* coef) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double b = __longlong_as_double((long long)*bound);
  const double a = b / ratio;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
  coef[0] = 1.0 / theta;
  if (k < 2) return;
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int j = 1; j < k; ++j) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    coef[2 * j] = rn * rho;
    coef[2 * j + 1] = 2.0 * rn / delta;
    rho = rn;
  }
}

CsrRows csr_rows(const HxLorMatrix& A) { return CsrRows{A.off, A.col, A.val}; }
StencilRows stencil_rows(const HxMgLevel& L) { return StencilRows{L.g, L.val}; }

// `degree` Chebyshev steps for A x = b on level L (x overwritten, or accumulated into)
template <typename Rows>
cudaError_t smooth(const Rows& A, const HxMgLevel& L, const double* dinv, const double* b, double* x, int degree,
                   const double* coef, int accumulate, const int* done, cudaStream_t s) {
  const unsigned g = grid_of(L.g.n);
  mg_cheb_first_kernel<<<g, kT, 0, s>>>(L.g.n, dinv, b, L.res, L.d0, x, coef, accumulate, done);
  cudaError_t e = cudaGetLastError();
  double* din = L.d0;
  double* dout = L.d1;
  for (int j = 1; j < degree && e == cudaSuccess; ++j) {
    mg_cheb_step_kernel<Rows><<<g, kT, 0, s>>>(A, L.g.n, dinv, din, dout, L.res, x, coef, j, done);
    e = cudaGetLastError();
    double* t = din;
    din = dout;
    dout = t;
  }
  return e;
}

template <typename Rows>
cudaError_t level_cycle(const HxMg& M, int l, const Rows& A, const double* dinv, const double* b, double* x,
                        const int* done, cudaStream_t s);

cudaError_t cycle_from(const HxMg& M, int l, const double* b, double* x, const int* done, cudaStream_t s) {
  return level_cycle(M, l, stencil_rows(M.levels[l]), M.levels[l].dinv, b, x, done, s);
}

template <typename Rows>
cudaError_t level_cycle(const HxMg& M, int l, const Rows& A, const double* dinv, const double* b, double* x,
                        const int* done, cudaStream_t s) {
  const HxMgLevel& L = M.levels[l];
  if (l == M.n_levels - 1) return smooth(A, L, dinv, b, x, M.coarse_degree, L.coef, 0, done, s);
  const HxMgLevel& C = M.levels[l + 1];
  const unsigned g = grid_of(L.g.n);
  cudaError_t e = smooth(A, L, dinv, b, x, M.smooth_degree, L.coef, 0, done, s);
  if (e != cudaSuccess) return e;
  mg_residual_kernel<Rows><<<g, kT, 0, s>>>(A, L.g.n, b, x, L.r, done);
  mg_restrict_kernel<<<grid_of(C.g.n), kT, 0, s>>>(L.g, L.dir, L.r, C.g, C.dir, C.b, done);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cycle_from(M, l + 1, C.b, C.x, done, s)) != cudaSuccess) return e;
  mg_prolong_kernel<<<g, kT, 0, s>>>(C.g, C.dir, C.x, L.g, L.dir, x, done);
  mg_residual_kernel<Rows><<<g, kT, 0, s>>>(A, L.g.n, b, x, L.r, done);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return smooth(A, L, dinv, L.r, x, M.smooth_degree, L.coef, 1, done, s);
}

}  // namespace

cudaError_t hx_mg_coarse_dir(const HxMgLevel& F, HxMgLevel& C, cudaStream_t s) {
  mg_coarse_dir_kernel<<<grid_of(C.g.n), kT, 0, s>>>(F.g, F.dir, C.g, C.dir_own);
  return cudaGetLastError();
}

// Galerkin operators, inverse diagonals, bounds and Chebyshev coefficients of every level
// (the fine level's matrix, inverse diagonal and bound come from the LOR assembly).
cudaError_t hx_mg_assemble(const HxMg& M, const HxLorMatrix& A0, const unsigned long long* bound0, cudaStream_t s) {
  // the fine level as a stencil (every LOR row couples only logical neighbours)
  mg_csr_to_stencil_kernel<<<grid_of(M.levels[0].g.n), kT, 0, s>>>(csr_rows(A0), M.levels[0].g, M.levels[0].val);
  cudaError_t e = cudaGetLastError();
  for (int l = 1; l < M.n_levels && e == cudaSuccess; ++l) {
    const HxMgLevel& F = M.levels[l - 1];
    const HxMgLevel& C = M.levels[l];
    const unsigned g = grid_of(C.g.n);
    mg_galerkin_kernel<StencilRows><<<g, kT, 0, s>>>(stencil_rows(F), F.g, F.dir, C.g, C.dir, C.val);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(C.bound, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      mg_diag_kernel<<<g, kT, 0, s>>>(stencil_rows(C), C.dinv, C.bound);
      e = cudaGetLastError();
    }
  }
  for (int l = 0; l < M.n_levels && e == cudaSuccess; ++l) {
    const HxMgLevel& L = M.levels[l];
    const bool coarsest = l == M.n_levels - 1;
    const int k = coarsest ? M.coarse_degree : M.smooth_degree;
    const double ratio = coarsest ? (double)k * k : M.smooth_ratio;
    mg_coef_kernel<<<1, 32, 0, s>>>(l == 0 ? bound0 : L.bound, k, ratio, L.coef);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t hx_mg_vcycle(const HxMg& M, const HxLorMatrix& A0, const double* r, double* z, const int* done,
                         cudaStream_t s) {
  return level_cycle(M, 0, stencil_rows(M.levels[0]), A0.dinv, r, z, done, s);
}

int hx_mg_vcycle_launches(const HxMg& M) {
  int k = 0;
  for (int l = 0; l < M.n_levels - 1; ++l) k += 2 * M.smooth_degree + 4;
  return k + M.coarse_degree;
}
