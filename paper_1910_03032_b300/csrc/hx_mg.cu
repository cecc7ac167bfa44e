// Geometric multigrid V-cycle on the low-order refined matrix of a structured mesh.
//
// The paper solves A_LOR with a structured geometric multigrid V-cycle (Sec. 5.2).  On a
// structured N^3 mesh of Q_p elements the LOR DoFs form a logical (pN+1)^3 grid, numbered
// lexicographically, and A_LOR couples each node with its 26 logical neighbours.  The grid is
// coarsened vertex-centred (every other node) while every dimension is odd and >= 5.
// Interpolation P is trilinear in the logical indices; its rows at Dirichlet fine nodes and
// its columns at Dirichlet coarse nodes are zero.  Coarse operators are Galerkin products
// P^T A P, stored as 27-point stencils ([27][n], neighbour k = (dz+1) 9 + (dy+1) 3 + (dx+1)),
// with identity rows at Dirichlet coarse nodes; the fine LOR matrix is assembled straight into
// the same structure-of-arrays form, so every smoother pass reads coalesced.  Smoothing: Chebyshev-Jacobi polynomials
// (the paper uses ordered ILU, a sequential method); the same polynomial before and after the
// coarse correction keeps the cycle a symmetric linear operator, as CG needs.
#include <cuda_runtime.h>

#include "hx_element.cuh"
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

// Every level: 27-point stencils on the logical grid (FP64; FP32 copies for the inner solver of
// mixed-precision solves).
template <typename Real>
struct StencilRowsT {
  HxGrid g;
  const Real* val;  // [27][n]
  // Row i times x.  FP64 rows are bound by the FP64 pipe (27 multiply-adds per 240 B); FP32 rows
  // by memory latency, so each z-plane's 9 stencil values (always in bounds: [27][n]) and 9
  // neighbours (an out-of-grid neighbour reads x[i] instead) are loaded before any is used and
  // the out-of-grid terms skipped afterwards, in the same order.
  __device__ __forceinline__ Real dot(long long i, const Real* __restrict__ x) const {
    int ix, iy, iz;
    coords(g, i, ix, iy, iz);
    const long long sy = g.mx, sz = (long long)g.mx * g.my;
    Real s = Real(0);
    if constexpr (sizeof(Real) == 4) {
      const bool okx[3] = {ix > 0, true, ix + 1 < g.mx}, oky[3] = {iy > 0, true, iy + 1 < g.my};
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        const bool okz = iz + dz >= 0 && iz + dz < g.mz;
        Real v[9], xv[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
          const int dx = a % 3 - 1, dy = a / 3 - 1;
          const bool ok = okz && oky[dy + 1] && okx[dx + 1];
          v[a] = __ldg(val + (long long)((dz + 1) * 9 + a) * g.n + i);
          xv[a] = __ldg(x + (ok ? i + dx + dy * sy + dz * sz : i));
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
          const int dx = a % 3 - 1, dy = a / 3 - 1;
          if (okz && oky[dy + 1] && okx[dx + 1]) s += v[a] * xv[a];
        }
      }
      return s;
    }
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
typedef StencilRowsT<double> StencilRows;

// ---- Chebyshev-Jacobi on one level (the recurrence of hx_lor.cu, accumulating into x) ----
template <typename Real>
__global__ void __launch_bounds__(kT) mg_cheb_first_kernel(long long n, const Real* __restrict__ dinv,
                                                           const Real* __restrict__ b, Real* __restrict__ res,
                                                           Real* __restrict__ d, Real* __restrict__ x,
                                                           const double* __restrict__ coef, int accumulate,
                                                           int more, const int* done) {
  if (done && *(volatile const int*)done) return;
  const Real c0 = Real(coef[0]);
  MG_STRIDE(i, n) {
    const Real s = dinv[i] * b[i];
    if (more) {  // the recurrence continues: keep its residual and direction
      res[i] = s;
      d[i] = c0 * s;
    }
    x[i] = accumulate ? x[i] + c0 * s : c0 * s;
  }
}

template <typename Real, typename Rows>
__global__ void __launch_bounds__(kT) mg_cheb_step_kernel(Rows A, long long n, const Real* __restrict__ dinv,
                                                          const Real* __restrict__ din, Real* __restrict__ dout,
                                                          Real* __restrict__ res, Real* __restrict__ x,
                                                          const double* __restrict__ coef, int j, const int* done) {
  if (done && *(volatile const int*)done) return;
  const Real c1 = Real(coef[2 * j]), c2 = Real(coef[2 * j + 1]);
  MG_STRIDE(i, n) {
    const Real rs = res[i] - dinv[i] * A.dot(i, din);
    res[i] = rs;
    const Real dn = c1 * din[i] + c2 * rs;
    dout[i] = dn;
    x[i] += dn;
  }
}

template <typename Real, typename Rows>
__global__ void __launch_bounds__(kT) mg_residual_kernel(Rows A, long long n, const Real* __restrict__ b,
                                                         const Real* __restrict__ x, Real* __restrict__ r,
                                                         const int* done) {
  if (done && *(volatile const int*)done) return;
  MG_STRIDE(i, n) { r[i] = b[i] - A.dot(i, x); }
}

// b_c = P^T r_f
// The transfer weights are powers of 1/2, exact in either precision: the restriction's are
// compile-time constants of the unrolled 27-point loop, and every term of a prolongation shares
// one weight (1/2 per odd coordinate of the fine node), applied once to the sum of the coarse
// values (scaling by a power of 2 is exact, so the sum is the same as term by term).
template <typename Real>
__global__ void __launch_bounds__(kT) mg_restrict_kernel(HxGrid fg, const unsigned char* __restrict__ fdir,
                                                         const Real* __restrict__ rf, HxGrid cg,
                                                         const unsigned char* __restrict__ cdir,
                                                         Real* __restrict__ bc, const int* done) {
  if (done && *(volatile const int*)done) return;
  const long long sy = fg.mx, sz = (long long)fg.mx * fg.my;
  MG_STRIDE(I, cg.n) {
    Real s = Real(0);
    if (!cdir[I]) {
      int X, Y, Z;
      coords(cg, I, X, Y, Z);
      const int cx = 2 * X, cy = 2 * Y, cz = 2 * Z;
      const long long c = index(fg, cx, cy, cz);
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        if (cz + dz < 0 || cz + dz >= fg.mz) continue;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          if (cy + dy < 0 || cy + dy >= fg.my) continue;
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            if (cx + dx < 0 || cx + dx >= fg.mx) continue;
            const long long i = c + dx + dy * sy + dz * sz;
            if (fdir[i]) continue;
            const Real w = Real(1) / Real(1 << ((dx != 0) + (dy != 0) + (dz != 0)));
            s += w * rf[i];
          }
        }
      }
    }
    bc[I] = s;
  }
}

// x_f += P x_c
template <typename Real>
__global__ void __launch_bounds__(kT) mg_prolong_kernel(HxGrid cg, const unsigned char* __restrict__ cdir,
                                                        const Real* __restrict__ xc, HxGrid fg,
                                                        const unsigned char* __restrict__ fdir,
                                                        Real* __restrict__ xf, const int* done) {
  if (done && *(volatile const int*)done) return;
  const long long sy = cg.mx, sz = (long long)cg.mx * cg.my;
  MG_STRIDE(i, fg.n) {
    if (fdir[i]) continue;
    int ix, iy, iz;
    coords(fg, i, ix, iy, iz);
    // coarse neighbours: (i/2) and, along an odd coordinate, (i/2) + 1 as well
    const int ox = ix & 1, oy = iy & 1, oz = iz & 1;
    const long long J0 = index(cg, ix >> 1, iy >> 1, iz >> 1);
    Real s = Real(0);
    for (int bz = 0; bz <= oz; ++bz)
      for (int by = 0; by <= oy; ++by)
        for (int bx = 0; bx <= ox; ++bx) {
          const long long J = J0 + bx + by * sy + bz * sz;
          if (!cdir[J]) s += xc[J];
        }
    const int k = ox + oy + oz;
    xf[i] += s * (k == 0 ? Real(1) : k == 1 ? Real(0.5) : k == 2 ? Real(0.25) : Real(0.125));
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

// The fine LOR stencil of a structured mesh, cell by cell.  A cell (cx, cy, cz) of the logical
// grid is sub-element (cx mod p, cy mod p, cz mod p) of element (cx / p, cy / p, cz / p); its Q1
// matrix (2 Gauss points per direction, the sub-element's Jacobian J_K(xi(eta)) diag(h) / 2) is
// computed once and added into the stencil rows of its 8 corners.  Cells of one parity class
// (ox, oy, oz) share no node, so each of the 8 passes adds without atomics, in a fixed order.
__global__ void __launch_bounds__(kT) mg_cell_kernel(const __grid_constant__ HxTables T, HxGrid g, int nx, int ny,
                                                     const double* __restrict__ X8,
                                                     const unsigned char* __restrict__ dir, double am, double nu,
                                                     int ox, int oy, int oz, double* __restrict__ v27) {
  const double g2 = 0.57735026918962576451;  // 2-point Gauss nodes +-1/sqrt(3), weights 1
  __shared__ double q1[8][8][4];             // Q1 shape functions and gradients at the 8 points
  if (threadIdx.x < 64) {
    const int qp = threadIdx.x >> 3, c = threadIdx.x & 7;
    double f[3], sg[3];
    for (int d = 0; d < 3; ++d) {
      sg[d] = ((c >> d) & 1) ? 1.0 : -1.0;
      f[d] = 0.5 * (1.0 + sg[d] * (((qp >> d) & 1) ? g2 : -g2));
    }
    q1[qp][c][0] = f[0] * f[1] * f[2];
    q1[qp][c][1] = 0.5 * sg[0] * f[1] * f[2];
    q1[qp][c][2] = 0.5 * sg[1] * f[0] * f[2];
    q1[qp][c][3] = 0.5 * sg[2] * f[0] * f[1];
  }
  __syncthreads();
  const int p = T.p;
  const int hxn = (g.mx - 1 - ox + 1) / 2, hyn = (g.my - 1 - oy + 1) / 2, hzn = (g.mz - 1 - oz + 1) / 2;
  const long long nc = (long long)hxn * hyn * hzn;
  const long long sy = g.mx, sz = (long long)g.mx * g.my;
  MG_STRIDE(t, nc) {
    const int ix = (int)(t % hxn), iy = (int)((t / hxn) % hyn), iz = (int)(t / ((long long)hxn * hyn));
    const int cx = 2 * ix + ox, cy = 2 * iy + oy, cz = 2 * iz + oz;
    const int ex = cx / p, ey = cy / p, ez = cz / p;
    const int s0 = cx - ex * p, t0 = cy - ey * p, u0 = cz - ez * p;
    const long long e = ex + (long long)nx * (ey + (long long)ny * ez);
    double cf[24];
    {
      double x8[24];
      for (int c = 0; c < 24; ++c) x8[c] = X8[e * 24 + c];
      hx::trilinear_coeffs(x8, cf);
    }
    const double hs = T.xn[s0 + 1] - T.xn[s0], ht = T.xn[t0 + 1] - T.xn[t0], hu = T.xn[u0 + 1] - T.xn[u0];
    double a[36];  // upper triangle of the symmetric 8 x 8 cell matrix (constant indices: registers)
#pragma unroll
    for (int k = 0; k < 36; ++k) a[k] = 0.0;
    for (int qp = 0; qp < 8; ++qp) {
      double j0[3], j1[3], j2[3], f[7];
      hx::trilinear_jacobian(cf, T.xn[s0] + 0.5 * (((qp & 1) ? g2 : -g2) + 1.0) * hs,
                             T.xn[t0] + 0.5 * (((qp & 2) ? g2 : -g2) + 1.0) * ht,
                             T.xn[u0] + 0.5 * (((qp & 4) ? g2 : -g2) + 1.0) * hu, j0, j1, j2);
      for (int d = 0; d < 3; ++d) {
        j0[d] *= 0.5 * hs;
        j1[d] *= 0.5 * ht;
        j2[d] *= 0.5 * hu;
      }
      hx::point_factors(j0, j1, j2, am, nu, f);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const double mc = f[0] * q1[qp][c][0];
        const double gx = q1[qp][c][1], gy = q1[qp][c][2], gz = q1[qp][c][3];
        const double G0 = f[1] * gx + f[2] * gy + f[3] * gz;
        const double G1 = f[2] * gx + f[4] * gy + f[5] * gz;
        const double G2 = f[3] * gx + f[5] * gy + f[6] * gz;
#pragma unroll
        for (int c2 = c; c2 < 8; ++c2)
          a[c * 8 - c * (c - 1) / 2 + (c2 - c)] +=
              mc * q1[qp][c2][0] + G0 * q1[qp][c2][1] + G1 * q1[qp][c2][2] + G2 * q1[qp][c2][3];
      }
    }
    const long long base = cx + sy * cy + sz * cz;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int dxc = c & 1, dyc = (c >> 1) & 1, dzc = (c >> 2) & 1;
      const long long i = base + dxc + sy * dyc + sz * dzc;
      if (dir[i]) continue;
#pragma unroll
      for (int c2 = 0; c2 < 8; ++c2) {
        const int dx = (c2 & 1) - dxc, dy = ((c2 >> 1) & 1) - dyc, dz = ((c2 >> 2) & 1) - dzc;
        const long long j = i + dx + sy * dy + sz * dz;
        if (dir[j]) continue;
        const int lo = c < c2 ? c : c2, hi = c < c2 ? c2 : c;
        const int k = lo * 8 - lo * (lo - 1) / 2 + (hi - lo);  // position of (lo, hi) in the upper triangle
        v27[(long long)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)) * g.n + i] += a[k];
      }
    }
  }
}

// Identity rows at Dirichlet nodes; the collocated mass (alpha Mc) added to the centre elsewhere.
__global__ void __launch_bounds__(kT) mg_fine_finish_kernel(HxGrid g, const unsigned char* __restrict__ dir,
                                                            const double* __restrict__ mc, double* __restrict__ v27) {
  MG_STRIDE(i, g.n) {
    if (dir[i]) {
      for (int k = 0; k < 27; ++k) v27[(long long)k * g.n + i] = (k == 13) ? 1.0 : 0.0;
    } else if (mc) {
      v27[13 * g.n + i] += mc[i];
    }
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

StencilRows stencil_rows(const HxMgLevel& L) { return StencilRows{L.g, L.val}; }

// What one V-cycle level works with, in the cycle's precision.
template <typename Real>
struct LevelView {
  HxGrid g;
  const unsigned char* dir;
  const Real* val;
  const Real* dinv;
  Real *b, *x, *r, *res, *d0, *d1;
  const double* coef;
};
LevelView<double> view(const HxMgLevel& L, double) {
  return LevelView<double>{L.g, L.dir, L.val, L.dinv, L.b, L.x, L.r, L.res, L.d0, L.d1, L.coef};
}
LevelView<float> view(const HxMgLevel& L, float) {
  return LevelView<float>{L.g, L.dir, L.val32, L.dinv32, L.b32, L.x32, L.r32, L.res32, L.d032, L.d132, L.coef};
}

// `degree` Chebyshev steps for A x = b on level L (x overwritten, or accumulated into)
template <typename Real>
cudaError_t smooth(const LevelView<Real>& L, const Real* b, Real* x, int degree, int accumulate, const int* done,
                   cudaStream_t s) {
  const StencilRowsT<Real> A{L.g, L.val};
  const unsigned g = grid_of(L.g.n);
  mg_cheb_first_kernel<Real><<<g, kT, 0, s>>>(L.g.n, L.dinv, b, L.res, L.d0, x, L.coef, accumulate, degree > 1,
                                              done);
  cudaError_t e = cudaGetLastError();
  Real* din = L.d0;
  Real* dout = L.d1;
  for (int j = 1; j < degree && e == cudaSuccess; ++j) {
    mg_cheb_step_kernel<Real, StencilRowsT<Real>><<<g, kT, 0, s>>>(A, L.g.n, L.dinv, din, dout, L.res, x, L.coef, j,
                                                                   done);
    e = cudaGetLastError();
    Real* t = din;
    din = dout;
    dout = t;
  }
  return e;
}

template <typename Real>
cudaError_t level_cycle(const HxMg& M, const LevelView<Real>* V, int l, const Real* b, Real* x, const int* done,
                        cudaStream_t s) {
  const LevelView<Real>& L = V[l];
  if (l == M.n_levels - 1) return smooth(L, b, x, M.coarse_degree, 0, done, s);
  const LevelView<Real>& C = V[l + 1];
  const StencilRowsT<Real> A{L.g, L.val};
  const unsigned g = grid_of(L.g.n);
  cudaError_t e = smooth(L, b, x, M.smooth_degree, 0, done, s);
  if (e != cudaSuccess) return e;
  mg_residual_kernel<Real, StencilRowsT<Real>><<<g, kT, 0, s>>>(A, L.g.n, b, x, L.r, done);
  mg_restrict_kernel<Real><<<grid_of(C.g.n), kT, 0, s>>>(L.g, L.dir, L.r, C.g, C.dir, C.b, done);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = level_cycle(M, V, l + 1, C.b, C.x, done, s)) != cudaSuccess) return e;
  mg_prolong_kernel<Real><<<g, kT, 0, s>>>(C.g, C.dir, C.x, L.g, L.dir, x, done);
  mg_residual_kernel<Real, StencilRowsT<Real>><<<g, kT, 0, s>>>(A, L.g.n, b, x, L.r, done);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return smooth(L, L.r, x, M.smooth_degree, 1, done, s);
}

template <typename Real>
cudaError_t vcycle(const HxMg& M, const Real* r, Real* z, const int* done, cudaStream_t s) {
  LevelView<Real> V[HX_MG_MAX_LEVELS];
  for (int l = 0; l < M.n_levels; ++l) V[l] = view(M.levels[l], Real(0));
  return level_cycle(M, V, 0, r, z, done, s);
}

}  // namespace

cudaError_t hx_mg_coarse_dir(const HxMgLevel& F, HxMgLevel& C, cudaStream_t s) {
  mg_coarse_dir_kernel<<<grid_of(C.g.n), kT, 0, s>>>(F.g, F.dir, C.g, C.dir_own);
  return cudaGetLastError();
}

// Galerkin operators, inverse diagonals, bounds and Chebyshev coefficients of every level
// (the fine level's matrix, inverse diagonal and bound come from the LOR assembly).
cudaError_t hx_mg_fine(const HxTables& T, int nx, int ny, const double* X8, double alpha, double nu, int collocated,
                       const double* mc, const HxMgLevel& L0, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(L0.val, 0, sizeof(double) * 27 * (size_t)L0.g.n, s);
  const double am = collocated ? 0.0 : alpha;  // the Q1 mass enters only in the consistent form
  const long long cells = (long long)(L0.g.mx - 1) * (L0.g.my - 1) * (L0.g.mz - 1);
  for (int c = 0; c < 8 && e == cudaSuccess; ++c) {
    mg_cell_kernel<<<grid_of(cells / 8 + 1), kT, 0, s>>>(T, L0.g, nx, ny, X8, L0.dir, am, nu, c & 1, (c >> 1) & 1,
                                                         (c >> 2) & 1, L0.val);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    mg_fine_finish_kernel<<<grid_of(L0.g.n), kT, 0, s>>>(L0.g, L0.dir, collocated ? mc : nullptr, L0.val);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t hx_mg_assemble(const HxMg& M, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(M.levels[0].bound, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    mg_diag_kernel<<<grid_of(M.levels[0].g.n), kT, 0, s>>>(stencil_rows(M.levels[0]), M.levels[0].dinv,
                                                           M.levels[0].bound);
    e = cudaGetLastError();
  }
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
    mg_coef_kernel<<<1, 32, 0, s>>>(L.bound, k, ratio, L.coef);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t hx_mg_vcycle(const HxMg& M, const double* r, double* z, const int* done, cudaStream_t s) {
  return vcycle<double>(M, r, z, done, s);
}

cudaError_t hx_mg_vcycle32(const HxMg& M, const float* r, float* z, const int* done, cudaStream_t s) {
  return vcycle<float>(M, r, z, done, s);
}

// FP32 copies of every level's stencil and inverse diagonal (the inner solver of mixed solves)
cudaError_t hx_mg_to_float(const HxMg& M, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < M.n_levels && e == cudaSuccess; ++l) {
    const HxMgLevel& L = M.levels[l];
    e = hx_launch_to_float(27 * L.g.n, L.val, L.val32, s);
    if (e == cudaSuccess) e = hx_launch_to_float(L.g.n, L.dinv, L.dinv32, s);
  }
  return e;
}

int hx_mg_vcycle_launches(const HxMg& M) {
  int k = 0;
  for (int l = 0; l < M.n_levels - 1; ++l) k += 2 * M.smooth_degree + 4;
  return k + M.coarse_degree;
}
