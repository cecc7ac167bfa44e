// Low-order refined (LOR) operator of Sec. 5.2 and a Chebyshev-Jacobi approximation of its
// inverse, used as the PCG preconditioner HX_PREC_LOR.
//
// A_LOR = alpha M_LOR + nu K_LOR is the Q1 discretization on the mesh that cuts every element
// along the Cartesian product of its Gauss-Lobatto points; the DoFs are those of the high-order
// space.  A sub-element is the image of a box [xn_s, xn_s+1] x [xn_t, xn_t+1] x [xn_u, xn_u+1]
// of the reference cube under the element's trilinear map, so its Jacobian at a point eta of its
// own reference cube is J_K(xi(eta)) diag(h_s, h_t, h_u) / 2 (h the Gauss-Lobatto spacings).
// Each sub-element matrix is integrated with 2 Gauss points per direction.
//
// The matrix is stored in CSR with the Dirichlet rows and columns eliminated (identity rows),
// built row by row without atomics: a row visits the (element, local node) pairs of its DoF
// through the transpose map and the (up to 8) sub-elements around each, in a fixed order, so
// pattern and values are deterministic.  The Chebyshev steps read a sliced-ELL copy (slices of
// 32 rows, column-major), refreshed from the CSR values whenever they change.
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

__device__ __forceinline__ int decode(int r) { return r >= 0 ? r : -r - 1; }

// Calls f(e, s, t, u, c) for every sub-element (s, t, u) of element e that has the local node of
// E-vector position v as its corner c = dx + 2 dy + 4 dz.
template <typename F>
__device__ __forceinline__ void for_sub_elements(int p, int v, F&& f) {
  const int n = p + 1, N3 = n * n * n;
  const int e = v / N3, l = v - e * N3;
  const int i = l % n, j = (l / n) % n, k = l / (n * n);
  for (int dz = 0; dz < 2; ++dz) {
    const int u = k - dz;
    if (u < 0 || u >= p) continue;
    for (int dy = 0; dy < 2; ++dy) {
      const int t = j - dy;
      if (t < 0 || t >= p) continue;
      for (int dx = 0; dx < 2; ++dx) {
        const int s = i - dx;
        if (s < 0 || s >= p) continue;
        f(e, s, t, u, dx + 2 * dy + 4 * dz);
      }
    }
  }
}

// global id of corner c of sub-element (s, t, u) of element e
__device__ __forceinline__ int corner_dof(const int* __restrict__ R, int p, int e, int s, int t, int u, int c) {
  const int n = p + 1;
  const int node = (s + (c & 1)) + n * (t + ((c >> 1) & 1)) + n * n * (u + ((c >> 2) & 1));
  return decode(__ldg(R + (long long)e * n * n * n + node));
}

// The sorted distinct columns of row g (Dirichlet rows: g alone; other rows skip Dirichlet
// columns).  Returns the count, or -1 when more than HX_LOR_MAX_NB.
__device__ int row_columns(int p, long long g, const int* __restrict__ toff, const int* __restrict__ tidx,
                           const int* __restrict__ R, const unsigned char* __restrict__ dir,
                           int (&cols)[HX_LOR_MAX_NB]) {
  if (dir[g]) {
    cols[0] = (int)g;
    return 1;
  }
  int nc = 0;
  bool overflow = false;
  for (int k = toff[g]; k < toff[g + 1]; ++k) {
    for_sub_elements(p, tidx[k], [&](int e, int s, int t, int u, int) {
      for (int c = 0; c < 8; ++c) {
        const int h = corner_dof(R, p, e, s, t, u, c);
        if (dir[h]) continue;
        bool found = false;
        for (int a = 0; a < nc; ++a) found |= (cols[a] == h);
        if (found) continue;
        if (nc == HX_LOR_MAX_NB) {
          overflow = true;
          continue;
        }
        int a = nc - 1;
        while (a >= 0 && cols[a] > h) {
          cols[a + 1] = cols[a];
          --a;
        }
        cols[a + 1] = h;
        ++nc;
      }
    });
  }
  return overflow ? -1 : nc;
}

__global__ void __launch_bounds__(kT) lor_count_kernel(int p, long long n, const int* __restrict__ toff,
                                                       const int* __restrict__ tidx, const int* __restrict__ R,
                                                       const unsigned char* __restrict__ dir,
                                                       long long* __restrict__ count, int* __restrict__ bad) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    int cols[HX_LOR_MAX_NB];
    const int nc = row_columns(p, g, toff, tidx, R, dir, cols);
    if (nc < 0) {
      atomicAdd(bad, 1);
      count[g] = 0;
    } else {
      count[g] = nc;
    }
  }
}

__global__ void __launch_bounds__(kT) lor_fill_kernel(int p, long long n, const int* __restrict__ toff,
                                                      const int* __restrict__ tidx, const int* __restrict__ R,
                                                      const unsigned char* __restrict__ dir,
                                                      const long long* __restrict__ off, int* __restrict__ col) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    int cols[HX_LOR_MAX_NB];
    const int nc = row_columns(p, g, toff, tidx, R, dir, cols);
    const long long o = off[g];
    for (int a = 0; a < nc && o + a < off[g + 1]; ++a) col[o + a] = cols[a];
  }
}

// Row g of A_LOR: for every sub-element around g (corner c), the row c of its Q1 element matrix
//   a_cc' = sum over the 8 points of w detJ (alpha phi_c phi_c' + nu (J^-T grad phi_c) . (J^-T grad phi_c')),
// added into the slots of the columns of the other corners.
__global__ void __launch_bounds__(kT) lor_values_kernel(const __grid_constant__ HxTables T, long long n,
                                                        const int* __restrict__ toff, const int* __restrict__ tidx,
                                                        const int* __restrict__ R, const unsigned char* __restrict__ dir,
                                                        const double* __restrict__ X8, double alpha, double nu,
                                                        int collocated, const long long* __restrict__ off,
                                                        const int* __restrict__ col, double* __restrict__ val) {
  const int p = T.p;
  const double am = collocated ? 0.0 : alpha;  // the Q1 mass enters only in the consistent form
  const double g2 = 0.57735026918962576451;  // 2-point Gauss nodes +-1/sqrt(3), weights 1
  // Q1 shape functions on the sub-element's cube, prod_d (1 + s_d eta_d) / 2, and their
  // gradients, at the 8 points: q1[qp][c] = (phi, dphi/deta_1, dphi/deta_2, dphi/deta_3)
  __shared__ double q1[8][8][4];
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
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    const long long o0 = off[g], o1 = off[g + 1];
    if (dir[g]) {
      for (long long o = o0; o < o1; ++o) val[o] = (col[o] == g) ? 1.0 : 0.0;
      continue;
    }
    for (long long o = o0; o < o1; ++o) val[o] = 0.0;
    for (int k = toff[g]; k < toff[g + 1]; ++k) {
      const int v = tidx[k];
      const int e = v / ((p + 1) * (p + 1) * (p + 1));
      double cf[24];
      {
        double x8[24];
        for (int c = 0; c < 24; ++c) x8[c] = X8[(long long)e * 24 + c];
        hx::trilinear_coeffs(x8, cf);
      }
      for_sub_elements(p, v, [&](int e_, int s, int t, int u, int c) {
        const double hs = T.xn[s + 1] - T.xn[s], ht = T.xn[t + 1] - T.xn[t], hu = T.xn[u + 1] - T.xn[u];
        double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int qp = 0; qp < 8; ++qp) {
          double j0[3], j1[3], j2[3], f[7];
          hx::trilinear_jacobian(cf, T.xn[s] + 0.5 * (((qp & 1) ? g2 : -g2) + 1.0) * hs,
                                 T.xn[t] + 0.5 * (((qp & 2) ? g2 : -g2) + 1.0) * ht,
                                 T.xn[u] + 0.5 * (((qp & 4) ? g2 : -g2) + 1.0) * hu, j0, j1, j2);
          for (int d = 0; d < 3; ++d) {
            j0[d] *= 0.5 * hs;
            j1[d] *= 0.5 * ht;
            j2[d] *= 0.5 * hu;
          }
          hx::point_factors(j0, j1, j2, am, nu, f);
          const double mc = f[0] * q1[qp][c][0];
          const double gx = q1[qp][c][1], gy = q1[qp][c][2], gz = q1[qp][c][3];
          const double G0 = f[1] * gx + f[2] * gy + f[3] * gz;
          const double G1 = f[2] * gx + f[4] * gy + f[5] * gz;
          const double G2 = f[3] * gx + f[5] * gy + f[6] * gz;
#pragma unroll
          for (int c2 = 0; c2 < 8; ++c2)
            a[c2] += mc * q1[qp][c2][0] + G0 * q1[qp][c2][1] + G1 * q1[qp][c2][2] + G2 * q1[qp][c2][3];
        }
        for (int c2 = 0; c2 < 8; ++c2) {
          const int h = corner_dof(R, p, e_, s, t, u, c2);
          if (dir[h]) continue;
          for (long long o = o0; o < o1; ++o)
            if (col[o] == h) {
              val[o] += a[c2];
              break;
            }
        }
      });
      if (collocated) {
        // alpha w_a w_b w_c detJ at the node: this pair's share of the collocated mass (Sec. 5.1)
        const int n = p + 1, l = v - e * n * n * n;
        const int ia = l % n, ib = (l / n) % n, ic = l / (n * n);
        double j0[3], j1[3], j2[3];
        hx::trilinear_jacobian(cf, T.xn[ia], T.xn[ib], T.xn[ic], j0, j1, j2);
        const double det = j0[0] * (j1[1] * j2[2] - j1[2] * j2[1]) + j0[1] * (j1[2] * j2[0] - j1[0] * j2[2]) +
                           j0[2] * (j1[0] * j2[1] - j1[1] * j2[0]);
        const double mc = alpha * T.wn[ia] * T.wn[ib] * T.wn[ic] * det;
        for (long long o = o0; o < o1; ++o)
          if (col[o] == g) {
            val[o] += mc;
            break;
          }
      }
    }
  }
}

// dinv = 1 / diag(A_LOR); bound = max_g sum_c |a_gc| / a_gg (Gershgorin: >= lambda_max(D^-1 A)).
// The bound is kept as the bit pattern of a non-negative double, whose integer order is its order.
__global__ void __launch_bounds__(kT) lor_diag_kernel(long long n, const long long* __restrict__ off,
                                                      const int* __restrict__ col, const double* __restrict__ val,
                                                      double* __restrict__ dinv, unsigned long long* bound) {
  double mx = 0.0;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    double d = 0.0, s = 0.0;
    for (long long o = off[g]; o < off[g + 1]; ++o) {
      s += fabs(val[o]);
      if (col[o] == g) d = val[o];
    }
    dinv[g] = 1.0 / d;
    mx = fmax(mx, s / d);
  }
  for (int w = 16; w > 0; w >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, w));
  if ((threadIdx.x & 31) == 0) atomicMax(bound, (unsigned long long)__double_as_longlong(mx));
}

// Chebyshev coefficients on [b / k^2, b], b the Gershgorin bound (Saad, Iterative Methods for Sparse
// Linear Systems, 2nd ed., Sec. 12.3, Algorithm 12.1): coef[0] = 1 / theta, and for j >= 1
// coef[2j] = rho_j rho_{j-1}, coef[2j+1] = 2 rho_j / delta.
__global__ void lor_coef_kernel(const unsigned long long* bound, int k, double* coef) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double b = __longlong_as_double((long long)*bound);
  const double a = b / (double)(k * k);
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

// res = D^-1 r, d = res / theta, z = d
__global__ void __launch_bounds__(kT) cheb_first_kernel(long long n, const double* __restrict__ dinv,
                                                        const double* __restrict__ r, double* __restrict__ res,
                                                        double* __restrict__ d, double* __restrict__ z,
                                                        const double* __restrict__ coef, const int* done) {
  if (done && *(volatile const int*)done) return;
  const double c0 = coef[0];
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    const double s = dinv[g] * r[g];
    res[g] = s;
    d[g] = c0 * s;
    z[g] = c0 * s;
  }
}

constexpr int kB = 9;  // entries per load batch in the Chebyshev step (27 = 3 batches on a hex mesh)

// res -= D^-1 A d_in, d_out = c1 d_in + c2 res, z += d_out.  One thread per row over the sliced-ELL
// copy; the grid stride is a multiple of 32, so a warp always covers one slice.
__global__ void __launch_bounds__(kT, 8) cheb_step_kernel(long long n, const long long* __restrict__ soff,
                                                       const int* __restrict__ scol, const double* __restrict__ sval,
                                                       const double* __restrict__ dinv, const double* __restrict__ din,
                                                       double* __restrict__ dout, double* __restrict__ res,
                                                       double* __restrict__ z, const double* __restrict__ coef, int j,
                                                       const int* done) {
  if (done && *(volatile const int*)done) return;
  const double c1 = coef[2 * j], c2 = coef[2 * j + 1];
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    const long long s0 = __ldg(soff + (g >> 5)), s1 = __ldg(soff + (g >> 5) + 1);
    const int w = (int)((s1 - s0) >> 5);
    const long long b = s0 + (g & 31);
    // batches of kB entries: all their column and value loads issue before the dependent
    // gathers of d_in, so each thread keeps several memory requests in flight
    double ad = 0.0;
    int k = 0;
    for (; k + kB <= w; k += kB) {
      int c[kB];
      double v[kB];
#pragma unroll
      for (int a = 0; a < kB; ++a) {
        c[a] = __ldg(scol + b + 32LL * (k + a));
        v[a] = __ldg(sval + b + 32LL * (k + a));
      }
#pragma unroll
      for (int a = 0; a < kB; ++a) ad += v[a] * __ldg(din + c[a]);
    }
    for (; k < w; ++k) ad += __ldg(sval + b + 32LL * k) * __ldg(din + __ldg(scol + b + 32LL * k));
    const double rs = res[g] - dinv[g] * ad;
    res[g] = rs;
    const double dn = c1 * din[g] + c2 * rs;
    dout[g] = dn;
    z[g] += dn;
  }
}

// count[t] = 32 x the longest row of slice t
__global__ void __launch_bounds__(kT) sell_count_kernel(long long n, const long long* __restrict__ off,
                                                        long long* __restrict__ count) {
  const long long ns = (n + 31) / 32;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ns; t += (long long)gridDim.x * blockDim.x) {
    long long w = 0;
    const long long g1 = (32 * t + 32 < n) ? 32 * t + 32 : n;
    for (long long g = 32 * t; g < g1; ++g) w = max(w, off[g + 1] - off[g]);
    count[t] = 32 * w;
  }
}

// one thread per (slice, lane) position: row g's entries in slice order, then the padding
__global__ void __launch_bounds__(kT) sell_copy_kernel(long long n, const long long* __restrict__ off,
                                                       const int* __restrict__ col, const double* __restrict__ val,
                                                       const long long* __restrict__ soff, int* __restrict__ scol,
                                                       double* __restrict__ sval) {
  const long long np = 32 * ((n + 31) / 32);
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < np; g += (long long)gridDim.x * blockDim.x) {
    const long long s0 = soff[g >> 5];
    const int w = (int)((soff[(g >> 5) + 1] - s0) >> 5);
    const long long b = s0 + (g & 31);
    const long long o0 = g < n ? off[g] : 0;
    const int len = g < n ? (int)(off[g + 1] - o0) : 0;
    for (int k = 0; k < w; ++k) {
      if (col) scol[b + 32LL * k] = k < len ? col[o0 + k] : (g < n ? (int)g : 0);
      if (val) sval[b + 32LL * k] = k < len ? val[o0 + k] : 0.0;
    }
  }
}

// ---- exclusive scan of n counts into off[0..n] (three passes, 2048 entries per block) ----
constexpr int kScanT = 1024, kScanPer = 2;
constexpr int kScanB = kScanT * kScanPer;

__device__ long long block_exclusive_scan(long long v, long long* sh, long long* total) {
  // inclusive warp scans, then a scan of the warp totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = (lane < (kScanT >> 5)) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  const long long before = (wid > 0 ? sh[wid - 1] : 0) + x - v;
  if (total) *total = sh[(kScanT >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kScanT) scan_sums_kernel(long long n, const long long* __restrict__ c,
                                                           long long* __restrict__ sums) {
  __shared__ long long sh[32];
  const long long base = (long long)blockIdx.x * kScanB + threadIdx.x * kScanPer;
  long long v = 0;
  for (int a = 0; a < kScanPer; ++a)
    if (base + a < n) v += c[base + a];
  long long tot;
  block_exclusive_scan(v, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanT) scan_top_kernel(long long nb, long long* __restrict__ sums,
                                                          long long* __restrict__ total) {
  __shared__ long long sh[32];
  long long carry = 0;
  for (long long b0 = 0; b0 < nb; b0 += kScanT) {
    const long long b = b0 + threadIdx.x;
    const long long v = (b < nb) ? sums[b] : 0;
    long long tot;
    const long long ex = block_exclusive_scan(v, sh, &tot);
    if (b < nb) sums[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanT) scan_apply_kernel(long long n, const long long* __restrict__ c,
                                                            const long long* __restrict__ sums,
                                                            long long* __restrict__ off) {
  __shared__ long long sh[32];
  const long long base = (long long)blockIdx.x * kScanB + threadIdx.x * kScanPer;
  long long v[kScanPer], s = 0;
  for (int a = 0; a < kScanPer; ++a) {
    v[a] = (base + a < n) ? c[base + a] : 0;
    s += v[a];
  }
  long long run = sums[blockIdx.x] + block_exclusive_scan(s, sh, nullptr);
  for (int a = 0; a < kScanPer; ++a) {
    if (base + a < n) off[base + a] = run;
    run += v[a];
  }
}

}  // namespace

cudaError_t hx_lor_count(const HxLorBuild& b, long long* count, int* bad, cudaStream_t s) {
  lor_count_kernel<<<grid_of(b.n), kT, 0, s>>>(b.p, b.n, b.toff, b.tidx, b.R, b.dir, count, bad);
  return cudaGetLastError();
}

// off[0..n] = exclusive prefix sums of count; off[n] = the total.  sums: >= hx_lor_scan_blocks(n) entries.
long long hx_lor_scan_blocks(long long n) { return (n + kScanB - 1) / kScanB; }

cudaError_t hx_lor_scan(long long n, const long long* count, long long* sums, long long* off, cudaStream_t s) {
  const long long nb = hx_lor_scan_blocks(n);
  if (nb == 0) return cudaMemsetAsync(off, 0, sizeof(long long), s);
  scan_sums_kernel<<<(unsigned)nb, kScanT, 0, s>>>(n, count, sums);
  scan_top_kernel<<<1, kScanT, 0, s>>>(nb, sums, off + n);
  scan_apply_kernel<<<(unsigned)nb, kScanT, 0, s>>>(n, count, sums, off);
  return cudaGetLastError();
}

cudaError_t hx_lor_fill(const HxLorBuild& b, const long long* off, int* col, cudaStream_t s) {
  lor_fill_kernel<<<grid_of(b.n), kT, 0, s>>>(b.p, b.n, b.toff, b.tidx, b.R, b.dir, off, col);
  return cudaGetLastError();
}

cudaError_t hx_lor_sell_count(long long n, const long long* off, long long* count, cudaStream_t s) {
  sell_count_kernel<<<grid_of((n + 31) / 32), kT, 0, s>>>(n, off, count);
  return cudaGetLastError();
}

cudaError_t hx_lor_sell_copy(const HxLorMatrix& A, const int* col, const double* val, cudaStream_t s) {
  sell_copy_kernel<<<grid_of(A.n), kT, 0, s>>>(A.n, A.off, col, val, A.soff, col ? A.scol : nullptr,
                                               val ? A.sval : nullptr);
  return cudaGetLastError();
}

cudaError_t hx_lor_values(const HxTables& T, const HxLorBuild& b, const double* X8, double alpha, double nu,
                          int collocated, const HxLorMatrix& A, unsigned long long* bound, cudaStream_t s) {
  lor_values_kernel<<<grid_of(b.n), kT, 0, s>>>(T, b.n, b.toff, b.tidx, b.R, b.dir, X8, alpha, nu, collocated, A.off,
                                                 A.col, A.val);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(bound, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  lor_diag_kernel<<<grid_of(b.n), kT, 0, s>>>(b.n, A.off, A.col, A.val, A.dinv, bound);
  e = cudaGetLastError();
  if (e != cudaSuccess || !A.sval) return e;
  return hx_lor_sell_copy(A, nullptr, A.val, s);
}

cudaError_t hx_lor_coefficients(const unsigned long long* bound, int degree, double* coef, cudaStream_t s) {
  lor_coef_kernel<<<1, 32, 0, s>>>(bound, degree, coef);
  return cudaGetLastError();
}

cudaError_t hx_lor_precondition(const HxLorMatrix& A, const HxChebWork& w, const double* r, double* z,
                                const int* done, cudaStream_t s) {
  const unsigned g = grid_of(A.n);
  cheb_first_kernel<<<g, kT, 0, s>>>(A.n, A.dinv, r, w.res, w.d0, z, w.coef, done);
  cudaError_t e = cudaGetLastError();
  double* din = w.d0;
  double* dout = w.d1;
  for (int j = 1; j < w.degree && e == cudaSuccess; ++j) {
    cheb_step_kernel<<<g, kT, 0, s>>>(A.n, A.soff, A.scol, A.sval, A.dinv, din, dout, w.res, z, w.coef, j, done);
    e = cudaGetLastError();
    double* t = din;
    din = dout;
    dout = t;
  }
  return e;
}

