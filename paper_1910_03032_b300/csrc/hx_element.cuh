// Element kernels of the matrix-free Q_p Helmholtz operator alpha M + nu K.
//
// One thread block processes NE elements.  Every stage is a loop over "line
// tasks" (one 1D contraction of one line of one element) spread over all NT
// threads, so warps stay full whatever p is; stages are separated by
// __syncthreads().  Per element, shared memory holds four q^3 regions
//   A: u at the quadrature points, then v = m u
//   B: du/dxi_1, then w_1, then (Dh^T w_1)
//   C: du/dxi_2, then w_2, then (Dh^T w_2)
//   D: the in-place pipeline x_E -> (B x) -> (B B x) -> ... and du/dxi_3
// all with strides (1, q, q^2), so each line of a stage is owned by one thread
// and can be overwritten in place.
//
// Sum factorization (Sec. 3.1, Eqs. (sumFactorized), (tensorGradient)):
//   u_q = (B x B x B) x_E, grad u_q = (Dh applied along each direction) u_q,
//   [v; w] = [m u_q; G grad u_q]  (pointwise, G = nu w detJ J^-1 J^-T, m = alpha w detJ),
//   y_E = (B x B x B)^T (v + sum_d Dh_d^T w_d).
// Each 1D contraction uses the even-odd folding of the symmetric 1D matrices
// (the symmetry the paper points out in Sec. 6).
#pragma once

#include <cuda_runtime.h>

#include "hx_internal.h"
#include "hx_tables.h"

namespace hx {

// y = S x for a centro-symmetric (SIGMA = +1) or centro-antisymmetric
// (SIGMA = -1) M x L matrix S given by its folded parts Se, So.
template <int L, int M, int SIGMA>
__device__ __forceinline__ void eo_apply(const double* __restrict__ Se, const double* __restrict__ So,
                                         const double (&x)[L], double (&y)[M]) {
  constexpr int HL = L / 2, CL = (L + 1) / 2, HM = M / 2;
  double ev[CL], od[HL];
#pragma unroll
  for (int b = 0; b < HL; ++b) {
    ev[b] = x[b] + x[L - 1 - b];
    od[b] = x[b] - x[L - 1 - b];
  }
  if (L & 1) ev[HL] = x[HL];
#pragma unroll
  for (int a = 0; a < HM; ++a) {
    double E = Se[a * CL] * ev[0];
#pragma unroll
    for (int b = 1; b < CL; ++b) E = fma(Se[a * CL + b], ev[b], E);
    double O = So[a * HL] * od[0];
#pragma unroll
    for (int b = 1; b < HL; ++b) O = fma(So[a * HL + b], od[b], O);
    y[a] = E + O;
    y[M - 1 - a] = (SIGMA > 0) ? (E - O) : (O - E);
  }
  if (M & 1) {
    constexpr int a = HM;
    if (SIGMA > 0) {
      double E = Se[a * CL] * ev[0];
#pragma unroll
      for (int b = 1; b < CL; ++b) E = fma(Se[a * CL + b], ev[b], E);
      y[a] = E;
    } else {
      double O = So[a * HL] * od[0];
#pragma unroll
      for (int b = 1; b < HL; ++b) O = fma(So[a * HL + b], od[b], O);
      y[a] = O;
    }
  }
}

template <int L>
__device__ __forceinline__ void load_line(const double* p, int stride, double (&v)[L]) {
#pragma unroll
  for (int i = 0; i < L; ++i) v[i] = p[i * stride];
}
template <int L>
__device__ __forceinline__ void store_line(double* p, int stride, const double (&v)[L]) {
#pragma unroll
  for (int i = 0; i < L; ++i) p[i * stride] = v[i];
}

// ---------------------------------------------------------------------------
// trilinear geometry: x(xi) = sum_c X_c prod_d (1 + s_cd xi_d)/2, J_ij = dx_i/dxi_j
// ---------------------------------------------------------------------------
// Monomial coefficients of the map per component: x = a0 + a1 xi1 + a2 xi2 + a3 xi3
// + a12 xi1 xi2 + a13 xi1 xi3 + a23 xi2 xi3 + a123 xi1 xi2 xi3, stored as
// cf[comp * 8 + m] with m in (0, 1, 2, 3, 12, 13, 23, 123) order.
__device__ __forceinline__ void trilinear_coeffs(const double* __restrict__ X8, double* cf) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double X[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) X[c] = X8[c * 3 + d];
    // corner c = cx + 2cy + 4cz, sign s = 2c - 1
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s12 = 0, s13 = 0, s23 = 0, s123 = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double sx = (c & 1) ? 1.0 : -1.0, sy = (c & 2) ? 1.0 : -1.0, sz = (c & 4) ? 1.0 : -1.0;
      s0 += X[c];
      s1 += sx * X[c];
      s2 += sy * X[c];
      s3 += sz * X[c];
      s12 += sx * sy * X[c];
      s13 += sx * sz * X[c];
      s23 += sy * sz * X[c];
      s123 += sx * sy * sz * X[c];
    }
    cf[d * 8 + 0] = 0.125 * s0;
    cf[d * 8 + 1] = 0.125 * s1;
    cf[d * 8 + 2] = 0.125 * s2;
    cf[d * 8 + 3] = 0.125 * s3;
    cf[d * 8 + 4] = 0.125 * s12;
    cf[d * 8 + 5] = 0.125 * s13;
    cf[d * 8 + 6] = 0.125 * s23;
    cf[d * 8 + 7] = 0.125 * s123;
  }
}

// Columns j0 = dx/dxi1, j1 = dx/dxi2, j2 = dx/dxi3 at (x1, x2, x3).
__device__ __forceinline__ void trilinear_jacobian(const double* cf, double x1, double x2, double x3,
                                                   double (&j0)[3], double (&j1)[3], double (&j2)[3]) {
  const double x23 = x2 * x3, x13 = x1 * x3, x12 = x1 * x2;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double* a = cf + d * 8;
    j0[d] = a[1] + a[4] * x2 + a[5] * x3 + a[7] * x23;
    j1[d] = a[2] + a[4] * x1 + a[6] * x3 + a[7] * x13;
    j2[d] = a[3] + a[5] * x1 + a[6] * x2 + a[7] * x12;
  }
}

__device__ __forceinline__ double trilinear_point(const double* cf, int d, double x1, double x2, double x3) {
  const double* a = cf + d * 8;
  return a[0] + a[1] * x1 + a[2] * x2 + a[3] * x3 + a[4] * x1 * x2 + a[5] * x1 * x3 + a[6] * x2 * x3 +
         a[7] * x1 * x2 * x3;
}

// Factors at one point: m = alpha w detJ and G = nu w detJ J^-1 J^-T.
// Rows of J^-1 are (j1 x j2, j2 x j0, j0 x j1) / detJ, so
// G_ik = (nu w / detJ) (c_i . c_k) with c the three cross products.
// Returns detJ.
__device__ __forceinline__ double point_factors(const double (&j0)[3], const double (&j1)[3],
                                                const double (&j2)[3], double alpha_w, double nu_w,
                                                double (&f)[7]) {
  double c0[3], c1[3], c2[3];
  c0[0] = j1[1] * j2[2] - j1[2] * j2[1];
  c0[1] = j1[2] * j2[0] - j1[0] * j2[2];
  c0[2] = j1[0] * j2[1] - j1[1] * j2[0];
  c1[0] = j2[1] * j0[2] - j2[2] * j0[1];
  c1[1] = j2[2] * j0[0] - j2[0] * j0[2];
  c1[2] = j2[0] * j0[1] - j2[1] * j0[0];
  c2[0] = j0[1] * j1[2] - j0[2] * j1[1];
  c2[1] = j0[2] * j1[0] - j0[0] * j1[2];
  c2[2] = j0[0] * j1[1] - j0[1] * j1[0];
  const double det = j0[0] * c0[0] + j0[1] * c0[1] + j0[2] * c0[2];
  const double s = nu_w / det;
  f[0] = alpha_w * det;
  f[1] = s * (c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]);
  f[2] = s * (c0[0] * c1[0] + c0[1] * c1[1] + c0[2] * c1[2]);
  f[3] = s * (c0[0] * c2[0] + c0[1] * c2[1] + c0[2] * c2[2]);
  f[4] = s * (c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]);
  f[5] = s * (c1[0] * c2[0] + c1[1] * c2[1] + c1[2] * c2[2]);
  f[6] = s * (c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2]);
  return det;
}

// ---------------------------------------------------------------------------
// stages shared by the apply and load-vector kernels
// ---------------------------------------------------------------------------
// After the z-direction transpose has left [kz][jq][iq] in region D: B^T along
// y, B^T along x, then a coalesced copy of the block's E-vector slab.
template <int N, int Q, int NE, int NT>
__device__ __forceinline__ void stage_transpose_y_x_store(const HxTables& T, double* smem, long long e0,
                                                          long long E, double* __restrict__ yE) {
  constexpr int Q3 = Q * Q * Q, N3 = N * N * N, SY = Q, SZ = Q * Q, R4 = 4 * Q3;
  for (int t = threadIdx.x; t < NE * N * Q; t += NT) {
    const int el = t / (N * Q), r = t - el * (N * Q);
    const int kz = r / Q, iq = r - kz * Q;
    double* line = smem + el * R4 + 3 * Q3 + kz * SZ + iq;
    double vin[Q], vout[N];
    load_line<Q>(line, SY, vin);
    eo_apply<Q, N, 1>(T.Bte, T.Bto, vin, vout);
    store_line<N>(line, SY, vout);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NE * N * N; t += NT) {
    const int el = t / (N * N), r = t - el * (N * N);
    const int kz = r / N, j = r - kz * N;
    double* line = smem + el * R4 + 3 * Q3 + kz * SZ + j * SY;
    double vin[Q], vout[N];
    load_line<Q>(line, 1, vin);
    eo_apply<Q, N, 1>(T.Bte, T.Bto, vin, vout);
    store_line<N>(line, 1, vout);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NE * N3; t += NT) {
    const int el = t / N3, l = t - el * N3;
    const long long e = e0 + el;
    if (e < E) {
      const int i = l % N, j = (l / N) % N, k = l / (N * N);
      yE[e * N3 + l] = smem[el * R4 + 3 * Q3 + k * SZ + j * SY + i];
    }
  }
}

// ---------------------------------------------------------------------------
// the operator kernel
// ---------------------------------------------------------------------------
template <int P, int Q, int NE, int NT, int GEOM, bool NUF>
__global__ void __launch_bounds__(NT) apply_kernel(const __grid_constant__ HxTables T, const HxApplyArgs A) {
  constexpr int N = P + 1, N3 = N * N * N, Q3 = Q * Q * Q, SY = Q, SZ = Q * Q, R4 = 4 * Q3;
  if (A.done != nullptr && *(volatile const int*)A.done) return;
  extern __shared__ double smem[];
  double* geo = smem + NE * R4;  // on-the-fly: NE x 24 map coefficients
  const long long e0 = (long long)blockIdx.x * NE;
  const int tid = threadIdx.x;

  if (GEOM == HX_KGEOM_ONTHEFLY) {
    for (int el = tid; el < NE; el += NT) {
      const long long e = e0 + el;
      double X8[24];
      for (int c = 0; c < 24; ++c) X8[c] = (e < A.E) ? A.X8[e * 24 + c] : 0.0;
      trilinear_coeffs(X8, geo + el * 24);
    }
  }
  // gather x_E = R x (Dirichlet DoFs read as zero for the constrained operator)
  for (int t = tid; t < NE * N3; t += NT) {
    const int el = t / N3, l = t - el * N3;
    const long long e = e0 + el;
    double v = 0.0;
    if (e < A.E) {
      const int g = __ldg(A.R + e * N3 + l);
      if (g >= 0) v = __ldg(A.x + g);
      else if (!A.constrained) v = __ldg(A.x + (-g - 1));
    }
    const int i = l % N, j = (l / N) % N, k = l / (N * N);
    smem[el * R4 + 3 * Q3 + k * SZ + j * SY + i] = v;
  }
  __syncthreads();
  // x-lines: [k][j][i] -> [k][j][iq]
  for (int t = tid; t < NE * N * N; t += NT) {
    const int el = t / (N * N), r = t - el * (N * N);
    const int k = r / N, j = r - k * N;
    double* line = smem + el * R4 + 3 * Q3 + k * SZ + j * SY;
    double vin[N], vout[Q];
    load_line<N>(line, 1, vin);
    eo_apply<N, Q, 1>(T.Be, T.Bo, vin, vout);
    store_line<Q>(line, 1, vout);
  }
  __syncthreads();
  // y-lines: [k][j][iq] -> [k][jq][iq]
  for (int t = tid; t < NE * N * Q; t += NT) {
    const int el = t / (N * Q), r = t - el * (N * Q);
    const int k = r / Q, iq = r - k * Q;
    double* line = smem + el * R4 + 3 * Q3 + k * SZ + iq;
    double vin[N], vout[Q];
    load_line<N>(line, SY, vin);
    eo_apply<N, Q, 1>(T.Be, T.Bo, vin, vout);
    store_line<Q>(line, SY, vout);
  }
  __syncthreads();
  // z-lines: [k][jq][iq] -> u at the points (region A) and du/dxi_3 (region D)
  for (int t = tid; t < NE * Q * Q; t += NT) {
    const int el = t / (Q * Q), r = t - el * (Q * Q);
    double* col = smem + el * R4 + 3 * Q3 + r;  // r = jq * q + iq
    double vin[N], u[Q], du[Q];
    load_line<N>(col, SZ, vin);
    eo_apply<N, Q, 1>(T.Be, T.Bo, vin, u);
    eo_apply<Q, Q, -1>(T.De, T.Do, u, du);
    store_line<Q>(smem + el * R4 + r, SZ, u);
    store_line<Q>(col, SZ, du);
  }
  __syncthreads();
  // du/dxi_1 (x-lines of A -> B) and du/dxi_2 (y-lines of A -> C)
  for (int t = tid; t < NE * 2 * Q * Q; t += NT) {
    const int el = t / (2 * Q * Q), r = t - el * (2 * Q * Q);
    const int dir = r >= Q * Q;
    const int rr = r - dir * Q * Q;
    const int a = rr / Q, b = rr - a * Q;
    const int off = dir ? (a * SZ + b) : (a * SZ + b * SY);
    const int stride = dir ? SY : 1;
    double u[Q], du[Q];
    load_line<Q>(smem + el * R4 + off, stride, u);
    eo_apply<Q, Q, -1>(T.De, T.Do, u, du);
    store_line<Q>(smem + el * R4 + (1 + dir) * Q3 + off, stride, du);
  }
  __syncthreads();
  // pointwise: v = m u, w = G grad u
  for (int t = tid; t < NE * Q3; t += NT) {
    const int el = t / Q3, pt = t - el * Q3;
    const long long e = e0 + el;
    double f[7];
    if (GEOM == HX_KGEOM_STORED) {
      if (e < A.E) {
        const double* fe = A.factors + e * 7 * Q3 + pt;
#pragma unroll
        for (int c = 0; c < 7; ++c) f[c] = __ldg(fe + c * Q3);
      } else {
#pragma unroll
        for (int c = 0; c < 7; ++c) f[c] = 0.0;
      }
    } else {
      const int iq = pt % Q, jq = (pt / Q) % Q, kq = pt / (Q * Q);
      double j0[3], j1[3], j2[3];
      trilinear_jacobian(geo + el * 24, T.xq[iq], T.xq[jq], T.xq[kq], j0, j1, j2);
      const double w = T.wq[iq] * T.wq[jq] * T.wq[kq];
      double nu = A.nu;
      if (NUF) nu = (e < A.E) ? __ldg(A.nu_q + e * Q3 + pt) : 0.0;
      point_factors(j0, j1, j2, A.alpha * w, nu * w, f);
      if (e >= A.E) {
#pragma unroll
        for (int c = 0; c < 7; ++c) f[c] = 0.0;
      }
    }
    double* s = smem + el * R4 + pt;
    const double u = s[0], u1 = s[Q3], u2 = s[2 * Q3], u3 = s[3 * Q3];
    s[0] = f[0] * u;
    s[Q3] = f[1] * u1 + f[2] * u2 + f[3] * u3;
    s[2 * Q3] = f[2] * u1 + f[4] * u2 + f[5] * u3;
    s[3 * Q3] = f[3] * u1 + f[5] * u2 + f[6] * u3;
  }
  __syncthreads();
  // Dh^T along x (B, in place) and along y (C, in place)
  for (int t = tid; t < NE * 2 * Q * Q; t += NT) {
    const int el = t / (2 * Q * Q), r = t - el * (2 * Q * Q);
    const int dir = r >= Q * Q;
    const int rr = r - dir * Q * Q;
    const int a = rr / Q, b = rr - a * Q;
    const int off = dir ? (a * SZ + b) : (a * SZ + b * SY);
    const int stride = dir ? SY : 1;
    double* line = smem + el * R4 + (1 + dir) * Q3 + off;
    double w[Q], tw[Q];
    load_line<Q>(line, stride, w);
    eo_apply<Q, Q, -1>(T.Dte, T.Dto, w, tw);
    store_line<Q>(line, stride, tw);
  }
  __syncthreads();
  // z-lines: V = v + t1 + t2 + Dh^T w3, then B^T along z -> D region [kz][jq][iq]
  for (int t = tid; t < NE * Q * Q; t += NT) {
    const int el = t / (Q * Q), r = t - el * (Q * Q);
    double* base = smem + el * R4 + r;
    double w3[Q], t3[Q], V[Q], out[N];
    load_line<Q>(base + 3 * Q3, SZ, w3);
    eo_apply<Q, Q, -1>(T.Dte, T.Dto, w3, t3);
#pragma unroll
    for (int kq = 0; kq < Q; ++kq) V[kq] = (base[kq * SZ] + base[Q3 + kq * SZ]) + (base[2 * Q3 + kq * SZ] + t3[kq]);
    eo_apply<Q, N, 1>(T.Bte, T.Bto, V, out);
    store_line<N>(base + 3 * Q3, SZ, out);
  }
  __syncthreads();
  stage_transpose_y_x_store<N, Q, NE, NT>(T, smem, e0, A.E, A.yE);
}

// Load vector: bE = (B x B x B)^T (w detJ f) per element.
template <int P, int Q, int NE, int NT>
__global__ void __launch_bounds__(NT) load_kernel(const __grid_constant__ HxTables T, const HxLoadArgs A) {
  constexpr int N = P + 1, Q3 = Q * Q * Q, SZ = Q * Q, R4 = 4 * Q3;
  extern __shared__ double smem[];
  double* geo = smem + NE * R4;
  const long long e0 = (long long)blockIdx.x * NE;
  const int tid = threadIdx.x;
  for (int el = tid; el < NE; el += NT) {
    const long long e = e0 + el;
    double X8[24];
    for (int c = 0; c < 24; ++c) X8[c] = (e < A.E) ? A.X8[e * 24 + c] : 0.0;
    trilinear_coeffs(X8, geo + el * 24);
  }
  __syncthreads();
  for (int t = tid; t < NE * Q3; t += NT) {
    const int el = t / Q3, pt = t - el * Q3;
    const long long e = e0 + el;
    double v = 0.0;
    if (e < A.E) {
      const int iq = pt % Q, jq = (pt / Q) % Q, kq = pt / (Q * Q);
      double j0[3], j1[3], j2[3];
      trilinear_jacobian(geo + el * 24, T.xq[iq], T.xq[jq], T.xq[kq], j0, j1, j2);
      const double det = j0[0] * (j1[1] * j2[2] - j1[2] * j2[1]) + j0[1] * (j1[2] * j2[0] - j1[0] * j2[2]) +
                         j0[2] * (j1[0] * j2[1] - j1[1] * j2[0]);
      v = T.wq[iq] * T.wq[jq] * T.wq[kq] * det * __ldg(A.fq + e * Q3 + pt);
    }
    smem[el * R4 + pt] = v;
  }
  __syncthreads();
  // z-lines: B^T along z from A into D
  for (int t = tid; t < NE * Q * Q; t += NT) {
    const int el = t / (Q * Q), r = t - el * (Q * Q);
    double V[Q], out[N];
    load_line<Q>(smem + el * R4 + r, SZ, V);
    eo_apply<Q, N, 1>(T.Bte, T.Bto, V, out);
    store_line<N>(smem + el * R4 + 3 * Q3 + r, SZ, out);
  }
  __syncthreads();
  stage_transpose_y_x_store<N, Q, NE, NT>(T, smem, e0, A.E, A.yE);
}

// Diagonal of the element matrices, sum-factorized:
// diag[k][j][i] = sum_{c,b,a} m (BB_ai BB_bj BB_ck) + G00 DD_ai BB_bj BB_ck + G11 BB_ai DD_bj BB_ck
//   + G22 BB_ai BB_bj DD_ck + 2 G01 BD_ai BD_bj BB_ck + 2 G02 BD_ai BB_bj BD_ck + 2 G12 BB_ai BD_bj BD_ck
// with BB = B.B, DD = D.D, BD = B.D (entrywise) and factors at point (a, b, c).
template <int P, int Q, int NE, int NT, int GEOM, bool NUF>
__global__ void __launch_bounds__(NT) diag_kernel(const __grid_constant__ HxTables T, const HxDiagArgs A) {
  constexpr int N = P + 1, N3 = N * N * N, Q3 = Q * Q * Q;
  constexpr int F1 = 7 * Q * Q * N, F2 = 7 * Q * N * N;
  constexpr int FA = (7 * Q3 > F2) ? 7 * Q3 : F2;  // factors, later reused by stage-2 output
  constexpr int PER = FA + F1;
  extern __shared__ double smem[];
  double* tab = smem + NE * PER;  // BB, DD, BD tables: 3 q n
  double* geo = tab + 3 * Q * N;  // NE x 24
  const long long e0 = (long long)blockIdx.x * NE;
  const int tid = threadIdx.x;
  for (int t = tid; t < Q * N; t += NT) {
    tab[t] = T.B[t] * T.B[t];
    tab[Q * N + t] = T.D[t] * T.D[t];
    tab[2 * Q * N + t] = T.B[t] * T.D[t];
  }
  if (GEOM == HX_KGEOM_ONTHEFLY) {
    for (int el = tid; el < NE; el += NT) {
      const long long e = e0 + el;
      double X8[24];
      for (int c = 0; c < 24; ++c) X8[c] = (e < A.E) ? A.X8[e * 24 + c] : 0.0;
      trilinear_coeffs(X8, geo + el * 24);
    }
    __syncthreads();
  }
  // factors into shared memory: F[f][c][b][a]
  for (int t = tid; t < NE * Q3; t += NT) {
    const int el = t / Q3, pt = t - el * Q3;
    const long long e = e0 + el;
    double f[7] = {0, 0, 0, 0, 0, 0, 0};
    if (e < A.E) {
      if (GEOM == HX_KGEOM_STORED) {
#pragma unroll
        for (int c = 0; c < 7; ++c) f[c] = A.factors[(e * 7 + c) * Q3 + pt];
      } else {
        const int iq = pt % Q, jq = (pt / Q) % Q, kq = pt / (Q * Q);
        double j0[3], j1[3], j2[3];
        trilinear_jacobian(geo + el * 24, T.xq[iq], T.xq[jq], T.xq[kq], j0, j1, j2);
        const double w = T.wq[iq] * T.wq[jq] * T.wq[kq];
        const double nu = NUF ? A.nu_q[e * Q3 + pt] : A.nu;
        point_factors(j0, j1, j2, A.alpha * w, nu * w, f);
      }
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) smem[el * PER + c * Q3 + pt] = f[c];
  }
  __syncthreads();
  const double* BB = tab;
  const double* DD = tab + Q * N;
  const double* BD = tab + 2 * Q * N;
  // stage 1: contract a -> T1[f][c][b][i]
  for (int t = tid; t < NE * Q * Q; t += NT) {
    const int el = t / (Q * Q), cb = t - el * (Q * Q);
    const double* F = smem + el * PER + cb * Q;
    double* T1 = smem + el * PER + FA + cb * N;
    for (int i = 0; i < N; ++i) {
      double s[7] = {0, 0, 0, 0, 0, 0, 0};
      for (int a = 0; a < Q; ++a) {
        const double bb = BB[a * N + i], dd = DD[a * N + i], bd = BD[a * N + i];
        s[0] += bb * F[0 * Q3 + a];
        s[1] += dd * F[1 * Q3 + a];
        s[2] += bd * F[2 * Q3 + a];
        s[3] += bd * F[3 * Q3 + a];
        s[4] += bb * F[4 * Q3 + a];
        s[5] += bb * F[5 * Q3 + a];
        s[6] += bb * F[6 * Q3 + a];
      }
      for (int f = 0; f < 7; ++f) T1[f * Q * Q * N + i] = s[f];
    }
  }
  __syncthreads();
  // stage 2: contract b -> T2[f][c][j][i] (reuses the factor space)
  for (int t = tid; t < NE * Q * N; t += NT) {
    const int el = t / (Q * N), r = t - el * (Q * N);
    const int c = r / N, i = r - c * N;
    const double* T1 = smem + el * PER + FA + c * Q * N + i;
    double* T2 = smem + el * PER + c * N * N + i;
    for (int j = 0; j < N; ++j) {
      double s[7] = {0, 0, 0, 0, 0, 0, 0};
      for (int b = 0; b < Q; ++b) {
        const double bb = BB[b * N + j], dd = DD[b * N + j], bd = BD[b * N + j];
        const double* src = T1 + b * N;
        s[0] += bb * src[0 * Q * Q * N];
        s[1] += bb * src[1 * Q * Q * N];
        s[2] += bd * src[2 * Q * Q * N];
        s[3] += bb * src[3 * Q * Q * N];
        s[4] += dd * src[4 * Q * Q * N];
        s[5] += bd * src[5 * Q * Q * N];
        s[6] += bb * src[6 * Q * Q * N];
      }
      for (int f = 0; f < 7; ++f) T2[f * Q * N * N + j * N] = s[f];
    }
  }
  __syncthreads();
  // stage 3: contract c -> element diagonal
  for (int t = tid; t < NE * N3; t += NT) {
    const int el = t / N3, l = t - el * N3;
    const int k = l / (N * N), ji = l - k * N * N;
    const long long e = e0 + el;
    const double* T2 = smem + el * PER + ji;
    double s = 0.0;
    for (int c = 0; c < Q; ++c) {
      const double bb = BB[c * N + k], dd = DD[c * N + k], bd = BD[c * N + k];
      const double* src = T2 + c * N * N;
      const int st = Q * N * N;
      s += bb * (src[0] + src[1 * st] + src[4 * st]) + dd * src[6 * st] + 2.0 * bd * (src[3 * st] + src[5 * st]) +
           2.0 * bb * src[2 * st];
    }
    if (e < A.E) A.dE[e * N3 + l] = s;
  }
}

// ---------------------------------------------------------------------------
// launch configuration per order
// ---------------------------------------------------------------------------
template <int P>
struct Config {
  // elements per block of the operator kernel (about 55-70 KB of shared memory)
  static constexpr int NE = P == 1 ? 64 : P == 2 ? 32 : P == 3 ? 16 : P == 4 ? 8 : P == 5 ? 6 : P == 6 ? 4 : P == 7 ? 3 : 2;
  static constexpr int NT = 256;
  static constexpr int NE_DIAG = P <= 2 ? 8 : P <= 4 ? 2 : 1;
};

template <int P, int Q, int GEOM, bool NUF>
cudaError_t launch_apply_impl(const HxTables& T, const HxApplyArgs& A, cudaStream_t s) {
  constexpr int NE = Config<P>::NE, NT = Config<P>::NT;
  const size_t shmem = sizeof(double) * (size_t)(NE * 4 * Q * Q * Q + (GEOM == HX_KGEOM_ONTHEFLY ? NE * 24 : 0));
  auto k = apply_kernel<P, Q, NE, NT, GEOM, NUF>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  if (err != cudaSuccess) return err;
  const long long blocks = (A.E + NE - 1) / NE;
  if (blocks == 0) return cudaSuccess;
  k<<<(unsigned)blocks, NT, shmem, s>>>(T, A);
  return cudaGetLastError();
}

template <int P, int Q>
cudaError_t launch_apply_q(const HxTables& T, const HxApplyArgs& A, int geom, cudaStream_t s) {
  if (geom == HX_KGEOM_STORED) return launch_apply_impl<P, Q, HX_KGEOM_STORED, false>(T, A, s);
  if (A.nu_q) return launch_apply_impl<P, Q, HX_KGEOM_ONTHEFLY, true>(T, A, s);
  return launch_apply_impl<P, Q, HX_KGEOM_ONTHEFLY, false>(T, A, s);
}

template <int P, int Q, int GEOM, bool NUF>
cudaError_t launch_diag_impl(const HxTables& T, const HxDiagArgs& A, cudaStream_t s) {
  constexpr int N = P + 1, NE = Config<P>::NE_DIAG, NT = 128;
  constexpr int F1 = 7 * Q * Q * N, F2 = 7 * Q * N * N;
  constexpr int FA = (7 * Q * Q * Q > F2) ? 7 * Q * Q * Q : F2;
  const size_t shmem = sizeof(double) * (size_t)(NE * (FA + F1) + 3 * Q * N + NE * 24);
  auto k = diag_kernel<P, Q, NE, NT, GEOM, NUF>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  if (err != cudaSuccess) return err;
  const long long blocks = (A.E + NE - 1) / NE;
  if (blocks == 0) return cudaSuccess;
  k<<<(unsigned)blocks, NT, shmem, s>>>(T, A);
  return cudaGetLastError();
}

template <int P, int Q>
cudaError_t launch_diag_q(const HxTables& T, const HxDiagArgs& A, int geom, cudaStream_t s) {
  if (geom == HX_KGEOM_STORED) return launch_diag_impl<P, Q, HX_KGEOM_STORED, false>(T, A, s);
  if (A.nu_q) return launch_diag_impl<P, Q, HX_KGEOM_ONTHEFLY, true>(T, A, s);
  return launch_diag_impl<P, Q, HX_KGEOM_ONTHEFLY, false>(T, A, s);
}

template <int P, int Q>
cudaError_t launch_load_q(const HxTables& T, const HxLoadArgs& A, cudaStream_t s) {
  constexpr int NE = Config<P>::NE, NT = Config<P>::NT;
  const size_t shmem = sizeof(double) * (size_t)(NE * 4 * Q * Q * Q + NE * 24);
  auto k = load_kernel<P, Q, NE, NT>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  if (err != cudaSuccess) return err;
  const long long blocks = (A.E + NE - 1) / NE;
  if (blocks == 0) return cudaSuccess;
  k<<<(unsigned)blocks, NT, shmem, s>>>(T, A);
  return cudaGetLastError();
}

}  // namespace hx

#define HX_DEFINE_ORDER(P)                                                                                 \
  cudaError_t hx_launch_apply_p##P(const HxTables& T, const HxApplyArgs& A, int geom, cudaStream_t s) {   \
    if (T.q == P + 1) return hx::launch_apply_q<P, P + 1>(T, A, geom, s);                                 \
    if (T.q == P + 2) return hx::launch_apply_q<P, P + 2>(T, A, geom, s);                                 \
    return cudaErrorInvalidValue;                                                                          \
  }                                                                                                        \
  cudaError_t hx_launch_diag_p##P(const HxTables& T, const HxDiagArgs& A, int geom, cudaStream_t s) {     \
    if (T.q == P + 1) return hx::launch_diag_q<P, P + 1>(T, A, geom, s);                                  \
    if (T.q == P + 2) return hx::launch_diag_q<P, P + 2>(T, A, geom, s);                                  \
    return cudaErrorInvalidValue;                                                                          \
  }                                                                                                        \
  cudaError_t hx_launch_load_p##P(const HxTables& T, const HxLoadArgs& A, cudaStream_t s) {               \
    if (T.q == P + 1) return hx::launch_load_q<P, P + 1>(T, A, s);                                        \
    if (T.q == P + 2) return hx::launch_load_q<P, P + 2>(T, A, s);                                        \
    return cudaErrorInvalidValue;                                                                          \
  }
