// Element kernels of the matrix-free Q_p Helmholtz operator alpha M + nu K.
//
// One thread block processes NE elements with NT >= NE q^2 threads, so that
// thread t owns z-column t (element t / q^2, column t % q^2) in the three
// "column" stages and keeps that column's data in registers between them.
// The other stages are loops over line tasks (one 1D contraction of one line
// of one element) spread over all threads, so warps stay full at every p.
// Stages are separated by __syncthreads().  Per element, shared memory holds
// three q^3 regions with strides (1, q, q^2):
//   D: the in-place pipeline x_E -> (B x) -> (B B x) -> u at the points,
//      later (B^T V) -> (B^T B^T V) -> y_E along the transposed directions
//   X: du/dxi_1, then w_1 = (G grad u)_1, then Dh^T w_1
//   Y: du/dxi_2, then w_2, then Dh^T w_2
// du/dxi_3, v = m u, w_3 and Dh^T w_3 never leave the column owner's registers.
//
// Sum factorization (Sec. 3.1, Eqs. (sumFactorized), (tensorGradient)):
//   u_q = (B x B x B) x_E, grad u_q = (Dh applied along each direction) u_q,
//   [v; w] = [m u_q; G grad u_q]  (pointwise, G = nu w detJ J^-1 J^-T, m = alpha w detJ),
//   y_E = (B x B x B)^T (v + sum_d Dh_d^T w_d).
// Each 1D contraction uses the even-odd folding of the centro-symmetric 1D
// matrices (the symmetry the paper points out in Sec. 6); along z the folded
// parts of one contraction feed the next one directly, without recombining.
#pragma once

#include <cuda_runtime.h>

#include "hx_internal.h"
#include "hx_tables.h"

namespace hx {

// sum_k S[k] v[k] (K >= 1 terms), first term a multiply
template <int K, typename Real>
__device__ __forceinline__ Real dotk(const Real* __restrict__ S, const Real* v) {
  Real s = S[0] * v[0];
#pragma unroll
  for (int k = 1; k < K; ++k) s = fma(S[k], v[k], s);
  return s;
}

// Even / odd parts of x: ev[b] = x[b] + x[L-1-b], od[b] = x[b] - x[L-1-b] (b < L/2),
// ev[L/2] = x[L/2] for odd L.
template <int L, typename Real>
__device__ __forceinline__ void fold(const Real (&x)[L], Real* ev, Real* od) {
  constexpr int HL = L / 2;
#pragma unroll
  for (int b = 0; b < HL; ++b) {
    ev[b] = x[b] + x[L - 1 - b];
    od[b] = x[b] - x[L - 1 - b];
  }
  if (L & 1) ev[HL] = x[HL];
}

// Folded products of a centro-(anti)symmetric M x L matrix with folded input:
// E[a] = sum_b Se[a][b] ev[b], O[a] = sum_b So[a][b] od[b] for a < M/2; for odd M the
// middle row has only its E part (SIGMA = +1) or only its O part (SIGMA = -1).
template <int L, int M, int SIGMA, typename Real>
__device__ __forceinline__ void products(const Real* __restrict__ Se, const Real* __restrict__ So,
                                         const Real* ev, const Real* od, Real* E, Real* O) {
  constexpr int HL = L / 2, CL = (L + 1) / 2, HM = M / 2;
#pragma unroll
  for (int a = 0; a < HM; ++a) {
    E[a] = dotk<CL>(Se + a * CL, ev);
    O[a] = dotk<HL>(So + a * HL, od);
  }
  if (M & 1) {
    if (SIGMA > 0) {
      E[HM] = dotk<CL>(Se + HM * CL, ev);
      O[HM] = Real(0);
    } else {
      O[HM] = dotk<HL>(So + HM * HL, od);
      E[HM] = Real(0);
    }
  }
}

// y from folded parts: y[a] = E + O, y[M-1-a] = SIGMA (E - O); middle as in products.
template <int M, int SIGMA, typename Real>
__device__ __forceinline__ void combine(const Real* E, const Real* O, Real (&y)[M]) {
  constexpr int HM = M / 2;
#pragma unroll
  for (int a = 0; a < HM; ++a) {
    y[a] = E[a] + O[a];
    y[M - 1 - a] = (SIGMA > 0) ? (E[a] - O[a]) : (O[a] - E[a]);
  }
  if (M & 1) y[HM] = (SIGMA > 0) ? E[HM] : O[HM];
}

// y = S x for a centro-symmetric (SIGMA = +1) or centro-antisymmetric
// (SIGMA = -1) M x L matrix S given by its folded parts Se, So.
template <int L, int M, int SIGMA, typename Real>
__device__ __forceinline__ void eo_apply(const Real* __restrict__ Se, const Real* __restrict__ So,
                                         const Real (&x)[L], Real (&y)[M]) {
  Real ev[(L + 1) / 2], od[(L + 1) / 2], E[(M + 1) / 2], O[(M + 1) / 2];
  fold<L>(x, ev, od);
  products<L, M, SIGMA>(Se, So, ev, od, E, O);
  combine<M, SIGMA>(E, O, y);
}

template <int L, typename Real>
__device__ __forceinline__ void load_line(const Real* p, int stride, Real (&v)[L]) {
#pragma unroll
  for (int i = 0; i < L; ++i) v[i] = p[i * stride];
}
template <int L, typename Real>
__device__ __forceinline__ void store_line(Real* p, int stride, const Real (&v)[L]) {
#pragma unroll
  for (int i = 0; i < L; ++i) p[i * stride] = v[i];
}

// ---------------------------------------------------------------------------
// trilinear geometry: x(xi) = sum_c X_c prod_d (1 + s_cd xi_d)/2, J_ij = dx_i/dxi_j
// ---------------------------------------------------------------------------
// Monomial coefficients of the map per component: x = a0 + a1 xi1 + a2 xi2 + a3 xi3
// + a12 xi1 xi2 + a13 xi1 xi3 + a23 xi2 xi3 + a123 xi1 xi2 xi3, stored as
// cf[comp * 8 + m] with m in (0, 1, 2, 3, 12, 13, 23, 123) order.
template <typename Real>
__device__ __forceinline__ void trilinear_coeffs(const double* __restrict__ X8, Real* cf) {
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
    cf[d * 8 + 0] = Real(0.125 * s0);
    cf[d * 8 + 1] = Real(0.125 * s1);
    cf[d * 8 + 2] = Real(0.125 * s2);
    cf[d * 8 + 3] = Real(0.125 * s3);
    cf[d * 8 + 4] = Real(0.125 * s12);
    cf[d * 8 + 5] = Real(0.125 * s13);
    cf[d * 8 + 6] = Real(0.125 * s23);
    cf[d * 8 + 7] = Real(0.125 * s123);
  }
}

// The same coefficients for the NE elements of a block, one (element, coefficient) pair per
// thread: the FP64 additions then run as warp instructions with all lanes busy (computed by one
// thread per element they cost as many FP64 warp instructions per element as there are
// additions, which made the FP32 kernels with recomputed geometry FP64-pipe bound).  Each
// coefficient sums its 8 corner terms in corner order, like trilinear_coeffs: the results
// are the same bits.  Call from all threads; a barrier must follow before geo is read.
template <typename Real>
__device__ __forceinline__ void trilinear_coeffs_block(const double* __restrict__ X8, long long e0, long long E,
                                                       int ne, Real* geo) {
  for (int t = threadIdx.x; t < ne * 24; t += blockDim.x) {
    const int el = t / 24, k = t - el * 24, d = k >> 3, m = k & 7;
    // axes of monomial m = (1, xi1, xi2, xi3, xi1 xi2, xi1 xi3, xi2 xi3, xi1 xi2 xi3) as bits
    const int axes = (0x76534210 >> (4 * m)) & 7;
    const long long e = e0 + el;
    double s = 0.0;
    if (e < E) {
      const double* X = X8 + e * 24 + d;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const double x = __ldg(X + c * 3);
        s += (__popc(axes & ~c) & 1) ? -x : x;  // sign: -1 per axis of the monomial where corner c sits at -1
      }
    }
    geo[el * 24 + k] = Real(0.125 * s);
  }
}

// Columns j0 = dx/dxi1, j1 = dx/dxi2, j2 = dx/dxi3 at (x1, x2, x3).
template <typename Real>
__device__ __forceinline__ void trilinear_jacobian(const Real* cf, Real x1, Real x2, Real x3, Real (&j0)[3],
                                                   Real (&j1)[3], Real (&j2)[3]) {
  const Real x23 = x2 * x3, x13 = x1 * x3, x12 = x1 * x2;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const Real* a = cf + d * 8;
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
template <typename Real>
__device__ __forceinline__ Real point_factors(const Real (&j0)[3], const Real (&j1)[3], const Real (&j2)[3],
                                              Real alpha_w, Real nu_w, Real (&f)[7]) {
  Real c0[3], c1[3], c2[3];
  c0[0] = j1[1] * j2[2] - j1[2] * j2[1];
  c0[1] = j1[2] * j2[0] - j1[0] * j2[2];
  c0[2] = j1[0] * j2[1] - j1[1] * j2[0];
  c1[0] = j2[1] * j0[2] - j2[2] * j0[1];
  c1[1] = j2[2] * j0[0] - j2[0] * j0[2];
  c1[2] = j2[0] * j0[1] - j2[1] * j0[0];
  c2[0] = j0[1] * j1[2] - j0[2] * j1[1];
  c2[1] = j0[2] * j1[0] - j0[0] * j1[2];
  c2[2] = j0[0] * j1[1] - j0[1] * j1[0];
  const Real det = j0[0] * c0[0] + j0[1] * c0[1] + j0[2] * c0[2];
  const Real s = nu_w / det;
  f[0] = alpha_w * det;
  f[1] = s * (c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]);
  f[2] = s * (c0[0] * c1[0] + c0[1] * c1[1] + c0[2] * c1[2]);
  f[3] = s * (c0[0] * c2[0] + c0[1] * c2[1] + c0[2] * c2[2]);
  f[4] = s * (c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]);
  f[5] = s * (c1[0] * c2[0] + c1[1] * c2[1] + c1[2] * c2[2]);
  f[6] = s * (c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2]);
  return det;
}

// 1 / d in FP64 by Newton-Raphson iteration y <- y (2 - d y) (quadratic convergence) from the
// hardware's approximate reciprocal: three steps take any start within 2^-10 relative below
// FP64 rounding, for a fraction of the cost of a correctly rounded division.
__device__ __forceinline__ double rcp_newton(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const double e = fma(-d, y, 1.0);
    y = fma(y, e, y);
  }
  return y;
}

template <typename Real>
__device__ __forceinline__ void cross3(const Real (&a)[3], const Real (&b)[3], Real (&c)[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// ---------------------------------------------------------------------------
// bulk asynchronous copies (TMA engine) into shared memory, completed on an mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  // make the initialized barrier visible to the asynchronous (bulk-copy) proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// global -> shared bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase 0 of `bar` with a bound on the attempts (each try_wait itself suspends
// for a while); false when the bound was reached.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, int limit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, 0u)) return true;
  return false;
}

// ---------------------------------------------------------------------------
// shared-memory layout of one element's q^3 region: [z][y][x] with row stride
// SY (q rounded up to odd, so x-line tasks of consecutive threads fall in
// different banks) and plane stride SZ = q SY
// ---------------------------------------------------------------------------
//
// FP32 (4-byte banks, shared-memory-bound kernel): rows are not padded (SY = q), so the
// column stages of consecutive threads read consecutive words; the plane stride SZ >= q^2 is
// the one that gives the fewest shared-memory wavefronts over all stages of the operator
// kernel's block (a count of the distinct words per bank of every warp access, taken for each
// q at its block shape; odd q^2 | 1 where no other stride does markedly better); and the
// element stride is padded so that the columns of the next element continue the bank
// sequence (R3 = q^2 mod 32) for warps that straddle elements.
template <int Q>
constexpr int f32_plane_stride() {
  return Q == 3 ? 14 : Q == 4 ? 27 : Q == 6 ? 39 : Q == 7 ? 72 : Q == 8 ? 73 : Q == 10 ? 107 : ((Q * Q) | 1);
}
template <int Q, typename Real = double>
struct Layout {
  static constexpr bool F32 = sizeof(Real) == 4;
  static constexpr int SY = F32 ? Q : ((Q % 2 == 0) ? Q + 1 : Q);
  static constexpr int SZ = F32 ? f32_plane_stride<Q>() : Q * SY;
  static_assert(SZ >= Q * SY, "planes must not overlap");
  static constexpr int RG = Q * SZ;  // one region
  // the three regions D, X, Y of one element (element stride)
  static constexpr int R3 = F32 ? 3 * RG + (((Q * Q - 3 * RG) % 32) + 32) % 32 : 3 * RG;
};

// ---------------------------------------------------------------------------
// stages shared by the apply and load-vector kernels (region D of each element)
// ---------------------------------------------------------------------------
// After the z-direction transpose has left [kz][jq][iq] in region D: B^T along
// y, then B^T along x into region X (free by now), and from there to the E-vector in the
// order of its layout, so that consecutive threads write consecutive words (whole element
// blocks for element-major E-vectors, the same x-line of the block's elements side by side
// for the line layout).
template <int N, int Q, int NE, int NT, typename Real>
__device__ __forceinline__ void transpose_y_x_store(const HxTablesT<Real>& T, Real* smem, long long e0, long long E,
                                                    Real* __restrict__ yE, const HxELayout& lay) {
  using Lt = Layout<Q, Real>;
  constexpr int N3 = N * N * N, SY = Lt::SY, SZ = Lt::SZ, R3 = Lt::R3, RG = Lt::RG;
  static_assert(RG >= N3, "an element's result fits in its region X");
  for (int t = threadIdx.x; t < NE * N * Q; t += NT) {
    const int el = t / (N * Q), r = t - el * (N * Q);
    const int kz = r / Q, iq = r - kz * Q;
    Real* line = smem + el * R3 + kz * SZ + iq;
    Real vin[Q], vout[N];
    load_line<Q>(line, SY, vin);
    eo_apply<Q, N, 1>(T.Bte, T.Bto, vin, vout);
    store_line<N>(line, SY, vout);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NE * N * N; t += NT) {
    const int el = t / (N * N), r = t - el * (N * N);
    const int kz = r / N, j = r - kz * N;
    Real vin[Q], vout[N];
    load_line<Q>(smem + el * R3 + kz * SZ + j * SY, 1, vin);
    eo_apply<Q, N, 1>(T.Bte, T.Bto, vin, vout);
    store_line<N>(smem + el * R3 + RG + r * N, 1, vout);
  }
  __syncthreads();
  const int nel = (E - e0) < NE ? (int)(E - e0) : NE;
  if (lay.nx == 0) {
    Real* out = yE + e0 * N3;  // the block's elements are one contiguous range
    for (int t = threadIdx.x; t < nel * N3; t += NT) {
      const int el = t / N3, l = t - el * N3;
      out[t] = smem[el * R3 + RG + l];
    }
  } else {
    for (int t = threadIdx.x; t < NE * N3; t += NT) {
      const int i = t % N, u = t / N, el = u % NE, r = u / NE;
      if (el < nel) yE[hx_eline(lay, e0 + el, r, N) + i] = smem[el * R3 + RG + r * N + i];
    }
  }
}

// ---------------------------------------------------------------------------
// the operator kernel
// ---------------------------------------------------------------------------
// The element work of block `blk` (elements blk NE .. blk NE + NE - 1) of one operator.
template <typename Real, int P, int Q, int NE, int NT, int GEOM, bool NUF>
__device__ __forceinline__ void apply_body(const HxTablesT<Real>& T, const HxApplyArgsT<Real>& A, long long blk) {
  using Lt = Layout<Q, Real>;
  constexpr int N = P + 1, N3 = N * N * N, Q2 = Q * Q, Q3 = Q2 * Q;
  constexpr int SY = Lt::SY, SZ = Lt::SZ, RG = Lt::RG, R3 = Lt::R3;
  constexpr int CQ = (Q + 1) / 2, CN = (N + 1) / 2;
  // FP32 stored factors are staged in shared memory by one bulk copy (TMA) per block, issued
  // before the forward contractions and waited for in the pointwise stage.  For p > 4 the
  // staging buffer would cut the resident blocks per SM, which costs more than it saves.
  constexpr bool STAGE = Lt::F32 && GEOM == HX_KGEOM_STORED && P <= 4;
  constexpr int FE = 7 * Q3;  // factors per element
  static_assert(NT >= NE * Q2, "one thread per z-column");
  if (A.done != nullptr && *(volatile const int*)A.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long fbar;  // completion barrier of the factor copy
  Real* smem = reinterpret_cast<Real*>(smem_raw);
  Real* geo = smem + NE * R3;  // on-the-fly: NE x 24 map coefficients
  Real* sf = smem + ((NE * R3 + 3) & ~3);  // staged factors (16-byte aligned)
  __shared__ int wait_failed;          // some thread's first wait for the factor copy gave up
  const long long e0 = blk * NE;
  const int tid = threadIdx.x;
  // the copy starts at the 16-byte boundary at or below element e0's first factor
  const int foff = STAGE ? (int)(((e0 * A.fstride * (long long)sizeof(Real)) & 15) / (long long)sizeof(Real)) : 0;

  if (STAGE) {
    if (tid == 0) {
      const long long nel = (A.E - e0) < NE ? (A.E - e0) : NE;
      const long long b0 = e0 * A.fstride * (long long)sizeof(Real), b1 = (e0 + nel) * A.fstride * (long long)sizeof(Real);
      const long long a0 = b0 & ~15LL, a1 = (b1 + 15) & ~15LL;  // the factor array has 16 bytes of slack
      wait_failed = 0;
      mbar_init(&fbar, 1);
      mbar_expect_tx(&fbar, (unsigned)(a1 - a0));
      bulk_load(sf, reinterpret_cast<const char*>(A.factors) + a0, (unsigned)(a1 - a0), &fbar);
    }
  } else if (GEOM == HX_KGEOM_STORED) {
    // pull this block's factors toward L2 while the forward contractions run
    const long long nel = (A.E - e0) < NE ? (A.E - e0) : NE;
    const char* base = reinterpret_cast<const char*>(A.factors + e0 * A.fstride);
    const long long bytes = nel * A.fstride * (long long)sizeof(Real);
    for (long long off = (long long)tid * 128; off < bytes; off += (long long)NT * 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
  } else {
    trilinear_coeffs_block(A.X8, e0, A.E, NE, geo);  // corner coordinates stay FP64 until here
  }
  // 1. gather x_E = R x (Dirichlet DoFs read as zero for A_c) and B along x: [k][j][i] -> [k][j][iq]
  for (int t = tid; t < NE * N * N; t += NT) {
    const int el = t / (N * N), r = t - el * (N * N);
    const long long e = e0 + el;
    Real vin[N];
    if (e < A.E) {
      const int* Rp = A.R + e * N3 + r * N;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int g = __ldg(Rp + i);
        vin[i] = (g >= 0) ? __ldg(A.x + g) : (A.constrained ? Real(0) : __ldg(A.x + (-g - 1)));
      }
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) vin[i] = Real(0);
    }
    const int k = r / N, j = r - k * N;
    Real vout[Q];
    eo_apply<N, Q, 1>(T.Be, T.Bo, vin, vout);
    store_line<Q>(smem + el * R3 + k * SZ + j * SY, 1, vout);
  }
  __syncthreads();
  // 2. B along y: [k][j][iq] -> [k][jq][iq]
  for (int t = tid; t < NE * N * Q; t += NT) {
    const int el = t / (N * Q), r = t - el * (N * Q);
    const int k = r / Q, iq = r - k * Q;
    Real* line = smem + el * R3 + k * SZ + iq;
    Real vin[N], vout[Q];
    load_line<N>(line, SY, vin);
    eo_apply<N, Q, 1>(T.Be, T.Bo, vin, vout);
    store_line<Q>(line, SY, vout);
  }
  __syncthreads();
  // 3. columns: B along z -> u (stored for the x/y derivatives);
  //    du/dxi_3 from the folded parts of that same contraction (kept in registers)
  const bool owner = tid < NE * Q2;
  const int cel = tid / Q2, c = tid - cel * Q2;         // element, column (jq, iq) = (c / q, c % q)
  // coefficients in the kernel's precision, converted once (an FP32 kernel would otherwise
  // convert them at every point on the FP64 pipe)
  const Real alpha_r = Real(A.alpha), nu_r = Real(A.nu);
  // on-the-fly geometry along this thread's z-column: for a trilinear map dx/dxi_3 does not
  // depend on xi_3 and the other two Jacobian columns are affine in it, so the map
  // coefficients are read once per column and each point costs two 3-vector updates
  // (+13-16% on the FP64 on-the-fly apply despite a few spilled registers)
  constexpr bool COLJ = true;
  // FP64 with on-the-fly geometry: the pointwise stage works with the cofactor rows directly
  constexpr bool COF = GEOM == HX_KGEOM_ONTHEFLY && sizeof(Real) == 8;
  Real P0[3], R0[3], P1[3], R1[3], J2[3];
  if (COLJ && !COF && GEOM == HX_KGEOM_ONTHEFLY && owner) {
    const Real* a = geo + cel * 24;
    const Real x1 = T.xq[c % Q], x2 = T.xq[c / Q];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const Real* ad = a + d * 8;
      P0[d] = ad[1] + ad[4] * x2;
      R0[d] = ad[5] + ad[7] * x2;
      P1[d] = ad[2] + ad[4] * x1;
      R1[d] = ad[6] + ad[7] * x1;
      J2[d] = ad[3] + ad[5] * x1 + (ad[6] + ad[7] * x1) * x2;
    }
  }
  const int cs = (c / Q) * SY + (c % Q);                // the column's offset in a region
  Real du[Q];
  if (owner) {
    Real* col = smem + cel * R3 + cs;
    Real vin[N], u[Q], ev[CN], od[CN], Eu[CQ], Ou[CQ], Ed[CQ], Od[CQ];
    load_line<N>(col, SZ, vin);
    fold<N>(vin, ev, od);
    products<N, Q, 1>(T.Be, T.Bo, ev, od, Eu, Ou);
    combine<Q, 1>(Eu, Ou, u);
    store_line<Q>(col, SZ, u);
    products<Q, Q, -1>(T.De2, T.Do2, Eu, Ou, Ed, Od);
    combine<Q, -1>(Ed, Od, du);
  }
  __syncthreads();
  // 4. du/dxi_1 (x-lines of D -> X) and du/dxi_2 (y-lines of D -> Y)
  for (int t = tid; t < NE * 2 * Q2; t += NT) {
    const int el = t / (2 * Q2), r = t - el * (2 * Q2);
    const int dir = r >= Q2;
    const int rr = r - dir * Q2;
    const int a = rr / Q, b = rr - a * Q;
    const int off = dir ? (a * SZ + b) : (a * SZ + b * SY);
    const int stride = dir ? SY : 1;
    Real uu[Q], d[Q];
    load_line<Q>(smem + el * R3 + off, stride, uu);
    eo_apply<Q, Q, -1>(T.De, T.Do, uu, d);
    store_line<Q>(smem + el * R3 + (1 + dir) * RG + off, stride, d);
  }
  __syncthreads();
  // 5. columns: pointwise v = m u (into D, over u), w = G grad u; then Dh^T along z of
  //    w_3 (folded parts kept in registers)
  Real Et[CQ], Ot[CQ];
  // a thread whose wait gave up raises the error flag and skips its pointwise work; after the
  // next barrier the whole block skips the remaining stages and stores nothing
  bool staged = true;
  if (STAGE && owner && !mbar_wait_bounded(&fbar, A.wait_limit)) {
    staged = false;
    wait_failed = 1;
    if (A.err) atomicExch(A.err, 1);
  }
  if (owner && staged) {
    const long long e = e0 + cel;
    Real* Dc = smem + cel * R3 + cs;
    Real* Xc = Dc + RG;
    Real* Yc = Xc + RG;
    Real w3[Q];
    if (COF) {
      // Rows of J^-1 are the cofactor rows c0 = j1 x j2, c1 = j2 x j0, c2 = j0 x j1 over detJ,
      // so G grad u = (nu w / detJ) sum_i c_i (c_i . t) with t = sum_k c_k du/dxi_k: no 3 x 3
      // factor matrix is formed.  Along the column j2 is constant and j0, j1 are affine in
      // z = xi_3 (coefficients once per column); detJ = j2 . c2, and 1/detJ by Newton-Raphson.
      const Real* ga = geo + cel * 24;
      const int iq = c % Q, jq = c / Q;
      const Real x1 = T.xq[iq], x2 = T.xq[jq];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const Real* ad = ga + d * 8;
        P0[d] = ad[1] + ad[4] * x2;
        R0[d] = ad[5] + ad[7] * x2;
        P1[d] = ad[2] + ad[4] * x1;
        R1[d] = ad[6] + ad[7] * x1;
        J2[d] = ad[3] + ad[5] * x1 + (ad[6] + ad[7] * x1) * x2;
      }
      const Real w12 = T.wq[iq] * T.wq[jq];
#pragma unroll
      for (int kq = 0; kq < Q; ++kq) {
        const Real z = T.xq[kq];
        Real j0[3], j1[3], c0[3], c1[3], c2[3], tt[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          j0[d] = P0[d] + z * R0[d];
          j1[d] = P1[d] + z * R1[d];
        }
        cross3(j1, J2, c0);
        cross3(J2, j0, c1);
        cross3(j0, j1, c2);
        const Real det = J2[0] * c2[0] + J2[1] * c2[1] + J2[2] * c2[2];
        const Real w = w12 * T.wq[kq];
        Real nu = nu_r;
        if (NUF) nu = (e < A.E) ? Real(__ldg(A.nu_q + e * Q3 + kq * Q2 + c)) : Real(0);
        const Real sc = (e < A.E) ? nu * w * rcp_newton(det) : Real(0);
        const Real ms = (e < A.E) ? alpha_r * w * det : Real(0);
        const Real u1 = Xc[kq * SZ], u2 = Yc[kq * SZ], u3 = du[kq];
#pragma unroll
        for (int d = 0; d < 3; ++d) tt[d] = c0[d] * u1 + c1[d] * u2 + c2[d] * u3;
        Dc[kq * SZ] = ms * Dc[kq * SZ];
        Xc[kq * SZ] = sc * (c0[0] * tt[0] + c0[1] * tt[1] + c0[2] * tt[2]);
        Yc[kq * SZ] = sc * (c1[0] * tt[0] + c1[1] * tt[1] + c1[2] * tt[2]);
        w3[kq] = sc * (c2[0] * tt[0] + c2[1] * tt[1] + c2[2] * tt[2]);
      }
    }
#pragma unroll
    for (int kq = 0; kq < Q && !COF; ++kq) {
      const int pt = kq * Q2 + c;
      Real f[7];
      if (STAGE) {
        if (e < A.E) {
          const Real* fe = sf + foff + cel * A.fstride + pt;
#pragma unroll
          for (int m = 0; m < 7; ++m) f[m] = fe[m * Q3];
        } else {
#pragma unroll
          for (int m = 0; m < 7; ++m) f[m] = Real(0);
        }
      } else if (GEOM == HX_KGEOM_STORED) {
        if (e < A.E) {
          const Real* fe = A.factors + e * A.fstride + pt;
#pragma unroll
          for (int m = 0; m < 7; ++m) f[m] = __ldg(fe + m * Q3);
        } else {
#pragma unroll
          for (int m = 0; m < 7; ++m) f[m] = Real(0);
        }
      } else {
        const int iq = c % Q, jq = c / Q;
        Real j0[3], j1[3], j2[3];
        if (COLJ) {
          const Real z = T.xq[kq];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            j0[d] = P0[d] + z * R0[d];
            j1[d] = P1[d] + z * R1[d];
            j2[d] = J2[d];
          }
        } else {
          trilinear_jacobian(geo + cel * 24, T.xq[iq], T.xq[jq], T.xq[kq], j0, j1, j2);
        }
        const Real w = T.wq[iq] * T.wq[jq] * T.wq[kq];
        Real nu = nu_r;
        if (NUF) nu = (e < A.E) ? Real(__ldg(A.nu_q + e * Q3 + pt)) : Real(0);
        point_factors(j0, j1, j2, alpha_r * w, nu * w, f);
        if (e >= A.E) {
#pragma unroll
          for (int m = 0; m < 7; ++m) f[m] = Real(0);
        }
      }
      const Real u1 = Xc[kq * SZ], u2 = Yc[kq * SZ], u3 = du[kq];
      Dc[kq * SZ] = f[0] * Dc[kq * SZ];
      Xc[kq * SZ] = f[1] * u1 + f[2] * u2 + f[3] * u3;
      Yc[kq * SZ] = f[2] * u1 + f[4] * u2 + f[5] * u3;
      w3[kq] = f[3] * u1 + f[5] * u2 + f[6] * u3;
    }
    Real ev[CQ], od[CQ];
    fold<Q>(w3, ev, od);
    products<Q, Q, -1>(T.Dte2, T.Dto2, ev, od, Et, Ot);  // rows doubled: (2E, 2O)
  }
  __syncthreads();
  if (STAGE && wait_failed) {
    // no copy may still be writing this block's shared memory when it exits: wait once more,
    // with a far larger bound than the first wait
    if (tid == 0) mbar_wait_bounded(&fbar, HX_WAIT_LIMIT_EXIT);
    return;
  }
  // 6. Dh^T along x (X, in place) and along y (Y, in place)
  for (int t = tid; t < NE * 2 * Q2; t += NT) {
    const int el = t / (2 * Q2), r = t - el * (2 * Q2);
    const int dir = r >= Q2;
    const int rr = r - dir * Q2;
    const int a = rr / Q, b = rr - a * Q;
    const int off = dir ? (a * SZ + b) : (a * SZ + b * SY);
    const int stride = dir ? SY : 1;
    Real* line = smem + el * R3 + (1 + dir) * RG + off;
    Real w[Q], tw[Q];
    load_line<Q>(line, stride, w);
    eo_apply<Q, Q, -1>(T.Dte, T.Dto, w, tw);
    store_line<Q>(line, stride, tw);
  }
  __syncthreads();
  // 7. columns: V = v + t1 + t2 + Dh^T w_3 formed directly in folded form, then B^T along z
  if (owner) {
    Real* Dc = smem + cel * R3 + cs;
    Real sv[Q], es[CQ], os[CQ], E[(N + 1) / 2], O[(N + 1) / 2], out[N];
#pragma unroll
    for (int kq = 0; kq < Q; ++kq) sv[kq] = Dc[kq * SZ] + Dc[RG + kq * SZ] + Dc[2 * RG + kq * SZ];
    fold<Q>(sv, es, os);
#pragma unroll
    for (int b = 0; b < CQ; ++b) es[b] += Ot[b];
#pragma unroll
    for (int b = 0; b < Q / 2; ++b) os[b] += Et[b];
    products<Q, N, 1>(T.Bte, T.Bto, es, os, E, O);
    combine<N, 1>(E, O, out);
    store_line<N>(Dc, SZ, out);
  }
  __syncthreads();
  transpose_y_x_store<N, Q, NE, NT>(T, smem, e0, A.E, A.yE, A.lay);
  // no copy may still be writing this block's shared memory when it exits (every owner's
  // first wait saw the copy complete, so this returns at once)
  if (STAGE && tid == 0) mbar_wait_bounded(&fbar, HX_WAIT_LIMIT_EXIT);
}

template <typename Real, int P, int Q, int NE, int NT, int MINB, int GEOM, bool NUF>
__global__ void __launch_bounds__(NT, MINB)
    apply_kernel(const __grid_constant__ HxTablesT<Real> T, const HxApplyArgsT<Real> A) {
  apply_body<Real, P, Q, NE, NT, GEOM, NUF>(T, A, blockIdx.x);
}

// Several operators of one order at once (the lock-step iterations of a batch): block b works
// on block b - blk_first[o] of operator o = blk_op[b], with that operator's arguments.
template <typename Real, int P, int Q, int NE, int NT, int MINB, int GEOM, bool NUF>
__global__ void __launch_bounds__(NT, MINB)
    apply_multi_kernel(const __grid_constant__ HxTablesT<Real> T, const HxApplyArgsT<Real>* __restrict__ args,
                       const int* __restrict__ blk_op, const int* __restrict__ blk_first) {
  const int o = __ldg(blk_op + blockIdx.x);
  const HxApplyArgsT<Real> A = args[o];
  apply_body<Real, P, Q, NE, NT, GEOM, NUF>(T, A, (long long)blockIdx.x - __ldg(blk_first + o));
}

// Load vector: bE = (B x B x B)^T (w detJ f) per element.
template <int P, int Q, int NE, int NT>
__global__ void __launch_bounds__(NT) load_kernel(const __grid_constant__ HxTables T, const HxLoadArgs A) {
  using Lt = Layout<Q>;
  constexpr int N = P + 1, Q2 = Q * Q, Q3 = Q2 * Q, SY = Lt::SY, SZ = Lt::SZ, R3 = Lt::R3;
  static_assert(NT >= NE * Q2, "one thread per z-column");
  extern __shared__ double smem[];
  double* geo = smem + NE * R3;
  const long long e0 = (long long)blockIdx.x * NE;
  const int tid = threadIdx.x;
  trilinear_coeffs_block(A.X8, e0, A.E, NE, geo);
  __syncthreads();
  if (tid < NE * Q2) {
    const int cel = tid / Q2, c = tid - cel * Q2;
    const int iq = c % Q, jq = c / Q;
    const long long e = e0 + cel;
    double V[Q], out[N];
#pragma unroll
    for (int kq = 0; kq < Q; ++kq) {
      double vv = 0.0;
      if (e < A.E) {
        double j0[3], j1[3], j2[3];
        trilinear_jacobian(geo + cel * 24, T.xq[iq], T.xq[jq], T.xq[kq], j0, j1, j2);
        const double det = j0[0] * (j1[1] * j2[2] - j1[2] * j2[1]) + j0[1] * (j1[2] * j2[0] - j1[0] * j2[2]) +
                           j0[2] * (j1[0] * j2[1] - j1[1] * j2[0]);
        vv = T.wq[iq] * T.wq[jq] * T.wq[kq] * det * (A.fq ? __ldg(A.fq + e * Q3 + kq * Q2 + c) : 1.0);
      }
      V[kq] = vv;
    }
    eo_apply<Q, N, 1>(T.Bte, T.Bto, V, out);
    store_line<N>(smem + cel * R3 + jq * SY + iq, SZ, out);
  }
  __syncthreads();
  transpose_y_x_store<N, Q, NE, NT>(T, smem, e0, A.E, A.yE, A.lay);
}

// Adjoint gradients at every quadrature point (not part of the paper's method):
//   dnu_q = -w_q detJ_q (J^-T grad lam)_q . (J^-T grad u)_q,   df_q = w_q detJ_q lam(x_q),
// the derivatives of L(u(nu, f)) through A_c lam = dL/du.  Both vectors go through the
// forward sum-factorized stages of the operator kernel side by side (six regions per
// element: D, X, Y for u, then for lam); the pointwise stage contracts the gradients
// with the geometric factor recomputed from the element vertices.
template <int P, int Q, int NE, int NT>
__global__ void __launch_bounds__(NT) grad_kernel(const __grid_constant__ HxTables T, const HxGradArgs A) {
  using Lt = Layout<Q>;
  constexpr int N = P + 1, N3 = N * N * N, Q2 = Q * Q, Q3 = Q2 * Q;
  constexpr int SY = Lt::SY, SZ = Lt::SZ, RG = Lt::RG, R6 = 6 * RG;
  constexpr int CQ = (Q + 1) / 2, CN = (N + 1) / 2;
  static_assert(NT >= NE * Q2, "one thread per z-column");
  extern __shared__ double smem[];
  double* geo = smem + NE * R6;
  const long long e0 = (long long)blockIdx.x * NE;
  const int tid = threadIdx.x;
  trilinear_coeffs_block(A.X8, e0, A.E, NE, geo);
  // 1. gather (Dirichlet entries as zero) and B along x, for u (v = 0) and lam (v = 1)
  for (int t = tid; t < 2 * NE * N * N; t += NT) {
    const int v = t / (NE * N * N), tt = t - v * NE * N * N;
    const int el = tt / (N * N), r = tt - el * (N * N);
    const long long e = e0 + el;
    const double* src = v ? A.lam : A.u;
    double vin[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int g = (e < A.E) ? __ldg(A.R + e * N3 + r * N + i) : -1;
      vin[i] = (g >= 0) ? __ldg(src + g) : 0.0;
    }
    const int k = r / N, j = r - k * N;
    double vout[Q];
    eo_apply<N, Q, 1>(T.Be, T.Bo, vin, vout);
    store_line<Q>(smem + el * R6 + v * 3 * RG + k * SZ + j * SY, 1, vout);
  }
  __syncthreads();
  // 2. B along y
  for (int t = tid; t < 2 * NE * N * Q; t += NT) {
    const int v = t / (NE * N * Q), tt = t - v * NE * N * Q;
    const int el = tt / (N * Q), r = tt - el * (N * Q);
    const int k = r / Q, iq = r - k * Q;
    double* line = smem + el * R6 + v * 3 * RG + k * SZ + iq;
    double vin[N], vout[Q];
    load_line<N>(line, SY, vin);
    eo_apply<N, Q, 1>(T.Be, T.Bo, vin, vout);
    store_line<Q>(line, SY, vout);
  }
  __syncthreads();
  // 3. columns: B along z (values kept in D) and d/dxi_3 (kept in registers), both vectors
  const bool owner = tid < NE * Q2;
  const int cel = tid / Q2, c = tid - cel * Q2;
  const int cs = (c / Q) * SY + (c % Q);
  double du[Q], dl[Q];
  if (owner) {
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      double* col = smem + cel * R6 + v * 3 * RG + cs;
      double vin[N], val[Q], ev[CN], od[CN], E[CQ], O[CQ], Ed[CQ], Od[CQ], d[Q];
      load_line<N>(col, SZ, vin);
      fold<N>(vin, ev, od);
      products<N, Q, 1>(T.Be, T.Bo, ev, od, E, O);
      combine<Q, 1>(E, O, val);
      store_line<Q>(col, SZ, val);
      products<Q, Q, -1>(T.De2, T.Do2, E, O, Ed, Od);
      combine<Q, -1>(Ed, Od, d);
#pragma unroll
      for (int k = 0; k < Q; ++k) (v ? dl : du)[k] = d[k];
    }
  }
  __syncthreads();
  // 4. d/dxi_1 and d/dxi_2 of both vectors
  for (int t = tid; t < 4 * NE * Q2; t += NT) {
    const int v = t / (2 * NE * Q2), tt = t - v * 2 * NE * Q2;
    const int el = tt / (2 * Q2), r = tt - el * (2 * Q2);
    const int dir = r >= Q2;
    const int rr = r - dir * Q2;
    const int a = rr / Q, b = rr - a * Q;
    const int off = dir ? (a * SZ + b) : (a * SZ + b * SY);
    const int stride = dir ? SY : 1;
    double* base = smem + el * R6 + v * 3 * RG;
    double uu[Q], d[Q];
    load_line<Q>(base + off, stride, uu);
    eo_apply<Q, Q, -1>(T.De, T.Do, uu, d);
    store_line<Q>(base + (1 + dir) * RG + off, stride, d);
  }
  __syncthreads();
  // 5. columns: the pointwise contractions, written with consecutive points in consecutive threads
  if (owner) {
    const long long e = e0 + cel;
    const double* U = smem + cel * R6 + cs;
    const double* Lm = U + 3 * RG;
    const int iq = c % Q, jq = c / Q;
#pragma unroll
    for (int kq = 0; kq < Q; ++kq) {
      double j0[3], j1[3], j2[3], f[7];
      trilinear_jacobian(geo + cel * 24, T.xq[iq], T.xq[jq], T.xq[kq], j0, j1, j2);
      const double w = T.wq[iq] * T.wq[jq] * T.wq[kq];
      point_factors(j0, j1, j2, w, w, f);  // f[0] = w detJ, f[1..6] = w detJ J^-1 J^-T
      const double u1 = U[RG + kq * SZ], u2 = U[2 * RG + kq * SZ], u3 = du[kq];
      const double l1 = Lm[RG + kq * SZ], l2 = Lm[2 * RG + kq * SZ], l3 = dl[kq];
      const double g1 = f[1] * u1 + f[2] * u2 + f[3] * u3;
      const double g2 = f[2] * u1 + f[4] * u2 + f[5] * u3;
      const double g3 = f[3] * u1 + f[5] * u2 + f[6] * u3;
      if (e < A.E) {
        const long long o = e * Q3 + kq * Q2 + c;
        A.dnu[o] = -(l1 * g1 + l2 * g2 + l3 * g3);
        A.df[o] = f[0] * Lm[kq * SZ];
      }
    }
  }
}

// Diagonal of the element matrices, sum-factorized:
// diag[k][j][i] = sum_{c,b,a} m (BB_ai BB_bj BB_ck) + G00 DD_ai BB_bj BB_ck + G11 BB_ai DD_bj BB_ck
//   + G22 BB_ai BB_bj DD_ck + 2 G01 BD_ai BD_bj BB_ck + 2 G02 BD_ai BB_bj BD_ck + 2 G12 BB_ai BD_bj BD_ck
// with BB = B.B, DD = D.D, BD = B.D (entrywise) and factors at point (a, b, c).  Terms that meet
// the same tables in the remaining directions are summed as soon as they do: after the
// a-contraction six sums remain (m and G00 share BB_bj BB_ck), after the b-contraction three
// (one per table along c), so the b and c stages contract 6 and 3 arrays instead of 7.
template <typename Real, int P, int Q, int NE, int NT, int GEOM, bool NUF>
__global__ void __launch_bounds__(NT) diag_kernel(const __grid_constant__ HxTablesT<Real> T, const HxDiagArgsT<Real> A) {
  constexpr int N = P + 1, N3 = N * N * N, Q3 = Q * Q * Q;
  constexpr int X1 = Q * Q * N;                       // one stage-1 array [c][b][i]
  constexpr int Y1 = Q * N * N;                       // one stage-2 array [c][j][i]
  constexpr int FA = (7 * Q3 > 3 * Y1) ? 7 * Q3 : 3 * Y1;  // factors, later reused by stage-2 output
  constexpr int PER = FA + 6 * X1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* smem = reinterpret_cast<Real*>(smem_raw);
  Real* tab = smem + NE * PER;  // BB, DD, BD tables: 3 q n
  Real* geo = tab + 3 * Q * N;  // NE x 24
  const long long e0 = (long long)blockIdx.x * NE;
  const int tid = threadIdx.x;
  for (int t = tid; t < Q * N; t += NT) {
    tab[t] = T.B[t] * T.B[t];
    tab[Q * N + t] = T.D[t] * T.D[t];
    tab[2 * Q * N + t] = T.B[t] * T.D[t];
  }
  if (GEOM == HX_KGEOM_ONTHEFLY) {
    trilinear_coeffs_block(A.X8, e0, A.E, NE, geo);
    __syncthreads();
  }
  // factors into shared memory: F[f][c][b][a]
  const Real alpha_r = Real(A.alpha), nu_r = Real(A.nu);
  for (int t = tid; t < NE * Q3; t += NT) {
    const int el = t / Q3, pt = t - el * Q3;
    const long long e = e0 + el;
    Real f[7] = {0, 0, 0, 0, 0, 0, 0};
    if (e < A.E) {
      if (GEOM == HX_KGEOM_STORED) {
#pragma unroll
        for (int c = 0; c < 7; ++c) f[c] = A.factors[e * A.fstride + c * Q3 + pt];
      } else {
        const int iq = pt % Q, jq = (pt / Q) % Q, kq = pt / (Q * Q);
        Real j0[3], j1[3], j2[3];
        trilinear_jacobian(geo + el * 24, T.xq[iq], T.xq[jq], T.xq[kq], j0, j1, j2);
        const Real w = T.wq[iq] * T.wq[jq] * T.wq[kq];
        const Real nu = NUF ? Real(A.nu_q[e * Q3 + pt]) : nu_r;
        point_factors(j0, j1, j2, alpha_r * w, nu * w, f);
      }
    }
    if (!(A.parts & 1)) f[0] = Real(0);  // the mass part left out
    if (!(A.parts & 2)) {               // the stiffness part left out
#pragma unroll
      for (int c = 1; c < 7; ++c) f[c] = Real(0);
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) smem[el * PER + c * Q3 + pt] = f[c];
  }
  __syncthreads();
  const Real* BB = tab;
  const Real* DD = tab + Q * N;
  const Real* BD = tab + 2 * Q * N;
  // stage 1: contract a -> X[s][c][b][i], s = (m + G00, G11, G22, G12 | BB_a or DD_a; G01, G02 | BD_a)
  for (int t = tid; t < NE * Q * Q * N; t += NT) {
    const int el = t / (Q * Q * N), r = t - el * (Q * Q * N);
    const int cb = r / N, i = r - cb * N;
    const Real* F = smem + el * PER + cb * Q;
    Real s[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const Real bb = BB[a * N + i], dd = DD[a * N + i], bd = BD[a * N + i];
      s[0] += bb * F[0 * Q3 + a] + dd * F[1 * Q3 + a];
      s[1] += bb * F[4 * Q3 + a];
      s[2] += bb * F[6 * Q3 + a];
      s[3] += bb * F[5 * Q3 + a];
      s[4] += bd * F[2 * Q3 + a];
      s[5] += bd * F[3 * Q3 + a];
    }
    Real* X = smem + el * PER + FA + cb * N + i;
#pragma unroll
    for (int f = 0; f < 6; ++f) X[f * X1] = s[f];
  }
  __syncthreads();
  // stage 2: contract b -> Y[s][c][j][i] (reusing the factor space), s = (BB_c, DD_c, 2 BD_c terms)
  for (int t = tid; t < NE * Q * N * N; t += NT) {
    const int el = t / (Q * N * N), r = t - el * (Q * N * N);
    const int c = r / (N * N), ji = r - c * (N * N);
    const int j = ji / N, i = ji - j * N;
    const Real* X = smem + el * PER + FA + c * Q * N + i;
    Real s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const Real bb = BB[b * N + j], dd = DD[b * N + j], bd = BD[b * N + j];
      const Real* src = X + b * N;
      s0 += bb * src[0 * X1] + dd * src[1 * X1] + Real(2) * bd * src[4 * X1];
      s1 += bb * src[2 * X1];
      s2 += bd * src[3 * X1] + bb * src[5 * X1];
    }
    Real* Y = smem + el * PER + c * N * N + ji;
    Y[0 * Y1] = s0;
    Y[1 * Y1] = s1;
    Y[2 * Y1] = s2;
  }
  __syncthreads();
  // stage 3: contract c -> element diagonal
  for (int t = tid; t < NE * N3; t += NT) {
    const int el = t / N3, l = t - el * N3;
    const int k = l / (N * N), ji = l - k * N * N;
    const long long e = e0 + el;
    const Real* Y = smem + el * PER + ji;
    Real s = Real(0);
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      const Real* src = Y + c * N * N;
      s += BB[c * N + k] * src[0] + DD[c * N + k] * src[Y1] + Real(2) * BD[c * N + k] * src[2 * Y1];
    }
    if (e < A.E) A.dE[hx_eline(A.lay, e, l / N, N) + l % N] = s;
  }
}

// ---------------------------------------------------------------------------
// launch configuration per order
// ---------------------------------------------------------------------------
template <int P, int Q, typename Real = double>
struct Config {
  // elements per block of the operator kernel (3 q^3 values each: ~40-75 KB per block);
  // FP32 blocks take twice the elements while the block stays within 1024 threads
  static constexpr int NE_D = P == 1 ? 64 : P == 2 ? 32 : P == 3 ? 16 : P == 4 ? 8 : P == 5 ? 6 : P == 6 ? 4 : P == 7 ? 3 : 2;
  // FP64 at p = 4 takes twice NE_D (16 elements, 576 threads, two blocks per SM): 1% faster
  // than 8 elements in a timing of 4, 8 and 16 elements per block on a 96^3 mesh
  static constexpr int NE = (sizeof(Real) == 4) ? (NE_D > 1 ? NE_D / 2 : 1) : (P == 4 ? 2 * NE_D : NE_D);
  // one thread per z-column, rounded up to whole warps
  static constexpr int NT = ((NE * Q * Q + 31) / 32) * 32;
  static_assert(NT <= 1024, "block too large");
  // resident blocks per SM the register budget is sized for (shared memory allows at least this)
  static constexpr int MINB_F = 65536 / (NT * 64) < 2 ? 2 : 65536 / (NT * 64) > 16 ? 16 : 65536 / (NT * 64);
  static constexpr int MINB = (sizeof(Real) == 4) ? MINB_F : (P >= 7) ? 3 : NT >= 512 ? 2 : NT >= 384 ? 3 : 4;
  static constexpr int NE_DIAG = P <= 2 ? 8 : P <= 4 ? 2 : 1;
};

// Block shape of the operator kernel.  FP32 with on-the-fly geometry keeps the larger blocks
// (twice the FP64 element count): its per-element map set-up amortizes better over them.
template <int P, int Q, typename Real, int GEOM>
struct ApplyConfig {
  using C = Config<P, Q, Real>;
  static constexpr bool BIG = sizeof(Real) == 4 && GEOM == HX_KGEOM_ONTHEFLY && 2 * C::NE_D * Q * Q <= 1024;
  static constexpr int NE = BIG ? 2 * C::NE_D : C::NE;
  static constexpr int NT = BIG ? ((NE * Q * Q + 31) / 32) * 32 : C::NT;
  static constexpr int MINB = BIG ? (NT >= 512 ? 2 : NT >= 384 ? 3 : 4) : C::MINB;
};

template <typename Real, int P, int Q, int GEOM, bool NUF>
cudaError_t launch_apply_impl(const HxTablesT<Real>& T, const HxApplyArgsT<Real>& A, cudaStream_t s) {
  using C = ApplyConfig<P, Q, Real, GEOM>;
  constexpr int NE = C::NE, NT = C::NT, MINB = C::MINB;
  using Lt = Layout<Q, Real>;
  constexpr bool STAGE = Lt::F32 && GEOM == HX_KGEOM_STORED && P <= 4;  // the kernel stages the factors
  // the copy rounds its start down and its end up to 16 bytes: up to 6 more words
  const size_t words = STAGE ? (size_t)((NE * Lt::R3 + 3) & ~3) + (size_t)NE * ((7 * Q * Q * Q + 3) & ~3) + 8
                             : (size_t)NE * Lt::R3 + (GEOM == HX_KGEOM_ONTHEFLY ? NE * 24 : 0);
  const size_t shmem = sizeof(Real) * words;
  auto k = apply_kernel<Real, P, Q, NE, NT, MINB, GEOM, NUF>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  if (err != cudaSuccess) return err;
  const long long blocks = (A.E + NE - 1) / NE;
  if (blocks == 0) return cudaSuccess;
  k<<<(unsigned)blocks, NT, shmem, s>>>(T, A);
  return cudaGetLastError();
}

template <int P, int Q, int GEOM, bool NUF>
cudaError_t launch_apply_multi_impl(const HxTables& T, const HxApplyArgs* args, const int* blk_op, const int* blk_first,
                                    long long blocks, cudaStream_t s) {
  using C = ApplyConfig<P, Q, double, GEOM>;
  constexpr int NE = C::NE, NT = C::NT, MINB = C::MINB;
  const size_t shmem = sizeof(double) * ((size_t)NE * Layout<Q>::R3 + (GEOM == HX_KGEOM_ONTHEFLY ? NE * 24 : 0));
  auto k = apply_multi_kernel<double, P, Q, NE, NT, MINB, GEOM, NUF>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  if (err != cudaSuccess || blocks == 0) return err;
  k<<<(unsigned)blocks, NT, shmem, s>>>(T, args, blk_op, blk_first);
  return cudaGetLastError();
}

template <int P, int Q>
cudaError_t launch_apply_multi_q(const HxTables& T, const HxApplyArgs* args, const int* blk_op, const int* blk_first,
                                 long long blocks, int geom, int nuf, cudaStream_t s) {
  if (geom == HX_KGEOM_STORED) return launch_apply_multi_impl<P, Q, HX_KGEOM_STORED, false>(T, args, blk_op, blk_first, blocks, s);
  if (nuf) return launch_apply_multi_impl<P, Q, HX_KGEOM_ONTHEFLY, true>(T, args, blk_op, blk_first, blocks, s);
  return launch_apply_multi_impl<P, Q, HX_KGEOM_ONTHEFLY, false>(T, args, blk_op, blk_first, blocks, s);
}

template <typename Real, int P, int Q>
cudaError_t launch_apply_q(const HxTablesT<Real>& T, const HxApplyArgsT<Real>& A, int geom, cudaStream_t s) {
  if (geom == HX_KGEOM_STORED) return launch_apply_impl<Real, P, Q, HX_KGEOM_STORED, false>(T, A, s);
  if (A.nu_q) return launch_apply_impl<Real, P, Q, HX_KGEOM_ONTHEFLY, true>(T, A, s);
  return launch_apply_impl<Real, P, Q, HX_KGEOM_ONTHEFLY, false>(T, A, s);
}

template <typename Real, int P, int Q, int GEOM, bool NUF>
cudaError_t launch_diag_impl(const HxTablesT<Real>& T, const HxDiagArgsT<Real>& A, cudaStream_t s) {
  constexpr int N = P + 1, NE = Config<P, Q>::NE_DIAG, NT = 128;
  constexpr int Y3 = 3 * Q * N * N;
  constexpr int FA = (7 * Q * Q * Q > Y3) ? 7 * Q * Q * Q : Y3;
  const size_t shmem = sizeof(Real) * (size_t)(NE * (FA + 6 * Q * Q * N) + 3 * Q * N + NE * 24);
  auto k = diag_kernel<Real, P, Q, NE, NT, GEOM, NUF>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  if (err != cudaSuccess) return err;
  const long long blocks = (A.E + NE - 1) / NE;
  if (blocks == 0) return cudaSuccess;
  k<<<(unsigned)blocks, NT, shmem, s>>>(T, A);
  return cudaGetLastError();
}

template <typename Real, int P, int Q>
cudaError_t launch_diag_q(const HxTablesT<Real>& T, const HxDiagArgsT<Real>& A, int geom, cudaStream_t s) {
  if (geom == HX_KGEOM_STORED) return launch_diag_impl<Real, P, Q, HX_KGEOM_STORED, false>(T, A, s);
  if (A.nu_q) return launch_diag_impl<Real, P, Q, HX_KGEOM_ONTHEFLY, true>(T, A, s);
  return launch_diag_impl<Real, P, Q, HX_KGEOM_ONTHEFLY, false>(T, A, s);
}

template <int P, int Q>
cudaError_t launch_grad_q(const HxTables& T, const HxGradArgs& A, cudaStream_t s) {
  constexpr int NE = Config<P, Q>::NE_D > 1 ? Config<P, Q>::NE_D / 2 : 1;
  constexpr int NT = ((NE * Q * Q + 31) / 32) * 32;
  const size_t shmem = sizeof(double) * (size_t)(NE * 6 * Layout<Q>::RG + NE * 24);
  auto k = grad_kernel<P, Q, NE, NT>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  if (err != cudaSuccess) return err;
  const long long blocks = (A.E + NE - 1) / NE;
  if (blocks == 0) return cudaSuccess;
  k<<<(unsigned)blocks, NT, shmem, s>>>(T, A);
  return cudaGetLastError();
}

template <int P, int Q>
cudaError_t launch_load_q(const HxTables& T, const HxLoadArgs& A, cudaStream_t s) {
  constexpr int NE = Config<P, Q>::NE, NT = Config<P, Q>::NT;
  const size_t shmem = sizeof(double) * (size_t)(NE * Layout<Q>::R3 + NE * 24);
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
    if (T.q == P + 1) return hx::launch_apply_q<double, P, P + 1>(T, A, geom, s);                         \
    if (T.q == P + 2) return hx::launch_apply_q<double, P, P + 2>(T, A, geom, s);                         \
    return cudaErrorInvalidValue;                                                                          \
  }                                                                                                        \
  cudaError_t hx_launch_apply32_p##P(const HxTablesF& T, const HxApplyArgsF& A, int geom, int kind,      \
                                     int tile, cudaStream_t s) {                                           \
    if (kind >= 3 && geom != HX_KGEOM_STORED) return cudaErrorInvalidValue;                                \
    if (T.q == P + 1)                                                                                      \
      return kind == 0   ? hx::launch_apply_q<float, P, P + 1>(T, A, geom, s)                              \
             : kind == 3 ? hx::launch_apply32_mma<P, P + 1, 1>(T, A, s)                                    \
             : kind == 4 ? hx::launch_apply32_mma<P, P + 1, 3>(T, A, s)                                    \
                         : hx::launch_apply32_q<P, P + 1>(T, A, geom, kind == 1, tile, s);                 \
    if (T.q == P + 2)                                                                                      \
      return kind == 0   ? hx::launch_apply_q<float, P, P + 2>(T, A, geom, s)                              \
             : kind == 3 ? hx::launch_apply32_mma<P, P + 2, 1>(T, A, s)                                    \
             : kind == 4 ? hx::launch_apply32_mma<P, P + 2, 3>(T, A, s)                                    \
                         : hx::launch_apply32_q<P, P + 2>(T, A, geom, kind == 1, tile, s);                 \
    return cudaErrorInvalidValue;                                                                          \
  }                                                                                                        \
  cudaError_t hx_launch_diag_p##P(const HxTables& T, const HxDiagArgs& A, int geom, cudaStream_t s) {     \
    if (T.q == P + 1) return hx::launch_diag_q<double, P, P + 1>(T, A, geom, s);                                  \
    if (T.q == P + 2) return hx::launch_diag_q<double, P, P + 2>(T, A, geom, s);                                  \
    return cudaErrorInvalidValue;                                                                          \
  }                                                                                                       \
  cudaError_t hx_launch_diag32_p##P(const HxTablesF& T, const HxDiagArgsF& A, int geom, cudaStream_t s) {     \
    if (T.q == P + 1) return hx::launch_diag_q<float, P, P + 1>(T, A, geom, s);                                  \
    if (T.q == P + 2) return hx::launch_diag_q<float, P, P + 2>(T, A, geom, s);                                  \
    return cudaErrorInvalidValue;                                                                          \
  }                                                                                                        \
  cudaError_t hx_launch_apply_multi_p##P(const HxTables& T, const HxApplyArgs* args, const int* blk_op,   \
                                         const int* blk_first, long long blocks, int geom, int nuf,       \
                                         cudaStream_t s) {                                                 \
    if (T.q == P + 1) return hx::launch_apply_multi_q<P, P + 1>(T, args, blk_op, blk_first, blocks, geom, nuf, s); \
    if (T.q == P + 2) return hx::launch_apply_multi_q<P, P + 2>(T, args, blk_op, blk_first, blocks, geom, nuf, s); \
    return cudaErrorInvalidValue;                                                                          \
  }                                                                                                        \
  int hx_apply32_block_elems_p##P(int q, int tile) {                                                      \
    return q == P + 1 ? hx::ne32_of_tile<P + 1>(tile) : hx::ne32_of_tile<P + 2>(tile);                    \
  }                                                                                                        \
  int hx_apply_block_elems_p##P(int q, int geom) {                                                         \
    if (q == P + 1)                                                                                        \
      return geom == HX_KGEOM_STORED ? hx::ApplyConfig<P, P + 1, double, HX_KGEOM_STORED>::NE              \
                                     : hx::ApplyConfig<P, P + 1, double, HX_KGEOM_ONTHEFLY>::NE;           \
    return geom == HX_KGEOM_STORED ? hx::ApplyConfig<P, P + 2, double, HX_KGEOM_STORED>::NE                \
                                   : hx::ApplyConfig<P, P + 2, double, HX_KGEOM_ONTHEFLY>::NE;             \
  }                                                                                                        \
  cudaError_t hx_launch_grad_p##P(const HxTables& T, const HxGradArgs& A, cudaStream_t s) {               \
    if (T.q == P + 1) return hx::launch_grad_q<P, P + 1>(T, A, s);                                        \
    if (T.q == P + 2) return hx::launch_grad_q<P, P + 2>(T, A, s);                                        \
    return cudaErrorInvalidValue;                                                                          \
  }                                                                                                        \
  cudaError_t hx_launch_load_p##P(const HxTables& T, const HxLoadArgs& A, cudaStream_t s) {               \
    if (T.q == P + 1) return hx::launch_load_q<P, P + 1>(T, A, s);                                        \
    if (T.q == P + 2) return hx::launch_load_q<P, P + 2>(T, A, s);                                        \
    return cudaErrorInvalidValue;                                                                          \
  }
