// Order-independent kernels: geometric factors (setup), point and node
// coordinates, the atomic-free E-to-L assembly, and the fused Jacobi-PCG
// vector kernels with deterministic reductions.
#include <cuda_runtime.h>

#include "hx_element.cuh"
#include "hx_internal.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum in a fixed order (deterministic); result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = (lane < NT / 32) ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// Last-block completion: every block writes NV partial sums to partial[v * G + block];
// the block that finishes last reduces them in a fixed order into out[v].
// Returns true in the last block (all threads), with out[] written by thread 0.
// (bid, G): the block's index among the G blocks that reduce together (a launch's whole grid, or
// one operator's share of a launch over several).
template <int NV>
__device__ bool last_block_reduce(const double (&v)[NV], double* partial, unsigned int* counter, double (&out)[NV],
                                  int bid, int G) {
  __shared__ double red[32];
  __shared__ bool is_last;
  for (int k = 0; k < NV; ++k) {
    const double s = block_sum<HX_RED_THREADS>(v[k], red);
    if (threadIdx.x == 0) partial[k * G + bid] = s;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    is_last = (ticket == (unsigned int)G - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < G; b += HX_RED_THREADS) s += __ldcg(partial + k * G + b);
    s = block_sum<HX_RED_THREADS>(s, red);
    if (threadIdx.x == 0) out[k] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

template <int NV>
__device__ bool last_block_reduce(const double (&v)[NV], double* partial, unsigned int* counter, double (&out)[NV]) {
  return last_block_reduce<NV>(v, partial, counter, out, blockIdx.x, gridDim.x);
}

// A thread's partial sum in the reduction passes of the CG.  FP64 vectors sum in FP64.  FP32
// vectors sum in FP32 with compensation (Kahan, "Further remarks on reducing truncation
// errors", 1965: the rounding error of each addition is carried to the next, so the error
// stays a few units of FP32 rounding however many terms a thread adds) and only the thread's
// result is widened to FP64: the FP64 pipe runs at 1/64 of the FP32 rate on this part, and
// widening and adding every term in FP64 made these passes FP64-bound.
template <typename Real>
struct PartialSum;
template <>
struct PartialSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double get() const { return s; }
};
template <>
struct PartialSum<float> {
  float s = 0.0f, c = 0.0f;  // c: minus the part of the terms not yet in s
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

template <int NV, typename Real>
__device__ bool last_block_reduce(const PartialSum<Real> (&v)[NV], double* partial, unsigned int* counter,
                                  double (&out)[NV], int bid, int G) {
  double d[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) d[k] = v[k].get();
  return last_block_reduce<NV>(d, partial, counter, out, bid, G);
}
template <int NV, typename Real>
__device__ bool last_block_reduce(const PartialSum<Real> (&v)[NV], double* partial, unsigned int* counter,
                                  double (&out)[NV]) {
  return last_block_reduce<NV, Real>(v, partial, counter, out, blockIdx.x, gridDim.x);
}

// 16-byte accesses of the CG vector passes (4 floats or 2 doubles): a quarter (a half) of the
// load instructions per byte, and more bytes in flight per thread.
template <typename Real>
struct Vec16 {
  static constexpr int W = 16 / (int)sizeof(Real);
};
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
__device__ __forceinline__ void ld16(float (&v)[4], const float* p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void ld16(double (&v)[2], const double* p) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  v[0] = t.x, v[1] = t.y;
}
__device__ __forceinline__ void st16(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st16(double* p, const double (&v)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// ---------------------------------------------------------------------------
// geometry setup: factors[e][c][pt], c = (m, G00, G01, G02, G11, G12, G22)
// ---------------------------------------------------------------------------
// One thread per z-column (element, iq, jq) of Gauss points: along the column dx/dxi_3 of the
// trilinear map is constant and the other two Jacobian columns are affine in xi_3, so each point
// costs two 3-vector updates instead of a full Jacobian evaluation.
__global__ void __launch_bounds__(kThreads) geometry_kernel(const __grid_constant__ HxTables T, long long E, int EB,
                                                             const double* __restrict__ X8,
                                                             const double* __restrict__ nu_q, double alpha, double nu,
                                                             double* __restrict__ factors, int* bad) {
  extern __shared__ double cf[];  // EB x 24
  const int q = T.q, Q2 = q * q, Q3 = Q2 * q;
  const long long e0 = (long long)blockIdx.x * EB;
  hx::trilinear_coeffs_block(X8, e0, E, EB, cf);
  __syncthreads();
  int nbad = 0;
  for (int t = threadIdx.x; t < EB * Q2; t += blockDim.x) {
    const int el = t / Q2, col = t - el * Q2;
    const long long e = e0 + el;
    if (e >= E) continue;
    const int iq = col % q, jq = col / q;
    const double x1 = T.xq[iq], x2 = T.xq[jq], w12 = T.wq[iq] * T.wq[jq];
    const double* a = cf + el * 24;
    double P0[3], R0[3], P1[3], R1[3], j2[3];
    for (int d = 0; d < 3; ++d) {
      const double* ad = a + d * 8;
      P0[d] = ad[1] + ad[4] * x2;
      R0[d] = ad[5] + ad[7] * x2;
      P1[d] = ad[2] + ad[4] * x1;
      R1[d] = ad[6] + ad[7] * x1;
      j2[d] = ad[3] + ad[5] * x1 + (ad[6] + ad[7] * x1) * x2;
    }
    // The rows of detJ J^-1 are the cross products c0 = j1 x j2, c1 = j2 x j0, c2 = j0 x j1
    // (G = nu w c c^T / detJ).  With j0 = P0 + z R0, j1 = P1 + z R1 and j2 fixed along the
    // column, c0 and c1 are affine in z, c2 and detJ = j0 . c0 quadratic: their coefficients are
    // formed once per column, and each point evaluates them (12 + 2 FMAs instead of two
    // Jacobian columns, nine cross-product entries and a dot product), with 1/detJ by the
    // Newton-Raphson reciprocal instead of a division.
    double A0[3], B0[3], A1[3], B1[3], C0[3], C1[3], C2[3], U[3], V[3];
    hx::cross3(P1, j2, A0);
    hx::cross3(R1, j2, B0);
    hx::cross3(j2, P0, A1);
    hx::cross3(j2, R0, B1);
    hx::cross3(P0, P1, C0);
    hx::cross3(P0, R1, U);
    hx::cross3(R0, P1, V);
    hx::cross3(R0, R1, C2);
    for (int d = 0; d < 3; ++d) C1[d] = U[d] + V[d];
    const double d0 = P0[0] * A0[0] + P0[1] * A0[1] + P0[2] * A0[2];
    const double d1 = P0[0] * B0[0] + P0[1] * B0[1] + P0[2] * B0[2] + R0[0] * A0[0] + R0[1] * A0[1] + R0[2] * A0[2];
    const double d2 = R0[0] * B0[0] + R0[1] * B0[1] + R0[2] * B0[2];
    for (int kq = 0; kq < q; ++kq) {
      const double z = T.xq[kq];
      double c0[3], c1[3], c2[3], f[7];
      for (int d = 0; d < 3; ++d) {
        c0[d] = A0[d] + z * B0[d];
        c1[d] = A1[d] + z * B1[d];
        c2[d] = C0[d] + z * (C1[d] + z * C2[d]);
      }
      const double det = d0 + z * (d1 + z * d2);
      const int pt = kq * Q2 + col;
      const double w = w12 * T.wq[kq];
      const double nuv = nu_q ? nu_q[e * Q3 + pt] : nu;
      const double s = nuv * w * hx::rcp_newton(det);
      f[0] = alpha * w * det;
      f[1] = s * (c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]);
      f[2] = s * (c0[0] * c1[0] + c0[1] * c1[1] + c0[2] * c1[2]);
      f[3] = s * (c0[0] * c2[0] + c0[1] * c2[1] + c0[2] * c2[2]);
      f[4] = s * (c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]);
      f[5] = s * (c1[0] * c2[0] + c1[1] * c2[1] + c1[2] * c2[2]);
      f[6] = s * (c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2]);
      if (!(det > 0.0)) ++nbad;
      for (int c = 0; c < 7; ++c) factors[(e * 7 + c) * Q3 + pt] = f[c];
    }
  }
  if (nbad) atomicAdd(bad, nbad);
}

__global__ void __launch_bounds__(kThreads) qpoint_kernel(const __grid_constant__ HxTables T, long long E, int EB,
                                                           const double* __restrict__ X8, double* __restrict__ xyz) {
  extern __shared__ double cf[];
  const int q = T.q, Q3 = q * q * q;
  const long long e0 = (long long)blockIdx.x * EB;
  hx::trilinear_coeffs_block(X8, e0, E, EB, cf);
  __syncthreads();
  for (int t = threadIdx.x; t < EB * Q3 * 3; t += blockDim.x) {
    const int el = t / (Q3 * 3), r = t - el * Q3 * 3;
    const int pt = r / 3, d = r - pt * 3;
    const long long e = e0 + el;
    if (e >= E) continue;
    const int iq = pt % q, jq = (pt / q) % q, kq = pt / (q * q);
    xyz[(e * Q3) * 3 + r] = hx::trilinear_point(cf + el * 24, d, T.xq[iq], T.xq[jq], T.xq[kq]);
  }
}

__global__ void __launch_bounds__(kThreads) node_kernel(const __grid_constant__ HxTables T, long long n_dof,
                                                         const int* __restrict__ off, const int* __restrict__ idx,
                                                         const double* __restrict__ X8, double* __restrict__ xyz) {
  const int n = T.p + 1, N3 = n * n * n;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n_dof; g += (long long)gridDim.x * blockDim.x) {
    const int v = idx[off[g]];  // first (element, node) holding g: deterministic owner
    const long long e = v / N3;
    const int l = v - (int)(e * N3);
    const int i = l % n, j = (l / n) % n, k = l / (n * n);
    double x8[24], cf[24];
    for (int c = 0; c < 24; ++c) x8[c] = X8[e * 24 + c];
    hx::trilinear_coeffs(x8, cf);
    for (int d = 0; d < 3; ++d) xyz[g * 3 + d] = hx::trilinear_point(cf, d, T.xn[i], T.xn[j], T.xn[k]);
  }
}

// Collocated mass at the local nodes (Sec. 5.1): the mass form integrated with the
// Gauss-Lobatto rule at the nodes of the nodal basis is diagonal,
//   dE[e][l] = alpha w_a w_b w_c detJ_e(xi_l),   l = (a, b, c).
__global__ void __launch_bounds__(kThreads) cmass_kernel(const __grid_constant__ HxTables T, long long E, int EB,
                                                          const double* __restrict__ X8, double alpha,
                                                          double* __restrict__ dE, const HxELayout lay) {
  extern __shared__ double cf[];
  const int n = T.p + 1, N3 = n * n * n;
  const long long e0 = (long long)blockIdx.x * EB;
  hx::trilinear_coeffs_block(X8, e0, E, EB, cf);
  __syncthreads();
  for (int t = threadIdx.x; t < EB * N3; t += blockDim.x) {
    const int el = t / N3, l = t - el * N3;
    const long long e = e0 + el;
    if (e >= E) continue;
    const int a = l % n, b = (l / n) % n, c = l / (n * n);
    double j0[3], j1[3], j2[3];
    hx::trilinear_jacobian(cf + el * 24, T.xn[a], T.xn[b], T.xn[c], j0, j1, j2);
    const double det = j0[0] * (j1[1] * j2[2] - j1[2] * j2[1]) + j0[1] * (j1[2] * j2[0] - j1[0] * j2[2]) +
                       j0[2] * (j1[0] * j2[1] - j1[1] * j2[0]);
    dE[hx_eline(lay, e, b + n * c, n) + a] = alpha * T.wn[a] * T.wn[b] * T.wn[c] * det;
  }
}

// ---------------------------------------------------------------------------
// E -> L assembly through the transpose map (atomic-free, fixed summation order)
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ Real gather_sum(long long g, const int* __restrict__ off, const int* __restrict__ idx,
                                           const Real* __restrict__ yE) {
  const int k0 = __ldg(off + g), k1 = __ldg(off + g + 1);
  Real s = Real(0);
  for (int k = k0; k < k1; ++k) s += __ldg(yE + __ldg(idx + k));
  return s;
}

// The same sums for a box mesh, its element entries found by index arithmetic, one x-run of
// nodes per thread.  Along each axis a node interior to an element row belongs to one element, a
// node between two elements to both (the lower one with local index p, the upper with 0).  Run
// t = ex + nx line (line = J + gy K, one DoF x-line) holds the nodes I = ex p + 1 .. ex p + p, and
// the run with ex = 0 also node I = 0: consecutive runs hold consecutive DoFs.  A node's entries
// are summed with the element index increasing (z, then y, then x outermost to innermost), the
// order of the transpose map.  The E-vector is in the line layout (rows of nx elements): entry
// (lx, ly, lz) of element (ex, ey, ez) at ((ey + ny ez) n^2 + ly + n lz) (nx n) + ex n + lx, so a
// run's entries for one (y, z) pair are n + 1 consecutive values.
__device__ __forceinline__ int fast_div(int n, unsigned m, int s) {
  return (int)(((unsigned long long)(unsigned)n * m) >> s);
}

// the elements (e) and local indices (l) of node X along an axis with ne elements; returns 1 or 2
__device__ __forceinline__ int grid_axis(int X, int ne, const HxGridAsm& G, int* e, int* l) {
  const int p = G.p, q = fast_div(X, G.mp, G.sp), r = X - q * p;
  if (r == 0 && q > 0 && q < ne) {  // between elements q - 1 and q
    e[0] = q - 1;
    l[0] = p;
    e[1] = q;
    l[1] = 0;
    return 2;
  }
  e[0] = q < ne ? q : ne - 1;
  l[0] = q < ne ? r : p;
  return 1;
}

__host__ __device__ __forceinline__ long long grid_runs(const HxGridAsm& G) {
  return (long long)G.nx * G.gy * ((long long)G.p * G.nz + 1);
}

// s[i] = the assembled entry of node ex p + i of run t (i >= *i0); returns the DoF of node ex p.
template <int P, typename Real>
__device__ __forceinline__ long long gather_run_grid(int t, const HxGridAsm& G, const Real* __restrict__ yE,
                                                     Real (&s)[P + 1], int* i0) {
  constexpr int n = P + 1;
  const int line = fast_div(t, G.mnx, G.snx), ex = t - line * G.nx;
  const int K = fast_div(line, G.mgy, G.sgy), J = line - K * G.gy;
  int ey[2], ly[2], ez[2], lz[2];
  const int cy = grid_axis(J, G.ny, G, ey, ly), cz = grid_axis(K, G.nz, G, ez, lz);
  const bool first = ex == 0, right = ex + 1 < G.nx;
  const long long xl = (long long)G.nx * n;  // one x-line of a row of elements
#pragma unroll
  for (int i = 0; i <= P; ++i) s[i] = Real(0);
  for (int a = 0; a < cz; ++a)
    for (int b = 0; b < cy; ++b) {
      const Real* L = yE + ((long long)(ey[b] + G.ny * ez[a]) * (n * n) + ly[b] + n * lz[a]) * xl + (long long)ex * n;
      if (first) s[0] += __ldg(L);
#pragma unroll
      for (int i = 1; i <= P; ++i) s[i] += __ldg(L + i);
      if (right) s[P] += __ldg(L + n);  // element ex + 1, local index 0
    }
  *i0 = first ? 0 : 1;
  return (long long)line * G.gx + (long long)ex * P;
}

#define HX_GRID_STRIDE(g, n) \
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < (n); g += (long long)gridDim.x * blockDim.x)
// the same over a virtual grid of nb blocks, this one being block bid
#define HX_VGRID_STRIDE(g, n, bid, nb) \
  for (long long g = (bid) * (long long)blockDim.x + threadIdx.x; g < (n); g += (long long)(nb) * blockDim.x)

template <typename Real>
__global__ void __launch_bounds__(kThreads) assemble_kernel(long long n, const HxGridAsm ga, const int* __restrict__ off,
                                                             const int* __restrict__ idx, const Real* __restrict__ yE,
                                                             const unsigned char* __restrict__ dir, int constrained,
                                                             const Real* __restrict__ x, double dir_const,
                                                             Real* __restrict__ y) {
  HX_GRID_STRIDE(g, n) {
    Real s;
    if (constrained && dir[g]) s = x ? x[g] : Real(dir_const);
    else s = gather_sum(g, off, idx, yE);
    y[g] = s;
  }
}

// the same for a box mesh, one x-run per thread
template <int P, typename Real>
__global__ void __launch_bounds__(kThreads) assemble_grid_kernel(long long runs, const HxGridAsm ga,
                                                                  const Real* __restrict__ yE,
                                                                  const unsigned char* __restrict__ dir,
                                                                  int constrained, const Real* __restrict__ x,
                                                                  double dir_const, Real* __restrict__ y) {
  HX_GRID_STRIDE(t, runs) {
    Real s[P + 1];
    int i0;
    const long long g0 = gather_run_grid<P>((int)t, ga, yE, s, &i0);
#pragma unroll
    for (int i = 0; i <= P; ++i) {
      if (i < i0) continue;
      const long long g = g0 + i;
      Real v = s[i];
      if (constrained && dir[g]) v = x ? x[g] : Real(dir_const);
      y[g] = v;
    }
  }
}

__global__ void __launch_bounds__(kThreads) dinv_kernel(long long n, const double* __restrict__ diag,
                                                         const unsigned char* __restrict__ dir, double* __restrict__ dinv) {
  HX_GRID_STRIDE(g, n) { dinv[g] = dir[g] ? 1.0 : 1.0 / diag[g]; }
}

__global__ void __launch_bounds__(kThreads) masked_copy_kernel(long long n, const double* __restrict__ src,
                                                                const unsigned char* __restrict__ dir, int constrained,
                                                                double value, double* __restrict__ dst) {
  HX_GRID_STRIDE(g, n) { dst[g] = (constrained && dir[g]) ? value : src[g]; }
}

// ---------------------------------------------------------------------------
// Jacobi-PCG (Sec. 5.3: CG on the SPD Helmholtz / Poisson systems), fused passes.
// Vectors in Real (double: the FP64 solver; float: the inner solver of the
// mixed-precision refinement); every reduction accumulates in double.
// ---------------------------------------------------------------------------
// x = P x0 (or 0), r = P b; sums ||P b||^2.
template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_init_kernel(HxCgBuffersT<Real> B, const Real* __restrict__ b,
                                                                  const Real* __restrict__ x0, double rtol, int max_it) {
  PartialSum<Real> acc[1];
  HX_GRID_STRIDE(g, B.n) {
    const bool d = B.dir[g];
    const Real bg = d ? Real(0) : (B.nullspace ? Real((double)b[g] - B.st->shift) : b[g]);
    B.r[g] = bg;
    B.x[g] = (x0 && !d) ? x0[g] : Real(0);
    acc[0].add(bg * bg);
  }
  double out[1];
  if (last_block_reduce<1>(acc, B.partial, &B.st->count[0], out) && threadIdx.x == 0) {
    HxCgState* s = B.st;
    s->bb = out[0];
    s->tol2 = rtol * rtol * out[0];
    s->iter = 0;
    s->max_it = max_it;
    s->done = 0;
    s->loops = 0;
    s->zmean = 0.0;
    s->status = 0;
    s->rz = s->alpha = s->beta = 0.0;
    s->rr = out[0];
  }
}

// r -= A_c x (after an apply of the initial guess into Ap).
template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_residual_kernel(HxCgBuffersT<Real> B) {
  HX_GRID_STRIDE(g, B.n) { B.r[g] -= B.Ap[g]; }
}

// z = D^-1 r, p = z; rz = (r, z), rr = (r, r); finishes at once if rr <= tol^2 ||b||^2, or
// as not converged if the iteration cap is 0.
// Null-space mode also sums z and r: the preconditioned residual is orthogonalized against
// the constants (z - mean z, Sec. 5.3) and p is finished by a direction pass with beta = 0.
template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_start_kernel(HxCgBuffersT<Real> B) {
  PartialSum<Real> acc[4];
  HX_GRID_STRIDE(g, B.n) {
    const Real r = B.r[g], z = B.z ? B.z[g] : B.dinv[g] * r;
    B.p[g] = z;
    acc[0].add(r * z);
    acc[1].add(r * r);
    acc[2].add(z);
    acc[3].add(r);
  }
  double out[4];
  if (last_block_reduce<4>(acc, B.partial, &B.st->count[1], out) && threadIdx.x == 0) {
    HxCgState* s = B.st;
    double rz = out[0];
    if (B.nullspace) {
      s->zmean = out[2] / (double)B.n;
      rz -= s->zmean * out[3];
      s->beta = 0.0;
    }
    s->rz = rz;
    s->rr = out[1];
    if (!isfinite(rz) || !isfinite(out[1])) {
      s->status = -6;  // HX_ERR_BREAKDOWN
      s->done = 1;
    } else if (out[1] <= s->tol2) {
      s->done = 1;
    } else if (s->max_it <= 0) {
      s->status = -5;  // HX_ERR_NOT_CONVERGED: no iteration allowed
      s->done = 1;
    }
  }
}

// st->shift = mean of v over all DoFs.
template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_mean_kernel(HxCgBuffersT<Real> B, const Real* __restrict__ v) {
  PartialSum<Real> acc[1];
  HX_GRID_STRIDE(g, B.n) { acc[0].add(v[g]); }
  double out[1];
  if (last_block_reduce<1>(acc, B.partial, &B.st->count[0], out) && threadIdx.x == 0) B.st->shift = out[0] / (double)B.n;
}

// The assembly of the pass for a box mesh, one x-run per thread; returns the thread's part of pAp.
template <int P, typename Real>
__device__ __forceinline__ PartialSum<Real> assemble_pap_runs(const HxCgBuffersT<Real>& B, int bid, int nb) {
  PartialSum<Real> acc;
  auto finish = [&](long long g0, const Real(&s)[P + 1], int i0) {
#pragma unroll
    for (int i = 0; i <= P; ++i) {
      if (i < i0) continue;
      const long long g = g0 + i;
      const Real pg = B.p[g];
      const Real ap = B.dir[g] ? pg : s[i];
      B.Ap[g] = ap;
      acc.add(pg * ap);
    }
  };
  HX_VGRID_STRIDE(t, grid_runs(B.ga), bid, nb) {
    Real s[P + 1];
    int i0;
    const long long g0 = gather_run_grid<P>((int)t, B.ga, B.yE, s, &i0);
    finish(g0, s, i0);
  }
  return acc;
}

// Ap = assemble(yE) with Dirichlet rows Ap = p; pAp = (p, Ap); alpha = rz / pAp.
// PG > 0: a box mesh of order PG (compile-time, so each order gets its own registers);
// PG = 0: the order read from the buffers (the lock-step kernels over several operators).
template <int PG, typename Real>
__device__ __forceinline__ void cg_assemble_pap_body(const HxCgBuffersT<Real>& B, int bid, int nb) {
  if (*(volatile int*)&B.st->done) return;
  PartialSum<Real> acc[1];
  if constexpr (PG > 0) acc[0] = assemble_pap_runs<PG>(B, bid, nb);
  else switch (B.ga.p) {
    case 0:
      HX_VGRID_STRIDE(g, B.n, bid, nb) {
        const Real pg = B.p[g];
        const Real ap = B.dir[g] ? pg : gather_sum(g, B.off, B.idx, B.yE);
        B.Ap[g] = ap;
        acc[0].add(pg * ap);
      }
      break;
    case 1: acc[0] = assemble_pap_runs<1>(B, bid, nb); break;
    case 2: acc[0] = assemble_pap_runs<2>(B, bid, nb); break;
    case 3: acc[0] = assemble_pap_runs<3>(B, bid, nb); break;
    case 4: acc[0] = assemble_pap_runs<4>(B, bid, nb); break;
    case 5: acc[0] = assemble_pap_runs<5>(B, bid, nb); break;
    case 6: acc[0] = assemble_pap_runs<6>(B, bid, nb); break;
    case 7: acc[0] = assemble_pap_runs<7>(B, bid, nb); break;
    default: acc[0] = assemble_pap_runs<8>(B, bid, nb); break;
  }
  double out[1];
  if (last_block_reduce<1>(acc, B.partial, &B.st->count[2], out, bid, nb) && threadIdx.x == 0) {
    HxCgState* s = B.st;
    if (!(out[0] > 0.0) || !isfinite(out[0])) {
      s->status = -6;  // HX_ERR_BREAKDOWN
      s->done = 1;
    } else {
      s->alpha = s->rz / out[0];
    }
  }
}

template <int PG, typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_assemble_pap_kernel(HxCgBuffersT<Real> B) {
  cg_assemble_pap_body<PG>(B, blockIdx.x, gridDim.x);
}

// x += alpha p, r -= alpha Ap, z = D^-1 r; rr = (r, r), rz' = (r, z); convergence test.
// Null-space mode: rz' = (r, z - mean z) and the mean is kept for the direction pass.
template <typename Real>
__device__ __forceinline__ void cg_update_body(const HxCgBuffersT<Real>& B, int bid, int nb) {
  if (*(volatile int*)&B.st->done) return;
  const Real a = Real(B.st->alpha);
  PartialSum<Real> acc[4];
  auto step = [&](Real pg, Real& xg, Real& rg, Real ag, Real dg) {
    xg += a * pg;
    const Real r = rg - a * ag;
    rg = r;
    acc[0].add(r * r);
    if (!B.z) {
      const Real z = dg * r;
      acc[1].add(r * z);
      if (B.nullspace) {  // the sums of z and r only serve the null-space projection
        acc[2].add(z);
        acc[3].add(r);
      }
    }
  };
  // 16-byte chunks over a virtual grid, then the n mod W tail entry by entry
  constexpr int W = Vec16<Real>::W;
  const bool vec = aligned16(B.x) && aligned16(B.r) && aligned16(B.p) && aligned16(B.Ap) && (B.z || aligned16(B.dinv));
  const long long nv = vec ? B.n / W : 0;
  HX_VGRID_STRIDE(v, nv, bid, nb) {
    const long long g = v * W;
    Real pv[W], xv[W], rv[W], av[W], dv[W];
    ld16(pv, B.p + g);
    ld16(xv, B.x + g);
    ld16(rv, B.r + g);
    ld16(av, B.Ap + g);
    if (!B.z) ld16(dv, B.dinv + g);
#pragma unroll
    for (int k = 0; k < W; ++k) step(pv[k], xv[k], rv[k], av[k], B.z ? Real(0) : dv[k]);
    st16(B.x + g, xv);
    st16(B.r + g, rv);
  }
  for (long long g = nv * W + (long long)bid * blockDim.x + threadIdx.x; g < B.n; g += (long long)nb * blockDim.x) {
    Real xg = B.x[g], rg = B.r[g];
    step(B.p[g], xg, rg, B.Ap[g], B.z ? Real(0) : B.dinv[g]);
    B.x[g] = xg;
    B.r[g] = rg;
  }
  double out[4];
  if (last_block_reduce<4>(acc, B.partial, &B.st->count[3], out, bid, nb) && threadIdx.x == 0) {
    HxCgState* s = B.st;
    s->iter += 1;
    s->rr = out[0];
    double rz = out[1];
    if (B.nullspace) {
      s->zmean = out[2] / (double)B.n;
      rz -= s->zmean * out[3];
    }
    if (!isfinite(out[0]) || !isfinite(rz)) {
      s->status = -6;
      s->done = 1;
    } else if (out[0] <= s->tol2) {
      s->done = 1;
    } else if (s->iter >= s->max_it) {
      s->status = -5;  // HX_ERR_NOT_CONVERGED
      s->done = 1;
    } else if (!B.z) {
      s->beta = rz / s->rz;
      s->rz = rz;
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_update_kernel(HxCgBuffersT<Real> B) {
  cg_update_body(B, blockIdx.x, gridDim.x);
}

// Preconditioner given as a vector z = M^-1 r (computed between the update and the direction
// passes): rz' = (r, z) (null-space mode: (r, z - mean z)), beta = rz' / rz.
template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_rz_kernel(HxCgBuffersT<Real> B) {
  if (*(volatile int*)&B.st->done) return;
  PartialSum<Real> acc[3];
  HX_GRID_STRIDE(g, B.n) {
    const Real r = B.r[g], z = B.z[g];
    acc[0].add(r * z);
    acc[1].add(z);
    acc[2].add(r);
  }
  double out[3];
  if (last_block_reduce<3>(acc, B.partial, &B.st->count[1], out) && threadIdx.x == 0) {
    HxCgState* s = B.st;
    double rz = out[0];
    if (B.nullspace) {
      s->zmean = out[1] / (double)B.n;
      rz -= s->zmean * out[2];
    }
    if (!isfinite(rz)) {
      s->status = -6;
      s->done = 1;
    } else {
      s->beta = rz / s->rz;
      s->rz = rz;
    }
  }
}

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// p = D^-1 r + beta p.
template <typename Real>
__device__ __forceinline__ void cg_direction_body(const HxCgBuffersT<Real>& B, int bid, int nb) {
  if (*(volatile int*)&B.st->done) return;
  const Real beta = Real(B.st->beta), zm = Real(B.st->zmean);
  // every rounding spelled out (a product rounded on its own, then one fused multiply-add), so
  // that the solo and the lock-step kernels, which both inline this, round alike
  auto dir = [&](Real pg, Real rg, Real dg, Real zg) -> Real {
    const Real z = B.z ? zg : mul_rn(dg, rg);
    return fma(beta, pg, z - zm);
  };
  constexpr int W = Vec16<Real>::W;
  const bool vec = aligned16(B.p) && (B.z ? aligned16(B.z) : (aligned16(B.r) && aligned16(B.dinv)));
  const long long nv = vec ? B.n / W : 0;
  HX_VGRID_STRIDE(v, nv, bid, nb) {
    const long long g = v * W;
    Real pv[W], rv[W], dv[W], zv[W];
    ld16(pv, B.p + g);
    if (B.z) {
      ld16(zv, B.z + g);
    } else {
      ld16(rv, B.r + g);
      ld16(dv, B.dinv + g);
    }
#pragma unroll
    for (int k = 0; k < W; ++k)
      pv[k] = B.z ? dir(pv[k], Real(0), Real(0), zv[k]) : dir(pv[k], rv[k], dv[k], Real(0));
    st16(B.p + g, pv);
  }
  for (long long g = nv * W + (long long)bid * blockDim.x + threadIdx.x; g < B.n; g += (long long)nb * blockDim.x)
    B.p[g] = B.z ? dir(B.p[g], Real(0), Real(0), B.z[g]) : dir(B.p[g], B.r[g], B.dinv[g], Real(0));
}

template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_direction_kernel(HxCgBuffersT<Real> B) {
  if (B.cond != 0ull && blockIdx.x == 0 && threadIdx.x == 0) {
    // last kernel of a CUDA-graph while-loop body: continue only while CG runs, and never
    // for more bodies than the iteration cap allows
    HxCgState* s = B.st;
    s->loops += 1;
    const bool stop = *(volatile int*)&s->done || s->loops > s->max_it + 1;
    cudaGraphSetConditional((cudaGraphConditionalHandle)B.cond, stop ? 0u : 1u);
  }
  cg_direction_body(B, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// lock-step CG iterations of several operators (a batch): one launch per pass over all of them.
// Block b works on share b - blk_first[o] of the blk_count[o] blocks given to operator
// o = blk_op[b], with that operator's buffers (the reductions finish per operator).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_assemble_pap_multi_kernel(const HxCgBuffersT<Real>* bufs,
                                                                                const int* __restrict__ blk_op,
                                                                                const int* __restrict__ blk_first,
                                                                                const int* __restrict__ blk_count) {
  const int o = __ldg(blk_op + blockIdx.x);
  const HxCgBuffersT<Real> B = bufs[o];
  cg_assemble_pap_body<0>(B, blockIdx.x - __ldg(blk_first + o), __ldg(blk_count + o));
}

template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_update_multi_kernel(const HxCgBuffersT<Real>* bufs,
                                                                          const int* __restrict__ blk_op,
                                                                          const int* __restrict__ blk_first,
                                                                          const int* __restrict__ blk_count) {
  const int o = __ldg(blk_op + blockIdx.x);
  const HxCgBuffersT<Real> B = bufs[o];
  cg_update_body(B, blockIdx.x - __ldg(blk_first + o), __ldg(blk_count + o));
}

template <typename Real>
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) cg_direction_multi_kernel(const HxCgBuffersT<Real>* bufs,
                                                                             const int* __restrict__ blk_op,
                                                                             const int* __restrict__ blk_first,
                                                                             const int* __restrict__ blk_count) {
  const int o = __ldg(blk_op + blockIdx.x);
  const HxCgBuffersT<Real> B = bufs[o];
  cg_direction_body(B, blockIdx.x - __ldg(blk_first + o), __ldg(blk_count + o));
}

// Last kernel of the lock-step while-loop body: every unfinished operator counts one more body;
// the loop continues while one of them runs and has not used up its cap of max_it + 1 bodies.
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) batch_condition_kernel(HxCgState* const* states, int n,
                                                                          unsigned long long cond) {
  __shared__ int live;
  if (threadIdx.x == 0) live = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    HxCgState* s = states[i];
    if (!*(volatile int*)&s->done) {
      s->loops += 1;
      if (s->loops <= s->max_it + 1) atomicOr(&live, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, live ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// mixed-precision iterative refinement (FP64 outer residual, FP32 inner CG)
// ---------------------------------------------------------------------------
// r = P b - Ax (FP64), out = ||r||^2.
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) ir_residual_kernel(long long n, const double* __restrict__ b,
                                                                      const double* __restrict__ Ax,
                                                                      const unsigned char* __restrict__ dir,
                                                                      double* __restrict__ r, double* partial,
                                                                      unsigned int* counter, double* out,
                                                                      const double* __restrict__ shift) {
  const double sh = shift ? *shift : 0.0;
  double acc[1] = {0.0};
  HX_GRID_STRIDE(g, n) {
    const double v = dir[g] ? 0.0 : (b[g] - sh) - Ax[g];
    r[g] = v;
    acc[0] += v * v;
  }
  double res[1];
  if (last_block_reduce<1>(acc, partial, counter, res) && threadIdx.x == 0) *out = res[0];
}

// r32 = r / ||r|| rounded to FP32 (||r||^2 read from the device).
__global__ void __launch_bounds__(kThreads) ir_scale_down_kernel(long long n, const double* __restrict__ r,
                                                                  const double* __restrict__ rn2, float* __restrict__ r32) {
  const double inv = (*rn2 > 0.0) ? 1.0 / sqrt(*rn2) : 0.0;
  HX_GRID_STRIDE(g, n) { r32[g] = (float)(r[g] * inv); }
}

// x += ||r|| d (FP64 accumulation of the FP32 correction).
__global__ void __launch_bounds__(kThreads) ir_update_kernel(long long n, double* __restrict__ x,
                                                              const float* __restrict__ d, const double* __restrict__ rn2) {
  const double s = sqrt(*rn2);
  HX_GRID_STRIDE(g, n) { x[g] += s * (double)d[g]; }
}

__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) sum_kernel(long long n, const double* __restrict__ v, double* partial,
                                                              unsigned int* counter, double* out) {
  double acc[1] = {0.0};
  HX_GRID_STRIDE(g, n) { acc[0] += v[g]; }
  double res[1];
  if (last_block_reduce<1>(acc, partial, counter, res) && threadIdx.x == 0) *out = res[0];
}

__global__ void __launch_bounds__(kThreads) shift_kernel(long long n, double* __restrict__ x, const double* __restrict__ num,
                                                          const double* __restrict__ den) {
  const double c = *num / *den;
  HX_GRID_STRIDE(g, n) { x[g] -= c; }
}

__global__ void __launch_bounds__(kThreads) to_float_kernel(long long n, const double* __restrict__ a,
                                                             float* __restrict__ b) {
  HX_GRID_STRIDE(g, n) { b[g] = (float)a[g]; }
}

__global__ void __launch_bounds__(kThreads) to_float_strided_kernel(long long E, int per, int stride,
                                                                     const double* __restrict__ a,
                                                                     float* __restrict__ b) {
  HX_GRID_STRIDE(g, E * stride) {
    const long long e = g / stride;
    const int k = (int)(g - e * stride);
    b[g] = (k < per) ? (float)a[e * per + k] : 0.0f;
  }
}

__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) dot_kernel(long long n, const double* __restrict__ a,
                                                              const double* __restrict__ c, double* partial,
                                                              unsigned int* counter, double* out) {
  double acc[1] = {0.0};
  HX_GRID_STRIDE(g, n) { acc[0] += a[g] * c[g]; }
  double res[1];
  if (last_block_reduce<1>(acc, partial, counter, res) && threadIdx.x == 0) *out = res[0];
}

// out = sum_g (dir[g] ? 0 : b[g] - Ax[g])^2
__global__ void __launch_bounds__(HX_RED_THREADS, HX_RED_MINB) resnorm_kernel(long long n, const double* __restrict__ b,
                                                                  const double* __restrict__ Ax,
                                                                  const unsigned char* __restrict__ dir,
                                                                  double* partial, unsigned int* counter, double* out,
                                                                  const double* __restrict__ shift) {
  const double sh = shift ? *shift : 0.0;
  double acc[1] = {0.0};
  HX_GRID_STRIDE(g, n) {
    const double r = dir[g] ? 0.0 : (b[g] - sh) - Ax[g];
    acc[0] += r * r;
  }
  double res[1];
  if (last_block_reduce<1>(acc, partial, counter, res) && threadIdx.x == 0) *out = res[0];
}

unsigned grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 148LL * 16) b = 148LL * 16;
  return (unsigned)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t hx_launch_geometry(const HxTables& T, long long E, const double* X8, const double* nu_q, double alpha,
                               double nu, double* factors, int* bad, cudaStream_t s) {
  const int Q2 = T.q * T.q;
  const int EB = Q2 >= kThreads ? 1 : kThreads / Q2;  // one thread per z-column
  const long long blocks = (E + EB - 1) / EB;
  if (blocks == 0) return cudaSuccess;
  geometry_kernel<<<(unsigned)blocks, kThreads, EB * 24 * sizeof(double), s>>>(T, E, EB, X8, nu_q, alpha, nu, factors, bad);
  return cudaGetLastError();
}

cudaError_t hx_launch_qpoint_coords(const HxTables& T, long long E, const double* X8, double* xyz, cudaStream_t s) {
  const int Q3 = T.q * T.q * T.q;
  const int EB = Q3 >= 1024 ? 1 : 1024 / Q3;
  const long long blocks = (E + EB - 1) / EB;
  if (blocks == 0) return cudaSuccess;
  qpoint_kernel<<<(unsigned)blocks, kThreads, EB * 24 * sizeof(double), s>>>(T, E, EB, X8, xyz);
  return cudaGetLastError();
}

cudaError_t hx_launch_node_coords(const HxTables& T, long long n_dof, const int* off, const int* idx, const double* X8,
                                  double* xyz, cudaStream_t s) {
  node_kernel<<<grid_for(n_dof), kThreads, 0, s>>>(T, n_dof, off, idx, X8, xyz);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_assemble(long long n, const HxGridAsm& ga, const int* off, const int* idx, const Real* yE,
                            const unsigned char* dir, int constrained, const Real* x, double dir_const, Real* y,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (ga.p == 0) {
    assemble_kernel<Real><<<grid_for(n), kThreads, 0, s>>>(n, ga, off, idx, yE, dir, constrained, x, dir_const, y);
    return cudaGetLastError();
  }
  const long long runs = grid_runs(ga);
  const unsigned gb = grid_for(runs);
  switch (ga.p) {
#define HX_ASM_CASE(P)                                                                                     \
  case P:                                                                                                  \
    assemble_grid_kernel<P, Real><<<gb, kThreads, 0, s>>>(runs, ga, yE, dir, constrained, x, dir_const, y); \
    break;
    HX_ASM_CASE(1)
    HX_ASM_CASE(2)
    HX_ASM_CASE(3)
    HX_ASM_CASE(4)
    HX_ASM_CASE(5)
    HX_ASM_CASE(6)
    HX_ASM_CASE(7)
    HX_ASM_CASE(8)
#undef HX_ASM_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t hx_launch_assemble(long long n, const HxGridAsm& ga, const int* off, const int* idx, const double* yE,
                               const unsigned char* dir,
                               int constrained, const double* x, double dir_const, double* y, cudaStream_t s) {
  return launch_assemble<double>(n, ga, off, idx, yE, dir, constrained, x, dir_const, y, s);
}

cudaError_t hx_launch_assemble32(long long n, const HxGridAsm& ga, const int* off, const int* idx, const float* yE,
                                 const unsigned char* dir,
                                 int constrained, const float* x, float* y, cudaStream_t s) {
  return launch_assemble<float>(n, ga, off, idx, yE, dir, constrained, x, 0.0, y, s);
}

// Stored factors after a change of constant coefficients (one warp per (element, component)
// row of q^3 points, so that the loads and stores are coalesced): m *= ra, G *= rk.
__global__ void __launch_bounds__(kThreads) scale_factors_kernel(long long rows, int Q3, double ra, double rk,
                                                                  double* __restrict__ f) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < rows; row += warps) {
    const double r = (row % 7 == 0) ? ra : rk;
    double* p = f + row * Q3;
    for (int i = lane; i < Q3; i += 32) p[i] *= r;
  }
}

template <typename Real>
__global__ void __launch_bounds__(kThreads) axpby_kernel(long long n, Real ra, const Real* __restrict__ a, Real rk,
                                                          const Real* __restrict__ b, Real* __restrict__ out) {
  HX_GRID_STRIDE(g, n) { out[g] = ra * a[g] + rk * b[g]; }
}

cudaError_t hx_launch_scale_factors(long long E, int Q3, double ra, double rk, double* factors, cudaStream_t s) {
  const long long rows = 7 * E;
  if (rows == 0) return cudaSuccess;
  long long b = (rows * 32 + kThreads - 1) / kThreads;
  if (b > 148LL * 16) b = 148LL * 16;
  scale_factors_kernel<<<(unsigned)b, kThreads, 0, s>>>(rows, Q3, ra, rk, factors);
  return cudaGetLastError();
}

cudaError_t hx_launch_axpby(long long n, double ra, const double* a, double rk, const double* b, double* out,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  axpby_kernel<double><<<grid_for(n), kThreads, 0, s>>>(n, ra, a, rk, b, out);
  return cudaGetLastError();
}

cudaError_t hx_launch_axpby32(long long n, float ra, const float* a, float rk, const float* b, float* out,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  axpby_kernel<float><<<grid_for(n), kThreads, 0, s>>>(n, ra, a, rk, b, out);
  return cudaGetLastError();
}

cudaError_t hx_launch_cmass(const HxTables& T, long long E, const double* X8, double alpha, double* dE,
                            const HxELayout& lay, cudaStream_t s) {
  const int EB = 8;
  const long long blocks = (E + EB - 1) / EB;
  if (blocks == 0) return cudaSuccess;
  cmass_kernel<<<(unsigned)blocks, kThreads, sizeof(double) * 24 * EB, s>>>(T, E, EB, X8, alpha, dE, lay);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kThreads) scale_kernel(long long n, const double* __restrict__ d,
                                                          const double* __restrict__ r, double* __restrict__ z) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x)
    z[g] = d[g] * r[g];
}

cudaError_t hx_launch_scale(long long n, const double* d, const double* r, double* z, cudaStream_t s) {
  scale_kernel<<<grid_for(n), kThreads, 0, s>>>(n, d, r, z);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kThreads) dinv32_kernel(long long n, const float* __restrict__ diag,
                                                           const unsigned char* __restrict__ dir, float* __restrict__ dinv) {
  HX_GRID_STRIDE(g, n) { dinv[g] = dir[g] ? 1.0f : 1.0f / diag[g]; }
}

cudaError_t hx_launch_dinv32(long long n, const float* diag, const unsigned char* dir, float* dinv, cudaStream_t s) {
  dinv32_kernel<<<grid_for(n), kThreads, 0, s>>>(n, diag, dir, dinv);
  return cudaGetLastError();
}

cudaError_t hx_launch_dinv(long long n, const double* diag, const unsigned char* dir, double* dinv, cudaStream_t s) {
  dinv_kernel<<<grid_for(n), kThreads, 0, s>>>(n, diag, dir, dinv);
  return cudaGetLastError();
}

cudaError_t hx_launch_masked_copy(long long n, const double* src, const unsigned char* dir, int constrained,
                                  double value, double* dst, cudaStream_t s) {
  masked_copy_kernel<<<grid_for(n), kThreads, 0, s>>>(n, src, dir, constrained, value, dst);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t hx_launch_cg_init(const HxCgBuffersT<Real>& b, const Real* bvec, const Real* x0, double rtol, int max_it,
                              cudaStream_t s) {
  cg_init_kernel<Real><<<(unsigned)hx_red_blocks(b.n), HX_RED_THREADS, 0, s>>>(b, bvec, x0, rtol, max_it);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t hx_launch_cg_residual(const HxCgBuffersT<Real>& b, cudaStream_t s) {
  cg_residual_kernel<Real><<<(unsigned)hx_red_blocks(b.n), HX_RED_THREADS, 0, s>>>(b);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t hx_launch_cg_start(const HxCgBuffersT<Real>& b, cudaStream_t s) {
  cg_start_kernel<Real><<<(unsigned)hx_red_blocks(b.n), HX_RED_THREADS, 0, s>>>(b);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t hx_launch_cg_assemble_pap(const HxCgBuffersT<Real>& b, cudaStream_t s) {
  const unsigned nb = (unsigned)hx_red_blocks(b.n);
  switch (b.ga.p) {
    case 1: cg_assemble_pap_kernel<1, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
    case 2: cg_assemble_pap_kernel<2, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
    case 3: cg_assemble_pap_kernel<3, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
    case 4: cg_assemble_pap_kernel<4, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
    case 5: cg_assemble_pap_kernel<5, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
    case 6: cg_assemble_pap_kernel<6, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
    case 7: cg_assemble_pap_kernel<7, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
    case 8: cg_assemble_pap_kernel<8, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
    default: cg_assemble_pap_kernel<0, Real><<<nb, HX_RED_THREADS, 0, s>>>(b); break;
  }
  return cudaGetLastError();
}
template <typename Real>
cudaError_t hx_launch_cg_update(const HxCgBuffersT<Real>& b, cudaStream_t s) {
  cg_update_kernel<Real><<<(unsigned)hx_red_blocks(b.n), HX_RED_THREADS, 0, s>>>(b);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t hx_launch_cg_rz(const HxCgBuffersT<Real>& b, cudaStream_t s) {
  cg_rz_kernel<Real><<<(unsigned)hx_red_blocks(b.n), HX_RED_THREADS, 0, s>>>(b);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t hx_launch_cg_direction(const HxCgBuffersT<Real>& b, cudaStream_t s) {
  cg_direction_kernel<Real><<<(unsigned)hx_red_blocks(b.n), HX_RED_THREADS, 0, s>>>(b);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t hx_launch_cg_mean(const HxCgBuffersT<Real>& b, const Real* v, cudaStream_t s) {
  cg_mean_kernel<Real><<<(unsigned)hx_red_blocks(b.n), HX_RED_THREADS, 0, s>>>(b, v);
  return cudaGetLastError();
}
cudaError_t hx_launch_sum(long long n, const double* v, double* partial, unsigned int* counter, double* out,
                          cudaStream_t s) {
  sum_kernel<<<HX_RED_BLOCKS, HX_RED_THREADS, 0, s>>>(n, v, partial, counter, out);
  return cudaGetLastError();
}
cudaError_t hx_launch_shift(long long n, double* x, const double* num, const double* den, cudaStream_t s) {
  shift_kernel<<<grid_for(n), kThreads, 0, s>>>(n, x, num, den);
  return cudaGetLastError();
}
#define HX_CG_INSTANTIATE(R)                                                                              \
  template cudaError_t hx_launch_cg_init<R>(const HxCgBuffersT<R>&, const R*, const R*, double, int, cudaStream_t); \
  template cudaError_t hx_launch_cg_residual<R>(const HxCgBuffersT<R>&, cudaStream_t);                 \
  template cudaError_t hx_launch_cg_start<R>(const HxCgBuffersT<R>&, cudaStream_t);                    \
  template cudaError_t hx_launch_cg_assemble_pap<R>(const HxCgBuffersT<R>&, cudaStream_t);             \
  template cudaError_t hx_launch_cg_update<R>(const HxCgBuffersT<R>&, cudaStream_t);                   \
  template cudaError_t hx_launch_cg_direction<R>(const HxCgBuffersT<R>&, cudaStream_t);                \
  template cudaError_t hx_launch_cg_rz<R>(const HxCgBuffersT<R>&, cudaStream_t);                       \
  template cudaError_t hx_launch_cg_mean<R>(const HxCgBuffersT<R>&, const R*, cudaStream_t);
HX_CG_INSTANTIATE(double)
HX_CG_INSTANTIATE(float)

cudaError_t hx_launch_cg_pass_multi(int pass, const HxCgBuffers* bufs, const int* blk_op, const int* blk_first,
                                    const int* blk_count, long long blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (pass == HX_PASS_ASSEMBLE_PAP)
    cg_assemble_pap_multi_kernel<double><<<(unsigned)blocks, HX_RED_THREADS, 0, s>>>(bufs, blk_op, blk_first, blk_count);
  else if (pass == HX_PASS_UPDATE)
    cg_update_multi_kernel<double><<<(unsigned)blocks, HX_RED_THREADS, 0, s>>>(bufs, blk_op, blk_first, blk_count);
  else
    cg_direction_multi_kernel<double><<<(unsigned)blocks, HX_RED_THREADS, 0, s>>>(bufs, blk_op, blk_first, blk_count);
  return cudaGetLastError();
}

cudaError_t hx_launch_batch_condition(HxCgState* const* states, int n, unsigned long long cond, cudaStream_t s) {
  batch_condition_kernel<<<1, HX_RED_THREADS, 0, s>>>(states, n, cond);
  return cudaGetLastError();
}

cudaError_t hx_launch_ir_residual(long long n, const double* b, const double* Ax, const unsigned char* dir, double* r,
                                  double* partial, unsigned int* counter, double* rn2, cudaStream_t s,
                                  const double* shift) {
  ir_residual_kernel<<<HX_RED_BLOCKS, HX_RED_THREADS, 0, s>>>(n, b, Ax, dir, r, partial, counter, rn2, shift);
  return cudaGetLastError();
}
cudaError_t hx_launch_ir_scale_down(long long n, const double* r, const double* rn2, float* r32, cudaStream_t s) {
  ir_scale_down_kernel<<<grid_for(n), kThreads, 0, s>>>(n, r, rn2, r32);
  return cudaGetLastError();
}
cudaError_t hx_launch_ir_update(long long n, double* x, const float* d, const double* rn2, cudaStream_t s) {
  ir_update_kernel<<<grid_for(n), kThreads, 0, s>>>(n, x, d, rn2);
  return cudaGetLastError();
}
cudaError_t hx_launch_to_float(long long n, const double* a, float* b, cudaStream_t s) {
  to_float_kernel<<<grid_for(n), kThreads, 0, s>>>(n, a, b);
  return cudaGetLastError();
}
cudaError_t hx_launch_to_float_strided(long long E, int per, int stride, const double* a, float* b,
                                       cudaStream_t s) {
  to_float_strided_kernel<<<grid_for(E * stride), kThreads, 0, s>>>(E, per, stride, a, b);
  return cudaGetLastError();
}
cudaError_t hx_launch_dot(long long n, const double* a, const double* c, double* partial, unsigned int* counter,
                          double* out, cudaStream_t s) {
  dot_kernel<<<HX_RED_BLOCKS, HX_RED_THREADS, 0, s>>>(n, a, c, partial, counter, out);
  return cudaGetLastError();
}
cudaError_t hx_launch_resnorm(long long n, const double* b, const double* Ax, const unsigned char* dir, double* partial,
                              unsigned int* counter, double* out, cudaStream_t s, const double* shift) {
  resnorm_kernel<<<HX_RED_BLOCKS, HX_RED_THREADS, 0, s>>>(n, b, Ax, dir, partial, counter, out, shift);
  return cudaGetLastError();
}
