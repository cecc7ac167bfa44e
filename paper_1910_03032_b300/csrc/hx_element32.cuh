// FP32 element kernel of the mixed-precision inner solver: y_E = A_e x_E for the operator
// alpha M + nu K in single precision, sum-factorized (Sec. 3.1, Eqs. (sumFactorized),
// (tensorGradient)) in the "B/D-direct" form:
//   u = (B x B x B) x_E,  du/dxi_1 = (B x B x D) x_E,  du/dxi_2 = (B x D x B) x_E,
//   du/dxi_3 = (D x B x B) x_E   (tensor factors listed z, y, x),
//   [v; w] = [m u; G grad u]  at every Gauss point,
//   y_E = (B x B x B)^T v + (B x B x D)^T w_1 + (B x D x B)^T w_2 + (D x B x B)^T w_3.
// Sharing the partial products, the forward pass is three contraction stages (x: B and D,
// y: three outputs, z: four outputs) and the transposed pass three more.  Against the
// collocated form of the FP64 kernel ("interpolate with B, differentiate with the q x q
// matrix Dh") this spends ~30% more FP32 flops -- cheap on this part -- to move less data
// through shared memory: every intermediate is written and read once (two planes of
// q n^2 and three of q^2 n values per element instead of repeated q^3 passes), and the
// whole pointwise stage and both z stages stay in the registers of the z-column's owner.
//
// Layout: NE elements per block (a power of two, at most 8; G = 32 / NE).  The contraction
// stages keep the NE elements interleaved word by word in shared memory: slot s of element
// el lives at word s NE + el, and the thread of element el and task m is t = el + NE m.  A
// warp then holds G consecutive tasks m of NE elements, and every stage addresses
// slot = SX m + const for its loop index (SX odd, >= n), so the 32 words a warp touches fall
// into 32 distinct banks.  Interleaved slots per element:
//   T1 (after x), 2 arrays:         j + SX (k + n iq)                 (SX n q each)
//   T2 (after y), 3 arrays:         k + SX (iq + q jq)                (SX q^2 each)
// The block's restriction indices (one contiguous range) arrive in shared memory by one bulk
// TMA copy at block start; the x-line stage gathers x_E from them and the transposed x-line
// stage stores y_E line by line.  Stored factors go the same way, one bulk copy per element
// into a slot of FE words (FE = G mod 32, so that the column owners of the NE elements read
// distinct banks), all completed on an mbarrier the column stage waits for.
#pragma once

#include "hx_element.cuh"

namespace hx {

// smallest value >= lo that is = r (mod 32) and a multiple of `mult`
constexpr int stride_mod32(int lo, int r, int mult) {
  int v = lo;
  while (v % 32 != r % 32 || v % mult != 0) ++v;
  return v;
}

template <int P, int Q, int NE>
struct Layout32 {
  static constexpr int N = P + 1;
  static constexpr int G = 32 / NE;               // tasks per warp and element
  static constexpr int SX = (N % 2) ? N : N + 1;  // odd line stride
  static constexpr int T1A = SX * N * Q;          // interleaved slots of one T1 array
  static constexpr int T2A = SX * Q * Q;          // interleaved slots of one T2 array
  static constexpr int FE32 = ((7 * Q * Q * Q) + 3) & ~3;                   // factor stride in HBM
  static constexpr int FE = stride_mod32(FE32, G, 4);                        // factor stride in shared memory
  // words of the T2 space (holding the block's restriction before stage 2), rounded up to
  // 16 bytes, and of T2 + T1
  static constexpr int T2S = (3 * NE * T2A + 3) & ~3;
  static constexpr int INT = T2S + 2 * NE * T1A;
};

// y = S1 x1 + S2 x2 for a centro-symmetric S1 (sigma = +1, folded S1e, S1o) and a
// centro-antisymmetric S2 (sigma = -1, folded S2e, S2o), both M x L: the folded products
// of the two combine as one centro-symmetric result (E1 + O2, O1 + E2).
template <int L, int M, typename Real>
__device__ __forceinline__ void eo_apply_sym_anti(const Real* __restrict__ S1e, const Real* __restrict__ S1o,
                                                  const Real* __restrict__ S2e, const Real* __restrict__ S2o,
                                                  const Real (&x1)[L], const Real (&x2)[L], Real (&y)[M]) {
  constexpr int CL = (L + 1) / 2, CM = (M + 1) / 2;
  Real e1[CL], o1[CL], e2[CL], o2[CL], E1[CM], O1[CM], E2[CM], O2[CM];
  fold<L>(x1, e1, o1);
  fold<L>(x2, e2, o2);
  products<L, M, 1>(S1e, S1o, e1, o1, E1, O1);
  products<L, M, -1>(S2e, S2o, e2, o2, E2, O2);
#pragma unroll
  for (int a = 0; a < CM; ++a) {
    E1[a] += O2[a];
    O1[a] += E2[a];
  }
  combine<M, 1>(E1, O1, y);
}

// Runs f(t) for the tasks t = tid, tid + NT, ... < TASKS, unrolled (TASKS, NT compile-time).
template <int TASKS, int NT, typename F>
__device__ __forceinline__ void for_tasks(int tid, F&& f) {
#pragma unroll
  for (int it = 0; it < (TASKS + NT - 1) / NT; ++it) {
    const int t = tid + it * NT;
    if (TASKS % NT == 0 || t < TASKS) f(t);
  }
}

template <int P, int Q, int NE, int NT, int MINB, int GEOM, bool NUF, bool STAGE>
__global__ void __launch_bounds__(NT, MINB)
    apply32_kernel(const __grid_constant__ HxTablesF T, const HxApplyArgsF A) {
  using L = Layout32<P, Q, NE>;
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N, Q2 = Q * Q, Q3 = Q2 * Q;
  constexpr int SX = L::SX, T1A = L::T1A, T2A = L::T2A, FE = L::FE;
  constexpr int CN = (N + 1) / 2, CQ = (Q + 1) / 2;
  static_assert((NE & (NE - 1)) == 0 && NE <= 8, "NE is a power of two, at most 8");
  static_assert(NT >= NE * Q2 && NT % 32 == 0, "one thread per z-column, whole warps");
  static_assert(!STAGE || GEOM == HX_KGEOM_STORED, "only stored factors are staged");
  static_assert(L::T2S >= NE * N3 + 8, "the restriction copy fits in the T2 space");
  if (A.done != nullptr && *(volatile const int*)A.done) return;
  extern __shared__ __align__(16) float sm[];
  __shared__ unsigned long long rbar;  // completion barrier of the restriction copy
  __shared__ unsigned long long fbar;  // completion barrier of the factor copies
  __shared__ int wait_failed;          // some thread's first wait for a copy gave up
  float* FS = sm;                              // staged factors: NE x FE (16-byte aligned)
  float* T2 = sm + (STAGE ? NE * FE : 0);      // 3 interleaved arrays
  float* T1 = T2 + L::T2S;                     // 2 interleaved arrays (16-byte aligned)
  int* RS = reinterpret_cast<int*>(T2);        // the block's restriction, until stage 1
  float* geo = T2 + L::INT;                    // on the fly: NE x 24 map coefficients
  const long long e0 = (long long)blockIdx.x * NE;
  const int tid = threadIdx.x;
  const int nel = (A.E - e0) < NE ? (int)(A.E - e0) : NE;
  // the restriction copy starts at the 16-byte boundary at or below element e0's first index
  const int roff = (int)((e0 * N3) & 3);

  if (tid == 0) {
    wait_failed = 0;
    // the block's restriction: one contiguous range (the array has 16 bytes of slack)
    const long long b0 = e0 * N3 * 4, b1 = (e0 + nel) * N3 * 4;
    const long long a0 = b0 & ~15LL, a1 = (b1 + 15) & ~15LL;
    mbar_init(&rbar, 1);
    mbar_expect_tx(&rbar, (unsigned)(a1 - a0));
    bulk_load(RS, reinterpret_cast<const char*>(A.R) + a0, (unsigned)(a1 - a0), &rbar);
    if (STAGE) {
      mbar_init(&fbar, 1);
      mbar_expect_tx(&fbar, (unsigned)(nel * L::FE32 * sizeof(float)));
      for (int el = 0; el < nel; ++el)
        bulk_load(FS + el * FE, A.factors + (e0 + el) * A.fstride, (unsigned)(L::FE32 * sizeof(float)), &fbar);
    }
  }
  if (!STAGE && GEOM == HX_KGEOM_STORED) {
    // pull this block's factors toward L2 while the gather and the first stages run
    const char* base = reinterpret_cast<const char*>(A.factors + e0 * A.fstride);
    const long long bytes = nel * A.fstride * (long long)sizeof(float);
    for (long long off = (long long)tid * 128; off < bytes; off += (long long)NT * 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
  } else if (GEOM == HX_KGEOM_ONTHEFLY) {
    trilinear_coeffs_block(A.X8, e0, A.E, NE, geo);  // corner coordinates stay FP64 until here
  }
  __syncthreads();  // the barriers are initialized before anyone waits on them
  // 1. gather x_E = R x (Dirichlet DoFs read as zero for A_c) line by line, and contract the
  //    x-lines (j, k): T1[0] = B x, T1[1] = D x along x
  {
    const bool ok = mbar_wait_bounded(&rbar, A.wait_limit);
    if (!ok) {
      wait_failed = 1;
      if (A.err) atomicExch(A.err, 1);
    }
    for_tasks<NE * N2, NT>(tid, [&](int t) {
      const int el = t % NE, r = t / NE;  // r = j + n k
      float xin[N], ev[CN], od[CN], E[CQ], O[CQ], out[Q];
      const int* rl = RS + roff + el * N3 + r * N;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        xin[i] = 0.0f;
        if (ok && el < nel) {
          const int g = rl[i];
          xin[i] = (g >= 0) ? __ldg(A.x + g) : (A.constrained ? 0.0f : __ldg(A.x + (-g - 1)));
        }
      }
      fold<N>(xin, ev, od);
      const int s1 = (r % N) + SX * (r / N);  // j + SX k
      products<N, Q, 1>(T.Be, T.Bo, ev, od, E, O);
      combine<Q, 1>(E, O, out);
#pragma unroll
      for (int iq = 0; iq < Q; ++iq) T1[(s1 + SX * N * iq) * NE + el] = out[iq];
      products<N, Q, -1>(T.Dne, T.Dno, ev, od, E, O);
      combine<Q, -1>(E, O, out);
#pragma unroll
      for (int iq = 0; iq < Q; ++iq) T1[(T1A + s1 + SX * N * iq) * NE + el] = out[iq];
    });
  }
  __syncthreads();
  if (wait_failed) {
    // no copy may still be writing this block's shared memory when it exits
    if (tid == 0) {
      mbar_wait_bounded(&rbar, HX_WAIT_LIMIT_EXIT);
      if (STAGE) mbar_wait_bounded(&fbar, HX_WAIT_LIMIT_EXIT);
    }
    return;
  }
  // 2. y-lines (k, iq): T2[0] = B_y B_x x, T2[1] = B_y D_x x, T2[2] = D_y B_x x
  for_tasks<NE * N * Q, NT>(tid, [&](int t) {
    const int el = t % NE, m = t / NE;  // m = k + n iq
    const int k = m % N, iq = m / N;
    float a[N], b[N], ev[CN], od[CN], E[CQ], O[CQ], out[Q];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      a[j] = T1[(SX * m + j) * NE + el];
      b[j] = T1[(T1A + SX * m + j) * NE + el];
    }
    const int s2 = k + SX * iq;
    fold<N>(a, ev, od);
    products<N, Q, 1>(T.Be, T.Bo, ev, od, E, O);
    combine<Q, 1>(E, O, out);
#pragma unroll
    for (int jq = 0; jq < Q; ++jq) T2[(s2 + SX * Q * jq) * NE + el] = out[jq];
    products<N, Q, -1>(T.Dne, T.Dno, ev, od, E, O);
    combine<Q, -1>(E, O, out);
#pragma unroll
    for (int jq = 0; jq < Q; ++jq) T2[(2 * T2A + s2 + SX * Q * jq) * NE + el] = out[jq];
    fold<N>(b, ev, od);
    products<N, Q, 1>(T.Be, T.Bo, ev, od, E, O);
    combine<Q, 1>(E, O, out);
#pragma unroll
    for (int jq = 0; jq < Q; ++jq) T2[(T2A + s2 + SX * Q * jq) * NE + el] = out[jq];
  });
  __syncthreads();
  // 3. z-columns c = iq + q jq: B_z and D_z forward, the pointwise factors, then
  //    A' = B_z^T v + D_z^T w_3, W1 = B_z^T w_1, W2 = B_z^T w_2 back into the column's slots
  if (tid < NE * Q2) {
    const int el = tid % NE, c = tid / NE;
    const long long e = e0 + el;
    const bool live = el < nel;
    float* col = T2 + (SX * c) * NE + el;
    float a[N], b[N], d[N], ev[CN], od[CN], E[CQ], O[CQ];
    float u[Q], ux[Q], uy[Q], uz[Q];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      a[k] = col[k * NE];
      b[k] = col[(T2A + k) * NE];
      d[k] = col[(2 * T2A + k) * NE];
    }
    fold<N>(a, ev, od);
    products<N, Q, 1>(T.Be, T.Bo, ev, od, E, O);
    combine<Q, 1>(E, O, u);
    products<N, Q, -1>(T.Dne, T.Dno, ev, od, E, O);
    combine<Q, -1>(E, O, uz);
    fold<N>(b, ev, od);
    products<N, Q, 1>(T.Be, T.Bo, ev, od, E, O);
    combine<Q, 1>(E, O, ux);
    fold<N>(d, ev, od);
    products<N, Q, 1>(T.Be, T.Bo, ev, od, E, O);
    combine<Q, 1>(E, O, uy);
    // a thread whose wait for the staged factors gives up raises the error flag and skips
    // its pointwise work; after the next barrier the whole block stops and stores nothing
    bool staged = true;
    if (STAGE && !mbar_wait_bounded(&fbar, A.wait_limit)) {
      staged = false;
      wait_failed = 1;
      if (A.err) atomicExch(A.err, 1);
    }
    if (staged) {
      // pointwise: v = m u, w = G grad u at the column's q points
      float P0[3], R0[3], P1[3], R1[3], J2[3], w12 = 0.0f;
      if (GEOM == HX_KGEOM_ONTHEFLY) {
        // for a trilinear map dx/dxi_3 is constant along the column and the other two
        // Jacobian columns are affine in xi_3: two 3-vector updates per point
        const float* gm = geo + el * 24;
        const int iq = c % Q, jq = c / Q;
        const float x1 = T.xq[iq], x2 = T.xq[jq];
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
          const float* ad = gm + dd * 8;
          P0[dd] = ad[1] + ad[4] * x2;
          R0[dd] = ad[5] + ad[7] * x2;
          P1[dd] = ad[2] + ad[4] * x1;
          R1[dd] = ad[6] + ad[7] * x1;
          J2[dd] = ad[3] + ad[5] * x1 + (ad[6] + ad[7] * x1) * x2;
        }
        w12 = T.wq[iq] * T.wq[jq];
      }
      // staged factors: element el's slot, bank = (el G + c) mod 32, distinct across the warp
      const float* fs = FS + el * FE + c;
      // unstaged factors: consecutive columns of one element are consecutive words
      const float* fe = A.factors + (live ? e : 0) * A.fstride + c;
#pragma unroll
      for (int kq = 0; kq < Q; ++kq) {
        float f[7];
        if (STAGE) {
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) f[mm] = fs[mm * Q3 + kq * Q2];
        } else if (GEOM == HX_KGEOM_STORED) {
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) f[mm] = live ? __ldg(fe + mm * Q3 + kq * Q2) : 0.0f;
        } else {
          const float z = T.xq[kq];
          float j0[3], j1[3], j2[3];
#pragma unroll
          for (int dd = 0; dd < 3; ++dd) {
            j0[dd] = P0[dd] + z * R0[dd];
            j1[dd] = P1[dd] + z * R1[dd];
            j2[dd] = J2[dd];
          }
          const float w = w12 * T.wq[kq];
          float nu = A.nu;
          if (NUF) nu = live ? float(__ldg(A.nu_q + e * Q3 + kq * Q2 + c)) : 0.0f;
          point_factors(j0, j1, j2, A.alpha * w, nu * w, f);
        }
        if (!live) {
#pragma unroll
          for (int mm = 0; mm < 7; ++mm) f[mm] = 0.0f;
        }
        const float g1 = ux[kq], g2 = uy[kq], g3 = uz[kq];
        u[kq] = f[0] * u[kq];
        ux[kq] = f[1] * g1 + f[2] * g2 + f[3] * g3;
        uy[kq] = f[2] * g1 + f[4] * g2 + f[5] * g3;
        uz[kq] = f[3] * g1 + f[5] * g2 + f[6] * g3;
      }
      float out[N];
      eo_apply_sym_anti<Q, N>(T.Bte, T.Bto, T.Dnte, T.Dnto, u, uz, out);
#pragma unroll
      for (int k = 0; k < N; ++k) col[k * NE] = out[k];
      eo_apply<Q, N, 1>(T.Bte, T.Bto, ux, out);
#pragma unroll
      for (int k = 0; k < N; ++k) col[(T2A + k) * NE] = out[k];
      eo_apply<Q, N, 1>(T.Bte, T.Bto, uy, out);
#pragma unroll
      for (int k = 0; k < N; ++k) col[(2 * T2A + k) * NE] = out[k];
    }
  }
  __syncthreads();
  if (STAGE && wait_failed) {
    // no copy may still be writing this block's shared memory when it exits: wait once more,
    // with a far larger bound than the first wait
    if (tid == 0) mbar_wait_bounded(&fbar, HX_WAIT_LIMIT_EXIT);
    return;
  }
  // 2T. y-lines (k, iq): P = B_y^T A' + D_y^T W2, R = B_y^T W1 at (iq, j, k) into T1
  for_tasks<NE * N * Q, NT>(tid, [&](int t) {
    const int el = t % NE, m = t / NE;  // m = k + n iq
    const int k = m % N, iq = m / N;
    const int s2 = k + SX * iq;
    float a[Q], w1[Q], w2[Q], out[N];
#pragma unroll
    for (int jq = 0; jq < Q; ++jq) {
      a[jq] = T2[(s2 + SX * Q * jq) * NE + el];
      w1[jq] = T2[(T2A + s2 + SX * Q * jq) * NE + el];
      w2[jq] = T2[(2 * T2A + s2 + SX * Q * jq) * NE + el];
    }
    eo_apply_sym_anti<Q, N>(T.Bte, T.Bto, T.Dnte, T.Dnto, a, w2, out);
#pragma unroll
    for (int j = 0; j < N; ++j) T1[(SX * m + j) * NE + el] = out[j];
    eo_apply<Q, N, 1>(T.Bte, T.Bto, w1, out);
#pragma unroll
    for (int j = 0; j < N; ++j) T1[(T1A + SX * m + j) * NE + el] = out[j];
  });
  __syncthreads();
  // 1T. x-lines (j, k): y = B_x^T P + D_x^T R, stored line by line into y_E
  for_tasks<NE * N2, NT>(tid, [&](int t) {
    const int el = t % NE, r = t / NE;  // r = j + n k
    const int s1 = (r % N) + SX * (r / N);
    float pp[Q], rr[Q], out[N];
#pragma unroll
    for (int iq = 0; iq < Q; ++iq) {
      pp[iq] = T1[(s1 + SX * N * iq) * NE + el];
      rr[iq] = T1[(T1A + s1 + SX * N * iq) * NE + el];
    }
    eo_apply_sym_anti<Q, N>(T.Bte, T.Bto, T.Dnte, T.Dnto, pp, rr, out);
    if (el < nel) {
      float* yl = A.yE + hx_eline(A.lay, e0 + el, r, N);
#pragma unroll
      for (int i = 0; i < N; ++i) yl[i] = out[i];
    }
  });
  // every owner's first wait saw the copies complete, so this returns at once
  if (STAGE && tid == 0) mbar_wait_bounded(&fbar, HX_WAIT_LIMIT_EXIT);
}

// Elements per block of the FP32 operator kernel: a power of two (at most 8) with
// NE q^2 <= 256 threads, at least 2.
template <int Q>
constexpr int ne32() {
  return (Q * Q * 8 <= 256) ? 8 : (Q * Q * 4 <= 256) ? 4 : 2;
}

// Elements per block of the tile variant `shift` (the default ne32 scaled by 2^shift), or 0 when
// that variant does not exist (NE outside 1..8, or more than 1024 threads).
template <int Q>
constexpr int ne32_tile(int shift) {
  const int ne = shift < 0 ? ne32<Q>() / 2 : shift > 0 ? ne32<Q>() * 2 : ne32<Q>();
  return (ne < 1 || ne > 8 || ((ne * Q * Q + 31) / 32) * 32 > 1024) ? 0 : ne;
}

template <int P, int Q, int GEOM, bool NUF, bool STAGE, int NE>
cudaError_t launch_apply32_impl(const HxTablesF& T, const HxApplyArgsF& A, cudaStream_t s) {
  if constexpr (NE == 0) {
    return cudaErrorInvalidValue;  // no such tile variant
  } else {
    using L = Layout32<P, Q, NE>;
    constexpr int NT = ((NE * Q * Q + 31) / 32) * 32;
    constexpr int RB = GEOM == HX_KGEOM_ONTHEFLY ? 96 : 64;  // registers per thread budgeted
    constexpr int MINB = 65536 / (NT * RB) < 1 ? 1 : 65536 / (NT * RB) > 16 ? 16 : 65536 / (NT * RB);
    // the bulk copies of staged factors move whole padded (16-byte) element ranges
    if (STAGE && A.fstride != L::FE32) return cudaErrorInvalidValue;
    const size_t shmem = sizeof(float) * ((STAGE ? (size_t)NE * L::FE : 0) + (size_t)L::INT +
                                          (GEOM == HX_KGEOM_ONTHEFLY ? NE * 24 : 0));
    if (shmem > 227 * 1024) return cudaErrorInvalidValue;
    auto k = apply32_kernel<P, Q, NE, NT, MINB, GEOM, NUF, STAGE>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    if (err != cudaSuccess) return err;
    const long long blocks = (A.E + NE - 1) / NE;
    if (blocks == 0) return cudaSuccess;
    k<<<(unsigned)blocks, NT, shmem, s>>>(T, A);
    return cudaGetLastError();
  }
}

// stage: stored factors arrive by bulk copies (else they are read from global memory);
// tile: -1, 0, +1 for half, the default and twice the elements per block (stored factors; the
// on-the-fly forms have the default only)
template <int P, int Q>
cudaError_t launch_apply32_q(const HxTablesF& T, const HxApplyArgsF& A, int geom, bool stage, int tile,
                             cudaStream_t s) {
  constexpr int NM = ne32_tile<Q>(-1), N0 = ne32_tile<Q>(0), NP = ne32_tile<Q>(1);
  if (geom == HX_KGEOM_STORED) {
    if (stage) {
      if (tile < 0) return launch_apply32_impl<P, Q, HX_KGEOM_STORED, false, true, NM>(T, A, s);
      if (tile > 0) return launch_apply32_impl<P, Q, HX_KGEOM_STORED, false, true, NP>(T, A, s);
      return launch_apply32_impl<P, Q, HX_KGEOM_STORED, false, true, N0>(T, A, s);
    }
    if (tile < 0) return launch_apply32_impl<P, Q, HX_KGEOM_STORED, false, false, NM>(T, A, s);
    if (tile > 0) return launch_apply32_impl<P, Q, HX_KGEOM_STORED, false, false, NP>(T, A, s);
    return launch_apply32_impl<P, Q, HX_KGEOM_STORED, false, false, N0>(T, A, s);
  }
  if (tile != 0) return cudaErrorInvalidValue;
  if (A.nu_q) return launch_apply32_impl<P, Q, HX_KGEOM_ONTHEFLY, true, false, N0>(T, A, s);
  return launch_apply32_impl<P, Q, HX_KGEOM_ONTHEFLY, false, false, N0>(T, A, s);
}

// elements per block of the direct FP32 kernel's tile variant (0: none)
template <int Q>
int ne32_of_tile(int tile) {
  return ne32_tile<Q>(tile);
}

}  // namespace hx
