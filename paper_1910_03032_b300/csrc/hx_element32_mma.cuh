// FP32 element operator with its 1D contractions on the tensor cores (not part of the paper's
// method): the B/D-direct form of apply32_kernel (hx_element32.cuh), every contraction stage
// done by warp-level mma.sync m16n8k16 with BF16 operands and FP32 accumulation.  A warp
// contracts 16 lines (rows) at a time; along the contracted index (K <= 16 per tile) the rows'
// inputs form the A operand, the 1D matrix (B, D or their transposes) the B operand, and the
// products land in FP32 accumulator fragments:
//   x-lines (j, k):   [B x, D x]                      K = n
//   y-lines (k, iq):  [B_y T1_0, D_y T1_0], B_y T1_1   K = n
//   z-columns:        [u, du/dxi_3] = [B_z, D_z] T2_0, du/dxi_1 = B_z T2_1, du/dxi_2 = B_z T2_2,
//                     the pointwise factors applied in the accumulator fragments, which are then
//                     the A operand (K = q) of A' = B_z^T v + D_z^T w_3, W1 = B_z^T w_1, W2 = B_z^T w_2
//   y-lines:          P = B_y^T A' + D_y^T W2, R = B_y^T W1     K = q
//   x-lines:          y = B_x^T P + D_x^T R                      K = q
// (the accumulator layout of an m16n8 tile pair is the A layout of an m16k16 tile, so the
// column stage chains its contractions in registers).  PASSES = 1 rounds every operand to
// BF16 (8 significant bits); PASSES = 3 splits each into hi + lo BF16 parts and accumulates
// hi*hi + hi*lo + lo*hi (about 16 significant bits).  Shared-memory layouts, the bulk TMA copies
// of restriction and factors and the bounded waits are those of apply32_kernel.
#pragma once

#include <cuda_bf16.h>

#include "hx_element32.cuh"

namespace hx {

__device__ __forceinline__ unsigned bf16x2(float lo_col, float hi_col) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo_col, hi_col);
  return *reinterpret_cast<unsigned*>(&h);
}

// hi = BF16 rounding of (a, b); lo = BF16 rounding of the remainders
__device__ __forceinline__ void split2(float a, float b, unsigned& hi, unsigned& lo) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  hi = *reinterpret_cast<unsigned*>(&h);
  lo = bf16x2(a - hf.x, b - hf.y);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A-operand fragment (rows ra = row0 + g, rb = ra + 8; K-tile columns 2t, 2t+1, 2t+8, 2t+9)
// from its 8 FP32 values v[0..7] = (ra,2t) (ra,2t+1) (rb,2t) (rb,2t+1) (ra,2t+8) (ra,2t+9)
// (rb,2t+8) (rb,2t+9), as hi (and lo) BF16 pairs.
template <int PASSES>
struct AFrag {
  unsigned hi[4], lo[4];
  __device__ __forceinline__ void set(const float (&v)[8]) {
    if (PASSES == 1) {
      hi[0] = bf16x2(v[0], v[1]);
      hi[1] = bf16x2(v[2], v[3]);
      hi[2] = bf16x2(v[4], v[5]);
      hi[3] = bf16x2(v[6], v[7]);
    } else {
      split2(v[0], v[1], hi[0], lo[0]);
      split2(v[2], v[3], hi[1], lo[1]);
      split2(v[4], v[5], hi[2], lo[2]);
      split2(v[6], v[7], hi[3], lo[3]);
    }
  }
};

// B-operand fragment of an (K-tile, N-tile) of M: element (k, n) = M(n_out = nt*8 + g, k_in)
// with k = kt*16 + {2t, 2t+1, 2t+8, 2t+9}
template <int PASSES>
struct BFrag {
  unsigned hi[2], lo[2];
  template <typename F>
  __device__ __forceinline__ void set(int lane, int kt, int nt, F&& M) {
    const int g = lane >> 2, t = lane & 3;
    const int n = nt * 8 + g, k0 = kt * 16 + 2 * t;
    const float v0 = M(n, k0), v1 = M(n, k0 + 1), v2 = M(n, k0 + 8), v3 = M(n, k0 + 9);
    if (PASSES == 1) {
      hi[0] = bf16x2(v0, v1);
      hi[1] = bf16x2(v2, v3);
    } else {
      split2(v0, v1, hi[0], lo[0]);
      split2(v2, v3, hi[1], lo[1]);
    }
  }
};

template <int PASSES>
__device__ __forceinline__ void mma_acc(float (&c)[4], const AFrag<PASSES>& a, const BFrag<PASSES>& b) {
  mma_bf16(c, a.hi, b.hi);
  if (PASSES == 3) {
    mma_bf16(c, a.hi, b.lo);
    mma_bf16(c, a.lo, b.hi);
  }
}

// the 8 values of an A fragment through in(row, k) (rows >= rows_total and k >= K read as 0)
template <typename F>
__device__ __forceinline__ void gather_a(int ra, int kt, int lane, int rows_total, int K, F&& in, float (&v)[8]) {
  const int t = lane & 3, rb = ra + 8;
  const int ks[4] = {kt * 16 + 2 * t, kt * 16 + 2 * t + 1, kt * 16 + 2 * t + 8, kt * 16 + 2 * t + 9};
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int k = ks[2 * h + s];
      v[4 * h + s] = (ra < rows_total && k < K) ? in(ra, k) : 0.0f;
      v[4 * h + 2 + s] = (rb < rows_total && k < K) ? in(rb, k) : 0.0f;
    }
}

// out(row, col, value) for the accumulator tile (rows ra, ra+8; columns nt*8 + 2t, +1),
// rows >= rows_total and columns >= NO skipped
template <typename F>
__device__ __forceinline__ void scatter_c(int ra, int nt, int lane, int rows_total, int NO, const float (&c)[4],
                                          F&& out) {
  const int t = lane & 3, col = nt * 8 + 2 * t;
  if (ra < rows_total) {
    if (col < NO) out(ra, col, c[0]);
    if (col + 1 < NO) out(ra, col + 1, c[1]);
  }
  if (ra + 8 < rows_total) {
    if (col < NO) out(ra + 8, col, c[2]);
    if (col + 1 < NO) out(ra + 8, col + 1, c[3]);
  }
}

template <int P, int Q, int NE, int NT, int PASSES>
__global__ void __launch_bounds__(NT, 1)
    apply32_mma_kernel(const __grid_constant__ HxTablesF T, const HxApplyArgsF A) {
  using L = Layout32<P, Q, NE>;
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N, Q2 = Q * Q, Q3 = Q2 * Q;
  constexpr int SX = L::SX, T1A = L::T1A, T2A = L::T2A, FE = L::FE;
  constexpr int NW = NT / 32;
  constexpr int NQT = (Q + 7) / 8, NNT = (N + 7) / 8;  // N-tiles over q and over n outputs
  static_assert(N <= 16 && Q <= 16, "one K-tile per contraction");
  static_assert(NT % 32 == 0, "whole warps");
  if (A.done != nullptr && *(volatile const int*)A.done) return;
  extern __shared__ __align__(16) float sm[];
  __shared__ unsigned long long rbar, fbar;
  __shared__ int wait_failed;
  float* FS = sm;
  float* T2 = sm + NE * FE;
  float* T1 = T2 + L::T2S;
  int* RS = reinterpret_cast<int*>(T2);
  const long long e0 = (long long)blockIdx.x * NE;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2;
  const int nel = (A.E - e0) < NE ? (int)(A.E - e0) : NE;
  const int roff = (int)((e0 * N3) & 3);
  auto Bm = [&](int o, int k) { return (o < Q && k < N) ? T.B[o * N + k] : 0.0f; };   // B[a][j]
  auto Dm = [&](int o, int k) { return (o < Q && k < N) ? T.D[o * N + k] : 0.0f; };   // D[a][j]
  auto Btm = [&](int j, int a) { return (j < N && a < Q) ? T.B[a * N + j] : 0.0f; };  // B^T[j][a]
  auto Dtm = [&](int j, int a) { return (j < N && a < Q) ? T.D[a * N + j] : 0.0f; };  // D^T[j][a]

  if (tid == 0) {
    wait_failed = 0;
    const long long b0 = e0 * N3 * 4, b1 = (e0 + nel) * N3 * 4;
    const long long a0 = b0 & ~15LL, a1 = (b1 + 15) & ~15LL;
    mbar_init(&rbar, 1);
    mbar_expect_tx(&rbar, (unsigned)(a1 - a0));
    bulk_load(RS, reinterpret_cast<const char*>(A.R) + a0, (unsigned)(a1 - a0), &rbar);
    mbar_init(&fbar, 1);
    mbar_expect_tx(&fbar, (unsigned)(nel * L::FE32 * sizeof(float)));
    for (int el = 0; el < nel; ++el)
      bulk_load(FS + el * FE, A.factors + (e0 + el) * A.fstride, (unsigned)(L::FE32 * sizeof(float)), &fbar);
  }
  __syncthreads();
  // forward fragments: [B | D] over q outputs, K = n
  BFrag<PASSES> fB[NQT], fD[NQT];
#pragma unroll
  for (int nt = 0; nt < NQT; ++nt) {
    fB[nt].set(lane, 0, nt, Bm);
    fD[nt].set(lane, 0, nt, Dm);
  }
  // 1. x-lines: rows (el, r = j + n k) interleaved as row = el + NE r; gather x_E from the copied
  //    restriction into the A fragments
  {
    const bool ok = mbar_wait_bounded(&rbar, A.wait_limit);
    if (!ok) {
      wait_failed = 1;
      if (A.err) atomicExch(A.err, 1);
    }
    constexpr int ROWS = NE * N2;
    for (int tile = warp; tile * 16 < ROWS; tile += NW) {
      const int ra = tile * 16 + g;
      float v[8];
      gather_a(ra, 0, lane, ROWS, N, [&](int row, int i) {
        const int el = row % NE, r = row / NE;
        if (!ok || el >= nel) return 0.0f;
        const int gg = RS[roff + el * N3 + r * N + i];
        return (gg >= 0) ? __ldg(A.x + gg) : (A.constrained ? 0.0f : __ldg(A.x + (-gg - 1)));
      }, v);
      AFrag<PASSES> a;
      a.set(v);
#pragma unroll
      for (int nt = 0; nt < NQT; ++nt) {
        float cb[4] = {0, 0, 0, 0}, cd[4] = {0, 0, 0, 0};
        mma_acc(cb, a, fB[nt]);
        mma_acc(cd, a, fD[nt]);
        auto st = [&](int arr) {
          return [&, arr](int row, int iq, float val) {
            const int el = row % NE, r = row / NE;
            const int s1 = (r % N) + SX * (r / N);
            T1[(arr * T1A + s1 + SX * N * iq) * NE + el] = val;
          };
        };
        scatter_c(ra, nt, lane, ROWS, Q, cb, st(0));
        scatter_c(ra, nt, lane, ROWS, Q, cd, st(1));
      }
    }
  }
  __syncthreads();
  if (wait_failed) {
    if (tid == 0) {
      mbar_wait_bounded(&rbar, HX_WAIT_LIMIT_EXIT);
      mbar_wait_bounded(&fbar, HX_WAIT_LIMIT_EXIT);
    }
    return;
  }
  // 2. y-lines: rows (el, m = k + n iq); T2_0 = B T1_0, T2_2 = D T1_0, T2_1 = B T1_1
  {
    constexpr int ROWS = NE * N * Q;
    for (int tile = warp; tile * 16 < ROWS; tile += NW) {
      const int ra = tile * 16 + g;
      float v[8];
      AFrag<PASSES> a0, a1;
      gather_a(ra, 0, lane, ROWS, N, [&](int row, int j) { return T1[(SX * (row / NE) + j) * NE + row % NE]; }, v);
      a0.set(v);
      gather_a(ra, 0, lane, ROWS, N, [&](int row, int j) { return T1[(T1A + SX * (row / NE) + j) * NE + row % NE]; },
               v);
      a1.set(v);
#pragma unroll
      for (int nt = 0; nt < NQT; ++nt) {
        float c0[4] = {0, 0, 0, 0}, c2[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0};
        mma_acc(c0, a0, fB[nt]);
        mma_acc(c2, a0, fD[nt]);
        mma_acc(c1, a1, fB[nt]);
        auto st = [&](int arr) {
          return [&, arr](int row, int jq, float val) {
            const int el = row % NE, m = row / NE;
            const int s2 = (m % N) + SX * (m / N);
            T2[(arr * T2A + s2 + SX * Q * jq) * NE + el] = val;
          };
        };
        scatter_c(ra, nt, lane, ROWS, Q, c0, st(0));
        scatter_c(ra, nt, lane, ROWS, Q, c1, st(1));
        scatter_c(ra, nt, lane, ROWS, Q, c2, st(2));
      }
    }
  }
  __syncthreads();
  // 3. z-columns: rows (el, c) interleaved as row = el + NE c
  {
    // warp-uniform: the tile loop below runs warp-wide mma.sync
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&fbar, A.wait_limit));
    if (!ok) {
      wait_failed = 1;
      if (A.err) atomicExch(A.err, 1);
    }
    // transposed fragments: K over the q points, outputs over n
    BFrag<PASSES> tB[NNT], tD[NNT];
#pragma unroll
    for (int nt = 0; nt < NNT; ++nt) {
      tB[nt].set(lane, 0, nt, Btm);
      tD[nt].set(lane, 0, nt, Dtm);
    }
    constexpr int ROWS = NE * Q2;
    const int t = lane & 3;
    for (int tile = warp; ok && tile * 16 < ROWS; tile += NW) {
      const int ra = tile * 16 + g;
      float v[8];
      AFrag<PASSES> a0, a1, a2;
      gather_a(ra, 0, lane, ROWS, N, [&](int row, int k) { return T2[(SX * (row / NE) + k) * NE + row % NE]; }, v);
      a0.set(v);
      gather_a(ra, 0, lane, ROWS, N, [&](int row, int k) { return T2[(T2A + SX * (row / NE) + k) * NE + row % NE]; },
               v);
      a1.set(v);
      gather_a(ra, 0, lane, ROWS, N,
               [&](int row, int k) { return T2[(2 * T2A + SX * (row / NE) + k) * NE + row % NE]; }, v);
      a2.set(v);
      // u, uz, ux, uy at (rows ra, ra + 8; points kq = nt*8 + 2t, +1), then v, w3, w1, w2 in place
      float u[2][4], uz[2][4], ux[2][4], uy[2][4];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int s = 0; s < 4; ++s) u[nt][s] = uz[nt][s] = ux[nt][s] = uy[nt][s] = 0.0f;
#pragma unroll
      for (int nt = 0; nt < NQT; ++nt) {
        mma_acc(u[nt], a0, fB[nt]);
        mma_acc(uz[nt], a0, fD[nt]);
        mma_acc(ux[nt], a1, fB[nt]);
        mma_acc(uy[nt], a2, fB[nt]);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int row = ra + ((s & 2) ? 8 : 0), kq = nt * 8 + 2 * t + (s & 1);
          const int el = row % NE, c = row / NE;
          float f[7] = {0, 0, 0, 0, 0, 0, 0};
          if (row < ROWS && kq < Q && el < nel) {
            const float* fs = FS + el * FE + kq * Q2 + c;
#pragma unroll
            for (int mm = 0; mm < 7; ++mm) f[mm] = fs[mm * Q3];
          }
          const float g1 = ux[nt][s], g2 = uy[nt][s], g3 = uz[nt][s];
          u[nt][s] = f[0] * u[nt][s];
          ux[nt][s] = f[1] * g1 + f[2] * g2 + f[3] * g3;
          uy[nt][s] = f[2] * g1 + f[4] * g2 + f[5] * g3;
          uz[nt][s] = f[3] * g1 + f[5] * g2 + f[6] * g3;
        }
      }
      // accumulator tiles (kq 0-7, 8-15) -> A fragments over K = kq
      auto chain = [&](const float (&cc)[2][4]) {
        const float vv[8] = {cc[0][0], cc[0][1], cc[0][2], cc[0][3], cc[1][0], cc[1][1], cc[1][2], cc[1][3]};
        AFrag<PASSES> a;
        a.set(vv);
        return a;
      };
      const AFrag<PASSES> av = chain(u), aw3 = chain(uz), aw1 = chain(ux), aw2 = chain(uy);
#pragma unroll
      for (int nt = 0; nt < NNT; ++nt) {
        float ca[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0}, c2[4] = {0, 0, 0, 0};
        mma_acc(ca, av, tB[nt]);
        mma_acc(ca, aw3, tD[nt]);
        mma_acc(c1, aw1, tB[nt]);
        mma_acc(c2, aw2, tB[nt]);
        auto st = [&](int arr) {
          return [&, arr](int row, int k, float val) {
            T2[(arr * T2A + SX * (row / NE) + k) * NE + row % NE] = val;
          };
        };
        scatter_c(ra, nt, lane, ROWS, N, ca, st(0));
        scatter_c(ra, nt, lane, ROWS, N, c1, st(1));
        scatter_c(ra, nt, lane, ROWS, N, c2, st(2));
      }
    }
  }
  __syncthreads();
  if (wait_failed) {
    if (tid == 0) mbar_wait_bounded(&fbar, HX_WAIT_LIMIT_EXIT);
    return;
  }
  BFrag<PASSES> tB[NNT], tD[NNT];
#pragma unroll
  for (int nt = 0; nt < NNT; ++nt) {
    tB[nt].set(lane, 0, nt, Btm);
    tD[nt].set(lane, 0, nt, Dtm);
  }
  // 2T. y-lines: rows (el, m = k + n iq); P = B^T A' + D^T W2, R = B^T W1 over K = jq
  {
    constexpr int ROWS = NE * N * Q;
    for (int tile = warp; tile * 16 < ROWS; tile += NW) {
      const int ra = tile * 16 + g;
      float v[8];
      AFrag<PASSES> aa, a1, a2;
      auto in = [&](int arr) {
        return [&, arr](int row, int jq) {
          const int m = row / NE;
          const int s2 = (m % N) + SX * (m / N);
          return T2[(arr * T2A + s2 + SX * Q * jq) * NE + row % NE];
        };
      };
      gather_a(ra, 0, lane, ROWS, Q, in(0), v);
      aa.set(v);
      gather_a(ra, 0, lane, ROWS, Q, in(1), v);
      a1.set(v);
      gather_a(ra, 0, lane, ROWS, Q, in(2), v);
      a2.set(v);
#pragma unroll
      for (int nt = 0; nt < NNT; ++nt) {
        float cp[4] = {0, 0, 0, 0}, cr[4] = {0, 0, 0, 0};
        mma_acc(cp, aa, tB[nt]);
        mma_acc(cp, a2, tD[nt]);
        mma_acc(cr, a1, tB[nt]);
        auto st = [&](int arr) {
          return [&, arr](int row, int j, float val) { T1[(arr * T1A + SX * (row / NE) + j) * NE + row % NE] = val; };
        };
        scatter_c(ra, nt, lane, ROWS, N, cp, st(0));
        scatter_c(ra, nt, lane, ROWS, N, cr, st(1));
      }
    }
  }
  __syncthreads();
  // 1T. x-lines: rows (el, r = j + n k); y = B^T P + D^T R over K = iq, stored line by line
  {
    constexpr int ROWS = NE * N2;
    for (int tile = warp; tile * 16 < ROWS; tile += NW) {
      const int ra = tile * 16 + g;
      float v[8];
      AFrag<PASSES> ap, ar;
      auto in = [&](int arr) {
        return [&, arr](int row, int iq) {
          const int r = row / NE;
          const int s1 = (r % N) + SX * (r / N);
          return T1[(arr * T1A + s1 + SX * N * iq) * NE + row % NE];
        };
      };
      gather_a(ra, 0, lane, ROWS, Q, in(0), v);
      ap.set(v);
      gather_a(ra, 0, lane, ROWS, Q, in(1), v);
      ar.set(v);
#pragma unroll
      for (int nt = 0; nt < NNT; ++nt) {
        float cy[4] = {0, 0, 0, 0};
        mma_acc(cy, ap, tB[nt]);
        mma_acc(cy, ar, tD[nt]);
        scatter_c(ra, nt, lane, ROWS, N, cy, [&](int row, int i, float val) {
          const int el = row % NE, r = row / NE;
          if (el < nel) A.yE[hx_eline(A.lay, e0 + el, r, N) + i] = val;
        });
      }
    }
  }
  if (tid == 0) mbar_wait_bounded(&fbar, HX_WAIT_LIMIT_EXIT);
}

template <int P, int Q, int PASSES>
cudaError_t launch_apply32_mma(const HxTablesF& T, const HxApplyArgsF& A, cudaStream_t s) {
  constexpr int NE = ne32<Q>();
  using L = Layout32<P, Q, NE>;
  constexpr int NT = ((NE * Q * Q + 31) / 32) * 32;
  if (A.fstride != L::FE32) return cudaErrorInvalidValue;  // whole padded element ranges are copied
  const size_t shmem = sizeof(float) * ((size_t)NE * L::FE + (size_t)L::INT);
  auto k = apply32_mma_kernel<P, Q, NE, NT, PASSES>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
  if (err != cudaSuccess) return err;
  const long long blocks = (A.E + NE - 1) / NE;
  if (blocks == 0) return cudaSuccess;
  k<<<(unsigned)blocks, NT, shmem, s>>>(T, A);
  return cudaGetLastError();
}

}  // namespace hx
