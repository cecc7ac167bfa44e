// Arithmetic-throughput probe (not part of the paper's method): the measured FP64 and FP32
// FMA rates that the roofline fractions of the FP64-pipe-bound kernels are compared with.
//
// Every thread runs 16 independent FMA chains x <- x a + c (0 < a < 1, so the values stay
// bounded and normal), enough independent work per warp to keep the FMA pipe issuing; the
// caller times one launch with CUDA events and divides the returned flop count by it.  The
// grid is one wave of resident blocks (at most 8 of 256 threads per SM).
#include <cuda_runtime.h>

#include "hx.h"
#include "hx_internal.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

__device__ double g_probe_sink[2];  // written only if the chains reach an impossible value

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(long long iters, T a, T c) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  // both multiplier and addend in registers (a constant-bank operand can slow the FMA issue)
  const bool never = threadIdx.x > 4096u;  // false for every thread (at most 256 per block)
  const T ar = never ? c : a, cr = never ? a : c;
#pragma unroll 4
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], ar, cr);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == T(-1)) g_probe_sink[sizeof(T) == 8 ? 0 : 1] = (double)s;  // keeps the chains live
}

}  // namespace

extern "C" hx_status hx_probe_fma(int fp64, int64_t iters, void* stream, double* flops) {
  if (iters < 1 || !flops) {
    hx_internal_set_error("hx_probe_fma: need iters >= 1 and a flops pointer");
    return HX_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    hx_internal_set_error(cudaGetErrorString(e));
    return HX_ERR_CUDA;
  }
  // exactly the blocks that are resident at once (one wave: no partly filled last wave)
  int per_sm = 0;
  if (e == cudaSuccess)
    e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<double>, kThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<float>, kThreads, 0);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    hx_internal_set_error("hx_probe_fma: occupancy query failed");
    return HX_ERR_CUDA;
  }
  const unsigned blocks = (unsigned)(sms * (per_sm < kBlocksPerSM ? per_sm : kBlocksPerSM));
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64)
    fma_probe_kernel<double><<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7);
  else
    fma_probe_kernel<float><<<blocks, kThreads, 0, s>>>(iters, 0.9999f, 1e-4f);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    hx_internal_set_error(cudaGetErrorString(e));
    return HX_ERR_CUDA;
  }
  *flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  return HX_OK;
}
