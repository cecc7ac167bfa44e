// Operator apply for callers that cannot allocate device memory.
//
// The regular path keeps the element-vector workspace of an apply inside an
// hx_op, which hx_op_create obtains with cudaMalloc.  Some callers cannot
// make that call: code inside a framework that owns all device memory through
// its own pool allocator (a cudaMalloc behind its back can fail or fragment
// the pool), services that fix their device memory budget at start-up, and
// latency-bound loops that cannot afford the device synchronization
// cudaMalloc / cudaFree imply.  hx_apply_noalloc serves them: every array is
// passed in by the caller, and the one scratch buffer the operator needs (the
// element vector between the element kernel and the assembly) is a
// fixed-size array in this file's static device memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "hx.h"
#include "hx_internal.h"

namespace {

// Element-vector scratch shared by every call on a device.  Each GPU that
// loads the library holds it (HX_NOALLOC_MAX_EVEC doubles, 32 MiB) until the
// process exits.  Host code must not pass this symbol to a kernel: on the host
// it only names a stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[HX_NOALLOC_MAX_EVEC];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;

// The scratch array's device address, cached per device together with the
// unique id of the CUDA context it was looked up in: a symbol's address
// belongs to a context, so a reset device (a new primary context) or another
// context made current by the caller triggers a new lookup.
struct ScratchSlot {
  unsigned long long ctx_id;
  double* addr;
};
ScratchSlot g_slot[kMaxDevices] = {};

// cuCtxGetCurrent / cuCtxGetId from the driver, reached through the runtime
// (the library does not link libcuda)
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

cudaError_t current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess) return e;
    if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
      return cudaErrorNotSupported;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
    get_id = reinterpret_cast<CtxGetIdFn>(f1);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (!ctx) {
    *id = 0;  // no context current yet: the runtime binds the primary context at the lookup
    return cudaSuccess;
  }
  return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch array in the current device's current context.
// The lookup (cudaGetSymbolAddress, with that device current) runs once per
// device and context; later calls reuse the cached address.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  unsigned long long id = 0;
  e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  if (id == 0 || g_slot[dev].ctx_id != id || !g_slot[dev].addr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (id == 0) {
      e = current_context_id(&id);  // the context the lookup just bound
      if (e != cudaSuccess) return e;
    }
    g_slot[dev].ctx_id = id;
    g_slot[dev].addr = static_cast<double*>(ptr);
  }
  *out = g_slot[dev].addr;
  return cudaSuccess;
}

cudaError_t launch_order(int p, const HxTables& T, const HxApplyArgs& A, cudaStream_t s) {
  switch (p) {
    case 1: return hx_launch_apply_p1(T, A, HX_KGEOM_ONTHEFLY, s);
    case 2: return hx_launch_apply_p2(T, A, HX_KGEOM_ONTHEFLY, s);
    case 3: return hx_launch_apply_p3(T, A, HX_KGEOM_ONTHEFLY, s);
    case 4: return hx_launch_apply_p4(T, A, HX_KGEOM_ONTHEFLY, s);
    case 5: return hx_launch_apply_p5(T, A, HX_KGEOM_ONTHEFLY, s);
    case 6: return hx_launch_apply_p6(T, A, HX_KGEOM_ONTHEFLY, s);
    case 7: return hx_launch_apply_p7(T, A, HX_KGEOM_ONTHEFLY, s);
    case 8: return hx_launch_apply_p8(T, A, HX_KGEOM_ONTHEFLY, s);
    default: return cudaErrorInvalidValue;
  }
}

hx_status noalloc_fail(hx_status s, const char* msg) {
  hx_internal_set_error(msg);
  return s;
}

}  // namespace

extern "C" hx_status hx_apply_noalloc(int p, int q, int64_t n_elem, int64_t n_dof, const double* X8,
                                      const int32_t* restriction, const int32_t* t_offsets,
                                      const int32_t* t_indices, double alpha, double nu, const double* x, double* y,
                                      void* stream) {
  if (p < 1 || p > HX_PMAX || (q != p + 1 && q != p + 2))
    return noalloc_fail(HX_ERR_UNSUPPORTED, "hx_apply_noalloc: need 1 <= p <= 8 and q in {p+1, p+2}");
  if (n_elem < 1 || n_dof < 1 || !X8 || !restriction || !t_offsets || !t_indices || !x || !y || x == y)
    return noalloc_fail(HX_ERR_ARG, "hx_apply_noalloc: bad size, NULL pointer, or x aliasing y");
  const long long n3 = (long long)(p + 1) * (p + 1) * (p + 1);
  if ((long double)n_elem * n3 > (long double)HX_NOALLOC_MAX_EVEC) {
    char buf[200];
    snprintf(buf, sizeof(buf),
             "hx_apply_noalloc: n_elem * (p+1)^3 = %lld exceeds the static scratch of %lld doubles",
             (long long)(n_elem * n3), (long long)HX_NOALLOC_MAX_EVEC);
    return noalloc_fail(HX_ERR_UNSUPPORTED, buf);
  }
  HxTables T;
  if (hx_build_tables(p, q, &T) != 0) return noalloc_fail(HX_ERR_UNSUPPORTED, "hx_apply_noalloc: no tables");
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(HX_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaStream_t s = (cudaStream_t)stream;
  // every entry of the scratch slab [0, n_elem (p+1)^3) is written by the element
  // kernel before the assembly reads it, so nothing has to be cleared first
  HxApplyArgs a;
  a.E = n_elem;
  a.R = restriction;
  a.x = x;
  a.yE = scratch;
  a.lay = HxELayout{0, 0u, 0};  // element-major: the caller's transpose map indexes it
  a.factors = nullptr;
  a.fstride = 0;
  a.X8 = X8;
  a.nu_q = nullptr;
  a.alpha = alpha;
  a.nu = nu;
  a.constrained = 0;
  a.done = nullptr;
  a.err = nullptr;
  a.wait_limit = HX_WAIT_LIMIT_DEFAULT;
  e = launch_order(p, T, a, s);
  const HxGridAsm no_grid = {};  // p = 0: the caller's transpose map is read
  if (e == cudaSuccess)
    e = hx_launch_assemble(n_dof, no_grid, t_offsets, t_indices, scratch, nullptr, 0, nullptr, 0.0, y, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(HX_ERR_CUDA, cudaGetErrorString(e));
  }
  return HX_OK;
}
