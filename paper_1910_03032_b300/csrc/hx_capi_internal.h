// Private declarations of the C ABI's implementation (include/hx.h is the public side):
// the mesh, operator and batch objects, the error helpers, and the functions the
// translation units hx_capi_*.cu share.  Nothing here is exported from libhx.so.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "hx.h"
#include "hx_internal.h"

namespace hxc {

// Sets the thread's last-error message (printf format) and returns s.
hx_status fail(hx_status s, const char* fmt, ...);
// Maps a CUDA error to HX_ERR_OOM / HX_ERR_CUDA with a message naming `what`.
hx_status cuda_fail(cudaError_t e, const char* what);
// The thread's last-error message (read and restored around calls that may overwrite it).
std::string& last_error();

#define HX_TRY(call, what)                             \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return hxc::cuda_fail(e_, what); \
  } while (0)

// Allocates *p unless it is already allocated: every buffer keeps one size for its owner's
// lifetime (a buffer to be resized is freed first), so a group of allocations that failed part
// way is completed, without leaks, by the next call.  Targets start as nullptr.
template <typename T>
hx_status dalloc(T** p, size_t count, const char* what) {
  if (*p) return HX_OK;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, what);
  }
  return HX_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

}  // namespace hxc

struct hx_mesh {
  int p = 0, q = 0, n = 0, N3 = 0, device = 0;
  long long E = 0, n_dof = 0;
  HxTables T;
  HxTablesF T32;  // FP32 rounding of T (inner solver of the mixed-precision refinement)
  int* R = nullptr;              // [E][n^3] (+4 ints of slack), g or -(g+1) for Dirichlet
  int* off = nullptr;            // [n_dof + 1] transpose offsets
  int* idx = nullptr;            // [E n^3] E-vector positions, increasing per DoF
  unsigned char* dir = nullptr;  // [n_dof]
  double* X8 = nullptr;          // [E][8][3]
  long long n_dirichlet = 0;     // Dirichlet DoFs (0: no boundary condition fixes the constants)
  long long grid[3] = {0, 0, 0}; // structured meshes: the logical (pN+1)-node grid of the DoFs
  HxGridAsm ga = {};  // box meshes: the grid the assembly indexes by arithmetic (ga.p = 0: none)
  HxELayout lay = {}; // layout of this mesh's E-vectors (line layout with ga, else element-major)
};

struct hx_op {
  hx_mesh* mesh = nullptr;
  double alpha = 0, nu = 0;
  int geom = 0;
  double* factors = nullptr;  // [E][7][Q3] (stored)
  double* nu_q = nullptr;     // [E][Q3] (on the fly with a field)
  bool use_field = false;     // on the fly: nu_q holds the current field
  double* yE = nullptr;       // E-vector, E n^3 values in the mesh's layout (mesh->lay)
  double* diag = nullptr;     // [n_dof] unconstrained diagonal
  // solver workspace (allocated at the first solve)
  double *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *dinv = nullptr, *partial = nullptr;
  double *hb = nullptr, *hx = nullptr;  // device staging for hx_solve_pcg_host
  double* scalars = nullptr;            // [2] device scalars (dot products)
  unsigned int* counters = nullptr;     // [2]
  HxCgState* st = nullptr;
  bool solver_ready = false;      // the whole solver workspace above and below exists
  HxCgState* st_host = nullptr;   // pinned
  cudaStream_t stream = nullptr;  // private non-blocking stream for solves
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;
  long long launches = 0;  // kernels enqueued by this operator so far (graph replays included)
  // FP32 inner solver of the mixed-precision refinement (allocated at the first mixed solve)
  float* factors32 = nullptr;  // [E][hx_f32_factor_stride(q)]: FP32 rounding of the stored factors,
                               // each element's 7 Q3 values padded to whole 16-byte units
  int* kerr = nullptr;         // device flag: a kernel's bounded wait gave up
  int wait_limit = HX_WAIT_LIMIT_DEFAULT;  // attempts of the FP32 kernel's first wait for its factors
  int f32_request = HX_F32_AUTO;  // FP32 element kernel asked for (hx_op_set_f32_kernel)
  int f32_kind = -1;              // FP32 element kernel in use (-1: not chosen yet)
  int f32_tile = 0;               // its tile variant (-1, 0, +1: half, default, twice the elements per block)
  int f32_tile_request = 0;       // tile asked for with a direct kind (hx_op_set_f32_tile)
  float f32_ms[3] = {-1.0f, -1.0f, -1.0f};  // autotuner: average time of each candidate (ms)
  float *yE32 = nullptr, *d32 = nullptr, *r32 = nullptr, *p32 = nullptr, *Ap32 = nullptr, *dinv32 = nullptr;
  double* rn2 = nullptr;        // device ||r||^2 of the outer FP64 residual
  HxCgState* st32 = nullptr;
  bool mixed_ready = false;     // the FP32 workspace above exists
  cudaGraphExec_t graph32 = nullptr;
  bool graph32_failed = false;
  bool mixed_stale = true;      // FP32 factors / diagonal need refreshing from the FP64 ones
  // pure Neumann Poisson (alpha = 0, no Dirichlet DoF): constants span the null space
  bool singular = false;
  double* m1 = nullptr;         // [n_dof] m1_i = int phi_i dx (mean-zero closure)
  double* vol = nullptr;        // [2] device: sum of m1 (the domain volume), and a dot-product slot
  // preconditioner: HX_PREC_JACOBI (dinv = 1 / diag A) or HX_PREC_COLLOCATED_MASS (1 / (alpha Mc))
  int prec = HX_PREC_JACOBI;
  double* pdiag = nullptr;      // [n_dof] alpha Mc (collocated mass)
  // the FP64 diagonal and the inverse preconditioner diagonal follow the coefficients lazily:
  // computed when a call needs them (a mixed-precision solve needs neither)
  bool diag_stale = true;
  bool dinv_stale = true;
  bool has_field = false;       // the coefficients include a per-point nu field
  // Constant-coefficient updates of stored factors: m is linear in alpha and G in nu, so a new
  // (alpha, nu), both nonzero, rescales the factors in place (rescales: in-place updates since
  // the geometry kernel last ran, bounded so that rounding cannot build up), and the diagonal is
  // alpha / alpha_d dm + nu / nu_d dk from its mass and stiffness parts dmk = [dm; dk], computed
  // once per geometry at (alpha_d, nu_d).
  double alpha_f = 0, nu_f = 0;  // the coefficients the stored factors hold
  bool factors_ok = false;       // stored factors computed without a nu field
  int rescales = 0;
  double* dmk = nullptr;         // [2][n_dof]
  double alpha_d = 0, nu_d = 0;
  bool dmk_ok = false;
  float* dmk32 = nullptr;        // the same for the FP32 operator of the mixed-precision solver
  double alpha_d32 = 0, nu_d32 = 0;
  bool dmk32_ok = false;
  // low-order refined operator (Sec. 5.2) and its Chebyshev-Jacobi inverse (HX_PREC_LOR)
  HxLorMatrix lor = {};
  long long lor_nnz = 0;
  bool lor_values_set = false;        // values of the current alpha, nu assembled
  int lor_collocated = 0;             // 1: alpha Mc + nu K_LOR (HX_PREC_LOR_MC)
  unsigned long long* lor_bound = nullptr;
  HxChebWork cheb = {0, nullptr, nullptr, nullptr, nullptr};
  double* zl = nullptr;               // [n_dof] preconditioned residual
  // geometric multigrid on the LOR matrix (HX_PREC_LOR_MG, structured meshes)
  HxMg mg = {};
  bool mg_built = false;
  double* mg_mc = nullptr;  // [n_dof] alpha Mc for the multigrid's fine stencil
  float* zl32 = nullptr;    // [n_dof] FP32 preconditioned residual (mixed solves with the multigrid)
  bool mg32 = false;        // FP32 copies of the multigrid levels allocated
};

struct hx_batch {
  int n = 0;
  std::vector<hx_op*> ops;
  std::vector<const double*> b;
  std::vector<double*> x;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t exec = nullptr;
  HxCgState* st_host = nullptr;  // pinned, n states
  double* rn2_host = nullptr;    // pinned, n true-residual norms
  double rtol = 0.0;             // stopping rule the graph was built with
  int max_it = 0;
  int lanes = 0;                 // lanes of the current graph (HX_BATCH_FUSED: lock-step mode)
  bool tune = false;             // pick the lanes by timing at the first solve
  // lock-step mode: element-kernel launches per (order, quadrature, geometry mode, nu field)
  struct Group {
    int p = 0, geom = 0, nuf = 0;
    HxTables T;
    int args_off = 0;                // the group's operators in Fused::args (and Fused::efirst)
    long long blk_off = 0, blocks = 0;  // the group's blocks in Fused::eop
  };
  struct Fused {
    bool built = false;
    std::vector<int> members;        // batch indices of the lock-step instances
    std::vector<Group> groups;
    HxCgBuffers* bufs = nullptr;     // per member: CG buffers (no loop handle)
    HxCgState** states = nullptr;    // per member: CG state
    int *vop = nullptr, *vfirst = nullptr, *vcount = nullptr;  // vector passes: block -> member
    long long vblocks = 0;
    HxApplyArgs* args = nullptr;     // per member, grouped: element-kernel arguments
    int *eop = nullptr, *efirst = nullptr;  // element blocks -> member within the group
  } fused;
};

namespace hxc {

// per-order kernel launchers (hx_capi_mesh.cu)
hx_apply_launcher apply_launcher(int p);
hx_diag_launcher diag_launcher(int p);
hx_load_launcher load_launcher(int p);

// operator (hx_capi_op.cu)
HxApplyArgs apply_args(const hx_op* op, const double* x, int constrained, const int* done);
cudaError_t element_apply(const hx_op* op, const double* x, int constrained, const int* done, cudaStream_t s);
hx_status check_kernel_flag(hx_op* op, cudaStream_t s);
hx_status ensure_diag(hx_op* op, cudaStream_t s, int* nl);
hx_status ensure_dinv(hx_op* op, cudaStream_t s);
void mg_free(hx_op* op);

// preconditioners (hx_capi_precond.cu)
hx_status lor_assemble(hx_op* op, cudaStream_t s, int* nl);

// Jacobi-PCG (hx_capi_solve.cu)
HxCgBuffers cg_buffers(const hx_op* op);
hx_status ensure_solver(hx_op* op);
cudaError_t apply_z(const hx_op* op, const double* r, double* z, const int* done, cudaStream_t s);
int z_launches(const hx_op* op);
cudaError_t cg_iteration(const hx_op* op, cudaStream_t s, unsigned long long cond = 0ull);
int iteration_launches(const hx_op* op);
cudaError_t precondition_start(const hx_op* op, cudaStream_t s);
bool build_while_graph(cudaStream_t s, const std::function<cudaError_t(unsigned long long)>& body,
                       cudaGraphExec_t* out);
constexpr int kMaxRescales = 64;  // in-place factor rescales before the geometry is recomputed
constexpr int kChunk = 16;  // CG iterations per launch of the fallback (non-conditional) path

}  // namespace hxc
