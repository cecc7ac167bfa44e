// C ABI of libhx.so (declared in include/hx.h): mesh and restriction setup,
// operator setup (geometric factors, diagonal), operator apply, load vector,
// and the graph-driven Jacobi-PCG solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "hx.h"
#include "hx_internal.h"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
namespace {

thread_local std::string g_err;

hx_status fail(hx_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

hx_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error
  if (e == cudaErrorMemoryAllocation) return fail(HX_ERR_OOM, "%s: out of device memory", what);
  return fail(HX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define HX_TRY(call, what)                             \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
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

}  // namespace

void hx_internal_set_error(const char* msg) { g_err = msg; }

struct hx_mesh {
  int p = 0, q = 0, n = 0, N3 = 0, device = 0;
  long long E = 0, n_dof = 0;
  HxTables T;
  HxTablesF T32;  // FP32 rounding of T (inner solver of the mixed-precision refinement)
  int* R = nullptr;              // [E][n^3], g or -(g+1) for Dirichlet
  int* off = nullptr;            // [n_dof + 1] transpose offsets
  int* idx = nullptr;            // [E n^3] E-vector positions, increasing per DoF
  unsigned char* dir = nullptr;  // [n_dof]
  double* X8 = nullptr;          // [E][8][3]
  long long n_dirichlet = 0;     // Dirichlet DoFs (0: no boundary condition fixes the constants)
  long long grid[3] = {0, 0, 0}; // structured meshes: the logical (pN+1)-node grid of the DoFs
};

struct hx_op {
  hx_mesh* mesh = nullptr;
  double alpha = 0, nu = 0;
  int geom = 0;
  double* factors = nullptr;  // [E][7][Q3] (stored)
  double* nu_q = nullptr;     // [E][Q3] (on the fly with a field)
  bool use_field = false;     // on the fly: nu_q holds the current field
  double* yE = nullptr;       // [E][n^3]
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
  float* factors32 = nullptr;  // [E][7][Q3] FP32 rounding of the stored factors (+16 bytes: the bulk
                               // copies of the element kernel round their end up to 16 bytes)
  int* kerr = nullptr;         // device flag: a kernel's bounded wait gave up
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

namespace {

// Frees every multigrid level, also the partial hierarchy of a failed set-up (the finest
// level's Chebyshev vectors belong to the LOR workspace and stay).
void mg_free(hx_op* op) {
  for (int l = 0; l < op->mg.n_levels; ++l) {
    HxMgLevel& L = op->mg.levels[l];
    dfree(L.r);
    dfree(L.coef);
    dfree(L.val);
    dfree(L.dinv);
    dfree(L.bound);
    if (l > 0) {
      dfree(L.dir_own);
      dfree(L.b);
      dfree(L.x);
      dfree(L.res);
      dfree(L.d0);
      dfree(L.d1);
    }
    dfree(L.val32);
    dfree(L.dinv32);
    dfree(L.b32);
    dfree(L.x32);
    dfree(L.r32);
    dfree(L.res32);
    dfree(L.d032);
    dfree(L.d132);
    L = HxMgLevel{};
  }
  op->mg.n_levels = 0;
  op->mg_built = false;
  op->mg32 = false;
  dfree(op->mg_mc);
}

hx_apply_launcher apply_launcher(int p) {
  static const hx_apply_launcher t[] = {nullptr, hx_launch_apply_p1, hx_launch_apply_p2, hx_launch_apply_p3,
                                        hx_launch_apply_p4, hx_launch_apply_p5, hx_launch_apply_p6,
                                        hx_launch_apply_p7, hx_launch_apply_p8};
  return t[p];
}
hx_diag_launcher diag_launcher(int p) {
  static const hx_diag_launcher t[] = {nullptr, hx_launch_diag_p1, hx_launch_diag_p2, hx_launch_diag_p3,
                                       hx_launch_diag_p4, hx_launch_diag_p5, hx_launch_diag_p6,
                                       hx_launch_diag_p7, hx_launch_diag_p8};
  return t[p];
}
hx_load_launcher load_launcher(int p) {
  static const hx_load_launcher t[] = {nullptr, hx_launch_load_p1, hx_launch_load_p2, hx_launch_load_p3,
                                       hx_launch_load_p4, hx_launch_load_p5, hx_launch_load_p6,
                                       hx_launch_load_p7, hx_launch_load_p8};
  return t[p];
}

hx_status check_order(int p, int q) {
  if (p < 1 || p > HX_PMAX) return fail(HX_ERR_UNSUPPORTED, "p = %d outside 1..%d", p, HX_PMAX);
  if (q != p + 1 && q != p + 2) return fail(HX_ERR_UNSUPPORTED, "q = %d not in {p+1, p+2} for p = %d", q, p);
  return HX_OK;
}

// Build the device mesh from host arrays.  restriction is [E][n^3] int64.
hx_status build_mesh(int p, int q, long long n_vert, const double* vert, long long E, const int64_t* ev,
                     long long n_dof, const int64_t* R, const uint8_t* dir, hx_mesh** out) {
  const int n = p + 1, N3 = n * n * n;
  if ((long double)E * N3 >= 2147483647.0L)
    return fail(HX_ERR_UNSUPPORTED, "n_elem * (p+1)^3 = %lld exceeds int32 indexing", (long long)E * N3);
  if (n_dof >= 2147483647LL) return fail(HX_ERR_UNSUPPORTED, "n_dof too large");
  // host-side restriction encoding and transpose (counting sort: deterministic order)
  std::vector<int> Renc((size_t)E * N3);
  std::vector<int> off((size_t)n_dof + 1, 0);
  for (long long k = 0; k < E * N3; ++k) {
    const long long g = R[k];
    if (g < 0 || g >= n_dof) return fail(HX_ERR_ARG, "restriction entry %lld = %lld outside [0, %lld)", k, g, n_dof);
    off[g + 1] += 1;
  }
  for (long long g = 0; g < n_dof; ++g) {
    if (off[g + 1] == 0) return fail(HX_ERR_ARG, "global DoF %lld belongs to no element", g);
    off[g + 1] += off[g];
  }
  std::vector<int> idx((size_t)E * N3), fill(off.begin(), off.end() - 1);
  for (long long k = 0; k < E * N3; ++k) {
    const long long g = R[k];
    idx[fill[g]++] = (int)k;
    Renc[k] = (dir && dir[g]) ? (int)(-g - 1) : (int)g;
  }
  std::vector<double> X8((size_t)E * 24);
  for (long long e = 0; e < E; ++e)
    for (int c = 0; c < 8; ++c) {
      const long long v = ev[e * 8 + c];
      if (v < 0 || v >= n_vert) return fail(HX_ERR_ARG, "elem_vert[%lld][%d] = %lld out of range", e, c, v);
      for (int d = 0; d < 3; ++d) X8[e * 24 + c * 3 + d] = vert[v * 3 + d];
    }
  std::vector<unsigned char> dmask((size_t)n_dof, 0);
  if (dir)
    for (long long g = 0; g < n_dof; ++g) dmask[g] = dir[g] ? 1 : 0;

  hx_mesh* m = new (std::nothrow) hx_mesh();
  if (!m) return fail(HX_ERR_OOM, "host allocation failed");
  m->p = p;
  m->q = q;
  m->n = n;
  m->N3 = N3;
  m->E = E;
  m->n_dof = n_dof;
  for (long long g = 0; g < n_dof; ++g) m->n_dirichlet += dmask[g];
  cudaGetDevice(&m->device);
  if (hx_build_tables(p, q, &m->T) == 0) hx_tables_to_float(m->T, &m->T32);
  else {
    delete m;
    return fail(HX_ERR_UNSUPPORTED, "cannot build tables for p=%d q=%d", p, q);
  }
  hx_status s;
  if ((s = dalloc(&m->R, Renc.size(), "mesh restriction")) || (s = dalloc(&m->off, off.size(), "mesh offsets")) ||
      (s = dalloc(&m->idx, idx.size(), "mesh transpose")) || (s = dalloc(&m->dir, dmask.size(), "mesh mask")) ||
      (s = dalloc(&m->X8, X8.size(), "mesh vertices"))) {
    hx_mesh_destroy(m);
    return s;
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(m->R, Renc.data(), Renc.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->dir, dmask.data(), dmask.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->X8, X8.data(), X8.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    hx_mesh_destroy(m);
    return cuda_fail(e, "mesh upload");
  }
  *out = m;
  return HX_OK;
}

}  // namespace

extern "C" {

int hx_version(void) { return 100; }

const char* hx_last_error(void) { return g_err.c_str(); }

hx_status hx_mesh_create(int p, int q, int64_t n_vert, const double* vert_xyz, int64_t n_elem,
                         const int64_t* elem_vert, int64_t n_dof, const int64_t* restriction, const uint8_t* dirichlet,
                         hx_mesh** out) {
  if (!out) return fail(HX_ERR_ARG, "out is NULL");
  *out = nullptr;
  hx_status s = check_order(p, q);
  if (s) return s;
  if (n_vert < 8 || n_elem < 1 || n_dof < 1 || !vert_xyz || !elem_vert || !restriction)
    return fail(HX_ERR_ARG, "bad sizes or NULL arrays");
  return build_mesh(p, q, n_vert, vert_xyz, n_elem, elem_vert, n_dof, restriction, dirichlet, out);
}

hx_status hx_mesh_create_box(int nx, int ny, int nz, int p, int q, const double* vert_xyz, int dirichlet_faces,
                             hx_mesh** out) {
  if (!out) return fail(HX_ERR_ARG, "out is NULL");
  *out = nullptr;
  hx_status s = check_order(p, q);
  if (s) return s;
  if (nx < 1 || ny < 1 || nz < 1 || !vert_xyz) return fail(HX_ERR_ARG, "bad grid size or NULL vertices");
  const int n = p + 1, N3 = n * n * n;
  const long long E = (long long)nx * ny * nz;
  const long long gx = (long long)p * nx + 1, gy = (long long)p * ny + 1, gz = (long long)p * nz + 1;
  const long long n_dof = gx * gy * gz;
  if ((long double)E * N3 >= 2147483647.0L) return fail(HX_ERR_UNSUPPORTED, "mesh too large for int32 indexing");
  const long long n_vert = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  std::vector<int64_t> ev((size_t)E * 8), R((size_t)E * N3);
  std::vector<uint8_t> dir((size_t)n_dof);
  const long long sx = nx + 1, sy = (long long)(nx + 1) * (ny + 1);
  long long e = 0;
  for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex, ++e) {
        for (int c = 0; c < 8; ++c)
          ev[e * 8 + c] = (ex + (c & 1)) + (ey + ((c >> 1) & 1)) * sx + (ez + ((c >> 2) & 1)) * sy;
        int l = 0;
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i, ++l)
              R[e * N3 + l] = ((long long)p * ex + i) + gx * (((long long)p * ey + j) + gy * ((long long)p * ez + k));
      }
  long long g = 0;
  for (long long K = 0; K < gz; ++K)
    for (long long J = 0; J < gy; ++J)
      for (long long I = 0; I < gx; ++I, ++g)
        dir[g] = (((dirichlet_faces & 1) && I == 0) || ((dirichlet_faces & 2) && I == gx - 1) ||
                  ((dirichlet_faces & 4) && J == 0) || ((dirichlet_faces & 8) && J == gy - 1) ||
                  ((dirichlet_faces & 16) && K == 0) || ((dirichlet_faces & 32) && K == gz - 1))
                     ? 1
                     : 0;
  s = build_mesh(p, q, n_vert, vert_xyz, E, ev.data(), n_dof, R.data(), dir.data(), out);
  if (s == HX_OK) {
    (*out)->grid[0] = gx;
    (*out)->grid[1] = gy;
    (*out)->grid[2] = gz;
  }
  return s;
}

hx_status hx_mesh_create_structured(int nx, int ny, int nz, int p, int q, const double* vert_xyz, hx_mesh** out) {
  return hx_mesh_create_box(nx, ny, nz, p, q, vert_xyz, 63, out);
}

void hx_mesh_destroy(hx_mesh* m) {
  if (!m) return;
  dfree(m->R);
  dfree(m->off);
  dfree(m->idx);
  dfree(m->dir);
  dfree(m->X8);
  delete m;
}

hx_status hx_mesh_info(const hx_mesh* m, int64_t* n_elem, int64_t* n_dof, int* p, int* q) {
  if (!m) return fail(HX_ERR_ARG, "mesh is NULL");
  if (n_elem) *n_elem = m->E;
  if (n_dof) *n_dof = m->n_dof;
  if (p) *p = m->p;
  if (q) *q = m->q;
  return HX_OK;
}

hx_status hx_mesh_qpoint_coords(const hx_mesh* m, double* xyz, void* stream) {
  if (!m || !xyz) return fail(HX_ERR_ARG, "NULL argument");
  HX_TRY(hx_launch_qpoint_coords(m->T, m->E, m->X8, xyz, (cudaStream_t)stream), "qpoint coords");
  return HX_OK;
}

hx_status hx_mesh_node_coords(const hx_mesh* m, double* xyz, void* stream) {
  if (!m || !xyz) return fail(HX_ERR_ARG, "NULL argument");
  HX_TRY(hx_launch_node_coords(m->T, m->n_dof, m->off, m->idx, m->X8, xyz, (cudaStream_t)stream), "node coords");
  return HX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// operator
// ---------------------------------------------------------------------------
namespace {

HxApplyArgs apply_args(const hx_op* op, const double* x, int constrained, const int* done) {
  const hx_mesh* m = op->mesh;
  HxApplyArgs a;
  a.E = m->E;
  a.R = m->R;
  a.x = x;
  a.yE = op->yE;
  a.factors = op->factors;
  a.X8 = m->X8;
  a.nu_q = op->use_field ? op->nu_q : nullptr;
  a.alpha = op->alpha;
  a.nu = op->nu;
  a.constrained = constrained;
  a.done = done;
  a.err = op->kerr;
  return a;
}

cudaError_t element_apply(const hx_op* op, const double* x, int constrained, const int* done, cudaStream_t s) {
  const HxApplyArgs a = apply_args(op, x, constrained, done);
  return apply_launcher(op->mesh->p)(op->mesh->T, a, op->geom, s);
}

}  // namespace

extern "C" {

void hx_op_destroy(hx_op* op) {
  if (!op) return;
  if (op->graph) cudaGraphExecDestroy(op->graph);
  if (op->ev) cudaEventDestroy(op->ev);
  if (op->stream) cudaStreamDestroy(op->stream);
  if (op->st_host) cudaFreeHost(op->st_host);
  dfree(op->factors);
  dfree(op->nu_q);
  dfree(op->yE);
  dfree(op->diag);
  dfree(op->x);
  dfree(op->r);
  dfree(op->p);
  dfree(op->Ap);
  dfree(op->dinv);
  dfree(op->partial);
  dfree(op->hb);
  dfree(op->hx);
  dfree(op->scalars);
  dfree(op->counters);
  dfree(op->st);
  if (op->graph32) cudaGraphExecDestroy(op->graph32);
  dfree(op->factors32);
  dfree(op->yE32);
  dfree(op->d32);
  dfree(op->r32);
  dfree(op->p32);
  dfree(op->Ap32);
  dfree(op->dinv32);
  dfree(op->rn2);
  dfree(op->st32);
  dfree(op->m1);
  dfree(op->vol);
  dfree(op->pdiag);
  dfree(op->kerr);
  dfree(op->lor.off);
  dfree(op->lor.col);
  dfree(op->lor.val);
  dfree(op->lor.dinv);
  dfree(op->lor.soff);
  dfree(op->lor.scol);
  dfree(op->lor.sval);
  dfree(op->lor_bound);
  dfree(op->cheb.res);
  dfree(op->cheb.d0);
  dfree(op->cheb.d1);
  dfree(op->cheb.coef);
  dfree(op->zl);
  mg_free(op);
  dfree(op->zl32);
  delete op;
}

}  // extern "C"

namespace {

// HX_ERR_CUDA when a kernel of this operator gave up a bounded wait since the last check
// (the flag is cleared).  Synchronizes s.
hx_status check_kernel_flag(hx_op* op, cudaStream_t s) {
  int flag = 0;
  HX_TRY(cudaMemcpyAsync(&flag, op->kerr, sizeof(int), cudaMemcpyDeviceToHost, s), "flag read");
  HX_TRY(cudaStreamSynchronize(s), "flag sync");
  if (flag) {
    HX_TRY(cudaMemsetAsync(op->kerr, 0, sizeof(int), s), "flag reset");
    return fail(HX_ERR_CUDA, "an element kernel's wait for its staged factors timed out");
  }
  return HX_OK;
}

// dinv = the inverse of the preconditioner's diagonal (Dirichlet rows 1): diag(A) for
// Jacobi, alpha Mc for the collocated mass (Sec. 5.1).  Counts its launches in *nl.
hx_status ensure_diag(hx_op* op, cudaStream_t s, int* nl) {
  if (!op->diag_stale) return HX_OK;
  const hx_mesh* m = op->mesh;
  HxDiagArgs d;
  d.E = m->E;
  d.factors = op->factors;
  d.X8 = m->X8;
  d.nu_q = op->use_field ? op->nu_q : nullptr;
  d.alpha = op->alpha;
  d.nu = op->nu;
  d.dE = op->yE;
  HX_TRY(diag_launcher(m->p)(m->T, d, op->geom, s), "diagonal kernel");
  HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, op->diag, s),
         "diagonal assembly");
  *nl += 2;
  op->diag_stale = false;
  return HX_OK;
}

hx_status refresh_dinv(hx_op* op, cudaStream_t s, int* nl) {
  const hx_mesh* m = op->mesh;
  const double* d = op->diag;
  if (op->prec != HX_PREC_COLLOCATED_MASS) {
    hx_status st = ensure_diag(op, s, nl);
    if (st) return st;
  }
  if (op->prec == HX_PREC_COLLOCATED_MASS) {
    if (!(op->alpha > 0.0)) return fail(HX_ERR_ARG, "the collocated mass preconditioner needs alpha > 0");
    HX_TRY(hx_launch_cmass(m->T, m->E, m->X8, op->alpha, op->yE, s), "collocated mass");
    HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, op->pdiag, s),
           "collocated mass assembly");
    *nl += 2;
    d = op->pdiag;
  }
  HX_TRY(hx_launch_dinv(m->n_dof, d, m->dir, op->dinv, s), "dinv");
  *nl += 1;
  op->dinv_stale = false;
  return HX_OK;
}

// the inverse preconditioner diagonal of the current coefficients (once the solver workspace exists)
hx_status ensure_dinv(hx_op* op, cudaStream_t s) {
  if (!op->dinv || !op->dinv_stale) return HX_OK;
  int nl = 0;
  hx_status st = refresh_dinv(op, s, &nl);
  op->launches += nl;
  return st;
}

HxLorBuild lor_build_args(const hx_op* op) {
  const hx_mesh* m = op->mesh;
  HxLorBuild b;
  b.p = m->p;
  b.n = m->n_dof;
  b.toff = m->off;
  b.tidx = m->idx;
  b.R = m->R;
  b.dir = m->dir;
  return b;
}

// Values of A_LOR for the current alpha, nu (the pattern exists), its inverse diagonal, the
// Gershgorin bound of D^-1 A_LOR and the Chebyshev coefficients.  Stream-ordered.
// CSR values of A_LOR (the Chebyshev forms and hx_op_lor_csr)
hx_status lor_csr_values(hx_op* op, cudaStream_t s, int* nl) {
  if (op->has_field) return fail(HX_ERR_UNSUPPORTED, "the LOR preconditioner takes a constant nu only");
  if (!op->lor.val) return HX_OK;  // pattern not built yet: assembled when the preconditioner is selected
  const hx_mesh* m = op->mesh;
  HX_TRY(hx_lor_values(m->T, lor_build_args(op), m->X8, op->alpha, op->nu, op->lor_collocated, op->lor, op->lor_bound,
                       s),
         "LOR values");
  HX_TRY(hx_lor_coefficients(op->lor_bound, op->cheb.degree, op->cheb.coef, s), "Chebyshev coefficients");
  *nl += 4;
  op->lor_values_set = true;
  return HX_OK;
}

// The multigrid hierarchy of the current alpha, nu: alpha Mc, the fine stencil of alpha Mc + nu K_LOR
// assembled cell by cell, then the Galerkin levels.
hx_status mg_values(hx_op* op, cudaStream_t s, int* nl) {
  if (op->has_field) return fail(HX_ERR_UNSUPPORTED, "the LOR preconditioner takes a constant nu only");
  const hx_mesh* m = op->mesh;
  const int nx = (int)((m->grid[0] - 1) / m->p), ny = (int)((m->grid[1] - 1) / m->p);
  HX_TRY(hx_launch_cmass(m->T, m->E, m->X8, op->alpha, op->yE, s), "collocated mass");
  HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, op->mg_mc, s),
         "collocated mass assembly");
  HX_TRY(hx_mg_fine(m->T, nx, ny, m->X8, op->alpha, op->nu, 1, op->mg_mc, op->mg.levels[0], s), "fine LOR stencil");
  HX_TRY(hx_mg_assemble(op->mg, s), "multigrid hierarchy");
  *nl += 2 + 10 + 3 * op->mg.n_levels;
  return HX_OK;
}

hx_status lor_assemble(hx_op* op, cudaStream_t s, int* nl) {
  if (op->prec == HX_PREC_LOR_MG) return mg_values(op, s, nl);
  return lor_csr_values(op, s, nl);
}

hx_status mg_alloc(hx_op* op, cudaStream_t s);

// The multigrid levels of a structured mesh (allocated once; values by hx_mg_assemble).  A
// failed allocation frees the partial hierarchy, so a later call starts from scratch.
hx_status mg_setup(hx_op* op, int smooth_degree, cudaStream_t s) {
  HxMg& M = op->mg;
  M.smooth_degree = smooth_degree;
  M.smooth_ratio = 10.0;
  M.coarse_degree = 16;
  if (op->mg_built) return HX_OK;
  const hx_status st = mg_alloc(op, s);
  if (st) mg_free(op);
  return st;
}

hx_status mg_alloc(hx_op* op, cudaStream_t s) {
  const hx_mesh* m = op->mesh;
  HxMg& M = op->mg;
  hx_status st = HX_OK;
  HxMgLevel& F = M.levels[0];
  F.g = HxGrid{(int)m->grid[0], (int)m->grid[1], (int)m->grid[2], m->n_dof};
  F.dir = m->dir;
  F.res = op->cheb.res;
  F.d0 = op->cheb.d0;
  F.d1 = op->cheb.d1;
  M.n_levels = 1;
  if ((st = dalloc(&F.r, (size_t)F.g.n, "MG residual")) || (st = dalloc(&F.coef, 2 * HX_LOR_MAX_DEGREE, "MG coefficients")) ||
      (st = dalloc(&F.val, 27 * (size_t)F.g.n, "MG fine stencil")) || (st = dalloc(&F.dinv, (size_t)F.g.n, "MG dinv")) ||
      (st = dalloc(&F.bound, 1, "MG bound")) || (st = dalloc(&op->mg_mc, (size_t)F.g.n, "MG collocated mass")))
    return st;
  while (M.n_levels < HX_MG_MAX_LEVELS) {
    const HxGrid& g = M.levels[M.n_levels - 1].g;
    if (!(g.mx % 2 == 1 && g.my % 2 == 1 && g.mz % 2 == 1 && g.mx >= 5 && g.my >= 5 && g.mz >= 5)) break;
    HxMgLevel& C = M.levels[M.n_levels];
    C.g = HxGrid{(g.mx + 1) / 2, (g.my + 1) / 2, (g.mz + 1) / 2, 0};
    C.g.n = (long long)C.g.mx * C.g.my * C.g.mz;
    const size_t n = (size_t)C.g.n;
    ++M.n_levels;  // counted before the allocations so that destroy frees a partial level
    if ((st = dalloc(&C.dir_own, n, "MG mask")) || (st = dalloc(&C.val, 27 * n, "MG stencil")) ||
        (st = dalloc(&C.dinv, n, "MG dinv")) || (st = dalloc(&C.b, n, "MG b")) || (st = dalloc(&C.x, n, "MG x")) ||
        (st = dalloc(&C.r, n, "MG r")) || (st = dalloc(&C.res, n, "MG res")) || (st = dalloc(&C.d0, n, "MG d0")) ||
        (st = dalloc(&C.d1, n, "MG d1")) || (st = dalloc(&C.coef, 2 * HX_LOR_MAX_DEGREE, "MG coefficients")) ||
        (st = dalloc(&C.bound, 1, "MG bound")))
      return st;
    C.dir = C.dir_own;
    HX_TRY(hx_mg_coarse_dir(M.levels[M.n_levels - 2], C, s), "MG coarse mask");
    op->launches += 1;
  }
  op->mg_built = true;
  return HX_OK;
}

// The preconditioned-residual vector and the Chebyshev workspace for `degree` steps.
hx_status lor_workspace(hx_op* op, int degree) {
  const long long n = op->mesh->n_dof;
  hx_status st = HX_OK;
  // each buffer on its own: a call after a failed allocation fills in only what is missing
  if ((!op->zl && (st = dalloc(&op->zl, (size_t)n, "preconditioned residual"))) ||
      (!op->cheb.res && (st = dalloc(&op->cheb.res, (size_t)n, "cheb res"))) ||
      (!op->cheb.d0 && (st = dalloc(&op->cheb.d0, (size_t)n, "cheb d0"))) ||
      (!op->cheb.d1 && (st = dalloc(&op->cheb.d1, (size_t)n, "cheb d1"))) ||
      (!op->cheb.coef && (st = dalloc(&op->cheb.coef, 2 * HX_LOR_MAX_DEGREE, "cheb coefficients"))))
    return st;
  op->cheb.degree = degree;
  return HX_OK;
}

// The LOR pattern (CSR, built once per operator) and the Chebyshev workspace for `degree`
// steps.  Synchronizes `s` once to size the column array.
hx_status lor_setup(hx_op* op, int degree, cudaStream_t s) {
  const hx_mesh* m = op->mesh;
  const long long n = m->n_dof;
  hx_status st = HX_OK;
  if (!op->lor.val) {
    long long* count = nullptr;
    long long* sums = nullptr;
    int* bad = nullptr;
    int nbad = 0;
    long long nnz = 0;
    do {
      if ((st = dalloc(&count, (size_t)n, "LOR counts")) || (st = dalloc(&sums, (size_t)hx_lor_scan_blocks(n) + 1, "scan")) ||
          (st = dalloc(&bad, 1, "flag")) || (st = dalloc(&op->lor.off, (size_t)n + 1, "LOR offsets")) ||
          (st = dalloc(&op->lor.dinv, (size_t)n, "LOR inverse diagonal")) ||
          (st = dalloc(&op->lor_bound, 1, "LOR bound")))
        break;
      cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
      const HxLorBuild b = lor_build_args(op);
      if (e == cudaSuccess) e = hx_lor_count(b, count, bad, s);
      if (e == cudaSuccess) e = hx_lor_scan(n, count, sums, op->lor.off, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, op->lor.off + n, sizeof(long long), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "LOR pattern");
        break;
      }
      if (nbad > 0) {
        st = fail(HX_ERR_UNSUPPORTED, "%d LOR rows have more than %d columns", nbad, HX_LOR_MAX_NB);
        break;
      }
      if ((st = dalloc(&op->lor.col, (size_t)nnz, "LOR columns")) || (st = dalloc(&op->lor.val, (size_t)nnz, "LOR values")))
        break;
      e = hx_lor_fill(b, op->lor.off, op->lor.col, s);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "LOR pattern fill");
        break;
      }
      // the sliced-ELL copy: slice widths, their offsets, then the columns
      const long long ns = (n + 31) / 32;
      long long sn = 0;
      if ((st = dalloc(&op->lor.soff, (size_t)ns + 1, "LOR slice offsets"))) break;
      e = hx_lor_sell_count(n, op->lor.off, count, s);
      if (e == cudaSuccess) e = hx_lor_scan(ns, count, sums, op->lor.soff, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&sn, op->lor.soff + ns, sizeof(long long), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "LOR slices");
        break;
      }
      if ((st = dalloc(&op->lor.scol, (size_t)sn, "LOR slice columns")) ||
          (st = dalloc(&op->lor.sval, (size_t)sn, "LOR slice values")))
        break;
      op->lor.n = n;
      e = hx_lor_sell_copy(op->lor, op->lor.col, nullptr, s);
      if (e != cudaSuccess) st = cuda_fail(e, "LOR slice columns");
      op->launches += 6 + 5;
    } while (0);
    dfree(count);
    dfree(sums);
    dfree(bad);
    if (st) {
      // nothing of a failed pattern survives: a later call starts from scratch (no leak)
      dfree(op->lor.off);
      dfree(op->lor.dinv);
      dfree(op->lor_bound);
      dfree(op->lor.col);
      dfree(op->lor.val);
      dfree(op->lor.soff);
      dfree(op->lor.scol);
      dfree(op->lor.sval);
      return st;
    }
    op->lor.n = n;
    op->lor_nnz = nnz;
  }
  return lor_workspace(op, degree);
}

// Coefficient-dependent setup, stream-ordered and allocation-free: stored
// factors (alpha, nu) and the assembled diagonal (and its inverse once the
// solver workspace exists).  `bad` (nullable) counts detJ <= 0 points.
hx_status setup_coefficients(hx_op* op, double alpha, double nu, const double* nu_q, int* bad, cudaStream_t s,
                             int* launches) {
  hx_mesh* m = op->mesh;
  const long long Q3 = (long long)m->q * m->q * m->q;
  int nl = 0;
  cudaError_t e;
  op->alpha = alpha;
  op->nu = nu;
  op->has_field = nu_q != nullptr;
  op->lor_values_set = false;
  // alpha = 0 with nothing fixed on the boundary: K alone, singular on the constants
  op->singular = (alpha == 0.0 && m->n_dirichlet == 0);
  if (op->geom == HX_GEOM_STORED) {
    HX_TRY(hx_launch_geometry(m->T, m->E, m->X8, nu_q, alpha, nu, op->factors, bad, s), "geometry kernel");
    ++nl;
  } else {
    op->use_field = nu_q != nullptr;
    if (nu_q && nu_q != op->nu_q) {
      e = cudaMemcpyAsync(op->nu_q, nu_q, sizeof(double) * m->E * Q3, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "nu copy");
    }
  }
  op->diag_stale = true;
  op->dinv_stale = true;
  if (launches) *launches = nl;
  if (op->prec == HX_PREC_LOR || op->prec == HX_PREC_LOR_MG) {
    hx_status st = lor_assemble(op, s, &nl);
    if (launches) *launches = nl;
    if (st) return st;
  }
  return HX_OK;
}

}  // namespace

extern "C" {

hx_status hx_op_create(hx_mesh* m, double alpha, double nu, const double* nu_q, int geom_mode, void* stream,
                       hx_op** out) {
  if (!out) return fail(HX_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!m) return fail(HX_ERR_ARG, "mesh is NULL");
  if (geom_mode != HX_GEOM_STORED && geom_mode != HX_GEOM_ONTHEFLY) return fail(HX_ERR_ARG, "bad geom_mode");
  cudaStream_t s = (cudaStream_t)stream;
  hx_op* op = new (std::nothrow) hx_op();
  if (!op) return fail(HX_ERR_OOM, "host allocation failed");
  op->mesh = m;
  op->geom = geom_mode;
  const long long Q3 = (long long)m->q * m->q * m->q;
  int* bad = nullptr;
  double* tmp = nullptr;
  hx_status st = HX_OK;
  int nbad = 0;
  cudaError_t e = cudaSuccess;
  do {
    if ((st = dalloc(&op->yE, (size_t)m->E * m->N3, "E-vector"))) break;
    if ((st = dalloc(&op->diag, (size_t)m->n_dof, "diagonal"))) break;
    if ((st = dalloc(&op->kerr, 1, "kernel error flag"))) break;
    if ((e = cudaMemsetAsync(op->kerr, 0, sizeof(int), s)) != cudaSuccess) { st = cuda_fail(e, "memset"); break; }
    if ((st = dalloc(&bad, 1, "flag"))) break;
    if ((e = cudaMemsetAsync(bad, 0, sizeof(int), s)) != cudaSuccess) { st = cuda_fail(e, "memset"); break; }
    if (geom_mode == HX_GEOM_STORED) {
      if ((st = dalloc(&op->factors, (size_t)m->E * 7 * Q3, "geometric factors"))) break;
    } else {
      if (nu_q && (st = dalloc(&op->nu_q, (size_t)m->E * Q3, "nu field"))) break;
      // detJ check through the factor kernel, a bounded slab of elements at a time
      const long long chunk = 65536;
      if ((st = dalloc(&tmp, (size_t)std::min(chunk, m->E) * 7 * Q3, "detJ check"))) break;
      for (long long e0 = 0; e0 < m->E && e == cudaSuccess; e0 += chunk) {
        const long long ne = std::min(chunk, m->E - e0);
        e = hx_launch_geometry(m->T, ne, m->X8 + e0 * 24, nullptr, 1.0, 1.0, tmp, bad, s);
      }
      if (e != cudaSuccess) { st = cuda_fail(e, "detJ check"); break; }
    }
    int nl = 0;
    if ((st = setup_coefficients(op, alpha, nu, nu_q, bad, s, &nl))) break;
    op->launches += nl;
    if (m->n_dirichlet == 0) {
      // m1_i = int phi_i dx and its sum (the volume), for the mean-zero closure of a
      // pure Neumann Poisson solve (Sec. 4.2, Eq. (meanZero))
      if ((st = dalloc(&op->m1, (size_t)m->n_dof, "mass row sums")) || (st = dalloc(&op->vol, 2, "volume"))) break;
      HxLoadArgs la;
      la.E = m->E;
      la.X8 = m->X8;
      la.fq = nullptr;
      la.yE = op->yE;
      e = load_launcher(m->p)(m->T, la, s);
      if (e == cudaSuccess) e = hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, op->m1, s);
      if (e != cudaSuccess) { st = cuda_fail(e, "mass row sums"); break; }
      op->launches += 2;
    }
    e = cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = cuda_fail(e, "operator setup"); break; }
    if (nbad > 0) st = fail(HX_ERR_INVALID_MESH, "detJ <= 0 at %d quadrature points", nbad);
  } while (0);
  dfree(bad);
  dfree(tmp);
  if (st != HX_OK) {
    hx_op_destroy(op);
    return st;
  }
  *out = op;
  return HX_OK;
}

hx_status hx_op_set_coefficients(hx_op* op, double alpha, double nu, const double* nu_q, void* stream) {
  if (!op) return fail(HX_ERR_ARG, "op is NULL");
  if (op->geom == HX_GEOM_ONTHEFLY && nu_q && !op->nu_q)
    return fail(HX_ERR_ARG, "on-the-fly operator created without a nu field cannot take one");
  if ((op->prec == HX_PREC_LOR || op->prec == HX_PREC_LOR_MG) && nu_q)
    return fail(HX_ERR_UNSUPPORTED, "the LOR preconditioner takes a constant nu only");
  if (op->prec == HX_PREC_COLLOCATED_MASS && !(alpha > 0.0))
    return fail(HX_ERR_ARG, "the collocated mass preconditioner needs alpha > 0");
  int nl = 0;
  hx_status st = setup_coefficients(op, alpha, nu, nu_q, nullptr, (cudaStream_t)stream, &nl);
  if (st == HX_OK) op->launches += nl;
  op->mixed_stale = true;
  if (op->graph32) {
    cudaGraphExecDestroy(op->graph32);
    op->graph32 = nullptr;
  }
  if (op->geom == HX_GEOM_ONTHEFLY && op->graph) {
    // the captured CG iterations carry alpha, nu (and the field pointer) as kernel
    // parameters: drop the graph so the next solve captures the new values
    cudaGraphExecDestroy(op->graph);
    op->graph = nullptr;
  }
  return st;
}

int64_t hx_op_launch_count(const hx_op* op) { return op ? op->launches : -1; }

hx_status hx_op_info(const hx_op* op, int64_t* n_elem, int64_t* n_dof, int* p, int* q) {
  if (!op) return fail(HX_ERR_ARG, "op is NULL");
  return hx_mesh_info(op->mesh, n_elem, n_dof, p, q);
}

hx_status hx_op_apply(hx_op* op, const double* x, double* y, int constrained, void* stream) {
  if (!op || !x || !y) return fail(HX_ERR_ARG, "NULL argument");
  if (x == y) return fail(HX_ERR_ARG, "x and y must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  const hx_mesh* m = op->mesh;
  HX_TRY(element_apply(op, x, constrained, nullptr, s), "element kernel");
  HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, constrained, x, 0.0, y, s), "assembly");
  op->launches += 2;
  return HX_OK;
}

hx_status hx_op_diagonal(hx_op* op, double* diag, int constrained, void* stream) {
  if (!op || !diag) return fail(HX_ERR_ARG, "NULL argument");
  int nl = 0;
  hx_status st = ensure_diag(op, (cudaStream_t)stream, &nl);
  op->launches += nl;
  if (st) return st;
  HX_TRY(hx_launch_masked_copy(op->mesh->n_dof, op->diag, op->mesh->dir, constrained, 1.0, diag,
                               (cudaStream_t)stream),
         "diagonal copy");
  op->launches += 1;
  return HX_OK;
}

hx_status hx_op_load_vector(hx_op* op, const double* f_q, double* b, void* stream) {
  if (!op || !f_q || !b) return fail(HX_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const hx_mesh* m = op->mesh;
  HxLoadArgs a;
  a.E = m->E;
  a.X8 = m->X8;
  a.fq = f_q;
  a.yE = op->yE;
  HX_TRY(load_launcher(m->p)(m->T, a, s), "load kernel");
  HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, b, s), "assembly");
  op->launches += 2;
  return HX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Jacobi-PCG
// ---------------------------------------------------------------------------
namespace {

HxCgBuffers cg_buffers(const hx_op* op) {
  const hx_mesh* m = op->mesh;
  HxCgBuffers b;
  b.n = m->n_dof;
  b.off = m->off;
  b.idx = m->idx;
  b.dir = m->dir;
  b.x = op->x;
  b.r = op->r;
  b.p = op->p;
  b.Ap = op->Ap;
  b.dinv = op->dinv;
  b.yE = op->yE;
  b.partial = op->partial;
  b.st = op->st;
  b.z = (op->prec == HX_PREC_LOR || op->prec == HX_PREC_LOR_MG) ? op->zl : nullptr;
  b.cond = 0ull;
  b.nullspace = op->singular ? 1 : 0;
  return b;
}

hx_status ensure_solver(hx_op* op) {
  if (op->solver_ready) return HX_OK;
  const long long n = op->mesh->n_dof;
  hx_status s;
  if ((s = dalloc(&op->x, n, "cg x")) || (s = dalloc(&op->r, n, "cg r")) || (s = dalloc(&op->p, n, "cg p")) ||
      (s = dalloc(&op->Ap, n, "cg Ap")) || (s = dalloc(&op->dinv, n, "cg dinv")) ||
      (s = dalloc(&op->partial, HX_RED_VALUES * HX_RED_BLOCKS, "cg partials")) || (s = dalloc(&op->scalars, 2, "scalars")) ||
      (s = dalloc(&op->counters, 2, "counters")) || (s = dalloc(&op->st, 1, "cg state")))
    return s;
  if (!op->st_host) HX_TRY(cudaMallocHost((void**)&op->st_host, sizeof(HxCgState)), "pinned state");
  if (!op->stream) HX_TRY(cudaStreamCreateWithFlags(&op->stream, cudaStreamNonBlocking), "solver stream");
  if (!op->ev) HX_TRY(cudaEventCreateWithFlags(&op->ev, cudaEventDisableTiming), "solver event");
  HX_TRY(cudaMemsetAsync(op->st, 0, sizeof(HxCgState), op->stream), "state init");
  HX_TRY(cudaMemsetAsync(op->counters, 0, 2 * sizeof(unsigned int), op->stream), "counter init");
  op->dinv_stale = true;  // computed by the first call that needs it
  op->solver_ready = true;
  return HX_OK;
}

// One CG iteration: element kernel on p, fused assembly + (p, Ap), update, direction.
// z = M^-1 r for the preconditioners that run outside the CG kernels (LOR forms)
cudaError_t apply_z(const hx_op* op, const double* r, double* z, const int* done, cudaStream_t s) {
  if (op->prec == HX_PREC_LOR_MG) return hx_mg_vcycle(op->mg, r, z, done, s);
  return hx_lor_precondition(op->lor, op->cheb, r, z, done, s);
}
int z_launches(const hx_op* op) {
  if (op->prec == HX_PREC_LOR_MG) return hx_mg_vcycle_launches(op->mg);
  if (op->prec == HX_PREC_LOR) return op->cheb.degree;
  return 0;
}

// One CG iteration: element kernel on p, fused assembly + (p, Ap), update, direction.
// cond: the conditional handle of an enclosing graph while loop (0 outside one).
cudaError_t cg_iteration(const hx_op* op, cudaStream_t s, unsigned long long cond = 0ull) {
  HxCgBuffers b = cg_buffers(op);
  b.cond = cond;
  cudaError_t e = element_apply(op, op->p, 1, &op->st->done, s);
  if (e == cudaSuccess) e = hx_launch_cg_assemble_pap(b, s);
  if (e == cudaSuccess) e = hx_launch_cg_update(b, s);
  if (e == cudaSuccess && b.z) {
    e = apply_z(op, op->r, op->zl, &op->st->done, s);
    if (e == cudaSuccess) e = hx_launch_cg_rz(b, s);
  }
  if (e == cudaSuccess) e = hx_launch_cg_direction(b, s);
  return e;
}

// kernels one CG iteration launches
int iteration_launches(const hx_op* op) { return z_launches(op) > 0 ? 4 + z_launches(op) + 1 : 4; }

// z = M^-1 r before the first direction (LOR preconditioner only; Jacobi is fused into cg_start)
cudaError_t precondition_start(const hx_op* op, cudaStream_t s) {
  if (op->prec != HX_PREC_LOR && op->prec != HX_PREC_LOR_MG) return cudaSuccess;
  return apply_z(op, op->r, op->zl, &op->st->done, s);
}

constexpr int kChunk = 16;  // CG iterations per launch of the fallback (non-conditional) path

// A graph holding one while node whose body is captured from body(handle); the body's
// last kernel keeps the loop going while its CG has not finished.  Returns false when
// the driver refuses conditional nodes (the caller then falls back to chunked launches).
bool build_while_graph(cudaStream_t s, const std::function<cudaError_t(unsigned long long)>& body,
                       cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  cudaGraphConditionalHandle h = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  // the parameter union has no default constructor: zero raw storage instead
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(raw);
  np->type = cudaGraphNodeTypeConditional;
  np->conditional.handle = h;
  np->conditional.type = cudaGraphCondTypeWhile;
  np->conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, np);
  if (e == cudaSuccess) {
    cudaGraph_t bodyg = np->conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t eb = body((unsigned long long)h);
      e = cudaStreamEndCapture(s, &bodyg);
      if (eb != cudaSuccess) e = eb;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return false;
  }
  return true;
}

void ensure_graph(hx_op* op) {
  if (op->graph || op->graph_failed) return;
  if (!build_while_graph(op->stream, [op](unsigned long long h) { return cg_iteration(op, op->stream, h); },
                         &op->graph))
    op->graph_failed = true;  // fall back to chunks of direct launches of the same kernels
}

hx_status solve_device(hx_op* op, const double* b, double* x, double rtol, int max_it, int use_x0,
                       cudaStream_t user, hx_solve_info* info) {
  const hx_mesh* m = op->mesh;
  hx_status s = ensure_solver(op);
  if (s) return s;
  ensure_graph(op);
  cudaStream_t st = op->stream;
  // order after the caller's prior work on `user`
  HX_TRY(cudaEventRecord(op->ev, user), "event record");
  HX_TRY(cudaStreamWaitEvent(st, op->ev, 0), "stream wait");
  if ((s = ensure_dinv(op, st))) return s;
  const HxCgBuffers buf = cg_buffers(op);
  const long long launches0 = op->launches;
  if (op->singular) {
    // pure Neumann: remove the mean of b (orthogonal to the constant null space, Sec. 5.3)
    HX_TRY(hx_launch_cg_mean(buf, b, st), "cg mean");
    op->launches += 1;
  }
  HX_TRY(hx_launch_cg_init(buf, b, use_x0 ? x : nullptr, rtol, max_it, st), "cg init");
  if (use_x0) {
    HX_TRY(element_apply(op, op->x, 1, nullptr, st), "cg x0 apply");
    HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, st), "cg x0 assembly");
    HX_TRY(hx_launch_cg_residual(buf, st), "cg residual");
    op->launches += 3;
  }
  HX_TRY(precondition_start(op, st), "first preconditioner");
  HX_TRY(hx_launch_cg_start(buf, st), "cg start");
  op->launches += 2 + z_launches(op);
  if (op->singular) {
    HX_TRY(hx_launch_cg_direction(buf, st), "cg first direction");  // p = z - mean z
    op->launches += 1;
  }
  if (op->graph) {
    // the whole iteration runs on the device: one graph launch, one synchronization
    HX_TRY(cudaGraphLaunch(op->graph, st), "graph launch");
    HX_TRY(cudaMemcpyAsync(op->st_host, op->st, sizeof(HxCgState), cudaMemcpyDeviceToHost, st), "state read");
    HX_TRY(cudaStreamSynchronize(st), "solver sync");
    op->launches += iteration_launches(op) * (long long)op->st_host->loops;
    if (!op->st_host->done) return fail(HX_ERR_CUDA, "CG graph loop ended before the solver finished");
  } else {
    for (;;) {
      HX_TRY(cudaMemcpyAsync(op->st_host, op->st, sizeof(HxCgState), cudaMemcpyDeviceToHost, st), "state read");
      HX_TRY(cudaStreamSynchronize(st), "solver sync");
      if (op->st_host->done) break;
      for (int i = 0; i < kChunk; ++i) HX_TRY(cg_iteration(op, st), "cg iteration");
      op->launches += iteration_launches(op) * kChunk;
    }
  }
  const HxCgState cs = *op->st_host;
  if (op->singular) {
    // mean-zero closure int x dx = m1 . x = 0 (Sec. 4.2, Eq. (meanZero)); K 1 = 0 keeps the residual
    HX_TRY(hx_launch_sum(m->n_dof, op->m1, op->partial, op->counters, op->vol, st), "volume");
    HX_TRY(hx_launch_dot(m->n_dof, op->m1, op->x, op->partial, op->counters, op->vol + 1, st), "mean");
    HX_TRY(hx_launch_shift(m->n_dof, op->x, op->vol + 1, op->vol, st), "mean shift");
    op->launches += 3;
  }
  // true residual ||P b - A_c x|| with one extra apply
  HX_TRY(element_apply(op, op->x, 1, nullptr, st), "residual apply");
  HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, st), "residual assembly");
  HX_TRY(hx_launch_resnorm(m->n_dof, b, op->Ap, m->dir, op->partial, op->counters, op->scalars, st,
                           op->singular ? &op->st->shift : nullptr),
         "residual norm");
  op->launches += 3;
  double rn2 = 0.0;
  HX_TRY(cudaMemcpyAsync(&rn2, op->scalars, sizeof(double), cudaMemcpyDeviceToHost, st), "residual read");
  HX_TRY(cudaMemcpyAsync(x, op->x, sizeof(double) * m->n_dof, cudaMemcpyDeviceToDevice, st), "solution copy");
  HX_TRY(cudaStreamSynchronize(st), "solver sync");
  const double bn = std::sqrt(cs.bb);
  hx_solve_info inf;
  inf.iterations = cs.iter;
  inf.status = cs.status;
  inf.b_norm = bn;
  inf.rel_residual = bn > 0 ? std::sqrt(cs.rr) / bn : 0.0;
  inf.true_rel_residual = bn > 0 ? std::sqrt(rn2) / bn : std::sqrt(rn2);
  inf.kernel_launches = (int)(op->launches - launches0);
  inf.refinements = 0;
  if (info) *info = inf;
  if (cs.status == HX_ERR_NOT_CONVERGED)
    return fail(HX_ERR_NOT_CONVERGED, "not converged in %d iterations (rel. residual %.3e)", cs.iter, inf.rel_residual);
  if (cs.status == HX_ERR_BREAKDOWN) return fail(HX_ERR_BREAKDOWN, "CG breakdown at iteration %d", cs.iter);
  return HX_OK;
}

}  // namespace

extern "C" {

hx_status hx_solve_pcg(hx_op* op, const double* b, double* x, double rtol, int max_it, int use_x0, void* stream,
                       hx_solve_info* info) {
  if (!op || !b || !x) return fail(HX_ERR_ARG, "NULL argument");
  if (!(rtol >= 0.0) || max_it < 0) return fail(HX_ERR_ARG, "rtol must be >= 0 and max_it >= 0");
  return solve_device(op, b, x, rtol, max_it, use_x0, (cudaStream_t)stream, info);
}

hx_status hx_solve_pcg_host(hx_op* op, const double* b_host, double* x_host, double rtol, int max_it, int use_x0,
                            void* stream, hx_solve_info* info) {
  if (!op || !b_host || !x_host) return fail(HX_ERR_ARG, "NULL argument");
  if (!(rtol >= 0.0) || max_it < 0) return fail(HX_ERR_ARG, "rtol must be >= 0 and max_it >= 0");
  const long long n = op->mesh->n_dof;
  hx_status s = ensure_solver(op);
  if (s) return s;
  if ((s = dalloc(&op->hb, n, "staging b")) || (s = dalloc(&op->hx, n, "staging x"))) return s;
  // the uploads run on the solver stream after the caller's prior work on `stream`
  HX_TRY(cudaEventRecord(op->ev, (cudaStream_t)stream), "event record");
  HX_TRY(cudaStreamWaitEvent(op->stream, op->ev, 0), "stream wait");
  HX_TRY(cudaMemcpyAsync(op->hb, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, op->stream), "b upload");
  if (use_x0)
    HX_TRY(cudaMemcpyAsync(op->hx, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, op->stream), "x0 upload");
  hx_status r = solve_device(op, op->hb, op->hx, rtol, max_it, use_x0, op->stream, info);
  if (r != HX_OK && r != HX_ERR_NOT_CONVERGED && r != HX_ERR_BREAKDOWN) return r;
  const std::string msg = g_err;
  HX_TRY(cudaMemcpyAsync(x_host, op->hx, sizeof(double) * n, cudaMemcpyDeviceToHost, op->stream), "x download");
  HX_TRY(cudaStreamSynchronize(op->stream), "solver sync");
  g_err = msg;
  return r;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mixed precision: FP64 iterative refinement around an FP32 Jacobi-PCG
// ---------------------------------------------------------------------------
namespace {

HxApplyArgsF apply_args32(const hx_op* op, const float* x, const int* done) {
  const hx_mesh* m = op->mesh;
  HxApplyArgsF a;
  a.E = m->E;
  a.R = m->R;
  a.x = x;
  a.yE = op->yE32;
  a.factors = op->factors32;
  a.X8 = m->X8;
  a.nu_q = op->use_field ? op->nu_q : nullptr;
  a.alpha = op->alpha;
  a.nu = op->nu;
  a.constrained = 1;
  a.done = done;
  a.err = op->kerr;
  return a;
}

cudaError_t element_apply32(const hx_op* op, const float* x, const int* done, cudaStream_t s) {
  static const hx_apply32_launcher t[] = {nullptr, hx_launch_apply32_p1, hx_launch_apply32_p2, hx_launch_apply32_p3,
                                          hx_launch_apply32_p4, hx_launch_apply32_p5, hx_launch_apply32_p6,
                                          hx_launch_apply32_p7, hx_launch_apply32_p8};
  const HxApplyArgsF a = apply_args32(op, x, done);
  return t[op->mesh->p](op->mesh->T32, a, op->geom, s);
}

HxCgBuffersF cg_buffers32(const hx_op* op) {
  const hx_mesh* m = op->mesh;
  HxCgBuffersF b;
  b.n = m->n_dof;
  b.off = m->off;
  b.idx = m->idx;
  b.dir = m->dir;
  b.x = op->d32;
  b.r = op->r32;
  b.p = op->p32;
  b.Ap = op->Ap32;
  b.dinv = op->dinv32;
  b.yE = op->yE32;
  b.partial = op->partial;
  b.st = op->st32;
  b.z = (op->prec == HX_PREC_LOR_MG) ? op->zl32 : nullptr;
  b.cond = 0ull;
  b.nullspace = op->singular ? 1 : 0;
  return b;
}

// FP32 workspace and the FP32 rounding of the stored factors and inverse diagonal.
hx_status ensure_mixed(hx_op* op) {
  const hx_mesh* m = op->mesh;
  const long long n = m->n_dof;
  hx_status s;
  if (!op->mixed_ready) {
    if ((s = dalloc(&op->yE32, (size_t)m->E * m->N3, "FP32 E-vector")) || (s = dalloc(&op->d32, n, "FP32 d")) ||
        (s = dalloc(&op->r32, n, "FP32 r")) || (s = dalloc(&op->p32, n, "FP32 p")) ||
        (s = dalloc(&op->Ap32, n, "FP32 Ap")) || (s = dalloc(&op->dinv32, n, "FP32 dinv")) ||
        (s = dalloc(&op->rn2, 1, "residual norm")) || (s = dalloc(&op->st32, 1, "FP32 state")))
      return s;
    if (op->geom == HX_GEOM_STORED &&
        (s = dalloc(&op->factors32, (size_t)m->E * 7 * m->q * m->q * m->q + 4, "FP32 factors")))
      return s;
    HX_TRY(cudaMemsetAsync(op->st32, 0, sizeof(HxCgState), op->stream), "FP32 state init");
    op->mixed_ready = true;
  }
  if (op->prec == HX_PREC_LOR_MG && !op->mg32) {
    // FP32 copies of the multigrid levels: stencils, inverse diagonals, work vectors
    for (int l = 0; l < op->mg.n_levels; ++l) {
      HxMgLevel& L = op->mg.levels[l];
      const size_t nl = (size_t)L.g.n;
      if ((s = dalloc(&L.val32, 27 * nl, "FP32 MG stencil")) || (s = dalloc(&L.dinv32, nl, "FP32 MG dinv")) ||
          (s = dalloc(&L.r32, nl, "FP32 MG r")) || (s = dalloc(&L.res32, nl, "FP32 MG res")) ||
          (s = dalloc(&L.d032, nl, "FP32 MG d0")) || (s = dalloc(&L.d132, nl, "FP32 MG d1")))
        return s;
      if (l > 0 && ((s = dalloc(&L.b32, nl, "FP32 MG b")) || (s = dalloc(&L.x32, nl, "FP32 MG x")))) return s;
    }
    if ((s = dalloc(&op->zl32, (size_t)n, "FP32 preconditioned residual"))) return s;
    op->mg32 = true;
    op->mixed_stale = true;
  }
  if (op->mixed_stale) {
    if (op->geom == HX_GEOM_STORED)
      HX_TRY(hx_launch_to_float((long long)m->E * 7 * m->q * m->q * m->q, op->factors, op->factors32, op->stream),
             "FP32 factors");
    if (op->prec == HX_PREC_LOR_MG) {
      HX_TRY(hx_mg_to_float(op->mg, op->stream), "FP32 multigrid levels");
      op->launches += 2 * op->mg.n_levels;
    } else if (op->prec == HX_PREC_JACOBI) {
      // the inner solver's Jacobi diagonal: the diagonal of the FP32 operator, computed in FP32
      static const hx_diag32_launcher t[] = {nullptr, hx_launch_diag32_p1, hx_launch_diag32_p2, hx_launch_diag32_p3,
                                             hx_launch_diag32_p4, hx_launch_diag32_p5, hx_launch_diag32_p6,
                                             hx_launch_diag32_p7, hx_launch_diag32_p8};
      HxDiagArgsF d;
      d.E = m->E;
      d.factors = op->factors32;
      d.X8 = m->X8;
      d.nu_q = op->use_field ? op->nu_q : nullptr;
      d.alpha = op->alpha;
      d.nu = op->nu;
      d.dE = op->yE32;
      HX_TRY(t[m->p](m->T32, d, op->geom, op->stream), "FP32 diagonal kernel");
      HX_TRY(hx_launch_assemble32(n, m->off, m->idx, op->yE32, m->dir, 0, nullptr, op->Ap32, op->stream),
             "FP32 diagonal assembly");
      HX_TRY(hx_launch_dinv32(n, op->Ap32, m->dir, op->dinv32, op->stream), "FP32 dinv");
      op->launches += 3;
    } else {
      if ((s = ensure_dinv(op, op->stream))) return s;
      HX_TRY(hx_launch_to_float(n, op->dinv, op->dinv32, op->stream), "FP32 dinv");
      op->launches += 1;
    }
    op->launches += (op->geom == HX_GEOM_STORED) ? 1 : 0;
    op->mixed_stale = false;
  }
  return HX_OK;
}

cudaError_t cg_iteration32(const hx_op* op, cudaStream_t s, unsigned long long cond = 0ull) {
  HxCgBuffersF b = cg_buffers32(op);
  b.cond = cond;
  cudaError_t e = element_apply32(op, op->p32, &op->st32->done, s);
  if (e == cudaSuccess) e = hx_launch_cg_assemble_pap(b, s);
  if (e == cudaSuccess) e = hx_launch_cg_update(b, s);
  if (e == cudaSuccess && b.z) {
    e = hx_mg_vcycle32(op->mg, op->r32, op->zl32, &op->st32->done, s);
    if (e == cudaSuccess) e = hx_launch_cg_rz(b, s);
  }
  if (e == cudaSuccess) e = hx_launch_cg_direction(b, s);
  return e;
}

void ensure_graph32(hx_op* op) {
  if (op->graph32 || op->graph32_failed) return;
  if (!build_while_graph(op->stream, [op](unsigned long long h) { return cg_iteration32(op, op->stream, h); },
                         &op->graph32))
    op->graph32_failed = true;
}

// FP64 residual r = P b - A_c x into op->r, ||r||^2 into op->rn2 (x in op->x).
hx_status outer_residual(hx_op* op, const double* b, bool x_is_zero, cudaStream_t st) {
  const double* shift = op->singular ? &op->st->shift : nullptr;  // pure Neumann: b minus its mean
  const hx_mesh* m = op->mesh;
  if (x_is_zero) {
    HX_TRY(cudaMemsetAsync(op->Ap, 0, sizeof(double) * m->n_dof, st), "zero");
  } else {
    HX_TRY(element_apply(op, op->x, 1, nullptr, st), "refinement apply");
    HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, st),
           "refinement assembly");
    op->launches += 2;
  }
  HX_TRY(hx_launch_ir_residual(m->n_dof, b, op->Ap, m->dir, op->r, op->partial, op->counters, op->rn2, st, shift),
         "refinement residual");
  op->launches += 1;
  return HX_OK;
}

hx_status solve_mixed(hx_op* op, const double* b, double* x, double rtol, int max_it, double inner_rtol,
                      cudaStream_t user, hx_solve_info* info) {
  const hx_mesh* m = op->mesh;
  if (op->prec == HX_PREC_LOR)
    return fail(HX_ERR_UNSUPPORTED, "mixed-precision solves take the Jacobi, collocated mass or multigrid preconditioner");
  hx_status s = ensure_solver(op);
  if (s) return s;
  cudaStream_t st = op->stream;
  HX_TRY(cudaEventRecord(op->ev, user), "event record");
  HX_TRY(cudaStreamWaitEvent(st, op->ev, 0), "stream wait");
  if ((s = ensure_mixed(op))) return s;
  ensure_graph32(op);
  const long long launches0 = op->launches;
  HX_TRY(cudaMemsetAsync(op->x, 0, sizeof(double) * m->n_dof, st), "x init");
  if (op->singular) {
    HX_TRY(hx_launch_cg_mean(cg_buffers(op), b, st), "mean of b");
    op->launches += 1;
  }
  if ((s = outer_residual(op, b, true, st))) return s;
  double rn2 = 0.0;
  HX_TRY(cudaMemcpyAsync(&rn2, op->rn2, sizeof(double), cudaMemcpyDeviceToHost, st), "norm read");
  HX_TRY(cudaStreamSynchronize(st), "solver sync");
  const double bn = std::sqrt(rn2);
  double rel = bn > 0 ? 1.0 : 0.0, prev = rel;
  int inner_total = 0, outer = 0, status = HX_OK, stalls = 0;
  const HxCgBuffersF buf = cg_buffers32(op);
  while (rel > rtol) {
    if (inner_total >= max_it) {
      status = HX_ERR_NOT_CONVERGED;
      break;
    }
    // inner FP32 Jacobi-PCG on A_c d = r / ||r|| from d = 0
    HX_TRY(hx_launch_ir_scale_down(m->n_dof, op->r, op->rn2, op->r32, st), "scale down");
    if (op->singular) {
      HX_TRY(hx_launch_cg_mean(buf, (const float*)op->r32, st), "inner mean");
      op->launches += 1;
    }
    HX_TRY(hx_launch_cg_init(buf, (const float*)op->r32, (const float*)nullptr, inner_rtol, max_it - inner_total, st),
           "inner init");
    if (op->prec == HX_PREC_LOR_MG) {
      HX_TRY(hx_mg_vcycle32(op->mg, op->r32, op->zl32, &op->st32->done, st), "inner first V-cycle");
      op->launches += hx_mg_vcycle_launches(op->mg);
    }
    HX_TRY(hx_launch_cg_start(buf, st), "inner start");
    op->launches += 3;
    if (op->singular) {
      HX_TRY(hx_launch_cg_direction(buf, st), "inner first direction");
      op->launches += 1;
    }
    if (op->graph32) {
      HX_TRY(cudaGraphLaunch(op->graph32, st), "graph launch");
      HX_TRY(cudaMemcpyAsync(op->st_host, op->st32, sizeof(HxCgState), cudaMemcpyDeviceToHost, st), "state read");
      HX_TRY(cudaStreamSynchronize(st), "solver sync");
      op->launches += iteration_launches(op) * (long long)op->st_host->loops;
      if (!op->st_host->done) return fail(HX_ERR_CUDA, "inner CG graph loop ended before the solver finished");
    } else {
      for (;;) {
        HX_TRY(cudaMemcpyAsync(op->st_host, op->st32, sizeof(HxCgState), cudaMemcpyDeviceToHost, st), "state read");
        HX_TRY(cudaStreamSynchronize(st), "solver sync");
        if (op->st_host->done) break;
        for (int i = 0; i < kChunk; ++i) HX_TRY(cg_iteration32(op, st), "inner iteration");
        op->launches += iteration_launches(op) * kChunk;
      }
    }
    const HxCgState cs = *op->st_host;
    inner_total += cs.iter;
    ++outer;
    if (cs.status == HX_ERR_BREAKDOWN) {
      status = HX_ERR_BREAKDOWN;
      break;
    }
    // x += ||r|| d in FP64, then the FP64 residual of the new x
    HX_TRY(hx_launch_ir_update(m->n_dof, op->x, op->d32, op->rn2, st), "refinement update");
    op->launches += 1;
    if ((s = outer_residual(op, b, false, st))) return s;
    HX_TRY(cudaMemcpyAsync(&rn2, op->rn2, sizeof(double), cudaMemcpyDeviceToHost, st), "norm read");
    HX_TRY(cudaStreamSynchronize(st), "solver sync");
    rel = bn > 0 ? std::sqrt(rn2) / bn : 0.0;
    if (!std::isfinite(rel)) {
      status = HX_ERR_BREAKDOWN;
      break;
    }
    // refinement that stops contracting (FP32 operator error above the target) ends the solve
    stalls = (rel > 0.5 * prev) ? stalls + 1 : 0;
    if (stalls >= 2 && rel > rtol) {
      status = HX_ERR_NOT_CONVERGED;
      break;
    }
    prev = rel;
  }
  if (op->singular) {
    HX_TRY(hx_launch_sum(m->n_dof, op->m1, op->partial, op->counters, op->vol, st), "volume");
    HX_TRY(hx_launch_dot(m->n_dof, op->m1, op->x, op->partial, op->counters, op->vol + 1, st), "mean");
    HX_TRY(hx_launch_shift(m->n_dof, op->x, op->vol + 1, op->vol, st), "mean shift");
    op->launches += 3;
  }
  HX_TRY(cudaMemcpyAsync(x, op->x, sizeof(double) * m->n_dof, cudaMemcpyDeviceToDevice, st), "solution copy");
  HX_TRY(cudaStreamSynchronize(st), "solver sync");
  if ((s = check_kernel_flag(op, st))) return s;
  hx_solve_info inf;
  inf.iterations = inner_total;
  inf.status = status;
  inf.b_norm = bn;
  inf.rel_residual = rel;
  inf.true_rel_residual = rel;
  inf.kernel_launches = (int)(op->launches - launches0);
  inf.refinements = outer;
  if (info) *info = inf;
  if (status == HX_ERR_NOT_CONVERGED)
    return fail(HX_ERR_NOT_CONVERGED, "mixed solve stopped at rel. residual %.3e after %d refinements", rel, outer);
  if (status == HX_ERR_BREAKDOWN) return fail(HX_ERR_BREAKDOWN, "mixed solve breakdown");
  return HX_OK;
}

}  // namespace

extern "C" {

hx_status hx_solve_pcg_mixed(hx_op* op, const double* b, double* x, double rtol, int max_it, double inner_rtol,
                             void* stream, hx_solve_info* info) {
  if (!op || !b || !x) return fail(HX_ERR_ARG, "NULL argument");
  if (!(rtol >= 0.0) || max_it < 0 || !(inner_rtol > 0.0 && inner_rtol < 1.0))
    return fail(HX_ERR_ARG, "need rtol >= 0, max_it >= 0 and 0 < inner_rtol < 1");
  return solve_mixed(op, b, x, rtol, max_it, inner_rtol, (cudaStream_t)stream, info);
}

hx_status hx_op_apply_f32(hx_op* op, const float* x, float* y, void* stream) {
  if (!op || !x || !y) return fail(HX_ERR_ARG, "NULL argument");
  if ((const void*)x == (void*)y) return fail(HX_ERR_ARG, "x and y must not alias");
  hx_status s = ensure_solver(op);
  if (s) return s;
  cudaStream_t us = (cudaStream_t)stream;
  // the FP32 set-up runs on the solver stream; order it with the caller's stream both ways
  HX_TRY(cudaEventRecord(op->ev, us), "event record");
  HX_TRY(cudaStreamWaitEvent(op->stream, op->ev, 0), "stream wait");
  if ((s = ensure_mixed(op))) return s;
  HX_TRY(cudaEventRecord(op->ev, op->stream), "event record");
  HX_TRY(cudaStreamWaitEvent(us, op->ev, 0), "stream wait");
  const hx_mesh* m = op->mesh;
  HX_TRY(element_apply32(op, x, nullptr, us), "FP32 element kernel");
  HX_TRY(hx_launch_assemble32(m->n_dof, m->off, m->idx, op->yE32, m->dir, 1, x, y, us), "FP32 assembly");
  op->launches += 2;
  return HX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batched solves: every instance's whole Jacobi-PCG is a branch of one graph
// ---------------------------------------------------------------------------
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
  int lanes = 0;                 // lanes of the current graph
  bool tune = false;             // pick the lanes by timing at the first solve
};

namespace {

// Capture `fn` (kernel launches on s) into a new graph and add it to G as a child node.
hx_status add_captured_child(cudaGraph_t G, cudaStream_t s, const cudaGraphNode_t* deps, size_t ndeps,
                             const std::function<cudaError_t()>& fn, cudaGraphNode_t* node) {
  cudaGraph_t g = nullptr;
  HX_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "batch capture");
  cudaError_t e = fn();
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e != cudaSuccess ? e : e2, "batch capture");
  }
  e = cudaGraphAddChildGraphNode(node, G, deps, ndeps, g);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "batch child node");
  return HX_OK;
}

hx_status build_batch_graph(hx_batch* B, double rtol, int max_it, int lanes) {
  cudaGraph_t G = nullptr;
  HX_TRY(cudaGraphCreate(&G, 0), "batch graph");
  hx_status s = HX_OK;
  cudaStream_t cs = B->stream;
  // instance i runs after instance i - lanes: `lanes` chains of solves run side by side
  std::vector<cudaGraphNode_t> tails((size_t)B->n, nullptr);
  for (int i = 0; i < B->n && s == HX_OK; ++i) {
    hx_op* op = B->ops[i];
    const hx_mesh* m = op->mesh;
    const double* bi = B->b[i];
    double* xi = B->x[i];
    const HxCgBuffers buf = cg_buffers(op);
    cudaGraphNode_t init = nullptr, loop = nullptr, tail = nullptr;
    // 1. initialization: r = P b (mean removed for pure Neumann), z = D^-1 r, p
    const cudaGraphNode_t* dep = (i >= lanes) ? &tails[(size_t)(i - lanes)] : nullptr;
    s = add_captured_child(G, cs, dep, dep ? 1 : 0, [&]() {
      cudaError_t e = cudaSuccess;
      if (op->singular) e = hx_launch_cg_mean(buf, bi, cs);
      if (e == cudaSuccess) e = hx_launch_cg_init(buf, bi, (const double*)nullptr, rtol, max_it, cs);
      if (e == cudaSuccess) e = precondition_start(op, cs);
      if (e == cudaSuccess) e = hx_launch_cg_start(buf, cs);
      if (e == cudaSuccess && op->singular) e = hx_launch_cg_direction(buf, cs);
      return e;
    }, &init);
    if (s) break;
    // 2. the CG iterations as a device-side while loop
    cudaGraphConditionalHandle h = 0;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault);
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(raw);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = h;
    np->conditional.type = cudaGraphCondTypeWhile;
    np->conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&loop, G, &init, nullptr, 1, np);
    if (e == cudaSuccess) {
      cudaGraph_t body = np->conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t eb = cg_iteration(op, cs, (unsigned long long)h);
        e = cudaStreamEndCapture(cs, &body);
        if (eb != cudaSuccess) e = eb;
      }
    }
    if (e != cudaSuccess) {
      s = cuda_fail(e, "batch while node");
      break;
    }
    // 3. mean-zero closure (pure Neumann), true residual, solution copy
    s = add_captured_child(G, cs, &loop, 1, [&]() {
      cudaError_t e3 = cudaSuccess;
      if (op->singular) {
        e3 = hx_launch_sum(m->n_dof, op->m1, op->partial, op->counters, op->vol, cs);
        if (e3 == cudaSuccess) e3 = hx_launch_dot(m->n_dof, op->m1, op->x, op->partial, op->counters, op->vol + 1, cs);
        if (e3 == cudaSuccess) e3 = hx_launch_shift(m->n_dof, op->x, op->vol + 1, op->vol, cs);
      }
      if (e3 == cudaSuccess) e3 = element_apply(op, op->x, 1, nullptr, cs);
      if (e3 == cudaSuccess)
        e3 = hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, cs);
      if (e3 == cudaSuccess)
        e3 = hx_launch_resnorm(m->n_dof, bi, op->Ap, m->dir, op->partial, op->counters, op->scalars, cs,
                               op->singular ? &op->st->shift : nullptr);
      if (e3 == cudaSuccess)
        e3 = cudaMemcpyAsync(xi, op->x, sizeof(double) * m->n_dof, cudaMemcpyDeviceToDevice, cs);
      return e3;
    }, &tail);
    tails[(size_t)i] = tail;
  }
  if (s == HX_OK) {
    cudaError_t e = cudaGraphInstantiate(&B->exec, G, 0);
    if (e != cudaSuccess) s = cuda_fail(e, "batch graph instantiate");
  }
  cudaGraphDestroy(G);
  return s;
}

// Autotuned lanes: one timed solve of the whole batch (CUDA events on its stream, the graph
// uploaded first) for each of 1, 2, 4, ... and n lanes; the fastest graph is kept.  The lanes
// only decide which solves overlap, never their arithmetic, so every run gives the same x.
hx_status tune_lanes(hx_batch* B) {
  std::vector<int> cand;
  for (int L = 1; L < B->n; L *= 2) cand.push_back(L);
  cand.push_back(B->n);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  hx_status s = HX_OK;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  int best = B->lanes;
  float best_ms = -1.0f;
  for (size_t k = 0; k < cand.size() && e == cudaSuccess; ++k) {
    const int L = cand[k];
    if (L != B->lanes) {
      cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
      if ((s = build_batch_graph(B, B->rtol, B->max_it, L))) break;
      B->lanes = L;
    }
    float ms = 0.0f;
    e = cudaGraphUpload(B->exec, B->stream);
    if (e == cudaSuccess) e = cudaEventRecord(t0, B->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, B->stream);
    if (e == cudaSuccess) e = cudaEventRecord(t1, B->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && (best_ms < 0.0f || ms < best_ms)) {
      best_ms = ms;
      best = L;
    }
  }
  if (e != cudaSuccess && s == HX_OK) s = cuda_fail(e, "batch lane timing");
  if (s == HX_OK && best != B->lanes) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    if ((s = build_batch_graph(B, B->rtol, B->max_it, best)) == HX_OK) B->lanes = best;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (s == HX_OK) B->tune = false;
  return s;
}

}  // namespace

extern "C" {

hx_status hx_batch_create(int n, hx_op* const* ops, const double* const* b, double* const* x, double rtol, int max_it,
                          int lanes, hx_batch** out) {
  if (!out) return fail(HX_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !ops || !b || !x) return fail(HX_ERR_ARG, "need n >= 1 and non-NULL arrays");
  if (!(rtol >= 0.0) || max_it < 0) return fail(HX_ERR_ARG, "rtol must be >= 0 and max_it >= 0");
  for (int i = 0; i < n; ++i)
    if (!ops[i] || !b[i] || !x[i]) return fail(HX_ERR_ARG, "instance %d: NULL operator or vector", i);
  hx_batch* B = new (std::nothrow) hx_batch();
  if (!B) return fail(HX_ERR_OOM, "host allocation failed");
  B->n = n;
  B->ops.assign(ops, ops + n);
  B->b.assign(b, b + n);
  B->x.assign(x, x + n);
  B->rtol = rtol;
  B->max_it = max_it;
  B->tune = lanes < 0;
  B->lanes = (lanes <= 0 || lanes > n) ? n : lanes;
  hx_status s = HX_OK;
  for (int i = 0; i < n && s == HX_OK; ++i) {
    s = ensure_solver(ops[i]);
    if (s == HX_OK && cudaStreamSynchronize(ops[i]->stream) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "sync");
  }
  cudaError_t e = cudaSuccess;
  if (s == HX_OK) e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && s == HX_OK) e = cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
  if (e == cudaSuccess && s == HX_OK) e = cudaMallocHost((void**)&B->st_host, sizeof(HxCgState) * n);
  if (e == cudaSuccess && s == HX_OK) e = cudaMallocHost((void**)&B->rn2_host, sizeof(double) * n);
  if (e != cudaSuccess && s == HX_OK) s = cuda_fail(e, "batch resources");
  if (s == HX_OK) s = build_batch_graph(B, rtol, max_it, B->lanes);
  if (s != HX_OK) {
    hx_batch_destroy(B);
    return s;
  }
  *out = B;
  return HX_OK;
}

hx_status hx_batch_solve(hx_batch* B, void* stream, hx_solve_info* infos) {
  if (!B) return fail(HX_ERR_ARG, "batch is NULL");
  HX_TRY(cudaEventRecord(B->ev, (cudaStream_t)stream), "event record");
  HX_TRY(cudaStreamWaitEvent(B->stream, B->ev, 0), "stream wait");
  for (int i = 0; i < B->n; ++i) {  // inverse diagonals of the operators' current coefficients
    hx_status st = ensure_dinv(B->ops[i], B->stream);
    if (st) return st;
  }
  if (B->tune) {
    hx_status st = tune_lanes(B);
    if (st) return st;
  }
  if (!B->exec) return fail(HX_ERR_CUDA, "the batch lost its graph in a failed rebuild");
  HX_TRY(cudaGraphLaunch(B->exec, B->stream), "batch graph launch");
  for (int i = 0; i < B->n; ++i) {
    HX_TRY(cudaMemcpyAsync(B->st_host + i, B->ops[i]->st, sizeof(HxCgState), cudaMemcpyDeviceToHost, B->stream),
           "state read");
    HX_TRY(cudaMemcpyAsync(B->rn2_host + i, B->ops[i]->scalars, sizeof(double), cudaMemcpyDeviceToHost, B->stream),
           "residual read");
  }
  HX_TRY(cudaStreamSynchronize(B->stream), "batch sync");
  hx_status worst = HX_OK;
  for (int i = 0; i < B->n; ++i) {
    const HxCgState& cs = B->st_host[i];
    const double bn = std::sqrt(cs.bb);
    B->ops[i]->launches += 4 * (long long)cs.loops + 8;
    if (infos) {
      hx_solve_info& inf = infos[i];
      inf.iterations = cs.iter;
      inf.status = cs.done ? cs.status : HX_ERR_CUDA;
      inf.b_norm = bn;
      inf.rel_residual = bn > 0 ? std::sqrt(cs.rr) / bn : 0.0;
      inf.true_rel_residual = bn > 0 ? std::sqrt(B->rn2_host[i]) / bn : std::sqrt(B->rn2_host[i]);
      inf.kernel_launches = 4 * cs.loops + 8;
      inf.refinements = 0;
    }
    if (!cs.done) worst = HX_ERR_CUDA;
    else if (cs.status != HX_OK && worst == HX_OK) worst = cs.status;
  }
  if (worst != HX_OK) return fail(worst, "at least one batch instance did not converge");
  return HX_OK;
}

int hx_batch_lanes(const hx_batch* B) { return B ? B->lanes : 0; }

void hx_batch_destroy(hx_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->ev) cudaEventDestroy(B->ev);
  if (B->stream) cudaStreamDestroy(B->stream);
  if (B->st_host) cudaFreeHost(B->st_host);
  if (B->rn2_host) cudaFreeHost(B->rn2_host);
  delete B;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// adjoint gradients
// ---------------------------------------------------------------------------
extern "C" hx_status hx_op_gradient(hx_op* op, const double* u, const double* lam, double* dnu_q, double* df_q,
                                    void* stream) {
  if (!op || !u || !lam || !dnu_q || !df_q) return fail(HX_ERR_ARG, "NULL argument");
  static const hx_grad_launcher t[] = {nullptr, hx_launch_grad_p1, hx_launch_grad_p2, hx_launch_grad_p3,
                                       hx_launch_grad_p4, hx_launch_grad_p5, hx_launch_grad_p6,
                                       hx_launch_grad_p7, hx_launch_grad_p8};
  const hx_mesh* m = op->mesh;
  HxGradArgs a;
  a.E = m->E;
  a.R = m->R;
  a.u = u;
  a.lam = lam;
  a.X8 = m->X8;
  a.dnu = dnu_q;
  a.df = df_q;
  HX_TRY(t[m->p](m->T, a, (cudaStream_t)stream), "gradient kernel");
  op->launches += 1;
  return HX_OK;
}

// ---------------------------------------------------------------------------
// preconditioners (Sec. 5.1)
// ---------------------------------------------------------------------------
extern "C" {

hx_status hx_op_collocated_mass(hx_op* op, double* diag, void* stream) {
  if (!op || !diag) return fail(HX_ERR_ARG, "NULL argument");
  const hx_mesh* m = op->mesh;
  cudaStream_t s = (cudaStream_t)stream;
  HX_TRY(hx_launch_cmass(m->T, m->E, m->X8, op->alpha, op->yE, s), "collocated mass");
  HX_TRY(hx_launch_assemble(m->n_dof, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, diag, s),
         "collocated mass assembly");
  op->launches += 2;
  return HX_OK;
}

hx_status hx_op_set_preconditioner(hx_op* op, int kind, int degree, void* stream) {
  if (!op) return fail(HX_ERR_ARG, "op is NULL");
  if (kind != HX_PREC_JACOBI && kind != HX_PREC_COLLOCATED_MASS && kind != HX_PREC_LOR && kind != HX_PREC_LOR_MC &&
      kind != HX_PREC_LOR_MG)
    return fail(HX_ERR_ARG, "unknown preconditioner");
  const bool lor = kind == HX_PREC_LOR || kind == HX_PREC_LOR_MC || kind == HX_PREC_LOR_MG;
  if (kind == HX_PREC_LOR_MG && op->mesh->grid[0] == 0)
    return fail(HX_ERR_UNSUPPORTED, "the multigrid preconditioner needs a structured mesh (hx_mesh_create_box)");
  cudaStream_t s = (cudaStream_t)stream;
  hx_status st = HX_OK;
  if (kind == HX_PREC_COLLOCATED_MASS) {
    if (!(op->alpha > 0.0)) return fail(HX_ERR_ARG, "the collocated mass preconditioner needs alpha > 0");
    if (!op->pdiag && (st = dalloc(&op->pdiag, (size_t)op->mesh->n_dof, "preconditioner diagonal"))) return st;
  }
  if (lor) {
    if (degree < 1 || degree > HX_LOR_MAX_DEGREE) return fail(HX_ERR_ARG, "degree must be in [1, %d]", HX_LOR_MAX_DEGREE);
    if (op->has_field) return fail(HX_ERR_UNSUPPORTED, "the LOR preconditioner takes a constant nu only");
    if (kind == HX_PREC_LOR_MG) {
      if ((st = lor_workspace(op, degree)) || (st = mg_setup(op, degree, s))) return st;
    } else if ((st = lor_setup(op, degree, s))) {
      return st;
    }
  }
  // the captured CG iterations differ between the preconditioners: capture again at the next solve
  if (op->graph) {
    cudaGraphExecDestroy(op->graph);
    op->graph = nullptr;
  }
  if (op->graph32) {
    cudaGraphExecDestroy(op->graph32);
    op->graph32 = nullptr;
  }
  op->graph_failed = false;
  op->graph32_failed = false;
  op->prec = (kind == HX_PREC_LOR_MC) ? HX_PREC_LOR : kind;  // one solver path for both Chebyshev forms
  op->mixed_stale = true;  // the FP32 inverse diagonal follows at the next mixed solve
  int nl = 0;
  if (lor) {
    op->cheb.degree = degree;
    op->lor_collocated = (kind == HX_PREC_LOR_MC || kind == HX_PREC_LOR_MG) ? 1 : 0;
    st = lor_assemble(op, s, &nl);
  } else {
    op->dinv_stale = true;
  }
  op->launches += nl;
  return st;
}

hx_status hx_op_precond_apply(hx_op* op, const double* r, double* z, void* stream) {
  if (!op || !r || !z) return fail(HX_ERR_ARG, "NULL argument");
  hx_status st = ensure_solver(op);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = ensure_dinv(op, op->stream))) return st;
  // the solver workspace is set up on the solver stream: order after it
  HX_TRY(cudaEventRecord(op->ev, op->stream), "event record");
  HX_TRY(cudaStreamWaitEvent(s, op->ev, 0), "stream wait");
  if (op->prec == HX_PREC_LOR || op->prec == HX_PREC_LOR_MG) {
    HX_TRY(apply_z(op, r, z, nullptr, s), "LOR preconditioner");
    op->launches += z_launches(op);
  } else {
    HX_TRY(hx_launch_scale(op->mesh->n_dof, op->dinv, r, z, s), "preconditioner apply");
    op->launches += 1;
  }
  return HX_OK;
}

hx_status hx_op_lor_csr(hx_op* op, int64_t* nnz, int64_t* row_off, int* col, double* val, void* stream) {
  if (!op || !nnz) return fail(HX_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  hx_status st = HX_OK;
  if (!op->lor.val) {
    if (op->has_field) return fail(HX_ERR_UNSUPPORTED, "the LOR operator takes a constant nu only");
    if ((st = lor_setup(op, op->cheb.degree > 0 ? op->cheb.degree : 1, s))) return st;
  }
  if (!op->lor_values_set) {
    if (op->cheb.degree == 0) op->cheb.degree = 1;
    int nl = 0;
    st = lor_csr_values(op, s, &nl);
    op->launches += nl;
    if (st) return st;
  }
  *nnz = op->lor_nnz;
  const long long n = op->mesh->n_dof;
  if (row_off)
    HX_TRY(cudaMemcpyAsync(row_off, op->lor.off, sizeof(long long) * (n + 1), cudaMemcpyDeviceToDevice, s), "copy");
  if (col) HX_TRY(cudaMemcpyAsync(col, op->lor.col, sizeof(int) * op->lor_nnz, cudaMemcpyDeviceToDevice, s), "copy");
  if (val)
    HX_TRY(cudaMemcpyAsync(val, op->lor.val, sizeof(double) * op->lor_nnz, cudaMemcpyDeviceToDevice, s), "copy");
  return HX_OK;
}

}  // extern "C"
