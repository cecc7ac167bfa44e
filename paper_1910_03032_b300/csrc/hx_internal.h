// Internal declarations shared by the C ABI (hx_capi_*.cu) and the kernel
// translation units.  Not part of the public interface (see include/hx.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hx_tables.h"

// Layout of an E-vector (n^3 values per element, local node l = i + n j + n^2 k, x-line r = j + n k).
// nx = 0: element-major, entry l of element e at e n^3 + l.  nx > 0 (box meshes, elements numbered
// x fastest in rows of nx): the x-lines of one row of elements lie side by side, line r of element
// e at ((e / nx) n^2 + r) (nx n) + (e mod nx) n, so that the entries a DoF-grid x-line gathers form
// one contiguous range (the two entries of a node between elements are neighbours).
struct HxELayout {
  int nx;
  unsigned m;  // e / nx = (e m) >> s for 0 <= e < 2^31
  int s;
};
// first entry of x-line r of element e
__host__ __device__ __forceinline__ long long hx_eline(const HxELayout& L, long long e, int r, int n) {
  if (L.nx == 0) return (e * n * n + r) * n;
  const long long row = (long long)(((unsigned long long)(unsigned)e * L.m) >> L.s);
  return (row * n * n + r) * ((long long)L.nx * n) + (e - row * L.nx) * n;
}

// Arguments of the element-operator kernel (gather -> contractions ->
// pointwise -> transposed contractions -> E-vector), in scalar type T
// (double: the operator; float: the inner solver of the mixed-precision refinement).
template <typename T>
struct HxApplyArgsT {
  long long E;            // number of elements
  const int* R;           // [E][n^3] restriction; g >= 0 free DoF, -(g+1) Dirichlet DoF
  const T* x;             // L-vector input
  T* yE;                  // E-vector output (E n^3 values)
  HxELayout lay;          // its layout
  const T* factors;       // stored geometry: [E][fstride], 7 planes of q^3 (m, G00, G01, G02, G11, G12, G22)
  long long fstride;      // element stride of `factors` (7 q^3, or the padded FP32 stride)
  const double* X8;       // [E][8][3] element corner coordinates (on-the-fly geometry)
  const double* nu_q;     // [E][q^3] per-point viscosity or null (on-the-fly geometry)
  T alpha, nu;            // Helmholtz coefficients (on-the-fly geometry), in the kernel's type:
                          // an FP64 value converted per point costs an FP64-pipe instruction
  int constrained;        // 1: Dirichlet DoFs of x read as zero
  const int* done;        // optional device flag: kernel returns at once when *done != 0
  int* err;               // optional device flag, set to 1 when a bounded wait gives up
  int wait_limit;         // try_wait attempts of the first wait for the staged factors (FP32 kernel)
};
typedef HxApplyArgsT<double> HxApplyArgs;
#define HX_WAIT_LIMIT_DEFAULT (1 << 16)  // attempts of the first bounded wait
#define HX_WAIT_LIMIT_EXIT (1 << 20)     // attempts of the wait before a block exits
typedef HxApplyArgsT<float> HxApplyArgsF;

// Element stride of the FP32 factor array: the 7 q^3 factors of an element rounded up to
// whole 16-byte units, so that every element's factors can be moved by one bulk copy.
inline long long hx_f32_factor_stride(int q) { return ((7LL * q * q * q) + 3) & ~3LL; }

// Arguments of the diagonal kernel (sum-factorized diag of the element matrices).
template <typename T>
struct HxDiagArgsT {
  long long E;
  const T* factors;       // stored geometry or null
  long long fstride;      // element stride of `factors`
  const double* X8;
  const double* nu_q;
  T alpha, nu;
  T* dE;                  // element diagonals (an E-vector)
  HxELayout lay;          // its layout
  int parts;              // terms summed: 1 the mass part (m), 2 the stiffness part (G), 3 both
};
typedef HxDiagArgsT<double> HxDiagArgs;
typedef HxDiagArgsT<float> HxDiagArgsF;

// Arguments of the load-vector kernel: bE = B^T (w detJ f) per element.
struct HxLoadArgs {
  long long E;
  const double* X8;
  const double* fq;       // [E][q^3] source values at the quadrature points (null: f = 1)
  double* yE;
  HxELayout lay;
};

// Arguments of the adjoint-gradient kernel: per-point dL/dnu and dL/df from u and lam.
struct HxGradArgs {
  long long E;
  const int* R;           // restriction (Dirichlet entries read as zero)
  const double* u;        // forward solution (L-vector)
  const double* lam;      // adjoint solution (L-vector)
  const double* X8;       // [E][8][3]
  double* dnu;            // [E][q^3] out: -w detJ (J^-T grad lam).(J^-T grad u)
  double* df;             // [E][q^3] out: w detJ lam(x_q)
};

enum { HX_KGEOM_STORED = 0, HX_KGEOM_ONTHEFLY = 1 };

// Per-order launchers (one translation unit per p; q in {p+1, p+2}).
typedef cudaError_t (*hx_apply_launcher)(const HxTables&, const HxApplyArgs&, int geom, cudaStream_t);
typedef cudaError_t (*hx_diag_launcher)(const HxTables&, const HxDiagArgs&, int geom, cudaStream_t);
typedef cudaError_t (*hx_diag32_launcher)(const HxTablesF&, const HxDiagArgsF&, int geom, cudaStream_t);
typedef cudaError_t (*hx_load_launcher)(const HxTables&, const HxLoadArgs&, cudaStream_t);
// kind: HX_F32_* (include/hx.h); tile: -1, 0, +1 (half, default, twice the elements per block of
// the direct kinds with stored factors)
typedef cudaError_t (*hx_apply32_launcher)(const HxTablesF&, const HxApplyArgsF&, int geom, int kind, int tile,
                                           cudaStream_t);
typedef cudaError_t (*hx_grad_launcher)(const HxTables&, const HxGradArgs&, cudaStream_t);
// the FP64 element kernel over several operators of one order: blocks -> (operator, block) by table
typedef cudaError_t (*hx_apply_multi_launcher)(const HxTables&, const HxApplyArgs*, const int* blk_op,
                                               const int* blk_first, long long blocks, int geom, int nuf,
                                               cudaStream_t);
typedef int (*hx_block_elems_fn)(int q, int geom);

#define HX_DECLARE_ORDER(P)                                                                        \
  cudaError_t hx_launch_apply_p##P(const HxTables&, const HxApplyArgs&, int, cudaStream_t);       \
  cudaError_t hx_launch_diag_p##P(const HxTables&, const HxDiagArgs&, int, cudaStream_t);         \
  cudaError_t hx_launch_diag32_p##P(const HxTablesF&, const HxDiagArgsF&, int, cudaStream_t);     \
  cudaError_t hx_launch_load_p##P(const HxTables&, const HxLoadArgs&, cudaStream_t);              \
  cudaError_t hx_launch_apply32_p##P(const HxTablesF&, const HxApplyArgsF&, int, int, int, cudaStream_t); \
  int hx_apply32_block_elems_p##P(int q, int tile);                                               \
  cudaError_t hx_launch_grad_p##P(const HxTables&, const HxGradArgs&, cudaStream_t);                     \
  cudaError_t hx_launch_apply_multi_p##P(const HxTables&, const HxApplyArgs*, const int*, const int*,     \
                                         long long, int, int, cudaStream_t);                              \
  int hx_apply_block_elems_p##P(int q, int geom);
HX_DECLARE_ORDER(1)
HX_DECLARE_ORDER(2)
HX_DECLARE_ORDER(3)
HX_DECLARE_ORDER(4)
HX_DECLARE_ORDER(5)
HX_DECLARE_ORDER(6)
HX_DECLARE_ORDER(7)
HX_DECLARE_ORDER(8)

// ---- order-independent kernels (hx_kernels.cu) ----
cudaError_t hx_launch_geometry(const HxTables& T, long long E, const double* X8, const double* nu_q,
                               double alpha, double nu, double* factors, int* bad_count, cudaStream_t s);
cudaError_t hx_launch_qpoint_coords(const HxTables& T, long long E, const double* X8, double* xyz,
                                    cudaStream_t s);
cudaError_t hx_launch_node_coords(const HxTables& T, long long n_dof, const int* off, const int* idx,
                                  const double* X8, double* xyz, cudaStream_t s);
// Logical grid of a box mesh (elements nx x ny x nz numbered x fastest, DoFs on the
// (p nx + 1) x (p ny + 1) x (p nz + 1) node grid, lexicographic local nodes): the assembly then
// finds a DoF's element entries by index arithmetic instead of reading the transpose map, in the
// map's order (increasing element index).  The E-vectors it reads are in the line layout with
// rows of nx elements (HxELayout).  p = 0: no such grid; element-major E-vectors, the map is read.
struct HxGridAsm {
  int p, nx, ny, nz, gx, gy;
  // n / d = (n m) >> s for 0 <= n < 2^31 (d = gx, gy, p, nx): multiply-shift instead of division
  unsigned mgx, mgy, mp, mnx;
  int sgx, sgy, sp, snx;
};
// Multiplier and shift of the division by d (1 <= d < 2^31) for dividends below 2^31:
// s = 31 + ceil(log2 d), m = floor(2^s / d) + 1 (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994: exact for every 31-bit dividend).
inline void hx_fastdiv_init(int d, unsigned* m, int* s) {
  int l = 0;
  while ((1LL << l) < d) ++l;
  *s = 31 + l;
  *m = (unsigned)((1ULL << *s) / (unsigned long long)d + 1ULL);
}
// the line layout of the E-vectors of a box mesh with rows of nx elements
inline HxELayout hx_elayout_rows(int nx) {
  HxELayout L = {nx, 0u, 0};
  hx_fastdiv_init(nx, &L.m, &L.s);
  return L;
}
inline HxGridAsm hx_grid_asm(int p, int nx, int ny, int nz, int gx, int gy) {
  HxGridAsm g = {p, nx, ny, nz, gx, gy, 0, 0, 0, 0, 0, 0, 0, 0};
  hx_fastdiv_init(gx, &g.mgx, &g.sgx);
  hx_fastdiv_init(gy, &g.mgy, &g.sgy);
  hx_fastdiv_init(p, &g.mp, &g.sp);
  hx_fastdiv_init(nx, &g.mnx, &g.snx);
  return g;
}
// y[g] = sum_{k in off[g]..off[g+1]} yE[idx[k]]; with `constrained`, Dirichlet rows
// (dir[g] != 0) take x[g] (x non-null) or dir_const.
cudaError_t hx_launch_assemble(long long n_dof, const HxGridAsm& ga, const int* off, const int* idx, const double* yE,
                               const unsigned char* dir, int constrained, const double* x,
                               double dir_const, double* y, cudaStream_t s);

// Jacobi-PCG state (device); scalars kept on the device between kernels.
struct HxCgState {
  double rz;        // (r, z)
  double alpha;     // step
  double beta;      // direction update
  double bb;        // ||P b||^2
  double rr;        // ||r||^2 of the last update
  double tol2;      // rtol^2 * bb
  int iter;         // completed iterations
  int max_it;
  int done;         // 0 running, 1 finished
  int loops;        // iterations of a graph while-loop body (a hard stop for the loop)
  double shift;     // null-space mode: mean of b, removed from the right-hand side
  double zmean;     // null-space mode: mean of D^-1 r, removed from the preconditioned residual
  int status;       // HX_OK / HX_ERR_NOT_CONVERGED / HX_ERR_BREAKDOWN
  unsigned int count[4];  // last-block counters, one per reduction kernel
};

// Grid of the reduction kernels: one wave of HX_RED_MINB blocks of HX_RED_THREADS on each of the
// 148 SMs (the kernels are compiled for that residency), so that no partly filled second wave
// stretches these memory-bound passes.
#define HX_RED_MINB 6
#define HX_RED_BLOCKS (HX_RED_MINB * 148)
#define HX_RED_VALUES 4     // partial sums per block at most (partial buffers hold HX_RED_VALUES x HX_RED_BLOCKS)
#define HX_RED_THREADS 256
// Blocks of a CG pass over n DoFs: about 4 entries per thread, at least 1, at most
// HX_RED_BLOCKS.  A solve's reductions sum over the same blocks whether its passes run alone or
// among the lock-step passes of a batch, so both give bit-identical results.
inline long long hx_red_blocks(long long n) {
  const long long b = (n + 4LL * HX_RED_THREADS - 1) / (4LL * HX_RED_THREADS);
  return b < 1 ? 1 : b > HX_RED_BLOCKS ? HX_RED_BLOCKS : b;
}

template <typename Real>
struct HxCgBuffersT {
  long long n;
  const int* off;
  const int* idx;
  const unsigned char* dir;
  Real* x;
  Real* r;
  Real* p;
  Real* Ap;
  Real* dinv;
  Real* yE;
  double* partial;  // [HX_RED_VALUES * HX_RED_BLOCKS]
  HxCgState* st;
  const Real* z;            // preconditioned residual computed outside the CG kernels, or NULL (Jacobi: dinv r)
  unsigned long long cond;  // CUDA graph conditional handle of the enclosing while loop, or 0
  int nullspace;            // 1: singular operator with the constants as null space (pure Neumann Poisson)
  HxGridAsm ga;             // logical grid of a box mesh (ga.p = 0: read the transpose map)
};
typedef HxCgBuffersT<double> HxCgBuffers;
typedef HxCgBuffersT<float> HxCgBuffersF;

cudaError_t hx_launch_cmass(const HxTables& T, long long E, const double* X8, double alpha, double* dE, const HxELayout& lay,
                            cudaStream_t s);
cudaError_t hx_launch_scale(long long n, const double* d, const double* r, double* z, cudaStream_t s);
cudaError_t hx_launch_dinv(long long n, const double* diag, const unsigned char* dir, double* dinv, cudaStream_t s);
// Stored factors [E][7][q^3] after a change of constant coefficients: m *= ra, G *= rk.
cudaError_t hx_launch_scale_factors(long long E, int Q3, double ra, double rk, double* factors, cudaStream_t s);
// out = ra a + rk b
cudaError_t hx_launch_axpby(long long n, double ra, const double* a, double rk, const double* b, double* out,
                            cudaStream_t s);
cudaError_t hx_launch_axpby32(long long n, float ra, const float* a, float rk, const float* b, float* out,
                              cudaStream_t s);
cudaError_t hx_launch_dinv32(long long n, const float* diag, const unsigned char* dir, float* dinv, cudaStream_t s);
cudaError_t hx_launch_masked_copy(long long n, const double* src, const unsigned char* dir, int constrained,
                                  double value, double* dst, cudaStream_t s);
template <typename Real>
cudaError_t hx_launch_cg_init(const HxCgBuffersT<Real>& b, const Real* bvec, const Real* x0, double rtol, int max_it,
                              cudaStream_t s);
template <typename Real>
cudaError_t hx_launch_cg_residual(const HxCgBuffersT<Real>& b, cudaStream_t s);
template <typename Real>
cudaError_t hx_launch_cg_start(const HxCgBuffersT<Real>& b, cudaStream_t s);
template <typename Real>
cudaError_t hx_launch_cg_assemble_pap(const HxCgBuffersT<Real>& b, cudaStream_t s);
template <typename Real>
cudaError_t hx_launch_cg_update(const HxCgBuffersT<Real>& b, cudaStream_t s);
template <typename Real>
cudaError_t hx_launch_cg_direction(const HxCgBuffersT<Real>& b, cudaStream_t s);
template <typename Real>
cudaError_t hx_launch_cg_rz(const HxCgBuffersT<Real>& b, cudaStream_t s);

// ---- low-order refined operator (Sec. 5.2) and its Chebyshev-Jacobi inverse ----
#define HX_LOR_MAX_NB 64  // distinct columns per LOR row at most (27 on structured meshes)
#define HX_LOR_MAX_DEGREE 64
struct HxLorBuild {
  int p;
  long long n;
  const int* toff;  // transpose map of the restriction
  const int* tidx;
  const int* R;
  const unsigned char* dir;
};
struct HxLorMatrix {
  long long n;
  long long* off;  // [n + 1]
  int* col;        // [nnz], sorted per row
  double* val;     // [nnz], Dirichlet rows and columns eliminated (identity rows)
  double* dinv;    // [n]
  // Sliced-ELL copy for the Chebyshev steps: rows in slices of 32, each slice stored column-major
  // over its longest row, so entry k of row g sits at soff[g / 32] + 32 k + g % 32 and a warp's
  // loads are coalesced.  Padding entries have value 0 (column g; column 0 past the last row).
  long long* soff; // [ceil(n / 32) + 1]
  int* scol;
  double* sval;
};
struct HxChebWork {
  int degree;      // Chebyshev steps (1: plain LOR-Jacobi)
  double* res;     // [n]
  double* d0;      // [n]
  double* d1;      // [n]
  double* coef;    // [2 degree]
};
cudaError_t hx_lor_count(const HxLorBuild& b, long long* count, int* bad, cudaStream_t s);
long long hx_lor_scan_blocks(long long n);
cudaError_t hx_lor_scan(long long n, const long long* count, long long* sums, long long* off, cudaStream_t s);
cudaError_t hx_lor_fill(const HxLorBuild& b, const long long* off, int* col, cudaStream_t s);
// Sliced-ELL pattern: count[t] = 32 x (the longest row of slice t), t < ceil(n / 32)
cudaError_t hx_lor_sell_count(long long n, const long long* off, long long* count, cudaStream_t s);
// Copies the CSR columns (col != nullptr) and/or values (val != nullptr) into the sliced-ELL arrays
// of A (A.soff set), with the padding entries.
cudaError_t hx_lor_sell_copy(const HxLorMatrix& A, const int* col, const double* val, cudaStream_t s);
// collocated = 0: alpha M_LOR + nu K_LOR; 1: alpha Mc + nu K_LOR (collocated Gauss-Lobatto mass)
cudaError_t hx_lor_values(const HxTables& T, const HxLorBuild& b, const double* X8, double alpha, double nu,
                          int collocated, const HxLorMatrix& A, unsigned long long* bound, cudaStream_t s);
cudaError_t hx_lor_coefficients(const unsigned long long* bound, int degree, double* coef, cudaStream_t s);
cudaError_t hx_lor_precondition(const HxLorMatrix& A, const HxChebWork& w, const double* r, double* z,
                                const int* done, cudaStream_t s);

// ---- geometric multigrid V-cycle on the LOR matrix of a structured mesh (hx_mg.cu) ----
struct HxGrid {
  int mx, my, mz;  // logical grid dimensions (x fastest)
  long long n;
};
struct HxMgLevel {
  HxGrid g;
  const unsigned char* dir;  // Dirichlet mask (the mesh's on the fine level)
  unsigned char* dir_own;    // coarse levels: owned mask
  double* val;               // [27][n] stencil (fine level: the LOR matrix; coarse: Galerkin)
  double* dinv;              // inverse diagonal
  double *b, *x, *r;         // right-hand side, solution, residual (b, x: coarse levels)
  double *res, *d0, *d1;     // Chebyshev work vectors
  double* coef;              // Chebyshev coefficients of this level's smoother (coarse solver)
  unsigned long long* bound; // Gershgorin bound of D^-1 A
  // FP32 copies for the inner solver of mixed-precision solves (allocated on first use)
  float *val32, *dinv32, *b32, *x32, *r32, *res32, *d032, *d132;
};
#define HX_MG_MAX_LEVELS 16
struct HxMg {
  int n_levels;
  int smooth_degree;     // Chebyshev steps before and after the coarse correction
  double smooth_ratio;   // smoothing interval [b / ratio, b]
  int coarse_degree;     // Chebyshev steps on the coarsest grid, interval [b / k^2, b]
  HxMgLevel levels[HX_MG_MAX_LEVELS];
};
cudaError_t hx_mg_coarse_dir(const HxMgLevel& F, HxMgLevel& C, cudaStream_t s);
// fine stencil of the LOR matrix (collocated = 1: alpha Mc + nu K_LOR, mc = alpha Mc assembled)
cudaError_t hx_mg_fine(const HxTables& T, int nx, int ny, const double* X8, double alpha, double nu, int collocated,
                       const double* mc, const HxMgLevel& L0, cudaStream_t s);
// inverse diagonals, bounds, Galerkin levels and Chebyshev coefficients from the fine stencil
cudaError_t hx_mg_assemble(const HxMg& M, cudaStream_t s);
cudaError_t hx_mg_vcycle(const HxMg& M, const double* r, double* z, const int* done, cudaStream_t s);
cudaError_t hx_mg_vcycle32(const HxMg& M, const float* r, float* z, const int* done, cudaStream_t s);
cudaError_t hx_mg_to_float(const HxMg& M, cudaStream_t s);
int hx_mg_vcycle_launches(const HxMg& M);
// mixed-precision refinement helpers
cudaError_t hx_launch_assemble32(long long n, const HxGridAsm& ga, const int* off, const int* idx, const float* yE,
                                 const unsigned char* dir, int constrained, const float* x, float* y, cudaStream_t s);
cudaError_t hx_launch_ir_residual(long long n, const double* b, const double* Ax, const unsigned char* dir, double* r,
                                  double* partial, unsigned int* counter, double* rn2, cudaStream_t s,
                                  const double* shift = nullptr);
cudaError_t hx_launch_ir_scale_down(long long n, const double* r, const double* rn2, float* r32, cudaStream_t s);
cudaError_t hx_launch_ir_update(long long n, double* x, const float* d, const double* rn2, cudaStream_t s);
cudaError_t hx_launch_to_float(long long n, const double* a, float* b, cudaStream_t s);
// b[e * stride + k] = a[e * per + k] for k < per, b[e * stride + k] = 0 for per <= k < stride
cudaError_t hx_launch_to_float_strided(long long E, int per, int stride, const double* a, float* b,
                                       cudaStream_t s);
cudaError_t hx_launch_dot(long long n, const double* a, const double* c, double* partial, unsigned int* counter,
                          double* out, cudaStream_t s);
cudaError_t hx_launch_resnorm(long long n, const double* b, const double* Ax, const unsigned char* dir, double* partial,
                              unsigned int* counter, double* out, cudaStream_t s, const double* shift = nullptr);
// lock-step CG passes over several operators (batches): block b works on share
// b - blk_first[o] of the blk_count[o] blocks of operator o = blk_op[b] (blk_count[o] <= HX_RED_BLOCKS)
enum { HX_PASS_ASSEMBLE_PAP = 0, HX_PASS_UPDATE = 1, HX_PASS_DIRECTION = 2 };
cudaError_t hx_launch_cg_pass_multi(int pass, const HxCgBuffers* bufs, const int* blk_op, const int* blk_first,
                                    const int* blk_count, long long blocks, cudaStream_t s);
// sets the while-loop condition `cond`: some operator unfinished and within its cap of bodies
cudaError_t hx_launch_batch_condition(HxCgState* const* states, int n, unsigned long long cond, cudaStream_t s);
// null-space (pure Neumann) helpers
template <typename Real>
cudaError_t hx_launch_cg_mean(const HxCgBuffersT<Real>& b, const Real* v, cudaStream_t s);
cudaError_t hx_launch_sum(long long n, const double* v, double* partial, unsigned int* counter, double* out,
                          cudaStream_t s);
// x -= (*num) / (*den)
cudaError_t hx_launch_shift(long long n, double* x, const double* num, const double* den, cudaStream_t s);

// Sets the message hx_last_error() returns on this thread (for entry points
// defined outside hx_capi.cu).
void hx_internal_set_error(const char* msg);
