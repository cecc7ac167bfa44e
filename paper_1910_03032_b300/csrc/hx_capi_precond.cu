// C ABI of libhx.so (include/hx.h): preconditioner selection and set-up -- collocated mass
// (Sec. 5.1), the low-order refined operator with its Chebyshev and multigrid inverses (Sec. 5.2).
#include "hx_capi_internal.h"

using namespace hxc;

namespace hxc {

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
  HX_TRY(hx_launch_cmass(m->T, m->E, m->X8, op->alpha, op->yE, m->lay, s), "collocated mass");
  HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, op->mg_mc, s),
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

}  // namespace hxc

// ---------------------------------------------------------------------------
// preconditioners (Sec. 5.1)
// ---------------------------------------------------------------------------
extern "C" {

hx_status hx_op_collocated_mass(hx_op* op, double* diag, void* stream) {
  if (!op || !diag) return fail(HX_ERR_ARG, "NULL argument");
  const hx_mesh* m = op->mesh;
  cudaStream_t s = (cudaStream_t)stream;
  HX_TRY(hx_launch_cmass(m->T, m->E, m->X8, op->alpha, op->yE, m->lay, s), "collocated mass");
  HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, diag, s),
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
