// C ABI of libhx.so (include/hx.h): the operator alpha M + nu K (Sec. 3.1) -- geometric
// factors, diagonal, apply, load vector -- and the adjoint gradients.
#include "hx_capi_internal.h"

using namespace hxc;

namespace hxc {

HxApplyArgs apply_args(const hx_op* op, const double* x, int constrained, const int* done) {
  const hx_mesh* m = op->mesh;
  HxApplyArgs a;
  a.E = m->E;
  a.R = m->R;
  a.x = x;
  a.yE = op->yE;
  a.lay = m->lay;
  a.factors = op->factors;
  a.fstride = 7LL * m->q * m->q * m->q;
  a.X8 = m->X8;
  a.nu_q = op->use_field ? op->nu_q : nullptr;
  a.alpha = op->alpha;
  a.nu = op->nu;
  a.constrained = constrained;
  a.done = done;
  a.err = op->kerr;
  a.wait_limit = op->wait_limit;
  return a;
}

cudaError_t element_apply(const hx_op* op, const double* x, int constrained, const int* done, cudaStream_t s) {
  const HxApplyArgs a = apply_args(op, x, constrained, done);
  return apply_launcher(op->mesh->p)(op->mesh->T, a, op->geom, s);
}

}  // namespace hxc

namespace hxc {

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

}  // namespace hxc

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
  dfree(op->dmk);
  dfree(op->dmk32);
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

namespace hxc {

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
  d.fstride = 7LL * m->q * m->q * m->q;
  d.X8 = m->X8;
  d.nu_q = op->use_field ? op->nu_q : nullptr;
  d.alpha = op->alpha;
  d.nu = op->nu;
  d.dE = op->yE;
  d.lay = m->lay;
  d.parts = 3;
  // stored factors of constant coefficients: the diagonal from its mass and stiffness parts
  const bool split = op->geom == HX_GEOM_STORED && op->factors_ok && op->alpha_f != 0.0 && op->nu_f != 0.0;
  if (split) {
    if (!op->dmk_ok) {
      hx_status st;
      if (!op->dmk && (st = dalloc(&op->dmk, 2 * (size_t)m->n_dof, "diagonal parts"))) return st;
      for (int part = 0; part < 2; ++part) {
        d.parts = 1 + part;
        HX_TRY(diag_launcher(m->p)(m->T, d, op->geom, s), "diagonal kernel");
        HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0,
                                  op->dmk + part * m->n_dof, s),
               "diagonal assembly");
      }
      *nl += 4;
      op->alpha_d = op->alpha_f;
      op->nu_d = op->nu_f;
      op->dmk_ok = true;
    }
    HX_TRY(hx_launch_axpby(m->n_dof, op->alpha / op->alpha_d, op->dmk, op->nu / op->nu_d, op->dmk + m->n_dof, op->diag,
                           s),
           "diagonal from its parts");
    *nl += 1;
  } else {
    HX_TRY(diag_launcher(m->p)(m->T, d, op->geom, s), "diagonal kernel");
    HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, op->diag, s),
           "diagonal assembly");
    *nl += 2;
  }
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
    HX_TRY(hx_launch_cmass(m->T, m->E, m->X8, op->alpha, op->yE, m->lay, s), "collocated mass");
    HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, op->pdiag, s),
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
    // constant coefficients, both nonzero before and after: the factors scale in place (a
    // bounded number of times in a row, then the geometry kernel recomputes them)
    if (!nu_q && op->factors_ok && op->alpha_f != 0.0 && op->nu_f != 0.0 && alpha != 0.0 && nu != 0.0 &&
        op->rescales < kMaxRescales) {
      HX_TRY(hx_launch_scale_factors(m->E, (int)Q3, alpha / op->alpha_f, nu / op->nu_f, op->factors, s),
             "factor rescale");
      ++op->rescales;
    } else {
      HX_TRY(hx_launch_geometry(m->T, m->E, m->X8, nu_q, alpha, nu, op->factors, bad, s), "geometry kernel");
      op->rescales = 0;
      op->dmk_ok = false;
      op->dmk32_ok = false;
    }
    op->alpha_f = alpha;
    op->nu_f = nu;
    op->factors_ok = nu_q == nullptr;
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

}  // namespace hxc

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
      la.lay = m->lay;
      e = load_launcher(m->p)(m->T, la, s);
      if (e == cudaSuccess) e = hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, op->m1, s);
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
  HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, constrained, x, 0.0, y, s), "assembly");
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
  a.lay = m->lay;
  HX_TRY(load_launcher(m->p)(m->T, a, s), "load kernel");
  HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 0, nullptr, 0.0, b, s), "assembly");
  op->launches += 2;
  return HX_OK;
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
