// C ABI of libhx.so (include/hx.h): mixed precision -- FP64 iterative refinement around an
// FP32 PCG with the FP32 operator (not part of the paper's method).
#include "hx_capi_internal.h"

using namespace hxc;

// ---------------------------------------------------------------------------
// mixed precision: FP64 iterative refinement around an FP32 Jacobi-PCG
// ---------------------------------------------------------------------------
namespace hxc {

HxApplyArgsF apply_args32(const hx_op* op, const float* x, const int* done) {
  const hx_mesh* m = op->mesh;
  HxApplyArgsF a;
  a.E = m->E;
  a.R = m->R;
  a.x = x;
  a.yE = op->yE32;
  a.lay = m->lay;
  a.factors = op->factors32;
  a.fstride = hx_f32_factor_stride(m->q);
  a.X8 = m->X8;
  a.nu_q = op->use_field ? op->nu_q : nullptr;
  a.alpha = op->alpha;
  a.nu = op->nu;
  a.constrained = 1;
  a.done = done;
  a.err = op->kerr;
  a.wait_limit = op->wait_limit;
  return a;
}

cudaError_t element_apply32(const hx_op* op, const float* x, const int* done, cudaStream_t s) {
  static const hx_apply32_launcher t[] = {nullptr, hx_launch_apply32_p1, hx_launch_apply32_p2, hx_launch_apply32_p3,
                                          hx_launch_apply32_p4, hx_launch_apply32_p5, hx_launch_apply32_p6,
                                          hx_launch_apply32_p7, hx_launch_apply32_p8};
  const HxApplyArgsF a = apply_args32(op, x, done);
  return t[op->mesh->p](op->mesh->T32, a, op->geom, op->f32_kind, op->f32_tile, s);
}

// Autotuned choice of the FP32 element kernel, shared by the operators of one process with the
// same order, quadrature, geometry mode and size class (log2 of the element count).
struct F32Key {
  int p, q, geom, field, size_class;
  bool operator<(const F32Key& o) const {
    return std::tie(p, q, geom, field, size_class) < std::tie(o.p, o.q, o.geom, o.field, o.size_class);
  }
};
std::mutex g_f32_mutex;
std::map<F32Key, std::pair<int, int>> g_f32_choice;  // (kind, tile)

// The FP32 element kernel this operator runs: the caller's choice (hx_op_set_f32_kernel, default
// tile), else the fastest candidate -- kernel form and tile shape (elements per block) -- for this
// order, quadrature and geometry mode, timed once per process and size class on this operator
// (one warm-up and three timed element-kernel launches each, CUDA events on the solver stream).
// The candidates compute the same operator; they differ in how the contractions are organized
// (collocated derivative or B/D-direct), in whether the stored factors arrive by bulk copies,
// and in how many elements a block holds.
hx_status tune_f32(hx_op* op) {
  if (op->f32_kind >= 0) return HX_OK;
  if (op->f32_request >= 0) {
    const bool direct = op->f32_request == HX_F32_DIRECT_STAGED || op->f32_request == HX_F32_DIRECT;
    const int tile = direct ? op->f32_tile_request : 0;
    if (direct && tile != 0) {
      static const hx_block_elems_fn t[] = {nullptr, hx_apply32_block_elems_p1, hx_apply32_block_elems_p2,
                                            hx_apply32_block_elems_p3, hx_apply32_block_elems_p4,
                                            hx_apply32_block_elems_p5, hx_apply32_block_elems_p6,
                                            hx_apply32_block_elems_p7, hx_apply32_block_elems_p8};
      if (t[op->mesh->p](op->mesh->q, tile) == 0)
        return fail(HX_ERR_UNSUPPORTED, "no FP32 tile variant %d for p = %d, q = %d", tile, op->mesh->p, op->mesh->q);
    }
    op->f32_kind = op->f32_request;
    op->f32_tile = tile;
    return HX_OK;
  }
  const hx_mesh* m = op->mesh;
  int size_class = 0;
  for (long long e = m->E; e > 1; e >>= 1) ++size_class;
  const F32Key key{m->p, m->q, op->geom, op->use_field ? 1 : 0, size_class};
  {
    std::lock_guard<std::mutex> lock(g_f32_mutex);
    auto it = g_f32_choice.find(key);
    if (it != g_f32_choice.end()) {
      op->f32_kind = it->second.first;
      op->f32_tile = it->second.second;
      return HX_OK;
    }
  }
  cudaStream_t st = op->stream;
  std::vector<std::pair<int, int>> cand;
  cand.push_back({HX_F32_COLLOCATED, 0});
  const int tiles = op->geom == HX_GEOM_STORED ? 1 : 0;  // tile variants only with stored factors
  for (int tl = -tiles; tl <= tiles; ++tl) {
    if (op->geom == HX_GEOM_STORED) cand.push_back({HX_F32_DIRECT_STAGED, tl});
    cand.push_back({HX_F32_DIRECT, tl});
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaMemsetAsync(op->p32, 0, sizeof(float) * m->n_dof, st);
  std::pair<int, int> best = cand[0];
  float best_ms = -1.0f;
  for (int i = 0; i < 3; ++i) op->f32_ms[i] = -1.0f;
  for (size_t k = 0; k < cand.size() && e == cudaSuccess; ++k) {
    op->f32_kind = cand[k].first;
    op->f32_tile = cand[k].second;
    // a tile variant that does not exist for this order (too many threads or too much shared
    // memory) is refused by its launcher before anything is enqueued: skip it
    if (element_apply32(op, op->p32, nullptr, st) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    e = cudaEventRecord(t0, st);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = element_apply32(op, op->p32, nullptr, st);
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    op->launches += 4;
    if (e != cudaSuccess) break;
    float& km = op->f32_ms[cand[k].first];
    if (km < 0.0f || ms / 3.0f < km) km = ms / 3.0f;  // per kind: its fastest tile
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best = cand[k];
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) {
    op->f32_kind = -1;
    return cuda_fail(e, "FP32 kernel timing");
  }
  op->f32_kind = best.first;
  op->f32_tile = best.second;
  std::lock_guard<std::mutex> lock(g_f32_mutex);
  g_f32_choice[key] = best;
  return HX_OK;
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
  b.ga = m->ga;
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
        (s = dalloc(&op->factors32, (size_t)m->E * hx_f32_factor_stride(m->q) + 4, "FP32 factors")))
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
      HX_TRY(hx_launch_to_float_strided(m->E, 7 * m->q * m->q * m->q, (int)hx_f32_factor_stride(m->q), op->factors,
                                        op->factors32, op->stream),
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
      d.fstride = hx_f32_factor_stride(m->q);
      d.X8 = m->X8;
      d.nu_q = op->use_field ? op->nu_q : nullptr;
      d.alpha = op->alpha;
      d.nu = op->nu;
      d.dE = op->yE32;
      d.lay = m->lay;
      d.parts = 3;
      // stored factors of constant coefficients: from its mass and stiffness parts, as in FP64
      const bool split = op->geom == HX_GEOM_STORED && op->factors_ok && op->alpha_f != 0.0 && op->nu_f != 0.0;
      if (split) {
        if (!op->dmk32_ok) {
          if (!op->dmk32 && (s = dalloc(&op->dmk32, 2 * (size_t)n, "FP32 diagonal parts"))) return s;
          for (int part = 0; part < 2; ++part) {
            d.parts = 1 + part;
            HX_TRY(t[m->p](m->T32, d, op->geom, op->stream), "FP32 diagonal kernel");
            HX_TRY(hx_launch_assemble32(n, m->ga, m->off, m->idx, op->yE32, m->dir, 0, nullptr, op->dmk32 + part * n,
                                        op->stream),
                   "FP32 diagonal assembly");
          }
          op->launches += 4;
          op->alpha_d32 = op->alpha_f;
          op->nu_d32 = op->nu_f;
          op->dmk32_ok = true;
        }
        HX_TRY(hx_launch_axpby32(n, (float)(op->alpha / op->alpha_d32), op->dmk32, (float)(op->nu / op->nu_d32),
                                 op->dmk32 + n, op->Ap32, op->stream),
               "FP32 diagonal from its parts");
      } else {
        HX_TRY(t[m->p](m->T32, d, op->geom, op->stream), "FP32 diagonal kernel");
        HX_TRY(hx_launch_assemble32(n, m->ga, m->off, m->idx, op->yE32, m->dir, 0, nullptr, op->Ap32, op->stream),
               "FP32 diagonal assembly");
        op->launches += 1;
      }
      HX_TRY(hx_launch_dinv32(n, op->Ap32, m->dir, op->dinv32, op->stream), "FP32 dinv");
      op->launches += 2;
    } else {
      if ((s = ensure_dinv(op, op->stream))) return s;
      HX_TRY(hx_launch_to_float(n, op->dinv, op->dinv32, op->stream), "FP32 dinv");
      op->launches += 1;
    }
    op->launches += (op->geom == HX_GEOM_STORED) ? 1 : 0;
    op->mixed_stale = false;
  }
  return tune_f32(op);
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
    HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, st),
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
  // the kernel error flag reports this solve only
  HX_TRY(cudaMemsetAsync(op->kerr, 0, sizeof(int), st), "flag reset");
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
      if (!op->st_host->done) {
        if ((s = check_kernel_flag(op, st))) return s;
        return fail(HX_ERR_CUDA, "inner CG graph loop ended before the solver finished");
      }
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

}  // namespace hxc

extern "C" {

hx_status hx_solve_pcg_mixed(hx_op* op, const double* b, double* x, double rtol, int max_it, double inner_rtol,
                             void* stream, hx_solve_info* info) {
  if (!op || !b || !x) return fail(HX_ERR_ARG, "NULL argument");
  if (!(rtol >= 0.0) || max_it < 0 || !(inner_rtol > 0.0 && inner_rtol < 1.0))
    return fail(HX_ERR_ARG, "need rtol >= 0, max_it >= 0 and 0 < inner_rtol < 1");
  return solve_mixed(op, b, x, rtol, max_it, inner_rtol, (cudaStream_t)stream, info);
}

hx_status hx_op_set_f32_kernel(hx_op* op, int kind) {
  if (!op) return fail(HX_ERR_ARG, "op is NULL");
  if (kind < HX_F32_AUTO || kind > HX_F32_MMA_BF16X3) return fail(HX_ERR_ARG, "unknown FP32 kernel kind %d", kind);
  if ((kind == HX_F32_DIRECT_STAGED || kind == HX_F32_MMA_BF16 || kind == HX_F32_MMA_BF16X3) &&
      op->geom != HX_GEOM_STORED)
    return fail(HX_ERR_UNSUPPORTED, "FP32 kernel kind %d needs stored factors", kind);
  op->f32_request = kind;
  op->f32_kind = -1;  // resolved (or tuned) at the next FP32 set-up
  if (op->graph32) {
    cudaGraphExecDestroy(op->graph32);
    op->graph32 = nullptr;
  }
  op->graph32_failed = false;
  return HX_OK;
}

hx_status hx_op_set_f32_tile(hx_op* op, int tile) {
  if (!op) return fail(HX_ERR_ARG, "op is NULL");
  if (tile < -1 || tile > 1) return fail(HX_ERR_ARG, "FP32 tile variant %d is not -1, 0 or 1", tile);
  if (tile != 0 && op->geom != HX_GEOM_STORED)
    return fail(HX_ERR_UNSUPPORTED, "FP32 tile variants need stored factors");
  op->f32_tile_request = tile;
  op->f32_kind = -1;  // resolved at the next FP32 set-up
  if (op->graph32) {
    cudaGraphExecDestroy(op->graph32);
    op->graph32 = nullptr;
  }
  op->graph32_failed = false;
  return HX_OK;
}

hx_status hx_op_f32_kernel(const hx_op* op, int* kind, int* block_elems, float* ms) {
  if (!op || !kind) return fail(HX_ERR_ARG, "NULL argument");
  *kind = op->f32_kind;
  if (block_elems) {
    static const hx_block_elems_fn t[] = {nullptr, hx_apply32_block_elems_p1, hx_apply32_block_elems_p2,
                                          hx_apply32_block_elems_p3, hx_apply32_block_elems_p4,
                                          hx_apply32_block_elems_p5, hx_apply32_block_elems_p6,
                                          hx_apply32_block_elems_p7, hx_apply32_block_elems_p8};
    const bool direct = op->f32_kind == HX_F32_DIRECT_STAGED || op->f32_kind == HX_F32_DIRECT;
    *block_elems = direct ? t[op->mesh->p](op->mesh->q, op->f32_tile) : -1;
  }
  if (ms)
    for (int i = 0; i < 3; ++i) ms[i] = op->f32_ms[i];  // the autotuner's candidates (kinds 0..2)
  return HX_OK;
}

hx_status hx_op_set_wait_limit(hx_op* op, int attempts) {
  if (!op) return fail(HX_ERR_ARG, "op is NULL");
  if (attempts < 0) return fail(HX_ERR_ARG, "attempts must be >= 0");
  op->wait_limit = attempts;
  // the captured inner CG carries the limit as a kernel parameter: capture again at the next solve
  if (op->graph32) {
    cudaGraphExecDestroy(op->graph32);
    op->graph32 = nullptr;
  }
  op->graph32_failed = false;
  return HX_OK;
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
  HX_TRY(hx_launch_assemble32(m->n_dof, m->ga, m->off, m->idx, op->yE32, m->dir, 1, x, y, us), "FP32 assembly");
  op->launches += 2;
  return HX_OK;
}

}  // extern "C"
