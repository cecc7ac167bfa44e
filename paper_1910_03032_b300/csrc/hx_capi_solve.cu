// C ABI of libhx.so (include/hx.h): the Jacobi-PCG solve (Sec. 5, Sec. 5.3), its iterations
// captured once into a CUDA graph with a device-side while loop.
#include "hx_capi_internal.h"

using namespace hxc;

// ---------------------------------------------------------------------------
// Jacobi-PCG
// ---------------------------------------------------------------------------
namespace hxc {

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
  b.ga = m->ga;
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
cudaError_t cg_iteration(const hx_op* op, cudaStream_t s, unsigned long long cond) {
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
    HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, st), "cg x0 assembly");
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
  HX_TRY(hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, st), "residual assembly");
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

}  // namespace hxc

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
  const std::string msg = last_error();
  HX_TRY(cudaMemcpyAsync(x_host, op->hx, sizeof(double) * n, cudaMemcpyDeviceToHost, op->stream), "x download");
  HX_TRY(cudaStreamSynchronize(op->stream), "solver sync");
  last_error() = msg;
  return r;
}

}  // extern "C"
