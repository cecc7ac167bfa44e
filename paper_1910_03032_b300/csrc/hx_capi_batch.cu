// C ABI of libhx.so (include/hx.h): batched solves of independent instances (the projection
// step's Helmholtz and Poisson solves, Sec. 4.2 and Sec. 5.3) in one graph.
#include "hx_capi_internal.h"

using namespace hxc;

// ---------------------------------------------------------------------------
// batched solves: every instance's whole Jacobi-PCG is a branch of one graph
// ---------------------------------------------------------------------------
namespace hxc {

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
        e3 = hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, cs);
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

}  // namespace hxc

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
