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

// The while-loop node of G (after `dep`) whose body is captured from body(handle).
hx_status add_while_node(cudaGraph_t G, cudaStream_t cs, cudaGraphNode_t dep,
                         const std::function<cudaError_t(unsigned long long)>& body, cudaGraphNode_t* loop) {
  cudaGraphConditionalHandle h = 0;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault);
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(raw);
  np->type = cudaGraphNodeTypeConditional;
  np->conditional.handle = h;
  np->conditional.type = cudaGraphCondTypeWhile;
  np->conditional.size = 1;
  if (e == cudaSuccess) e = cudaGraphAddNode(loop, G, &dep, nullptr, 1, np);
  if (e == cudaSuccess) {
    cudaGraph_t bodyg = np->conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t eb = body((unsigned long long)h);
      e = cudaStreamEndCapture(cs, &bodyg);
      if (eb != cudaSuccess) e = eb;
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch while node");
  return HX_OK;
}

// Instance i's solve before its iterations: r = P b (mean removed for pure Neumann), z, p.
cudaError_t instance_init(hx_batch* B, int i, double rtol, int max_it, cudaStream_t cs) {
  hx_op* op = B->ops[i];
  const HxCgBuffers buf = cg_buffers(op);
  const double* bi = B->b[i];
  cudaError_t e = cudaSuccess;
  if (op->singular) e = hx_launch_cg_mean(buf, bi, cs);
  if (e == cudaSuccess) e = hx_launch_cg_init(buf, bi, (const double*)nullptr, rtol, max_it, cs);
  if (e == cudaSuccess) e = precondition_start(op, cs);
  if (e == cudaSuccess) e = hx_launch_cg_start(buf, cs);
  if (e == cudaSuccess && op->singular) e = hx_launch_cg_direction(buf, cs);
  return e;
}

// Instance i's solve after its iterations: mean-zero closure (pure Neumann), true residual,
// solution copy.
cudaError_t instance_tail(hx_batch* B, int i, cudaStream_t cs) {
  hx_op* op = B->ops[i];
  const hx_mesh* m = op->mesh;
  cudaError_t e = cudaSuccess;
  if (op->singular) {
    e = hx_launch_sum(m->n_dof, op->m1, op->partial, op->counters, op->vol, cs);
    if (e == cudaSuccess) e = hx_launch_dot(m->n_dof, op->m1, op->x, op->partial, op->counters, op->vol + 1, cs);
    if (e == cudaSuccess) e = hx_launch_shift(m->n_dof, op->x, op->vol + 1, op->vol, cs);
  }
  if (e == cudaSuccess) e = element_apply(op, op->x, 1, nullptr, cs);
  if (e == cudaSuccess)
    e = hx_launch_assemble(m->n_dof, m->ga, m->off, m->idx, op->yE, m->dir, 1, op->x, 0.0, op->Ap, cs);
  if (e == cudaSuccess)
    e = hx_launch_resnorm(m->n_dof, B->b[i], op->Ap, m->dir, op->partial, op->counters, op->scalars, cs,
                          op->singular ? &op->st->shift : nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->x[i], op->x, sizeof(double) * m->n_dof, cudaMemcpyDeviceToDevice, cs);
  return e;
}

// Instance i's whole solve as a branch of G after `dep` (may be null); its tail node out.
hx_status add_instance_branch(cudaGraph_t G, hx_batch* B, int i, double rtol, int max_it, const cudaGraphNode_t* dep,
                              cudaGraphNode_t* tail) {
  cudaStream_t cs = B->stream;
  hx_op* op = B->ops[i];
  cudaGraphNode_t init = nullptr, loop = nullptr;
  hx_status s = add_captured_child(G, cs, dep, dep ? 1 : 0, [&]() { return instance_init(B, i, rtol, max_it, cs); },
                                   &init);
  if (s == HX_OK)
    s = add_while_node(G, cs, init, [&](unsigned long long h) { return cg_iteration(op, cs, h); }, &loop);
  if (s == HX_OK) s = add_captured_child(G, cs, &loop, 1, [&]() { return instance_tail(B, i, cs); }, tail);
  return s;
}

// Lock-step mode: the instances with a diagonal preconditioner iterate together, one loop body
// per CG iteration for all of them, each pass one launch over a work list (element kernel: one
// launch per order, quadrature and geometry mode; vector passes: one launch for all).
bool fusable(const hx_op* op) { return op->prec == HX_PREC_JACOBI || op->prec == HX_PREC_COLLOCATED_MASS; }

hx_status build_fused_tables(hx_batch* B, double rtol, int max_it) {
  (void)rtol;
  (void)max_it;
  hx_batch::Fused& F = B->fused;
  if (F.built) return HX_OK;
  std::vector<int> ids;
  for (int i = 0; i < B->n; ++i)
    if (fusable(B->ops[i])) ids.push_back(i);
  F.members = ids;
  const int nf = (int)ids.size();
  if (nf == 0) {
    F.built = true;
    return HX_OK;
  }
  // vector passes: each instance gets the blocks its solo passes use (the reductions finish per
  // instance over its own blocks, in the same order as in a solo solve)
  std::vector<HxCgBuffers> bufs(nf);
  std::vector<HxCgState*> states(nf);
  std::vector<int> vop, vfirst(nf), vcount(nf);
  for (int k = 0; k < nf; ++k) {
    const hx_op* op = B->ops[ids[k]];
    bufs[k] = cg_buffers(op);
    bufs[k].cond = 0ull;
    states[k] = op->st;
    const long long nb = hx_red_blocks(op->mesh->n_dof);  // the blocks of its solo passes
    vfirst[k] = (int)vop.size();
    vcount[k] = (int)nb;
    for (long long b = 0; b < nb; ++b) vop.push_back(k);
  }
  // element kernel: one group per (p, q, geometry mode, nu field)
  std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
  for (int k = 0; k < nf; ++k) {
    const hx_op* op = B->ops[ids[k]];
    groups[std::make_tuple(op->mesh->p, op->mesh->q, op->geom, op->use_field ? 1 : 0)].push_back(k);
  }
  static const hx_block_elems_fn nel_fn[] = {nullptr, hx_apply_block_elems_p1, hx_apply_block_elems_p2,
                                             hx_apply_block_elems_p3, hx_apply_block_elems_p4,
                                             hx_apply_block_elems_p5, hx_apply_block_elems_p6,
                                             hx_apply_block_elems_p7, hx_apply_block_elems_p8};
  std::vector<HxApplyArgs> args;
  std::vector<int> eop, efirst;
  F.groups.clear();
  for (auto& kv : groups) {
    hx_batch::Group g;
    g.p = std::get<0>(kv.first);
    g.geom = std::get<2>(kv.first);
    g.nuf = std::get<3>(kv.first);
    g.T = B->ops[ids[kv.second[0]]]->mesh->T;
    g.args_off = (int)args.size();
    g.blk_off = (long long)eop.size();
    const int ne = nel_fn[g.p](std::get<1>(kv.first), g.geom);
    for (size_t j = 0; j < kv.second.size(); ++j) {
      const hx_op* op = B->ops[ids[kv.second[j]]];
      args.push_back(apply_args(op, op->p, 1, &op->st->done));
      efirst.push_back((int)(eop.size() - g.blk_off));
      const long long nb = (op->mesh->E + ne - 1) / ne;
      for (long long b = 0; b < nb; ++b) eop.push_back((int)j);
    }
    g.blocks = (long long)eop.size() - g.blk_off;
    F.groups.push_back(g);
  }
  hx_status s;
  if ((s = dalloc(&F.bufs, bufs.size(), "batch buffers")) || (s = dalloc(&F.states, states.size(), "batch states")) ||
      (s = dalloc(&F.vop, vop.size(), "batch pass table")) || (s = dalloc(&F.vfirst, vfirst.size(), "batch pass table")) ||
      (s = dalloc(&F.vcount, vcount.size(), "batch pass table")) || (s = dalloc(&F.args, args.size(), "batch arguments")) ||
      (s = dalloc(&F.eop, eop.size(), "batch block table")) || (s = dalloc(&F.efirst, efirst.size(), "batch block table")))
    return s;
  F.vblocks = (long long)vop.size();
  HX_TRY(cudaMemcpy(F.bufs, bufs.data(), sizeof(HxCgBuffers) * bufs.size(), cudaMemcpyHostToDevice), "batch tables");
  HX_TRY(cudaMemcpy(F.states, states.data(), sizeof(HxCgState*) * states.size(), cudaMemcpyHostToDevice),
         "batch tables");
  HX_TRY(cudaMemcpy(F.vop, vop.data(), sizeof(int) * vop.size(), cudaMemcpyHostToDevice), "batch tables");
  HX_TRY(cudaMemcpy(F.vfirst, vfirst.data(), sizeof(int) * vfirst.size(), cudaMemcpyHostToDevice), "batch tables");
  HX_TRY(cudaMemcpy(F.vcount, vcount.data(), sizeof(int) * vcount.size(), cudaMemcpyHostToDevice), "batch tables");
  HX_TRY(cudaMemcpy(F.args, args.data(), sizeof(HxApplyArgs) * args.size(), cudaMemcpyHostToDevice), "batch tables");
  HX_TRY(cudaMemcpy(F.eop, eop.data(), sizeof(int) * eop.size(), cudaMemcpyHostToDevice), "batch tables");
  HX_TRY(cudaMemcpy(F.efirst, efirst.data(), sizeof(int) * efirst.size(), cudaMemcpyHostToDevice), "batch tables");
  F.built = true;
  return HX_OK;
}

// One lock-step CG iteration of the fused instances (h: the enclosing while loop's handle).
cudaError_t fused_iteration(hx_batch* B, unsigned long long h) {
  static const hx_apply_multi_launcher t[] = {nullptr, hx_launch_apply_multi_p1, hx_launch_apply_multi_p2,
                                              hx_launch_apply_multi_p3, hx_launch_apply_multi_p4,
                                              hx_launch_apply_multi_p5, hx_launch_apply_multi_p6,
                                              hx_launch_apply_multi_p7, hx_launch_apply_multi_p8};
  hx_batch::Fused& F = B->fused;
  cudaStream_t cs = B->stream;
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < F.groups.size() && e == cudaSuccess; ++k) {
    const hx_batch::Group& g = F.groups[k];
    e = t[g.p](g.T, F.args + g.args_off, F.eop + g.blk_off, F.efirst + g.args_off, g.blocks, g.geom, g.nuf, cs);
  }
  if (e == cudaSuccess) e = hx_launch_cg_pass_multi(HX_PASS_ASSEMBLE_PAP, F.bufs, F.vop, F.vfirst, F.vcount, F.vblocks, cs);
  if (e == cudaSuccess) e = hx_launch_cg_pass_multi(HX_PASS_UPDATE, F.bufs, F.vop, F.vfirst, F.vcount, F.vblocks, cs);
  if (e == cudaSuccess) e = hx_launch_cg_pass_multi(HX_PASS_DIRECTION, F.bufs, F.vop, F.vfirst, F.vcount, F.vblocks, cs);
  if (e == cudaSuccess) e = hx_launch_batch_condition(F.states, (int)F.members.size(), h, cs);
  return e;
}

hx_status build_batch_graph(hx_batch* B, double rtol, int max_it, int lanes) {
  cudaGraph_t G = nullptr;
  HX_TRY(cudaGraphCreate(&G, 0), "batch graph");
  hx_status s = HX_OK;
  cudaStream_t cs = B->stream;
  if (lanes == HX_BATCH_FUSED) {
    s = build_fused_tables(B, rtol, max_it);
    // instances the lock-step loop cannot take (preconditioners applied outside the CG
    // kernels) are branches of their own, running beside it
    for (int i = 0; i < B->n && s == HX_OK; ++i) {
      if (fusable(B->ops[i])) continue;
      cudaGraphNode_t tail = nullptr;
      s = add_instance_branch(G, B, i, rtol, max_it, nullptr, &tail);
    }
    const std::vector<int>& mem = B->fused.members;
    if (s == HX_OK && !mem.empty()) {
      cudaGraphNode_t init = nullptr, loop = nullptr, tail = nullptr;
      s = add_captured_child(G, cs, nullptr, 0, [&]() {
        cudaError_t e = cudaSuccess;
        for (size_t k = 0; k < mem.size() && e == cudaSuccess; ++k) e = instance_init(B, mem[k], rtol, max_it, cs);
        return e;
      }, &init);
      if (s == HX_OK) s = add_while_node(G, cs, init, [&](unsigned long long h) { return fused_iteration(B, h); }, &loop);
      if (s == HX_OK)
        s = add_captured_child(G, cs, &loop, 1, [&]() {
          cudaError_t e = cudaSuccess;
          for (size_t k = 0; k < mem.size() && e == cudaSuccess; ++k) e = instance_tail(B, mem[k], cs);
          return e;
        }, &tail);
    }
  } else {
    // instance i runs after instance i - lanes: `lanes` chains of solves run side by side
    std::vector<cudaGraphNode_t> tails((size_t)B->n, nullptr);
    for (int i = 0; i < B->n && s == HX_OK; ++i) {
      const cudaGraphNode_t* dep = (i >= lanes) ? &tails[(size_t)(i - lanes)] : nullptr;
      s = add_instance_branch(G, B, i, rtol, max_it, dep, &tails[(size_t)i]);
    }
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
  cand.push_back(HX_BATCH_FUSED);
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
  B->tune = lanes < 0 && lanes != HX_BATCH_FUSED;
  B->lanes = lanes == HX_BATCH_FUSED ? HX_BATCH_FUSED : (lanes <= 0 || lanes > n) ? n : lanes;
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
  hx_batch::Fused& F = B->fused;
  dfree(F.bufs);
  dfree(F.states);
  dfree(F.vop);
  dfree(F.vfirst);
  dfree(F.vcount);
  dfree(F.args);
  dfree(F.eop);
  dfree(F.efirst);
  delete B;
}

}  // extern "C"
