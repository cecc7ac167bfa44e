"""Benchmark: FP64 matrix-free Q_p Helmholtz operator and Jacobi-PCG on one B300 (per rank).

One step = one pass of the whole hot path on the resident problem:
  coefficient setup (geometric factors m = alpha w detJ, G = nu w detJ J^-1 J^-T,
  and the sum-factorized diagonal), then Jacobi-PCG to a 1e-10 relative
  residual, each iteration one matrix-free apply (gather, sum-factorized
  contractions, pointwise factors, transposed contractions, atomic-free
  assembly) plus the fused vector updates; one more apply checks the true
  residual.

Workload (default): perturbed 96^3 hexahedral mesh of the unit cube, Q_4
(57,066,625 DoFs), 6^3 Gauss points per element, alpha = 1/dt = 1000,
nu = 1e-2, homogeneous Dirichlet boundary, manufactured right-hand side
f = (alpha + 3 pi^2 nu) sin(pi x) sin(pi y) sin(pi z), stored factors.

value = DoF-applies per second: n_dof x (applies per solve) / step time, in
GDoF/s, summed over ranks (each rank solves its own replica; there is no
data-path collective).  The JSON line also carries the PCG time, the
isolated apply throughput, the roofline of the element kernel, the
end-to-end number through host buffers, the CPU oracle baseline, and the
SM clocks sampled during the timed region.

The default run also carries a bounded per-order sweep (p = 2..8 on the FP64 sweep meshes:
FP64 apply, FP32 apply, on-the-fly apply, FP64 set-up + PCG step and mixed-precision step,
each timed with CUDA events) and the measured FP64 / FP32 FMA rates of the device.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hx|reference]
                       [--p P] [--n N] [--geom stored|onthefly] [--no-cpu] [--no-mixed]
                       [--no-sweep] [--sweep-reps R] [--f32-kernel K] [--grad] [--precond]
                       [--batch [--batch-reps R]]
       python bench.py --vcycle [--p P] [--n N]     (the LOR multigrid V-cycle alone)
       python bench.py --cheb [--p P] [--n N]       (the LOR-Chebyshev preconditioner alone)
       python bench.py --peaks                      (the FP64 / FP32 FMA-rate probe alone)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "Helmholtz apply GDoF/s & PCG time, p=2-8; mixed/batched vs FP64 at 1e-10"
ALPHA, NU, RTOL = 1000.0, 1e-2, 1e-10
SWEEP_N = {2: 160, 3: 96, 4: 96, 5: 64, 6: 64, 7: 48, 8: 48}
def _measured_hbm_gbs(fallback=6400.0):
    """The measured copy bandwidth of the B300 (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return fallback


HBM_GBS = _measured_hbm_gbs()
# FP64 peak of the B300 from the unit count: 2 DFMA per clock per SM x 148 SMs x 2032 MHz x
# 2 flops (the library's FMA-rate probe reaches 506 G DFMA/s = 1.68 per clock per SM; every
# default run measures it again and reports the fraction of both).
FP64_PEAK_TFLOPS = 148 * 2.032e9 * 2 * 2 / 1e12
# dram__bytes_read.sum + dram__bytes_write.sum of one element-kernel launch, keyed by
# (p, N, geom): the 32^3 capture of the current kernel (16 elements per block, line-layout
# E-vector; 457.9 MB read + 28.7 MB written) scaled by the element count (27x at 96^3);
# traffic grows in proportion to the elements.
NCU_TRAFFIC = {(4, 96, "stored"): (457.918976e6 + 28.729088e6) * 27}
# sm__pipe_fp64_cycles_active (% of peak sustained) of the same capture: the FP64 pipe's
# own utilization, which the algorithmic-flop fraction overstates (the even-odd folding
# executes fewer flops than the algorithmic count)
NCU_FP64_PIPE = {(4, 96, "stored"): 0.828}
# FP32 element kernels of the mixed-precision solve (include/hx.h HX_F32_*)
F32_KERNELS = {0: "collocated", 1: "direct_staged", 2: "direct", 3: "mma_bf16", 4: "mma_bf16x3"}


def alg_flops_per_element(p: int, q: int) -> int:
    """Algorithmic flops of one element apply: the cheaper of the two sum-factorized
    formulations (B/D-direct, or interpolate then q x q collocated derivative), forward
    plus transpose, and ~20 flops per point for the stored pointwise factors."""
    n = p + 1
    direct = 2 * (4 * q * n ** 3 + 6 * q * q * n * n + 8 * q ** 3 * n)
    coll = 2 * (2 * (q * n ** 3 + q * q * n * n + q ** 3 * n) + 6 * q ** 4)
    return min(direct, coll) + 20 * q ** 3


def alg_bytes_per_apply(p: int, q: int, E: int, n_dof: int, geom: str) -> int:
    """Algorithmic minimum HBM bytes of one apply: x in, y out, restriction indices,
    and the stored factors (7 doubles per point) or 8 vertices per element."""
    n = p + 1
    geo = 7 * 8 * q ** 3 * E if geom == "stored" else 24 * 8 * E
    return 16 * n_dof + 4 * n ** 3 * E + geo


# ---------------------------------------------------------------------------
# measured arithmetic rates (the FMA-throughput probe of the library)
# ---------------------------------------------------------------------------
def measure_peaks(hx, torch, index=0):
    """FP64 and FP32 FMA rates of this device: one probe launch each (16 independent FMA
    chains per thread, one wave of resident 256-thread blocks), timed with CUDA events on the
    launching stream after one warm-up launch, SM clocks sampled meanwhile."""
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    with ClockSampler(index) as clk:
        for name, fp64, iters in (("fp64", 1, 1 << 15), ("fp32", 0, 1 << 21)):
            hx.hx_probe_fma(fp64, max(1, iters // 16))
            torch.cuda.synchronize()
            e0.record(s)
            flops = hx.hx_probe_fma(fp64, iters)
            e1.record(s)
            e1.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            out[name + "_tflops"] = flops / t / 1e12
            out[name + "_ms"] = 1e3 * t
    out["clocks"] = clk.summary()
    out["kernel"] = "fma_probe_kernel (paper_1910_03032_b300/csrc/hx_probe.cu), via hx_probe_fma"
    return out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: one independent problem per rank)
# ---------------------------------------------------------------------------
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:  # host-only runs (the reference arm, CPU tests of this plumbing)
            dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# problem set-up through the library
# ---------------------------------------------------------------------------
def make_problem(hx, torch, p: int, N: int, geom: str):
    q = p + 2
    V = S.structured_vertices(N, N, N, 0.1, S.DEFAULT_MESH_SEED)
    mesh = hx.Mesh.structured(N, N, N, p, q, V)
    gm = hx.HX_GEOM_STORED if geom == "stored" else hx.HX_GEOM_ONTHEFLY
    op = hx.Operator(mesh, ALPHA, NU, geom_mode=gm)
    xq = mesh.qpoint_coords()
    f = (ALPHA + 3 * math.pi ** 2 * NU) * torch.sin(math.pi * xq[..., 0]) * torch.sin(math.pi * xq[..., 1]) * \
        torch.sin(math.pi * xq[..., 2])
    del xq
    b = op.load_vector(f.contiguous())
    del f
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return mesh, op, b


def time_applies(op, torch, x, reps=20, warm=3, constrained=True):
    """Average device time of hx_op_apply (element kernel + assembly) with CUDA events on its stream."""
    y = torch.empty_like(x)
    s = torch.cuda.current_stream()
    for _ in range(warm):
        op.apply(x, y, constrained=constrained)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(reps):
        e0.record(s)
        op.apply(x, y, constrained=constrained)
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(times)), float(np.mean(times))


def run_step(op, b, x):
    """Coefficient set-up, then a cold-started (x0 = 0) Jacobi-PCG solve into x."""
    import paper_1910_03032_b300 as hx
    op.set_coefficients(ALPHA, NU)
    return hx.hx_solve_pcg(op.handle, b, x, RTOL, 20000, use_x0=False)


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def oracle_sample_throughput(p: int, n_apply: int, ns: int):
    """Oracle DoF-applies per second on an ns^3-element piece of the workload: the
    oracle builds its explicit element matrices once, then applies them n_apply times."""
    from oracle import fem
    q = p + 2
    V = S.structured_vertices(ns, ns, ns, 0.1, S.DEFAULT_MESH_SEED)
    om = fem.StructuredMesh(ns, ns, ns, p, q, V, S.structured_elem_vert(ns, ns, ns))
    t0 = time.perf_counter()
    op = fem.Operator(om, ALPHA, NU)
    t1 = time.perf_counter()
    x = S.random_vector(om.n_dof, S.DEFAULT_VECTOR_SEED)
    reps = 3
    for _ in range(reps):
        op.apply(x, constrained=True)
    t2 = time.perf_counter()
    t_setup, t_apply = t1 - t0, (t2 - t1) / reps
    dofs = om.n_dof
    t_solve = t_setup + n_apply * t_apply
    return {"gdofs": dofs * n_apply / t_solve / 1e9, "t_setup": t_setup, "t_apply": t_apply, "n_dof": dofs,
            "n_elem": om.n_elem}


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        th = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if th:
            return int(max(th))
    except Exception:
        pass
    return len(os.sched_getaffinity(0))


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    """The oracle as the reference arm: each step = oracle set-up + PCG-length applies on a sample."""
    if rank != 0:
        return
    p = args.p
    its = args.ref_iterations
    ns = args.ref_elems
    for _ in range(args.warmup):
        oracle_sample_throughput(p, its + 1, ns)
    vals, times = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle_sample_throughput(p, its + 1, ns)
        times.append(time.perf_counter() - t0)
        vals.append(r["gdofs"])
    v = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": v, "unit": "GDoF/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"{ns}^3 elements of the same p/q/perturbation; explicit element matrices "
                                   f"built once, then {its + 1} applies (the GPU arm's PCG applies per solve)"},
        "e2e": {"value": v, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    p, N = args.p, args.n
    return {"workload": f"FP64 Helmholtz alpha*M+nu*K (alpha=1/dt=1000, nu=1e-2) on a perturbed {N}^3 hex mesh, "
                        f"Q_{p} GLL, q={p + 2} Gauss; coefficient update + Jacobi-PCG to 1e-10 on the "
                        f"manufactured RHS", "p": p, "q": p + 2, "mesh": f"{N}^3", "n_dof": (p * N + 1) ** 3,
            "geometry": args.geom, "l2": "inputs larger than L2 (geometric factors stream from HBM every apply)"}


def run_hx(args, world, rank, local):
    import torch
    import paper_1910_03032_b300 as hx
    torch.cuda.set_device(local)
    p, N = args.p, args.n
    mesh, op, b = make_problem(hx, torch, p, N, args.geom)
    n_dof, E, q = mesh.n_dof, mesh.n_elem, mesh.q
    x = torch.zeros_like(b)
    # warm-up
    for _ in range(args.warmup):
        info = run_step(op, b, x)
    torch.cuda.synchronize()
    barrier(world)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    l0 = op.launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(args.steps):
            infos.append(run_step(op, b, x))
        e1.record(s)
        torch.cuda.synchronize()
    launches = op.launch_count() - l0
    barrier(world)
    t_local = e0.elapsed_time(e1) / 1e3
    t = reduce_max(t_local, world)
    applies = sum(i["iterations"] + 1 for i in infos)
    value = world * n_dof * applies / t / 1e9
    its = infos[-1]["iterations"]

    # isolated apply and roofline of the element kernel (dominant kernel)
    t_apply_med, t_apply_mean = time_applies(op, torch, b)
    flops = alg_flops_per_element(p, q) * E
    achieved = flops / t_apply_mean / 1e12
    bytes_alg = alg_bytes_per_apply(p, q, E, n_dof, args.geom)
    traffic = NCU_TRAFFIC.get((p, N, args.geom))

    # end to end through host buffers (pinned), public API, copies inside the timed region
    bh = b.cpu().pin_memory()
    xh = torch.zeros(n_dof, dtype=torch.float64).pin_memory()
    e2e_steps = min(args.steps, 5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        op.set_coefficients(ALPHA, NU)
        info_h = hx.hx_solve_pcg_host(op.handle, bh, xh, RTOL, 20000, False)
    torch.cuda.synchronize()
    t_e2e = reduce_max(time.perf_counter() - t0, world)
    e2e = world * n_dof * e2e_steps * (info_h["iterations"] + 1) / t_e2e / 1e9
    clocks = clk.summary()
    del bh, xh

    mixed = measure_mixed(hx, torch, op, b, x, args, t / args.steps, world) if not args.no_mixed else None
    peaks = measure_peaks(hx, torch, local)

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu:
            # free the device problem first; the oracle runs on the host cores
            r = oracle_sample_throughput(p, its + 1, args.cpu_elems)
            cpu = {"value": r["gdofs"], "unit": "GDoF/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"{args.cpu_elems}^3 elements ({r['n_dof']} DoFs) of the same p, q and perturbation: "
                             f"explicit element matrices built once ({r['t_setup']:.2f} s), then {its + 1} applies "
                             f"at {r['t_apply']:.3f} s each (the GPU's applies per solve)"}
        line = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "pcg_time_s": t / args.steps, "pcg_iterations": its,
            "true_rel_residual": infos[-1]["true_rel_residual"],
            "apply_gdofs": n_dof / t_apply_mean / 1e9, "apply_ms": 1e3 * t_apply_mean,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                         "kernel": f"apply_kernel<P={p},Q={q}> (+ assembly, timed together)",
                         "peak_source": "FP64 pipe: 2 DFMA/clk/SM x 148 SMs x 2032 MHz (derived)",
                         "probe_tflops": peaks["fp64_tflops"],
                         "frac_of_probe": achieved / peaks["fp64_tflops"],
                         "fp64_pipe_ncu": NCU_FP64_PIPE.get((p, N, args.geom)),
                         "alg_flops_per_launch": flops, "alg_bytes_per_launch": bytes_alg,
                         "hbm_gbs": bytes_alg / t_apply_mean / 1e9,
                         "hbm_frac": bytes_alg / t_apply_mean / 1e9 / HBM_GBS},
            "e2e": {"value": e2e, "unit": "GDoF/s", "h2d_bytes_per_step": 8 * n_dof, "d2h_bytes_per_step": 8 * n_dof,
                    "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "mixed": mixed,
            "peaks_probe": peaks,
        }
    del op, mesh, b, x
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_sweep:
        line["sweep"] = run_sweep(hx, torch, args, peaks)
    if rank == 0 and args.grad:
        line["grad"] = run_grad(hx, torch, args)
    if rank == 0 and args.precond:
        line["precond"] = run_precond(hx, torch, args)
    if rank == 0 and args.batch:
        line["batch"] = run_batch(hx, torch, args)
    if rank == 0:
        print(json.dumps(line), flush=True)


def time_applies_f32(op, torch, x32, reps=20, warm=3, group=5):
    """Average device time of the FP32 apply (element kernel + assembly) with CUDA events: groups
    of `group` back-to-back applies between two events, so that the host's launch latency before
    the first kernel of a group is spread over the group (an apply takes only ~1 ms)."""
    s = torch.cuda.current_stream()
    for _ in range(warm):
        op.apply_f32(x32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(max(1, reps // group)):
        e0.record(s)
        for _ in range(group):
            op.apply_f32(x32)
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3 / group)
    return float(np.mean(times))


def measure_mixed(hx, torch, op, b, x64, args, t_fp64, world):
    """Mixed precision on the same problem: FP64 refinement around FP32 Jacobi-PCG to the same 1e-10."""
    p, q = args.p, args.p + 2
    E, n_dof = hx.hx_op_info(op.handle)[:2]
    xm = torch.empty_like(b)
    op.set_f32_kernel(args.f32_kernel)

    def step():
        op.set_coefficients(ALPHA, NU)
        return hx.hx_solve_pcg_mixed(op.handle, b, xm, RTOL, 100000, args.inner_rtol)

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        info = step()
    e1.record(s)
    torch.cuda.synchronize()
    t_mix = reduce_max(e0.elapsed_time(e1) / 1e3, world) / args.steps
    err = float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64))
    kind, block_elems, tune_ms = op.f32_kernel()
    t32 = time_applies_f32(op, torch, b.float())
    n = p + 1
    geo = 7 * 4 * q ** 3 * E if args.geom == "stored" else 24 * 8 * E
    bytes32 = 8 * n_dof + 4 * n ** 3 * E + geo
    # the element kernel alone (its launches timed with CUDA events by the autotuner on this
    # operator): x in, restriction and factors in, E-vector out
    k_ms = tune_ms[kind] if 0 <= kind < len(tune_ms) and tune_ms[kind] > 0 else None
    kbytes = 4 * n_dof + 8 * n ** 3 * E + geo
    kernel_only = None if k_ms is None else {
        "ms": k_ms, "alg_bytes_per_launch": kbytes, "achieved": kbytes / (k_ms * 1e-3) / 1e9,
        "frac": kbytes / (k_ms * 1e-3) / 1e9 / HBM_GBS,
        "timing": "mean of 3 back-to-back launches after 1 warm-up, CUDA events (the FP32 kernel autotuner)"}
    return {"solve_time_s": t_mix, "speedup_vs_fp64": t_fp64 / t_mix, "refinements": info["refinements"],
            "inner_iterations": info["iterations"], "inner_rtol": args.inner_rtol,
            "rel_residual_fp64": info["rel_residual"], "rel_diff_vs_fp64_solution": err,
            "apply_f32_gdofs": n_dof / t32 / 1e9, "apply_f32_ms": 1e3 * t32,
            "f32_kernel": F32_KERNELS.get(kind, kind), "f32_block_elems": block_elems,
            "f32_autotune_ms": {F32_KERNELS[k]: v for k, v in enumerate(tune_ms) if v >= 0},
            "roofline_f32": {"bound": "hbm", "achieved": bytes32 / t32 / 1e9, "peak": HBM_GBS, "unit": "GB/s",
                             "frac": bytes32 / t32 / 1e9 / HBM_GBS, "alg_bytes_per_launch": bytes32,
                             "kernel": f"FP32 element kernel ({F32_KERNELS.get(kind, kind)}, P={p}, Q={q}) "
                                       "+ assembly, timed together",
                             "element_kernel_only": kernel_only}}


def batch_specs(seed=4444, n=64):
    """64 seeded instances: N in [8, 32] elements per direction, p in {2..8}, alpha 0 (Poisson) or
    1/dt with dt log-uniform in [1e-4, 1e-2], nu log-uniform in [1e-4, 1]."""
    u = (S.uniform_pm1(seed, 5 * n).reshape(n, 5) + 1.0) / 2.0  # U[0, 1)
    specs = []
    for i in range(n):
        N = 8 + int(u[i, 0] * 25)
        p = 2 + int(u[i, 1] * 7)
        alpha = 0.0 if u[i, 2] < 0.5 else 1.0 / (10.0 ** (-4 + 2 * u[i, 3]))
        nu = 10.0 ** (-4 + 4 * u[i, 4])
        specs.append((N, p, alpha, nu))
    return specs


def run_batch(hx, torch, args):
    """64 independent instances (8^3..32^3, p = 2..8) in one graph launch vs one solve after another, plus the
    projection-step set (3 velocity Helmholtz + 1 pure-Neumann pressure Poisson, 64^3, p = 5; the
    Poisson instance with the LOR multigrid preconditioner)."""
    def build(specs, faces_of, prec_of=lambda k: (hx.HX_PREC_JACOBI, 0)):
        ops, bs, xs = [], [], []
        for k, (N, p, a, nu) in enumerate(specs):
            V = S.structured_vertices(N, N, N, 0.1, S.DEFAULT_MESH_SEED + k)
            mesh = hx.Mesh.box(N, N, N, p, p + 2, V, dirichlet_faces=faces_of(k))
            op = hx.Operator(mesh, a, nu)
            op.set_preconditioner(*prec_of(k))
            xq = mesh.qpoint_coords()
            f = torch.sin(math.pi * xq[..., 0]) * torch.sin(math.pi * xq[..., 1]) * torch.cos(math.pi * xq[..., 2])
            ops.append(op)
            bs.append(op.load_vector(f.contiguous()))
            xs.append(torch.zeros_like(bs[-1]))
            del xq, f
        return ops, bs, xs

    def timed(fn, reps):
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(reps):
            out = fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps, out

    res = {}
    # the projection step: 3 velocity Helmholtz solves (Jacobi) and the pure-Neumann pressure
    # Poisson, whose Jacobi-PCG needs ~2800 iterations, with the LOR multigrid preconditioner
    for name, specs, faces_of, prec_of in [
            ("batch64", batch_specs(), lambda k: 63, lambda k: (hx.HX_PREC_JACOBI, 0)),
            ("batch64_mg", batch_specs(), lambda k: 63,
             lambda k: (hx.HX_PREC_LOR_MG, 1) if batch_specs()[k][2] == 0.0 else (hx.HX_PREC_JACOBI, 0)),
            ("projection_step", [(64, 5, 1000.0, 1e-2)] * 3 + [(64, 5, 0.0, 1.0)], lambda k: 63 if k < 3 else 0,
             lambda k: (hx.HX_PREC_JACOBI, 0) if k < 3 else (hx.HX_PREC_LOR_MG, 1))]:
        ops, bs, xs = build(specs, faces_of, prec_of)
        seq = lambda: [hx.hx_solve_pcg(o.handle, b, x, RTOL, 20000, False) for o, b, x in zip(ops, bs, xs)]
        seq()
        t_seq, infos_seq = timed(seq, args.batch_reps)
        # lanes: how many chains of solves the graph runs side by side; the best is reported
        by_lanes = {}
        for lanes in ([0, 8, 2, hx.HX_BATCH_FUSED] if len(ops) > 8 else [0, 1, hx.HX_BATCH_FUSED]):
            batch = hx.Batch(ops, bs, xs, rtol=RTOL, max_it=20000, lanes=lanes)
            batch.solve()
            by_lanes[lanes] = timed(batch.solve, args.batch_reps)
            del batch
        best = min(by_lanes, key=lambda k: by_lanes[k][0])
        t_bat, infos = by_lanes[best]
        dof_applies = sum(o.n_dof * (i["iterations"] + 1) for o, i in zip(ops, infos))
        if name == "projection_step":
            # the same step with every solve in mixed precision (FP32 inner CG, FP64 refinement),
            # one solve after another
            mixed = lambda: [o.solve_mixed(b, rtol=RTOL) for o, b in zip(ops, bs)]
            mixed()
            t_mix, infos_mix = timed(mixed, args.batch_reps)
            res["projection_step_mixed"] = {
                "instances": len(ops), "solve_s": t_mix, "speedup_vs_fp64_batched": t_bat / t_mix,
                "inner_iterations": [i["iterations"] for _, i in infos_mix],
                "refinements": [i["refinements"] for _, i in infos_mix],
                "max_rel_residual": max(i["rel_residual"] for _, i in infos_mix),
                "converged": all(i["status"] == 0 for _, i in infos_mix),
                "timing": f"{args.batch_reps} reps after 1 warm-up, sequential"}
        res[name] = {"instances": len(ops), "n_dof_total": sum(o.n_dof for o in ops),
                     "iterations_total": sum(i["iterations"] for i in infos),
                     "converged": all(i["status"] == 0 for i in infos),
                     "max_true_rel_residual": max(i["true_rel_residual"] for i in infos),
                     "batched_s": t_bat, "sequential_s": t_seq, "speedup": t_seq / t_bat,
                     "lanes": "fused" if best == hx.HX_BATCH_FUSED else best,
                     "batched_s_by_lanes": {("fused" if k == hx.HX_BATCH_FUSED else str(k)): v[0]
                                            for k, v in by_lanes.items()},
                     "batched_gdofs": dof_applies / t_bat / 1e9, "timing": f"{args.batch_reps} reps after 1 warm-up"}
        del ops, bs, xs
        torch.cuda.empty_cache()
    return res


def run_grad(hx, torch, args):
    """Forward solve + adjoint solve + gradient contraction of L = 1/2 (u - u*)^T M (u - u*) on a
    perturbed 32^3 mesh, p = 4: nu log-normal (median 1e-2, sigma 0.5) per quadrature point, f a sum
    of Fourier modes up to wavenumber 4, u* = 0.  Times the whole differentiable step and the
    gradient kernel alone."""
    import paper_1910_03032_b300.autograd as ag
    N, p = 32, 4
    q = p + 2
    V = S.structured_vertices(N, N, N, 0.1, S.DEFAULT_MESH_SEED)
    mesh = hx.Mesh.structured(N, N, N, p, q, V)
    E = mesh.n_elem
    nu = torch.as_tensor(np.exp(np.log(1e-2) + 0.5 * S.uniform_pm1(91, E * q ** 3)).reshape(E, q ** 3),
                         device="cuda")
    xq = mesh.qpoint_coords()
    f = torch.zeros(E, q ** 3, dtype=torch.float64, device="cuda")
    amp = S.uniform_pm1(92, 64)
    for k in range(1, 5):
        for a in range(3):
            c = amp[4 * (k - 1) + a]
            f += c * torch.sin(math.pi * k * xq[..., a]) * torch.cos(math.pi * (k - 1) * xq[..., (a + 1) % 3])
    del xq
    alpha = 1000.0
    op = hx.Operator(mesh, alpha, 0.0, nu)
    mass = hx.Operator(mesh, 1.0, 0.0)

    def step():
        nu_t = nu.clone().requires_grad_(True)
        f_t = f.clone().requires_grad_(True)
        u = ag.solve(op, alpha, nu_t, f_t, rtol=RTOL)
        L = 0.5 * torch.dot(u, ag.apply(mass, u))
        L.backward()
        return L, nu_t.grad, f_t.grad

    for _ in range(2):
        step()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        L, gnu, gf = step()
    e1.record(s)
    torch.cuda.synchronize()
    t_step = e0.elapsed_time(e1) / 1e3 / reps
    u, _ = op.solve(op.load_vector(f), rtol=RTOL)
    lam = mass.apply(u)
    dnu = torch.empty_like(nu)
    dff = torch.empty_like(nu)
    for _ in range(3):
        hx.hx_op_gradient(op.handle, u, lam, dnu, dff)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(20):
        hx.hx_op_gradient(op.handle, u, lam, dnu, dff)
    e1.record(s)
    torch.cuda.synchronize()
    t_k = e0.elapsed_time(e1) / 1e3 / 20
    bytes_k = 8 * (2 * mesh.n_dof + 2 * E * q ** 3 + 24 * E) + 4 * E * (p + 1) ** 3
    return {"mesh": f"{N}^3", "p": p, "q": q, "n_dof": mesh.n_dof, "loss": L.item(),
            "step_s": t_step, "grad_kernel_ms": 1e3 * t_k,
            "grad_kernel_gbs": bytes_k / t_k / 1e9, "grad_kernel_bytes": bytes_k,
            "timing": f"{reps} steps after 2 warm-up; kernel: 20 launches after 3"}


def run_precond(hx, torch, args):
    """Preconditioners on two solves: the projection step's pure-Neumann pressure Poisson (64^3,
    p = 5) and the headline Helmholtz (96^3, p = 4, alpha = 1000, nu = 1e-2), both to 1e-10.
    Per preconditioner: set-up time (selection: LOR pattern + values), solve time, iterations."""
    cases = [("poisson_neumann_64_p5", 64, 5, 0.0, 1.0, 0), ("helmholtz_96_p4", 96, 4, 1000.0, 1e-2, 63)]
    precs = [("jacobi", hx.HX_PREC_JACOBI, 0), ("lor_mc_k8", hx.HX_PREC_LOR_MC, 8),
             ("lor_mc_k16", hx.HX_PREC_LOR_MC, 16), ("lor_mg_s1", hx.HX_PREC_LOR_MG, 1),
             ("lor_mg_s2", hx.HX_PREC_LOR_MG, 2)]
    out = {}
    s = torch.cuda.current_stream()
    for name, N, p, alpha, nu, faces in cases:
        V = S.structured_vertices(N, N, N, 0.1, S.DEFAULT_MESH_SEED)
        mesh = hx.Mesh.box(N, N, N, p, p + 2, V, dirichlet_faces=faces)
        op = hx.Operator(mesh, alpha, nu)
        xq = mesh.qpoint_coords()
        f = torch.sin(math.pi * xq[..., 0]) * torch.sin(math.pi * xq[..., 1]) * torch.cos(math.pi * xq[..., 2])
        b = op.load_vector(f.contiguous())
        del xq, f
        res = {"n_dof": mesh.n_dof}
        for pname, kind, k in precs:
            if alpha > 0 and pname == "lor_mc_k16":
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            op.set_preconditioner(kind, max(k, 1))
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - t0
            x, info = op.solve(b, rtol=RTOL, max_it=20000)  # warm-up (graph capture)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            x, info = op.solve(b, rtol=RTOL, max_it=20000)
            e1.record(s)
            torch.cuda.synchronize()
            res[pname] = {"setup_s": t_setup, "solve_s": e0.elapsed_time(e1) / 1e3, "iterations": info["iterations"],
                          "true_rel_residual": info["true_rel_residual"], "status": info["status"]}
            if pname in ("jacobi", "lor_mg_s1"):
                # the same preconditioner inside the mixed-precision refinement (FP32 inner CG)
                xm, infom = op.solve_mixed(b, rtol=RTOL)
                e0.record(s)
                xm, infom = op.solve_mixed(b, rtol=RTOL)
                e1.record(s)
                torch.cuda.synchronize()
                res[pname + "_mixed"] = {"solve_s": e0.elapsed_time(e1) / 1e3, "inner_iterations": infom["iterations"],
                                         "refinements": infom["refinements"], "rel_residual": infom["rel_residual"],
                                         "status": infom["status"]}
        out[name] = res
        del op, mesh, b, x
        torch.cuda.empty_cache()
    return out


def run_vcycle(args):
    """The LOR multigrid preconditioner alone: one V-cycle (smoothing degree 1) against one
    high-order apply on the pure-Neumann Poisson of an N^3, Q_p mesh (the projection step's
    pressure solve); CUDA events, 3 warm-up calls, 10 timed.  Then the FP64 MG-PCG solve and
    the mixed-precision solve with the FP32 V-cycle, each timed on its second call."""
    import torch
    import paper_1910_03032_b300 as hx
    N, p = args.n, args.p
    V = S.structured_vertices(N, N, N, 0.1, S.DEFAULT_MESH_SEED)
    mesh = hx.Mesh.box(N, N, N, p, p + 2, V, dirichlet_faces=0)
    op = hx.Operator(mesh, 0.0, 1.0)
    r = torch.as_tensor(S.uniform_pm1(5, mesh.n_dof), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op.set_preconditioner(hx.HX_PREC_LOR_MG, 1)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, fn in (("vcycle_ms", lambda: op.precond_apply(r)), ("apply_ms", lambda: op.apply(r, constrained=True))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(10):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / 10
    # the two solves that use it, to 1e-10: FP64 MG-PCG and the mixed-precision refinement
    # (FP32 inner CG with the FP32 V-cycle); the second call of each is timed
    b = r - r.mean()
    for name, fn in (("solve", lambda: op.solve(b, rtol=RTOL)), ("solve_mixed", lambda: op.solve_mixed(b, rtol=RTOL))):
        fn()
        e0.record(s)
        x, info = fn()
        e1.record(s)
        torch.cuda.synchronize()
        out[name + "_s"] = e0.elapsed_time(e1) / 1e3
        out[name + "_iterations"] = info["iterations"]
    print(json.dumps({"probe": "lor_multigrid_vcycle", "mesh": f"{N}^3", "p": p, "n_dof": mesh.n_dof,
                      "setup_s": t_setup, **out}), flush=True)


def run_cheb(args):
    """The LOR-Chebyshev preconditioner (HX_PREC_LOR_MC) alone on the pure-Neumann Poisson of an
    N^3, Q_p mesh: one application at degree 1 (the Jacobi step) and at degree 16; the 15
    Chebyshev steps (one sliced-ELL SpMV each) take the difference.  Algorithmic bytes of a step:
    12 B per stored entry (value + column) + 56 B per row (own d_in, D^-1, res read/write, d_out,
    z read/write); the gathered neighbours of d_in are taken as cache hits.  CUDA events, 3 warm-up
    calls, 10 timed."""
    import torch
    import paper_1910_03032_b300 as hx
    N, p = args.n, args.p
    V = S.structured_vertices(N, N, N, 0.1, S.DEFAULT_MESH_SEED)
    mesh = hx.Mesh.box(N, N, N, p, p + 2, V, dirichlet_faces=0)
    op = hx.Operator(mesh, 0.0, 1.0)
    r = torch.as_tensor(S.uniform_pm1(5, mesh.n_dof), device="cuda")
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for k in (1, 16):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op.set_preconditioner(hx.HX_PREC_LOR_MC, k)
        torch.cuda.synchronize()
        out[f"setup_k{k}_s"] = time.perf_counter() - t0
        for _ in range(3):
            op.precond_apply(r)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(10):
            op.precond_apply(r)
        e1.record(s)
        torch.cuda.synchronize()
        out[f"k{k}_ms"] = e0.elapsed_time(e1) / 10
    nnz = op.lor_csr()[1].numel()
    step_ms = (out["k16_ms"] - out["k1_ms"]) / 15
    step_bytes = 12 * nnz + 56 * mesh.n_dof
    print(json.dumps({"probe": "lor_chebyshev", "mesh": f"{N}^3", "p": p, "n_dof": mesh.n_dof, "nnz": nnz, **out,
                      "step_ms": step_ms, "step_bytes": step_bytes, "step_gbs": step_bytes / step_ms / 1e6}),
          flush=True)


def run_sweep(hx, torch, args, peaks):
    """p = 2..8 on the FP64 sweep meshes (stored factors): per order the FP64 apply (GDoF/s, fraction
    of the derived and of the probed FP64 peak), the FP32 apply (fraction of the measured HBM
    bandwidth), the on-the-fly FP64 apply on the same mesh, the FP64 step (set-up + Jacobi-PCG to
    1e-10) and the mixed-precision step (set-up + FP64 refinement around FP32 PCG to 1e-10) with its
    refinements and its relative difference from the FP64 solution.  Applies: 10 timed after 3
    warm-up; steps: args.sweep_reps timed after one warm-up; CUDA events on the current stream."""
    out = {}
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(reps):
            r = fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps, r

    for p in range(2, 9):
        N = SWEEP_N[p]
        q = p + 2
        mesh, op, b = make_problem(hx, torch, p, N, "stored")
        E, n_dof = mesh.n_elem, mesh.n_dof
        t_app = time_applies(op, torch, b, reps=10)[1]
        flops = alg_flops_per_element(p, q) * E
        t32 = time_applies_f32(op, torch, b.float(), reps=10)
        bytes32 = 8 * n_dof + 4 * (p + 1) ** 3 * E + 7 * 4 * q ** 3 * E
        x = torch.zeros_like(b)
        t_fp64, info = timed(lambda: run_step(op, b, x), args.sweep_reps)
        xm = torch.empty_like(b)

        def mixed_step():
            op.set_coefficients(ALPHA, NU)
            return hx.hx_solve_pcg_mixed(op.handle, b, xm, RTOL, 100000, args.inner_rtol)

        t_mix, infom = timed(mixed_step, args.sweep_reps)
        diff = float(torch.linalg.norm(xm - x) / torch.linalg.norm(x))
        kind, block_elems, tune_ms = op.f32_kernel()
        del op, x, xm
        torch.cuda.empty_cache()
        otf = hx.Operator(mesh, ALPHA, NU, geom_mode=hx.HX_GEOM_ONTHEFLY)
        t_otf = time_applies(otf, torch, b, reps=10)[1]
        del otf
        out[str(p)] = {
            "mesh": f"{N}^3", "q": q, "n_dof": n_dof,
            "apply_ms": 1e3 * t_app, "apply_gdofs": n_dof / t_app / 1e9,
            "apply_fp64_frac": flops / t_app / 1e12 / FP64_PEAK_TFLOPS,
            "apply_fp64_frac_of_probe": flops / t_app / 1e12 / peaks["fp64_tflops"],
            "apply_f32_ms": 1e3 * t32, "apply_f32_gdofs": n_dof / t32 / 1e9,
            "apply_f32_hbm_frac": bytes32 / t32 / 1e9 / HBM_GBS,
            "f32_kernel": F32_KERNELS.get(kind, kind), "f32_block_elems": block_elems,
            "f32_autotune_ms": {F32_KERNELS[k]: v for k, v in enumerate(tune_ms) if v >= 0},
            "apply_onthefly_gdofs": n_dof / t_otf / 1e9, "onthefly_vs_stored": t_app / t_otf,
            "fp64_step_s": t_fp64, "fp64_iterations": info["iterations"],
            "fp64_true_rel_residual": info["true_rel_residual"],
            "fp64_step_gdofs": n_dof * (info["iterations"] + 1) / t_fp64 / 1e9,
            "mixed_step_s": t_mix, "mixed_speedup": t_fp64 / t_mix, "mixed_refinements": infom["refinements"],
            "mixed_inner_iterations": infom["iterations"], "mixed_rel_residual": infom["rel_residual"],
            "mixed_rel_diff_vs_fp64": diff,
        }
        del mesh, b
        torch.cuda.empty_cache()
    out["timing"] = (f"applies: 10 timed after 3 warm-up; steps (set-up + solve to 1e-10): {args.sweep_reps} "
                     "timed after 1 warm-up; CUDA events")
    return out


def run_peaks(args):
    import torch
    import paper_1910_03032_b300 as hx
    print(json.dumps({"probe": "fma_rates", **measure_peaks(hx, torch)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hx", choices=["hx", "reference"])
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--n", type=int, default=96)
    ap.add_argument("--geom", default="stored", choices=["stored", "onthefly"])
    ap.add_argument("--no-sweep", action="store_true", help="skip the per-order sweep (p = 2..8)")
    ap.add_argument("--sweep-reps", type=int, default=3)
    ap.add_argument("--peaks", action="store_true", help="run the FP64 / FP32 FMA-rate probe alone and exit")
    ap.add_argument("--batch", action="store_true", help="add the batched-solve measurement (64 instances; projection-step set)")
    ap.add_argument("--precond", action="store_true", help="add the preconditioner comparison (Jacobi vs LOR)")
    ap.add_argument("--vcycle", action="store_true",
                    help="time one LOR multigrid V-cycle against one apply (pure-Neumann Poisson, --p, --n) and exit")
    ap.add_argument("--cheb", action="store_true",
                    help="time the LOR-Chebyshev preconditioner at degrees 1 and 16 (pure-Neumann Poisson, --p, --n) and exit")
    ap.add_argument("--grad", action="store_true", help="add the adjoint-gradient measurement (32^3, p = 4)")
    ap.add_argument("--batch-reps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--inner-rtol", type=float, default=1e-5)
    ap.add_argument("--f32-kernel", type=int, default=-1,
                    help="FP32 element kernel of the mixed-precision measurement: -1 autotuned (default), "
                         "0 collocated, 1 direct staged, 2 direct, 3 tensor-core BF16, 4 tensor-core BF16x3")
    ap.add_argument("--cpu-elems", type=int, default=14)
    ap.add_argument("--ref-elems", type=int, default=6)
    ap.add_argument("--ref-iterations", type=int, default=100)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.vcycle:
        run_vcycle(args)
        return
    if args.peaks:
        run_peaks(args)
        return
    if args.cheb:
        run_cheb(args)
        return
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_hx(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
