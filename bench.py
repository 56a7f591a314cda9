"""Benchmark of the SIP Helmholtz apply on one GB300 (or N replicas).

Default workload: the 64x64 quad mesh of [0,1]^2 with interior vertices
jittered by +-0.15h (seed 1) and element orders i.i.d. in {2..6}, lambda = 1,
tau_F = 2 (max(P-,P+)+1)^2 / h_F; x ~ N(0,1) per DOF (seed 0).

One step = one FP64 apply y = A x (trace kernel + main kernel) on inputs
already resident in HBM; the L2 cache is flushed (a 256 MiB write) before every
timed step, outside the timed events.  value = DOFs / second summed over
ranks (GDoF/s).  The JSON line also carries the FP32 apply, the CG solves to a
1e-10 relative residual (FP64 CG and FP32-apply CG in FP64 refinement) on this
workload and on the 32^3 hex workload (the precision comparison), the
rooflines of the main kernels against peaks measured on this GPU, the
end-to-end number through the public API with host buffers, clocks sampled
during the timed region and the oracle's throughput on all host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]
                  [--faces shared|p2p] [--rule gauss|gll] [--force-interp]
                  [--tiling FILE | --save-tiling FILE] [--no-cg] [--no-cpu] [--no-precision-config]
  python bench.py --sweep orders|dofs|traces   (hex throughput sweeps, one JSON line per mesh)

The batched 24^3 workload applies to (and solves for) its 32 right-hand sides in
one call; its GDoF/s count every right-hand side's DOFs.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sip_inputs as si  # noqa: E402

WORKLOAD = "c2_2d_64x64_jitter_p2to6"
PRECISION_WORKLOAD = "c3_3d_32cube_p4"
METRIC = "SIP apply GDoF/s (FP64 vs FP32-refined) and CG time to 1e-10 residual"

# right-hand sides per apply: the batched 24^3 workload applies to a batch of 32
# N(0,1) vectors (seed 4) in one launch pair; the others to one vector (seed 0)
NRHS = {"c4_3d_24cube_jitter_p2to7": 32}

# DRAM bytes (read + write) per launch of the FP64 main kernel, from one ncu
# capture of that workload with the current kernels and the schedule the
# autotuner picks for it (shared-rule faces, Gauss points); workloads without
# such a capture report null
NCU_MAIN_TRAFFIC: dict[str, float] = {"c2_2d_64x64_jitter_p2to6": 11170048.0,
                                        "c3_3d_32cube_p4": 186371584.0 + 24141312.0}


def peaks():
    p = {"hbm_gbs": 6800.0, "src": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        p["hbm_gbs"] = float(d.get("hbm_gbs", 6800.0))
        p["src"] = "measured"
    return p


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t_local: float, world: int, device=None) -> float:
    """Step time of the slowest rank (the job's time); plain value when world == 1."""
    if world <= 1:
        return float(t_local)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(units_per_rank: int, world: int, t_max: float) -> float:
    """Whole-job units per second: every rank processes its own replica of the
    workload (weak scaling), the job takes the slowest rank's time."""
    return world * units_per_rank / t_max


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"sip_clocks_{os.getpid()}_{id(self)}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle baseline on the host cores
# The oracle as it stands (one process per host core, each building rows of A for
# its share of the elements from the local blocks and applying them to x), on a
# bounded sample of the workload; rate = DOF-columns of all workers / wall time.

_ORC = {}


def _oracle_worker_init(mesh, nrhs):
    from oracle import SipOracle
    orc = SipOracle(mesh, lam=mesh.lam)
    x = si.random_vector(orc.ndof, 0) if nrhs == 1 else si.random_rhs_batch(nrhs, orc.ndof, 4).T.copy()
    _ORC["orc"], _ORC["x"], _ORC["nrhs"] = orc, x, nrhs


def _oracle_worker_run(elems, budget_s):
    orc, x, nrhs = _ORC["orc"], _ORC["x"], _ORC["nrhs"]
    t0 = time.perf_counter()
    done, nel = 0, 0
    for i in range(0, len(elems), 4):
        R = orc.rows_for_elements(elems[i:i + 4])
        _ = R @ x
        done += R.shape[0] * nrhs
        nel += len(elems[i:i + 4])
        if time.perf_counter() - t0 > budget_s:
            break
    return done, nel, time.perf_counter() - t0


class OraclePool:
    """One spawned worker process per host core (spawned, so that it is safe
    after CUDA has been initialised), each holding the oracle of the workload."""

    def __init__(self, mesh, nrhs, workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.workers = workers or len(os.sched_getaffinity(0))
        self.mesh, self.nrhs = mesh, nrhs
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"          # one thread per worker process: the pool supplies the parallelism
        try:
            self.ex = cf.ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"),
                                             initializer=_oracle_worker_init, initargs=(mesh, nrhs))
            list(self.ex.map(_oracle_worker_run, [[0]] * self.workers, [0.0] * self.workers))  # warm the workers
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, budget_s, seed):
        """One bounded run: every worker takes its share of a random element
        order and works for about budget_s.  Returns (DOF-columns/s, DOF-columns,
        elements, wall seconds)."""
        order = np.random.default_rng(seed).permutation(self.mesh.n_elem).tolist()
        shares = [order[w::self.workers] for w in range(self.workers)]
        t0 = time.perf_counter()
        res = list(self.ex.map(_oracle_worker_run, shares, [budget_s] * self.workers))
        wall = time.perf_counter() - t0
        done = sum(r[0] for r in res)
        return done / wall, done, sum(r[1] for r in res), wall

    def close(self):
        self.ex.shutdown()


def oracle_baseline(mesh, nrhs, runs=5, budget_s=3.0):
    """Median of `runs` bounded runs of the oracle on all host cores."""
    pool = OraclePool(mesh, nrhs)
    try:
        rs = [pool.run(budget_s, seed=k) for k in range(runs)]
    finally:
        pool.close()
    med = sorted(rs, key=lambda r: r[0])[len(rs) // 2]
    return {"value": med[0] / 1e9, "unit": "GDoF/s", "cores": pool.workers, "kind": "oracle",
            "sample": f"median of {runs} runs; each: {pool.workers} worker processes (one per host core) build "
                      f"rows of A from local blocks for their share of a random element order and apply them, "
                      f"about {budget_s:.0f} s; median run {med[2]} of {mesh.n_elem} elements, "
                      f"{med[1]} DOF-columns ({nrhs} right-hand side(s)) in {med[3]:.1f} s"}


def run_reference(args):
    """The reference arm: the oracle as it stands, on all host cores (one
    worker process per core), each step a bounded run on the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    mesh = si.workload(args.workload)
    nrhs = NRHS.get(args.workload, 1)
    budget = max(1.0, min(6.0, 90.0 / max(1, args.steps + args.warmup)))
    pool = OraclePool(mesh, nrhs)
    try:
        rates = []
        for k in range(args.warmup + args.steps):
            r = pool.run(budget, seed=k)
            if k >= args.warmup:
                rates.append(r)
    finally:
        pool.close()
    val = statistics.median(r[0] for r in rates) / 1e9
    med = sorted(rates, key=lambda r: r[0])[len(rates) // 2]
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GDoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(r[3] for r in rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "nrhs": nrhs, "precision": "fp64", "l2": "n/a (host)"},
        "cpu_baseline": {"value": val, "unit": "GDoF/s", "cores": pool.workers, "kind": "oracle",
                         "sample": f"per step: {pool.workers} worker processes (one per host core) build rows "
                                   f"of A from local blocks for their share of a random element order and "
                                   f"apply them for about {budget:.0f} s (median step: {med[2]} elements, "
                                   f"{med[1]} DOF-columns)"},
        "e2e": {"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _handle_options(g, args):
    kw = {}
    if args.faces == "p2p":
        kw["face_scheme"] = g.SIP_FACES_P2P
    if args.rule == "gll":
        kw["quad_rule"] = g.SIP_RULE_GLL
    if args.force_interp:
        kw["force_interp"] = 1
    return g.options(**kw) if kw else None


def timed_cg(g, op, bvec, nrhs, rtol=1e-10):
    """FP64 CG and FP32-apply CG in FP64 refinement to rtol: wall time of the
    second of two identical solves (the first captures the CUDA graphs; a
    32-column batch stops its first solve early, one batched solve being long)."""
    import torch
    warm_rtol = rtol if nrhs == 1 else 1e-4
    res = {}
    for name, mode in (("fp64", g.SIP_CG_FP64), ("fp32_refined", g.SIP_CG_FP32_REFINED)):
        op.cg_solve(bvec, mode=mode, rtol=warm_rtol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = op.cg_solve(bvec, mode=mode, rtol=rtol)
        torch.cuda.synchronize()
        res[name] = {"seconds": time.perf_counter() - t0, "nrhs": nrhs, "iterations": st["iterations"],
                     "refinements": st["refinements"], "rel_residual": st["rel_residual"]}
    res["speedup_fp32_refined"] = res["fp64"]["seconds"] / res["fp32_refined"]["seconds"]
    return res


def manufactured_rhs(op, mesh):
    """Load vector of the manufactured solution prod_k sin(pi x_k)."""
    import torch
    xq = op.quad_points()
    f = (mesh.lam + mesh.dim * np.pi ** 2) * torch.prod(torch.sin(np.pi * xq), dim=1)
    return op.iproduct(f.contiguous())


def run_gb300(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_2504_03573_gb300 as g

    mesh = si.workload(args.workload)
    p2p = args.faces == "p2p"
    op = g.SipOperator.from_mesh(mesh, opts=_handle_options(g, args))
    n = op.ndof
    nrhs = NRHS.get(args.workload, 1)
    if p2p:
        args.no_cg = True   # CG needs the symmetric shared-rule operator
    # tile shapes chosen by the library's autotuner (set-up, outside the timed region)
    precs = {"fp64": g.SIP_FP64, "fp32": g.SIP_FP32}
    if args.tiling:
        # a schedule saved by an earlier run (--save-tiling), e.g. to profile exactly it
        saved = json.load(open(args.tiling))
        tiling = {k: op.set_tiling(precs[k], v["epb_by_order"], v["ctas_per_sm"], v["persistent"], v["threads"],
                                   v.get("cta_layout", 0))
                  for k, v in saved.items()}
    elif not args.no_tune:
        tiling = {k: op.autotune(p) for k, p in precs.items()}
    else:
        tiling = None
    if args.save_tiling:
        with open(args.save_tiling, "w") as f:
            json.dump({k: op.tiling(p) for k, p in precs.items()}, f)
    xhost = si.random_vector(n, 0) if nrhs == 1 else si.random_rhs_batch(nrhs, n, 4)
    x = torch.tensor(xhost, device="cuda")
    y = torch.empty_like(x)
    x32 = x.float()
    y32 = torch.empty_like(x32)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed_applies(xin, yout, steps, warmup, kernel_times=False, label="timed"):
        for _ in range(warmup):
            op.apply(xin, out=yout)
        op.set_timing(kernel_times)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        kt = []
        barrier()
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push(label)   # lets ncu --nvtx-include select the timed launches
        if not kernel_times:
            # a head start for the host: the GPU spins ~0.1 ms per step before the
            # first step, while the host queues every step, so that no step's
            # events also time the host's launch latency
            torch.cuda._sleep(int(steps * 100e-6 * 2.1e9))
        for i in range(steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            op.apply(xin, out=yout)
            evs[i][1].record(stream)
            if kernel_times:
                kt.append(op.last_kernel_ms())
        torch.cuda.nvtx.range_pop()
        barrier()
        wall = time.perf_counter() - t0
        op.set_timing(False)
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, kt, wall

    # ---- arithmetic peaks of this GPU, measured by the library (FMA chains on every SM)
    with ClockSampler(local) as clk_peak:
        fp64_peak = g.fp_peak(g.SIP_FP64, 1 << 14)
        fp32_peak = g.fp_peak(g.SIP_FP32, 1 << 18)
    clocks_peak = clk_peak.summary()

    # ---- headline: FP64 apply (the two kernels back to back, as the solver runs them)
    with ClockSampler(local) as clk:
        ms, _, wall = timed_applies(x, y, args.steps, args.warmup, label="timed_fp64")
    clocks = clk.summary()
    t_step = sum(ms) / len(ms) / 1e3
    t_max = max_over_ranks(t_step, world, device="cuda")
    value = job_throughput(nrhs * n, world, t_max) / 1e9
    # per-kernel times for the roofline: a second pass with events around each
    # kernel (which also keeps the next kernel from starting early)
    _, kt, _ = timed_applies(x, y, args.steps, 0, kernel_times=True, label="kernels_fp64")

    # ---- FP32 apply (same protocol)
    ms32, _, _ = timed_applies(x32, y32, args.steps, args.warmup, label="timed_fp32")
    t32 = sum(ms32) / len(ms32) / 1e3
    _, kt32, _ = timed_applies(x32, y32, args.steps, 0, kernel_times=True, label="kernels_fp32")

    # ---- rooflines of the dominant kernel (the main kernel)
    w64 = op.work_model(g.SIP_FP64)
    w32 = op.work_model(g.SIP_FP32)
    trace_ms = statistics.mean(a for a, _ in kt)
    main_ms = statistics.mean(b for _, b in kt)
    main32_ms = statistics.mean(b for _, b in kt32)
    trace32_ms = statistics.mean(a for a, _ in kt32)
    pk = peaks()
    ach = nrhs * w64["flops_main"] / (main_ms / 1e3) / 1e12
    apply_tf = nrhs * (w64["flops_main"] + w64["flops_trace"]) / t_step / 1e12
    bytes64 = nrhs * (w64["bytes_x"] + w64["bytes_y"]) + w64["bytes_geometry"]
    roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": ach / fp64_peak,
            "traffic": None if (p2p or args.rule != "gauss" or args.force_interp) else NCU_MAIN_TRAFFIC.get(args.workload),
            "kernel": f"k_main<double,{mesh.dim},{'true' if p2p else 'false'},{1 if args.rule == 'gll' else 0}>",
            "peak_src": "measured (sip_fp_peak: FP64 FMA chains on every SM, CUDA events), of measured",
            "kernel_ms": main_ms, "trace_kernel_ms": trace_ms,
            "whole_apply": {"achieved": apply_tf, "frac": apply_tf / fp64_peak,
                            "note": "trace + main flops of the work model / headline apply time"},
            "hbm_frac": bytes64 / t_step / (pk["hbm_gbs"] * 1e9)}
    ach32 = nrhs * w32["flops_main"] / (main32_ms / 1e3) / 1e12
    bytes32 = nrhs * (w32["bytes_x"] + w32["bytes_y"]) + w32["bytes_geometry"]
    roof32 = {"bound": "hbm" if mesh.n_elem and nrhs == 1 and args.workload in ("c2_2d_64x64_jitter_p2to6",)
              else "alu",
              "hbm": {"achieved": bytes32 / t32 / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                      "frac": bytes32 / t32 / (pk["hbm_gbs"] * 1e9),
                      "bytes": bytes32, "note": "x, y and volume / face geometry per apply / apply time"},
              "alu": {"achieved": ach32, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach32 / fp32_peak,
                      "kernel": "main", "kernel_ms": main32_ms},
              "peak_src": "HBM: MEASURED_PEAKS.json; FP32: sip_fp_peak, of measured"}

    # ---- end to end through the C ABI with host buffers: sip_apply_host moves x in,
    # applies and moves y out (pinned buffers: the kernels read x and write y in place
    # over the host link), all inside the timed region
    xh = torch.tensor(xhost).pin_memory()
    yh = torch.empty(xh.shape, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        op.apply_host(xh, out=yh)
    barrier()
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        op.apply_host(xh, out=yh)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    barrier()
    e2e_val = world * nrhs * n / (statistics.mean(e2e_ms) / 1e3) / 1e9

    # ---- CG solves to 1e-10 (manufactured right-hand side, or the 32 N(0,1) columns)
    cg = None
    if not args.no_cg:
        bvec = manufactured_rhs(op, mesh) if nrhs == 1 else x
        cg = timed_cg(g, op, bvec, nrhs)
    del op
    torch.cuda.empty_cache()

    # ---- the precision comparison on the 32^3 hex workload: FP64 CG against
    # FP32-apply CG in FP64 refinement, both to a 1e-10 relative residual
    prec_cfg = None
    if rank == 0 and world == 1 and not args.no_precision_config and not p2p and args.workload != PRECISION_WORKLOAD:
        m3 = si.workload(PRECISION_WORKLOAD)
        op3 = g.SipOperator.from_mesh(m3, opts=_handle_options(g, args))
        for p in (g.SIP_FP64, g.SIP_FP32):
            op3.autotune(p, reps=3)
        prec_cfg = {"workload": PRECISION_WORKLOAD, "ndof": op3.ndof, **timed_cg(g, op3, manufactured_rhs(op3, m3), 1)}
        del op3
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_baseline(mesh, nrhs)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "ndof": n, "nrhs": nrhs, "n_elem": mesh.n_elem, "precision": "fp64",
                       "faces": args.faces, "rule": args.rule, "force_interp": bool(args.force_interp),
                       "l2": "flushed before every step (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "tiling": tiling},
            "fp32_apply": {"value": world * nrhs * n / t32 / 1e9, "unit": "GDoF/s", "ms_per_step": t32 * 1e3,
                           "main_kernel_ms": main32_ms, "trace_kernel_ms": trace32_ms, "roofline": roof32},
            "cg": cg,
            "precision_config": prec_cfg,
            "roofline": roof,
            "peaks_measured": {"fp64_tflops": fp64_peak, "fp32_tflops": fp32_peak, "clocks": clocks_peak},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "GDoF/s", "h2d_bytes_per_step": 8 * nrhs * n,
                    "d2h_bytes_per_step": 8 * nrhs * n},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
            "wall_s_timed_region": wall,
            "hbm_peak_src": pk["src"],
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _time_apply(op, prec, steps, warmup, flush, g):
    """Median apply time (CUDA events, L2 flushed before every apply) and the
    per-kernel medians of a second pass with the library's events."""
    import torch
    stream = torch.cuda.current_stream()
    dt = torch.float64 if prec == g.SIP_FP64 else torch.float32
    x = torch.tensor(si.random_vector(op.ndof, 0), device="cuda", dtype=dt)
    y = torch.empty_like(x)
    for _ in range(warmup):
        op.apply(x, out=y)
    ms = []
    for i in range(steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        op.apply(x, out=y)
        b.record(stream)
        ms.append((a, b))
    torch.cuda.synchronize()
    t = statistics.median(a.elapsed_time(b) for a, b in ms) / 1e3
    op.set_timing(True)
    kt = []
    for i in range(steps):
        flush.fill_(float(i))
        op.apply(x, out=y)
        kt.append(op.last_kernel_ms())
    op.set_timing(False)
    return t, statistics.median(m for _, m in kt), statistics.median(tr for tr, _ in kt)


def run_sweep(args):
    """Throughput sweeps shaped like the paper's CPU measurements (Sec. 5.2),
    on uniform hex meshes of [0,1]^3 (affine elements, one order each), one JSON
    line per mesh:

    orders: P = 1..10 at about 1.1e7 DOFs each (the paper's sub-operator study
            uses 1.1e7 DOFs per order), FP64 and FP32;
    dofs:   P = 4 from about 1e4 to 1e8 DOFs (the paper's size sweep), FP64 and FP32;
    traces: the trace schemes on the same mesh (Sec. 5.2's forced-interpolation
            comparison): Gauss points (traces evaluated from the element),
            Gauss-Lobatto points (traces gathered, fluxes scattered), and each
            with interpolation forced on every face; P = 2, 4, 6 at about 4e6
            DOFs and the 64x64 jittered quads, FP64 and FP32."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_03573_gb300 as g
    fp64_peak = g.fp_peak(g.SIP_FP64, 1 << 14)
    fp32_peak = g.fp_peak(g.SIP_FP32, 1 << 18)
    gauss = dict()
    variants = {"gauss": gauss}
    if args.sweep == "orders":
        cases = [(p, max(2, round(1.1e7 ** (1 / 3) / (p + 1)))) for p in range(1, 11)]
    elif args.sweep == "dofs":
        cases = [(4, n) for n in (4, 8, 16, 24, 32, 48, 64, 90)]
    else:
        cases = [(p, round(4e6 ** (1 / 3) / (p + 1))) for p in (2, 4, 6)] + [("c2", None)]
        variants = {"gauss": gauss, "gauss_forced": dict(force_interp=1),
                    "gll_gather": dict(quad_rule=g.SIP_RULE_GLL),
                    "gll_forced": dict(quad_rule=g.SIP_RULE_GLL, force_interp=1)}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for p, n in cases:
        mesh = si.workload(WORKLOAD) if p == "c2" else si.structured_mesh(3, n, order=p)
        line = {"sweep": args.sweep, "order": p, "n": n, "n_elem": mesh.n_elem,
                "unit": "GDoF/s", "l2": "flushed before every step (256 MiB write)",
                "peaks_measured_tflops": {"fp64": fp64_peak, "fp32": fp32_peak}}
        for vname, kw in variants.items():
            op = g.SipOperator.from_mesh(mesh, opts=g.options(**kw) if kw else None)
            line["ndof"] = op.ndof
            res = {}
            for name, prec, peak in (("fp64", g.SIP_FP64, fp64_peak), ("fp32", g.SIP_FP32, fp32_peak)):
                op.autotune(prec, reps=3)
                t, main_ms, trace_ms = _time_apply(op, prec, args.steps, args.warmup, flush, g)
                w = op.work_model(prec)
                res[name] = {"value": op.ndof / t / 1e9, "ms_per_apply": t * 1e3, "main_kernel_ms": main_ms,
                             "trace_kernel_ms": trace_ms,
                             "main_tflops": w["flops_main"] / (main_ms / 1e3) / 1e12,
                             "apply_tflops": (w["flops_main"] + w["flops_trace"]) / t / 1e12}
                res[name]["main_frac_of_peak"] = res[name]["main_tflops"] / peak
                res[name]["apply_frac_of_peak"] = res[name]["apply_tflops"] / peak
            if len(variants) == 1:
                line.update(res)
            else:
                line[vname] = res
            del op
            torch.cuda.empty_cache()
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=list(si.WORKLOADS))
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--tiling", default=None, help="install the schedule saved by --save-tiling instead of tuning")
    ap.add_argument("--save-tiling", default=None, help="write the schedule in use to this JSON file")
    ap.add_argument("--no-precision-config", action="store_true",
                    help="skip the FP64 vs FP32-refined CG comparison on the 32^3 hex workload")
    ap.add_argument("--rule", default="gauss", choices=["gauss", "gll"],
                    help="volume and face points: Gauss-Legendre (traces evaluated from the element) or "
                         "Gauss-Lobatto-Legendre (traces gathered, fluxes scattered)")
    ap.add_argument("--force-interp", action="store_true",
                    help="interpolate to the shared rule on every face, also conforming ones")
    ap.add_argument("--faces", default="shared", choices=["shared", "p2p"],
                    help="interior-face flux: one shared rule per face (the method) or point-to-point "
                         "interpolation between the two sides' own rules (the comparison variant)")
    ap.add_argument("--sweep", default=None, choices=["orders", "dofs", "traces"],
                    help="throughput sweep on uniform hex meshes instead of the benchmark line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.sweep:
        return run_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
