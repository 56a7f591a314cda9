"""Benchmark of the SIP Helmholtz apply on one GB300 (or N replicas).

Default workload: the 64x64 quad mesh of [0,1]^2 with interior vertices
jittered by +-0.15h (seed 1) and element orders i.i.d. in {2..6}, lambda = 1,
tau_F = 2 (max(P-,P+)+1)^2 / h_F; x ~ N(0,1) per DOF (seed 0).

One step = one FP64 apply y = A x (trace kernel + main kernel) on inputs
already resident in HBM; the L2 cache is flushed (a 256 MiB write) before every
timed step, outside the timed events.  value = DOFs / second summed over
ranks (GDoF/s).  The JSON line also carries the FP32 apply, the CG solves to a
1e-10 relative residual (FP64 CG and FP32-apply CG in FP64 refinement), the
roofline of the dominant kernel, the end-to-end number through the public API
with host buffers, clocks sampled during the timed region and the oracle's
throughput on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]
                  [--faces shared|p2p] [--tiling FILE | --save-tiling FILE] [--no-cg] [--no-cpu]
  python bench.py --sweep orders|dofs      (hex throughput sweeps, one JSON line per mesh)

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
METRIC = "SIP apply GDoF/s (FP64 vs FP32-refined) and CG time to 1e-10 residual"

# FP64 arithmetic peak of one GB300: 1.25 TFLOP/s dense (vendor figure; the FP64
# units of this part are a small fraction of B200's).  FP32: 152 SMs x 128 lanes
# x 2 flop x 2.07 GHz = 80.5 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# right-hand sides per apply: the batched 24^3 workload applies to a batch of 32
# N(0,1) vectors (seed 4) in one launch pair; the others to one vector (seed 0)
NRHS = {"c4_3d_24cube_jitter_p2to7": 32}

# DRAM bytes (read + write) per launch of the FP64 main kernel, from one ncu capture
# of that workload with the current kernels (profiles/apply_<workload>.md)
NCU_MAIN_TRAFFIC = {"c2_2d_64x64_jitter_p2to6": 10.929664e6, "c3_3d_32cube_p4": 183.096576e6 + 22.797568e6}


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
        self.path = os.path.join("/tmp", f"sip_clocks_{os.getpid()}.csv")

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


def oracle_apply_rate(mesh, budget_s=12.0, seed=0, nrhs=1):
    """The oracle as it stands on a bounded sample: rows of A for a prefix of a
    shuffled element list, built from the local blocks and applied to x (nrhs
    columns), until the time budget is spent.  Returns (DOF/s counted per
    right-hand side, dofs done, elements, seconds, cores)."""
    from oracle import SipOracle
    orc = SipOracle(mesh, lam=mesh.lam)
    x = si.random_vector(orc.ndof, 0) if nrhs == 1 else si.random_rhs_batch(nrhs, orc.ndof, 4).T.copy()
    order = np.random.default_rng(seed).permutation(mesh.n_elem)
    t0 = time.perf_counter()
    c0 = time.process_time()
    done, nel = 0, 0
    for i in range(0, mesh.n_elem, 8):
        els = order[i:i + 8]
        R = orc.rows_for_elements(els)
        _ = R @ x
        done += R.shape[0] * nrhs
        nel += len(els)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = (time.process_time() - c0) / dt     # threads actually busy, on average
    return done / dt, done, nel, dt, cores


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    mesh = si.workload(args.workload)
    nrhs = NRHS.get(args.workload, 1)
    budget = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    rates = []
    for k in range(args.warmup + args.steps):
        r, done, nel, dt, cores = oracle_apply_rate(mesh, budget_s=budget, seed=k, nrhs=nrhs)
        if k >= args.warmup:
            rates.append((r, done, nel, dt, cores))
    val = statistics.median(r[0] for r in rates) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GDoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(r[3] for r in rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "nrhs": nrhs, "precision": "fp64", "l2": "n/a (host)"},
        "cpu_baseline": {"value": val, "unit": "GDoF/s", "cores": round(max(r[4] for r in rates), 2),
                         "kind": "oracle",
                         "sample": f"rows of {rates[0][2]} elements ({rates[0][1]} DOF-columns) per step, "
                                   f"{budget:.0f} s budget; cores = CPU time / wall time"},
        "e2e": {"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


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
    op = g.SipOperator.from_mesh(mesh, opts=g.options(face_scheme=g.SIP_FACES_P2P) if p2p else None)
    n = op.ndof
    nrhs = NRHS.get(args.workload, 1)
    if p2p:
        args.no_cg = True   # CG needs the symmetric shared-rule operator
    # tile shapes chosen by the library's autotuner (set-up, outside the timed region)
    precs = {"fp64": g.SIP_FP64, "fp32": g.SIP_FP32}
    if args.tiling:
        # a schedule saved by an earlier run (--save-tiling), e.g. to profile exactly it
        saved = json.load(open(args.tiling))
        tiling = {k: op.set_tiling(precs[k], v["epb_by_order"], v["ctas_per_sm"], v["persistent"], v["threads"])
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

    # ---- roofline of the dominant kernel (the main kernel), FP64
    w64 = op.work_model(g.SIP_FP64)
    w32 = op.work_model(g.SIP_FP32)
    trace_ms = statistics.mean(a for a, _ in kt)
    main_ms = statistics.mean(b for _, b in kt)
    main32_ms = statistics.mean(b for _, b in kt32)
    trace32_ms = statistics.mean(a for a, _ in kt32)
    pk = peaks()
    ach = nrhs * w64["flops_main"] / (main_ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None if p2p else NCU_MAIN_TRAFFIC.get(args.workload),
            "kernel": f"k_main<double,{mesh.dim},{'true' if p2p else 'false'}>",
            "peak_src": "FP64 vendor figure 1.25 TFLOP/s (dense)",
            "kernel_ms": main_ms, "trace_kernel_ms": trace_ms,
            "hbm_frac": (nrhs * (w64["bytes_x"] + w64["bytes_y"] + w64["bytes_trace"]) + w64["bytes_geometry"])
            / ((main_ms + trace_ms) / 1e3) / (pk["hbm_gbs"] * 1e9)}
    ach32 = nrhs * w32["flops_main"] / (main32_ms / 1e3) / 1e12

    # ---- end to end through the C ABI with host buffers: sip_apply_host copies x
    # in, applies and copies y out, all inside the timed region
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

    # ---- CG solves to 1e-10 (manufactured right-hand side)
    cg = None
    if not args.no_cg:
        if nrhs == 1:
            # manufactured right-hand side of sin(pi x) sin(pi y) (sin(pi z))
            xq = op.quad_points()
            f = (mesh.lam + mesh.dim * np.pi ** 2) * torch.prod(torch.sin(np.pi * xq), dim=1)
            bvec = op.iproduct(f.contiguous())
        else:
            bvec = x   # the batch of N(0,1) right-hand sides
        # warm-up solve (graph capture); the 32-column batch stops it early, since
        # one full batched solve takes about a minute
        warm_rtol = 1e-10 if nrhs == 1 else 1e-4
        res = {}
        for name, mode in (("fp64", g.SIP_CG_FP64), ("fp32_refined", g.SIP_CG_FP32_REFINED)):
            op.cg_solve(bvec, mode=mode, rtol=warm_rtol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = op.cg_solve(bvec, mode=mode, rtol=1e-10)
            torch.cuda.synchronize()
            res[name] = {"seconds": time.perf_counter() - t0, "nrhs": nrhs, "iterations": st["iterations"],
                         "refinements": st["refinements"], "rel_residual": st["rel_residual"]}
        res["speedup_fp32_refined"] = res["fp64"]["seconds"] / res["fp32_refined"]["seconds"]
        cg = res

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        r, done, nel, dt, cores = oracle_apply_rate(mesh, budget_s=args.cpu_budget, nrhs=nrhs)
        cpu = {"value": r / 1e9, "unit": "GDoF/s", "cores": round(cores, 2), "kind": "oracle",
               "sample": f"rows of {nel} of {mesh.n_elem} elements ({done} DOF-columns, {nrhs} right-hand "
                         f"side(s)) built from local blocks and applied, {dt:.1f} s; cores = CPU time / wall time"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "ndof": n, "nrhs": nrhs, "n_elem": mesh.n_elem, "precision": "fp64",
                       "faces": args.faces,
                       "l2": "flushed before every step (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "tiling": tiling},
            "fp32_apply": {"value": world * nrhs * n / t32 / 1e9, "unit": "GDoF/s", "ms_per_step": t32 * 1e3,
                           "main_kernel_ms": main32_ms, "trace_kernel_ms": trace32_ms,
                           "main_tflops": ach32, "main_frac_of_fp32_peak": ach32 / FP32_PEAK_TFLOPS},
            "cg": cg,
            "roofline": roof,
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


def run_sweep(args):
    """Throughput sweeps shaped like the paper's CPU measurements (Sec. 5.2):
    uniform hex meshes of [0,1]^3 (affine elements, one order each), FP64 and
    FP32 applies, one JSON line per mesh.

    orders: P = 1..8 at about 1.1e7 DOFs each (the paper's sub-operator study
            uses 1.1e7 DOFs per order);
    dofs:   P = 4 from about 1e4 to 1e8 DOFs (the paper's size sweep)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_03573_gb300 as g
    if args.sweep == "orders":
        cases = [(p, max(2, round(1.1e7 ** (1 / 3) / (p + 1)))) for p in range(1, 9)]
    else:
        cases = [(4, n) for n in (4, 8, 16, 24, 32, 48, 64, 90)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for p, n in cases:
        mesh = si.structured_mesh(3, n, order=p)
        op = g.SipOperator.from_mesh(mesh)
        line = {"sweep": args.sweep, "order": p, "n": n, "n_elem": mesh.n_elem, "ndof": op.ndof,
                "unit": "GDoF/s", "l2": "flushed before every step (256 MiB write)"}
        for name, prec, dt in (("fp64", g.SIP_FP64, torch.float64), ("fp32", g.SIP_FP32, torch.float32)):
            op.autotune(prec, reps=3)
            x = torch.tensor(si.random_vector(op.ndof, 0), device="cuda", dtype=dt)
            y = torch.empty_like(x)
            for _ in range(args.warmup):
                op.apply(x, out=y)
            op.set_timing(True)
            ms, kt = [], []
            for i in range(args.steps):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                op.apply(x, out=y)
                b.record(stream)
                kt.append(op.last_kernel_ms())
                ms.append((a, b))
            torch.cuda.synchronize()
            op.set_timing(False)
            t = statistics.median(a.elapsed_time(b) for a, b in ms) / 1e3
            main_ms = statistics.median(m for _, m in kt)
            w = op.work_model(prec)
            line[name] = {"value": op.ndof / t / 1e9, "ms_per_apply": t * 1e3, "main_kernel_ms": main_ms,
                          "trace_kernel_ms": statistics.median(tr for tr, _ in kt),
                          "main_tflops": w["flops_main"] / (main_ms / 1e3) / 1e12}
        line["fp64"]["main_frac_of_fp64_peak"] = line["fp64"]["main_tflops"] / FP64_PEAK_TFLOPS
        line["fp32"]["main_frac_of_fp32_peak"] = line["fp32"]["main_tflops"] / FP32_PEAK_TFLOPS
        print(json.dumps(line), flush=True)
        del op
        torch.cuda.empty_cache()
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
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--faces", default="shared", choices=["shared", "p2p"],
                    help="interior-face flux: one shared rule per face (the method) or point-to-point "
                         "interpolation between the two sides' own rules (the comparison variant)")
    ap.add_argument("--sweep", default=None, choices=["orders", "dofs"],
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
