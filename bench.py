#!/usr/bin/env python
"""Benchmark of the method's hot path on one GB300 (or N replicas under torchrun).

One step = one pass of the whole path on one geometry with inputs resident in
HBM: plan creation (stereographic projection and per-node precompute, Morton
quadtree and interaction lists, the multiplier-potential lists and the inverse
Schur complement of the border), the left-preconditioned GMRES solve to a 1e-10
relative residual (by default with FP32-FMM inner solves and FP64 iterative
refinement of the residual; --precision fp64 applies the FP64 FMM in every
iteration), and the evaluation of u at off-curve targets.  The headline value is the operator throughput inside the
solve: N x (operator applications, both precisions) / step time, in Mpts/s.

Workload (default): 1024 star-cap islands x 1024 nodes (N = 1,048,576), seed 3,
Green's-function pair data with sources in islands 0 and 1, 256 targets.

--impl reference times the oracle (plain FP64 C, host cores) on a bounded
sample of rows of the same operator, in the same unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM matvec Mpts/s and GMRES solve time at 1e-10 rel err; fraction of FP64 peak"
FP64_PEAK_TFLOPS = 1.25   # nominal dense FP64 of one GB300 (recipe table)
FP32_PEAK_TFLOPS = 80.6   # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
DF64_FLOPS_PER_FLOP = 9.5  # float flops per double-float flop (fma 18/2, mul 10, add 11)
WORKLOADS = {
    "C3-256": dict(M=256, nodes=1024),
    "C3-1024": dict(M=1024, nodes=1024),
    "C3-2048": dict(M=2048, nodes=1024),
    "C2": dict(M=16, nodes=512),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="C3-1024", choices=sorted(WORKLOADS) + ["C4"])
    ap.add_argument("--instances", type=int, default=512, help="C4: independent geometries")
    ap.add_argument("--loop-instances", type=int, default=48,
                    help="C4: instances timed in the plain FP64 loop (a bounded sample)")
    ap.add_argument("--workers", type=int, default=16, help="C4: scheduler threads/streams")
    ap.add_argument("--sweep", action="store_true",
                    help="C3 matvec sweep: one line per island count (K_ONLY operator)")
    ap.add_argument("--sweep-m", default="64,128,256,1024,2048,4096,8192,16384")
    ap.add_argument("--precision", default="fp32r", choices=["fp64", "fp32r"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--p", type=int, default=None)
    ap.add_argument("--p32", type=int, default=None)
    ap.add_argument("--leaf", type=int, default=None)
    ap.add_argument("--inner-tol", type=float, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--targets", type=int, default=256)
    return ap.parse_args()


def make_inputs(name):
    import numpy as np
    import workloads as wl

    w = WORKLOADS[name]
    if name.startswith("C3"):
        g = wl.star_caps(3, w["M"], w["nodes"])
    else:
        g = wl.config_geometry("C2")
    src, gam, _ = wl.pair_sources(g, 0, 1)
    return g, src, gam, np


def workload_config(name, g, T, tol, precision):
    w = WORKLOADS[name]
    return {"workload": f"{name}: {w['M']} star-cap islands x {w['nodes']} nodes "
                        f"(N={g.N}), Green's-pair data, GMRES(50) tol {tol:g}, {T} targets",
            "islands": g.M, "nodes": g.N, "targets": T, "precision": precision,
            "accurate_operator_arithmetic": "double-float FMM (pairs of floats), double elsewhere",
            "l2": f"working set larger than L2: the Krylov basis alone is 51 x {g.N + g.M} doubles "
                  f"({51 * (g.N + g.M) * 8 / 1e6:.0f} MB), streamed every iteration"}


# ---- clocks -------------------------------------------------------------------------

class Clocks:
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        except OSError:
            rows = []
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = max(mx, float(r[1]))
            except (ValueError, IndexError):
                continue
            for nme, v in zip(names, r[2:6]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nme)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- oracle baseline (host cores) -------------------------------------------------

def oracle_rate(g, np, rows=256, seed=11):
    """The oracle's direct matvec (entries computed on the fly, OpenMP rows) on a
    sample of rows; returns (Mpts/s of a full N-row matvec, seconds, threads, rows)."""
    import oracle

    oracle.build()
    sig = np.random.default_rng(seed).standard_normal(g.N)
    idx = np.sort(np.random.default_rng(seed + 1).choice(g.N, rows, replace=False))
    t0 = time.perf_counter()
    oracle.apply_rows(g, sig, idx, op=1)
    dt = time.perf_counter() - t0
    full = dt * g.N / rows
    return g.N / full / 1e6, dt, oracle.num_threads(), rows


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g, src, gam, np = make_inputs(args.workload)
    rows = 2048 if g.N > 100000 else 256
    for _ in range(args.warmup):
        oracle_rate(g, np, rows)
    vals, dts = [], []
    for _ in range(args.steps):
        v, dt, cores, rows = oracle_rate(g, np, rows)
        vals.append(v)
        dts.append(dt)
    val = statistics.median(vals)
    sample = f"{rows} rows of the N={g.N} density block (I+K), entries computed on the fly"
    line = {"metric": METRIC, "value": val, "unit": "Mpts/s", "impl": "reference", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(dts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args.workload, g, args.targets, args.tol, "fp64"),
            "cpu_baseline": {"value": val, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---- our arm ---------------------------------------------------------------------------

def src_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1306_0612_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def kernel_work(name, c, bc, P, P32, N):
    """(algorithmic work of one operator application, unit) per the FMM's
    operation counts: 11 flops per near pair, 8(p+1) per node for P2M and L2P and
    per (node, box) for M2P/P2L, 8(p+1)^2 per translation, 10 per node to combine.
    Multiplier potential: 8 flops per local-expansion term evaluated at a node
    (one expansion per node in double, one per ancestor level >= 2 in float),
    8 per (node, centre) pair summed directly (log counted as one flop, like the
    division of P2P), 10 per node to combine."""
    f32 = name.endswith("32")
    base = name[:-2] if f32 else name
    Q = P32 if f32 else P
    if base == "leaf":
        return 11 * c["p2p_pairs"] + 8 * Q * N + 8 * Q * c["w_pairs"] + 10 * N, "TFLOP/s"
    if base == "down":
        return 8 * Q * Q * (c["m2l"] + c["l2l"]) + 8 * Q * c["x_pairs"], "TFLOP/s"
    if base == "up":
        return 8 * Q * N + 8 * Q * Q * c["m2m"], "TFLOP/s"
    if base == "direct":
        return 11 * N * (N - 1), "TFLOP/s"
    if base == "esum" and bc:
        terms = 8 * bc["terms32"] * bc["walk_expansions"] if f32 else 8 * bc["terms"] * N
        return (terms + 8 * bc["direct_pairs"] + 8 * bc["global_centres"] * N + 10 * N,
                "TFLOP/s")
    return None, None


def measured_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def aggregate(ms, units, world, device):
    """Whole-job numbers of one timed region over the ranks: the slowest rank's time and
    the units every rank processed (each rank runs its own replica)."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1306_0612_gb300 import lbfmm as L
    import __graft_entry__

    __graft_entry__.build()
    g, src, gam, np = make_inputs(args.workload)
    import workloads as wl

    T = args.targets
    tg = wl.targets_off_islands(g, T, seed=17)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(dev)
    x, dx, d2x, cen, tgt = t(g.x), t(g.dx), t(g.d2x), t(g.centres), t(tg)
    srcd, gamd = t(src), t(gam)
    data = torch.empty(g.N, dtype=torch.float64, device=dev)
    L.lbf_green_sum(x, srcd, gamd, data)
    uex = torch.empty(T, dtype=torch.float64, device=dev)
    L.lbf_green_sum(tgt, srcd, gamd, uex)
    kw = dict(tol=args.tol)
    if args.precision == "fp32r":
        kw["precision"] = L.LBF_PRECISION_FP32_REFINE
    for k, v in (("p", args.p), ("p32", args.p32), ("leaf_size", args.leaf), ("inner_tol", args.inner_tol)):
        if v:
            kw[k] = v
    opt = L.lbf_default_options(**kw)
    sig = torch.empty(g.N, dtype=torch.float64, device=dev)
    a = torch.empty(g.M, dtype=torch.float64, device=dev)
    u = torch.empty(T, dtype=torch.float64, device=dev)
    holder = {}

    def step():
        plan = L.lbf_plan_create(g.island_ptr, x, dx, d2x, cen, opt=opt)
        rc, its, rr = L.lbf_gmres_solve(plan, data, sig, a)
        L.lbf_evaluate(plan, sig, a, tgt, u)
        holder["plan"] = plan
        return rc, its, rr, L.lbf_solve_stats(plan)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    L.lbf_profile_reset()
    L.lbf_profile_enable(True)
    n0 = L.lbf_launch_count()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = dict(arnoldi=0, fp64_applies=0, fp32_applies=0, refine_steps=0)
    rcs = []
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            rc, its, rr, st = step()
            rcs.append(rc)
            for k in tot:
                tot[k] += st[k]
        ev1.record(stream)
        torch.cuda.synchronize()
    L.lbf_profile_enable(False)
    launches = L.lbf_launch_count() - n0
    ms = ev0.elapsed_time(ev1)
    ms, units = aggregate(ms, float(g.N * (tot["fp64_applies"] + tot["fp32_applies"])), world, dev)
    clocks = clk.summary()
    plan = holder["plan"]
    info = plan.info()
    counts = L.lbf_plan_counts(plan)
    P, P32 = info["p"] + 1, opt.p32 + 1
    # per-kernel device time over the timed region (CUDA events on the launch stream)
    prof = {}
    for kid, name in enumerate(L.KERNEL_NAMES):
        n, tms = L.lbf_profile_read(kid)
        if n:
            prof[name] = {"launches": n, "ms": tms}
    L.lbf_profile_reset()
    dom = max((k for k in prof if not k.startswith("plan_")), key=lambda k: prof[k]["ms"])
    # applications that did work (launches queued past convergence return at once)
    n64, n32 = tot["fp64_applies"], tot["fp32_applies"]
    applies = (n64 + n32) / args.steps
    bcounts = L.lbf_border_counts(plan)
    work, unit = kernel_work(dom, counts, bcounts, P, P32, g.N)
    roofline = None
    if work is not None:
        n_app = n32 if dom.endswith("32") else n64
        rate = work * n_app / (prof[dom]["ms"] / 1e3)
        if unit == "GB/s":
            peak, src_p = measured_hbm()
            ach, bound = rate / 1e9, "hbm"
        else:
            f32 = dom.endswith("32")
            peak = FP32_PEAK_TFLOPS if f32 else FP64_PEAK_TFLOPS
            src_p = ("FP32 derived from unit counts and the 2.07 GHz clock" if f32 else
                     "nominal FP64 (recipe table; MEASURED_PEAKS.json has no FP64 entry)")
            if not f32 and dom in ("up", "down", "leaf") and opt.fmm64:
                src_p += ("; this kernel runs double-float arithmetic on the FP32 pipes, whose "
                          f"own ceiling is {FP32_PEAK_TFLOPS / DF64_FLOPS_PER_FLOP:.2f} TFLOP/s of "
                          "double flops (FP32 peak / 9.5 float flops per double flop)")
            ach, bound = rate / 1e12, "alu"
        traffic = None
        tp = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tp):
            tj = json.load(open(tp))
            if tj.get("src_hash") == src_hash() and dom in tj.get("kernels", {}):
                traffic = tj["kernels"][dom].get("bytes_per_launch")
        roofline = {"bound": bound, "kernel": dom, "achieved": ach, "peak": peak, "unit": unit,
                    "frac": ach / peak, "traffic": traffic, "peak_source": src_p}
    err = float((u - uex).abs().max() / uex.abs().max())
    # pure operator throughput of the FMM K-block apply in both precisions
    vin = torch.randn(g.N, dtype=torch.float64, device=dev,
                      generator=torch.Generator(device=dev).manual_seed(1))
    vout = torch.empty_like(vin)
    apply_ms = {}
    ops = [("fp64", L.LBF_OP_K_ONLY)]
    if args.precision == "fp32r":
        ops.append(("fp32", L.LBF_OP_K_ONLY | L.LBF_OP_FP32))
    ref64 = torch.empty_like(vin)
    L.lbf_apply(plan, L.LBF_OP_K_ONLY, vin, ref64)
    apply_err = {}
    for nm, op in ops:
        for _ in range(2):
            L.lbf_apply(plan, op, vin, vout)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            L.lbf_apply(plan, op, vin, vout)
        e1.record(stream)
        torch.cuda.synchronize()
        apply_ms[nm] = e0.elapsed_time(e1) / 5
        apply_err[nm] = float((vout - ref64).norm() / ref64.norm())
    value = units / (ms / 1e3) / 1e6

    # end to end through the public API, host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        pin = lambda a_: torch.from_numpy(np.ascontiguousarray(a_, dtype=np.float64).reshape(-1)).pin_memory()
        hx, hdx, hd2x, hc, ht = pin(g.x), pin(g.dx), pin(g.d2x), pin(g.centres), pin(tg)
        hg = data.cpu().pin_memory()
        hu = torch.empty(T, dtype=torch.float64).pin_memory()
        bi = 8 * (hx.numel() + hdx.numel() + hd2x.numel() + hc.numel() + ht.numel() + hg.numel())
        bo = 8 * T

        def e2e_step():
            dx_ = hx.to(dev, non_blocking=True)
            ddx = hdx.to(dev, non_blocking=True)
            dd2 = hd2x.to(dev, non_blocking=True)
            dc = hc.to(dev, non_blocking=True)
            dt_ = ht.to(dev, non_blocking=True)
            dg = hg.to(dev, non_blocking=True)
            pl = L.lbf_plan_create(g.island_ptr, dx_, ddx, dd2, dc, opt=opt)
            s_ = torch.empty(g.N, dtype=torch.float64, device=dev)
            a_ = torch.empty(g.M, dtype=torch.float64, device=dev)
            u_ = torch.empty(T, dtype=torch.float64, device=dev)
            L.lbf_gmres_solve(pl, dg, s_, a_)
            L.lbf_evaluate(pl, s_, a_, dt_, u_)
            hu.copy_(u_, non_blocking=True)
            st = L.lbf_solve_stats(pl)
            return st["fp64_applies"] + st["fp32_applies"]

        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ap_e = 0
        for _ in range(args.steps):
            ap_e += e2e_step()
        f1.record(stream)
        torch.cuda.synchronize()
        ems, units_e = aggregate(f0.elapsed_time(f1), float(g.N * ap_e), world, dev)
        e2e = {"value": units_e / (ems / 1e3) / 1e6, "unit": "Mpts/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": ems / args.steps}

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        v, dt, cores, rows = oracle_rate(g, np, 2048 if g.N > 100000 else 256)
        cpu = {"value": v, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
               "sample": f"{rows} rows of the N={g.N} density block (I+K), {dt:.1f} s wall"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32+f64",
                "data": "synthetic",
                "config": workload_config(args.workload, g, T, args.tol, args.precision),
                "solve": {"status": rcs, "applies_per_step": applies,
                          "fp64_applies": n64 / args.steps, "fp32_applies": n32 / args.steps,
                          "refine_steps": tot["refine_steps"] / args.steps, "rel_residual": rr,
                          "solution_max_rel_err": err, "step_ms": ms / args.steps,
                          "apply_ms": apply_ms, "apply_rel_err_vs_fp64": apply_err,
                          "apply_mpts": {k: g.N / v / 1e3 for k, v in apply_ms.items()},
                          "tree": info, "counts": counts, "border_counts": bcounts},
                "kernels_ms": {k: round(v["ms"] / args.steps, 3) for k, v in prof.items()},
                "kernel_launches": {k: v["launches"] / args.steps for k, v in prof.items()},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """C4: independent geometries of uneven size (1-64 islands, 64-1024 nodes per
    island, log-uniform), 16 Green's-pair right-hand sides each, solved to 1e-10 and
    evaluated at off-curve targets.  Batched arm: the native scheduler (worker
    streams, FP32 FMM with FP64 refinement).  Baseline arm: the plain FP64 loop over
    instances on one stream (plan, 16 solves, evaluations), on a bounded sample."""
    import numpy as np
    import torch
    import workloads as wl
    from paper_1306_0612_gb300 import lbfmm as L
    import __graft_entry__

    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    T = 32
    inst = []
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(dev)
    for g, pairs in wl.batch_instances(seed=4, count=args.instances, nrhs=16):
        x = t(g.x)
        data = torch.empty((len(pairs), g.N), dtype=torch.float64, device=dev)
        tg = t(wl.targets_off_islands(g, T, seed=5))
        uex = torch.empty((len(pairs), T), dtype=torch.float64, device=dev)
        for k, (pp, gam) in enumerate(pairs):
            L.lbf_green_sum(x, t(pp), t(gam), data[k])
            L.lbf_green_sum(tg, t(pp), t(gam), uex[k])
        inst.append(dict(island_ptr=g.island_ptr, x=x, dx=t(g.dx), d2x=t(g.d2x),
                         centres=t(g.centres), g=data, targets=tg, uex=uex, N=g.N, M=g.M))
    torch.cuda.synchronize()
    nsolve = sum(i["g"].shape[0] for i in inst)
    nodes = sum(i["N"] for i in inst)

    def err(res, sub):
        e = []
        for ins, r in zip(sub, res):
            d = (r["u"] - ins["uex"]).abs().amax(dim=1) / ins["uex"].abs().amax(dim=1)
            e.extend(d.tolist())
        return float(np.max(e)), float(np.median(e))

    def batched(precision, sub):
        kw = dict(inner_tol=args.inner_tol) if args.inner_tol else {}
        opt = L.lbf_default_options(tol=args.tol, precision=precision, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = L.lbf_batch_run(sub, opt=opt, nworkers=args.workers)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = [r["status"] for r in res]
        return dt, res, st

    # warm-up on a few instances (library load, attributes, allocator)
    batched(L.LBF_PRECISION_FP32_REFINE, inst[:args.workers])
    dt32, res32, st32 = batched(L.LBF_PRECISION_FP32_REFINE, inst)
    e32 = err(res32, inst)
    dt64b, res64b, st64b = batched(L.LBF_PRECISION_FP64, inst)
    e64b = err(res64b, inst)
    # plain FP64 loop over instances, one stream, on a bounded sample
    sub = inst[:min(args.loop_instances, len(inst))]
    opt64 = L.lbf_default_options(tol=args.tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nloop = 0
    loop_err = []
    for ins in sub:
        plan = L.lbf_plan_create(ins["island_ptr"], ins["x"], ins["dx"], ins["d2x"], ins["centres"],
                                 opt=opt64)
        sig = torch.empty(ins["N"], dtype=torch.float64, device=dev)
        a = torch.empty(ins["M"], dtype=torch.float64, device=dev)
        u = torch.empty(T, dtype=torch.float64, device=dev)
        for k in range(ins["g"].shape[0]):
            L.lbf_gmres_solve(plan, ins["g"][k], sig, a)
            L.lbf_evaluate(plan, sig, a, ins["targets"], u)
            loop_err.append(float((u - ins["uex"][k]).abs().max() / ins["uex"][k].abs().max()))
            nloop += 1
        del plan
    torch.cuda.synchronize()
    dtl = time.perf_counter() - t0
    loop_rate = nloop / dtl
    line = {"metric": "batched uneven solves: solves per second (plan + GMRES to 1e-10 + evaluation)",
            "value": nsolve / dt32, "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic",
            "config": {"workload": f"C4: {len(inst)} star-cap geometries, 1-64 islands, 64-1024 nodes "
                                   f"per island (log-uniform), 16 Green's-pair right-hand sides each, "
                                   f"{T} targets", "instances": len(inst), "solves": nsolve,
                       "nodes": nodes, "workers": args.workers, "tol": args.tol},
            "batched_fp32r": {"wall_s": dt32, "solves_per_s": nsolve / dt32,
                              "statuses_ok": st32.count(0), "solution_err_max": e32[0],
                              "solution_err_median": e32[1],
                              "fp32_applies": sum(r["fp32_applies"] for r in res32),
                              "fp64_applies": sum(r["fp64_applies"] for r in res32)},
            "batched_fp64": {"wall_s": dt64b, "solves_per_s": nsolve / dt64b,
                             "statuses_ok": st64b.count(0), "solution_err_max": e64b[0],
                             "solution_err_median": e64b[1]},
            "loop_fp64": {"instances": len(sub), "solves": nloop, "wall_s": dtl,
                          "solves_per_s": loop_rate, "solution_err_max": float(np.max(loop_err)),
                          "note": "plain FP64 loop over instances on one stream, timed on the "
                                  "first instances of the same list"},
            "speedup_vs_loop_fp64": (nsolve / dt32) / loop_rate}
    print(json.dumps(line))
    return 0


def run_sweep(args):
    """C3 sweep: the density operator (I + 2K) sigma, sigma ~ N(0, 1), on 2^k islands x
    1024 nodes; FP64 and FP32 FMM applies (median of 5 after 3 warm-ups, CUDA events),
    per-kernel algorithmic rates, the FP32 error against FP64, and (N <= 262144) the FMM
    against the GPU's tiled direct sum, with the direct sum's own time."""
    import numpy as np
    import torch
    import workloads as wl
    from paper_1306_0612_gb300 import lbfmm as L
    import __graft_entry__

    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(dev)

    def timed(plan, op, vin, vout, reps=5):
        for _ in range(3):
            L.lbf_apply(plan, op, vin, vout)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.lbf_apply(plan, op, vin, vout)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for M in [int(v) for v in args.sweep_m.split(",")]:
        g = wl.star_caps(3, M, 1024)
        x, dx, d2x, cen = t(g.x), t(g.dx), t(g.d2x), t(g.centres)
        opt = L.lbf_default_options(border=0, precision=L.LBF_PRECISION_FP32_REFINE)
        plan = L.lbf_plan_create(g.island_ptr, x, dx, d2x, cen, opt=opt)
        vin = t(wl.random_density(g.N, seed=1))
        o64, o32 = torch.empty_like(vin), torch.empty_like(vin)
        ms64 = timed(plan, L.LBF_OP_K_ONLY, vin, o64)
        ms32 = timed(plan, L.LBF_OP_K_ONLY | L.LBF_OP_FP32, vin, o32)
        counts = L.lbf_plan_counts(plan)
        info = plan.info()
        P, P32 = info["p"] + 1, opt.p32 + 1
        L.lbf_profile_reset()
        L.lbf_profile_enable(True)
        L.lbf_apply(plan, L.LBF_OP_K_ONLY, vin, o64)
        L.lbf_apply(plan, L.LBF_OP_K_ONLY | L.LBF_OP_FP32, vin, o32)
        torch.cuda.synchronize()
        L.lbf_profile_enable(False)
        kern = {}
        for kid, name in enumerate(L.KERNEL_NAMES):
            n, tms = L.lbf_profile_read(kid)
            if n and name in ("up", "down", "leaf", "up32", "down32", "leaf32"):
                work, _ = kernel_work(name, counts, None, P, P32, g.N)
                peak = FP32_PEAK_TFLOPS if name.endswith("32") else FP64_PEAK_TFLOPS
                ach = work / (tms / 1e3) / 1e12
                kern[name] = {"ms": round(tms, 3), "tflops": ach, "frac": ach / peak}
        L.lbf_profile_reset()
        line = {"sweep": "C3", "islands": M, "N": g.N, "tree": info,
                "fp64": {"apply_ms": ms64, "mpts": g.N / ms64 / 1e3},
                "fp32": {"apply_ms": ms32, "mpts": g.N / ms32 / 1e3,
                         "rel_l2_vs_fp64": float((o32 - o64).norm() / o64.norm())},
                "kernels": kern}
        if g.N <= 262144:
            od = torch.empty_like(vin)
            pd = L.lbf_plan_create(g.island_ptr, x, dx, d2x, cen,
                                   opt=L.lbf_default_options(border=0, matvec=L.LBF_MATVEC_DIRECT))
            msd = timed(pd, L.LBF_OP_K_ONLY, vin, od, reps=3)
            line["direct"] = {"apply_ms": msd, "mpts": g.N / msd / 1e3,
                              "pairs_per_s": g.N * (g.N - 1) / (msd / 1e3)}
            line["fp64"]["rel_l2_vs_direct"] = float((o64 - od).norm() / od.norm())
            line["fp32"]["rel_l2_vs_direct"] = float((o32 - od).norm() / od.norm())
            del pd
        print(json.dumps(line), flush=True)
        del plan
        torch.cuda.empty_cache()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.workload == "C4":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
