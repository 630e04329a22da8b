#!/usr/bin/env python
"""Benchmark of the method's hot path on one GB300 (or N replicas under torchrun).

One step = one pass of the whole path on one geometry, inputs resident in HBM: plan
creation (stereographic projection and per-node precompute, Morton quadtree and
interaction lists, the multiplier-potential lists, the Schur complement of the border
and its factorisation), the left-preconditioned GMRES(50) solve to a 1e-10 relative
residual, and the evaluation of u at 256 off-curve targets.

Default workload: 16,384 star-cap islands x 1024 nodes (N = 16,777,216, seed 3),
Green's-pair data with sources in islands 0 and 1, every operator application in native
double (--precision fp64).  value = N x operator applications per step / step time
(Mpts/s: the FP64 FMM matvec rate of the whole step, plan and evaluation included).
Extra keys: the pure matvec rate of each arithmetic, the same step with the
double-float operator and with FP32 inner solves under FP64 refinement (each with its
error against the exact solution and against the FP64 result), and the other
workloads: one island (solve latency), 16 islands (matvec and solve latency), the
gradient at 256 islands x 512 nodes, and batched uneven solves against the plain FP64
loop over instances.

--impl reference times the oracle (plain FP64 C, host cores) on a bounded sample of
rows of the same operator, in the same unit.
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
FP64_PEAK_TFLOPS = 1.25   # nominal dense FP64 of one GB300 (recipe table); no measured entry
FP32_PEAK_TFLOPS = 80.6   # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
DF64_FLOPS_PER_FLOP = 9.5  # float flops per double-float flop (fma 18/2, mul 10, add 11)
WORKLOADS = {
    "C3-16384": dict(M=16384, nodes=1024),
    "C3-4096": dict(M=4096, nodes=1024),
    "C3-1024": dict(M=1024, nodes=1024),
    "C3-256": dict(M=256, nodes=1024),
    "C2": dict(M=16, nodes=512),
}
DEFAULT_WORKLOAD = "C3-16384"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["C4"])
    ap.add_argument("--instances", type=int, default=512, help="C4: independent geometries")
    ap.add_argument("--workers", type=int, default=16, help="C4: scheduler threads/streams")
    ap.add_argument("--arms", default="all",
                    help="C4: comma list of fp32r, fp32r_seq, fp64, fp64_lockstep, loop (default all)")
    ap.add_argument("--sweep", action="store_true",
                    help="C3 matvec sweep: one line per island count (K_ONLY operator)")
    ap.add_argument("--sweep-m", default="64,128,256,1024,2048,4096,8192,16384")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "df64", "fp32r"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--p", type=int, default=None)
    ap.add_argument("--p32", type=int, default=None)
    ap.add_argument("--leaf", type=int, default=None)
    ap.add_argument("--inner-tol", type=float, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="steps of the end-to-end region (at most --steps)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the variant arithmetics and the other workloads")
    ap.add_argument("--targets", type=int, default=256)
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (p, leaf size and near-field tile at their defaults)")
    ap.add_argument("--tune-target", type=float, default=1e-10,
                    help="the autotuner's bound on the operator's rel-l2 error")
    ap.add_argument("--warps", type=int, default=None, help="near-field tile (warps per block)")
    ap.add_argument("--apply", action="store_true",
                    help="one density-operator application on the workload's plan, for kernel profiling")
    return ap.parse_args()


def precision_options(L, name):
    """Options of one arithmetic of the step."""
    if name == "fp64":
        return dict(fmm64=0)
    if name == "df64":
        return dict(fmm64=1)
    return dict(precision=L.LBF_PRECISION_FP32_REFINE, fmm64=0)


def make_geometry(name):
    import workloads as wl

    w = WORKLOADS[name]
    if name.startswith("C3"):
        g = wl.star_caps(3, w["M"], w["nodes"])
    else:
        g = wl.config_geometry("C2")
    src, gam, _ = wl.pair_sources(g, 0, 1)
    return g, src, gam


def workload_config(name, g, T, tol, precision):
    w = WORKLOADS[name]
    arith = {"fp64": "native double throughout",
             "df64": "double-float FMM (pairs of floats), double elsewhere",
             "fp32r": "float FMM in the inner solves, native double residuals (refinement)"}[precision]
    return {"workload": f"{name}: {w['M']} star-cap islands x {w['nodes']} nodes "
                        f"(N={g.N}), Green's-pair data, GMRES(50) tol {tol:g}, {T} targets",
            "islands": g.M, "nodes": g.N, "targets": T, "precision": precision,
            "operator_arithmetic": arith,
            "value": "N x operator applications per step / step time (plan, solve, "
                     "evaluation in the step)",
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

def oracle_rate(g, rows, seed=11):
    """The oracle's direct matvec (entries computed on the fly, OpenMP rows) on a
    sample of rows; returns (Mpts/s of a full N-row matvec, seconds, threads, rows)."""
    import numpy as np

    import oracle

    oracle.build()
    sig = np.random.default_rng(seed).standard_normal(g.N)
    idx = np.sort(np.random.default_rng(seed + 1).choice(g.N, rows, replace=False))
    t0 = time.perf_counter()
    oracle.apply_rows(g, sig, idx, op=1)
    dt = time.perf_counter() - t0
    full = dt * g.N / rows
    return g.N / full / 1e6, dt, oracle.num_threads(), rows


def reference_rows(g):
    # a bounded sample: about 2e9 kernel entries (a few seconds on the machine's cores)
    return max(16, min(g.N, int(2e9 // max(g.N, 1))))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = DEFAULT_WORKLOAD if args.workload == "C4" else args.workload
    g, _, _ = make_geometry(name)
    rows = reference_rows(g)
    for _ in range(args.warmup):
        oracle_rate(g, rows)
    vals, dts = [], []
    cores = None
    for _ in range(args.steps):
        v, dt, cores, rows = oracle_rate(g, rows)
        vals.append(v)
        dts.append(dt)
    val = statistics.median(vals)
    sample = f"{rows} rows of the N={g.N} density block (I+K), entries computed on the fly"
    line = {"metric": METRIC, "value": val, "unit": "Mpts/s", "impl": "reference", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(dts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(name, g, args.targets, args.tol, "fp64"),
            "cpu_baseline": {"value": val, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---- our arm ---------------------------------------------------------------------------

# the sources that decide the memory traffic of the FMM passes (up, down, leaf: their
# kernels, launch shapes, tree and lists); the DRAM bytes of profiles/traffic.json are
# keyed to them
# inner tolerance of the batched refinement: on 128 of the 512 geometries, 1e-5 needs two
# refinement rounds where 3e-4 (the library's default) needs three, with fewer float applies
# too (51,663 and 4,174 FP64 against 58,486 and 6,133): 1.41 s against 1.64 s; 1e-4 and 3e-5
# were slower (1.71, 1.91 s: more float applies, the same rounds).  (Not the library's default:
# on the 16,384-island step 1e-5 took five rounds and 67 float applies, 2.41 s, against four
# and 39, 1.72 s.)
C4_INNER_TOL = 1e-5

FMM_SOURCES = ("lbf_fmm_tpl.cuh", "lbf_fmm.cu", "lbf_tree.cu", "lbf_df64.cuh", "lbf_internal.cuh")


def src_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1306_0612_gb300", "csrc")
    for f in FMM_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def kernel_work(name, c, bc, P, P32, N):
    """(algorithmic work of one operator application, unit) per the FMM's
    operation counts, Q = p + 1 terms: 11 flops per near pair, 8Q per node for P2M and
    L2P and per (node, box) for M2P/P2L, 10 per node to combine; a translation in the
    binomial factorisation the kernels use: the real binomial matrix on the complex
    coefficients (4 flops an entry) between two diagonal complex scalings (6Q and 8Q),
    so 4Q^2 + 14Q for M2L and 2Q(Q+1) + 14Q for M2M and L2L, whose binomial matrix is
    triangular.  Multiplier potential: 8 flops per local-expansion term evaluated at a
    node (one expansion per node in double, one per ancestor level >= 2 in float), 8 per
    (node, centre) pair summed directly (log counted as one flop, like the division of
    P2P), 10 per node to combine."""
    f32 = name.endswith("32")
    base = name[:-2] if f32 else name
    Q = P32 if f32 else P
    m2l = 4 * Q * Q + 14 * Q
    tri = 2 * Q * (Q + 1) + 14 * Q
    if base == "leaf":
        return 11 * c["p2p_pairs"] + 8 * Q * N + 8 * Q * c["w_pairs"] + 10 * N, "TFLOP/s"
    if base == "down":
        return m2l * c["m2l"] + tri * c["l2l"] + 8 * Q * c["x_pairs"], "TFLOP/s"
    if base == "up":
        return 8 * Q * N + tri * c["m2m"], "TFLOP/s"
    if base == "direct":
        return 11 * N * (N - 1), "TFLOP/s"
    if base == "esum" and bc:
        if f32:
            terms = 8 * bc["terms32"] * bc["walk_expansions"]
        else:  # P2L per (box, centre) pair, L2L per box, L2P per node
            Pe = bc["terms"]
            terms = 8 * Pe * bc["p2l_pairs"] + (2 * Pe * (Pe + 1) + 14 * Pe) * c["l2l"] + 8 * Pe * N
        return (terms + 8 * bc["direct_pairs"] + 8 * bc["global_centres"] * N + 10 * N,
                "TFLOP/s")
    return None, None


def peak_fractions(line):
    """The FMM matvec's and the whole GMRES solve's algorithmic FP64 rate against the
    roofline's FP64 peak (native-double runs): the operator's work by kernel_work (upward,
    downward and leaf passes; the solve adds each preconditioned application's multiplier
    potential E y) over the measured apply and solve times.  The Arnoldi steps, the
    preconditioner's S^-1 and the vector work count as no work, so the solve's fraction is
    a lower bound.  None when the line lacks what it needs."""
    try:
        s, rf = line["solve"], line["roofline"]
        c, bc, N = s["counts"], s["border_counts"], s["counts"]["N"]
        P = s["tree"]["p"] + 1
        if rf.get("unit") != "TFLOP/s" or not line["matvec"].get("fp64"):
            return None
        w = {k: kernel_work(k, c, bc, P, 0, N)[0] for k in ("up", "down", "leaf", "esum")}
        k_apply = w["up"] + w["down"] + w["leaf"]
        mv_ms = line["matvec"]["fp64"]["ms"]
        work = s["fp64_applies"] * (k_apply + (w["esum"] or 0))
        peak = rf["peak"]

        def rate(flop, ms):
            a = flop / (ms * 1e-3) / 1e12
            return {"gflop": flop / 1e9, "ms": ms, "achieved": a, "frac": a / peak}

        return {"unit": "TFLOP/s", "peak": peak, "peak_source": rf.get("peak_source"),
                "matvec": rate(k_apply, mv_ms), "solve": rate(work, s["solve_ms"])}
    except (KeyError, TypeError, AttributeError, ZeroDivisionError):
        return None


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


class Step:
    """One pass of the path on device-resident inputs (plan, solve, evaluation)."""

    def __init__(self, L, g, inputs, opt):
        import torch

        self.L, self.g, self.inp, self.opt = L, g, inputs, opt
        dev = inputs["x"].device
        self.sig = torch.empty(g.N, dtype=torch.float64, device=dev)
        self.a = torch.empty(g.M, dtype=torch.float64, device=dev)
        self.u = torch.empty(inputs["tgt"].numel() // 3, dtype=torch.float64, device=dev)
        self.plan = None

    def __call__(self):
        L, i = self.L, self.inp
        self.plan = None  # the previous plan (and its workspace) goes first
        self.plan = L.lbf_plan_create(self.g.island_ptr, i["x"], i["dx"], i["d2x"], i["cen"],
                                      opt=self.opt)
        rc, its, rr = L.lbf_gmres_solve(self.plan, i["data"], self.sig, self.a)
        L.lbf_evaluate(self.plan, self.sig, self.a, i["tgt"], self.u)
        return rc, its, rr, L.lbf_solve_stats(self.plan)


def timed(fn, stream, n):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = [fn() for _ in range(n)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def apply_rate(L, plan, op, vin, vout, stream, reps=5):
    import torch

    for _ in range(2):
        L.lbf_apply(plan, op, vin, vout)
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.lbf_apply(plan, op, vin, vout)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def traced(L, fn):
    """Per-kernel device time of one call of fn (CUDA events around each traced launch
    on its stream), in a pass of its own: the timed regions run untraced."""
    import torch

    torch.cuda.synchronize()
    L.lbf_profile_reset()
    L.lbf_profile_enable(True)
    fn()
    torch.cuda.synchronize()
    L.lbf_profile_enable(False)
    prof = {}
    for kid, name in enumerate(L.KERNEL_NAMES):
        n, tms = L.lbf_profile_read(kid)
        if n:
            prof[name] = {"launches": n, "ms": tms}
    L.lbf_profile_reset()
    return prof


def traffic_for(kernel, p, leaf):
    """DRAM bytes per launch of an FMM pass from the ncu captures in profiles/traffic.json,
    for the same kernel sources, expansion order and leaf size; else None."""
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tp):
        return None
    tj = json.load(open(tp))
    if tj.get("src_hash") != src_hash():
        return None
    return tj.get("kernels", {}).get(f"{kernel}@p{p}/leaf{leaf}", {}).get("bytes_per_launch")


def roofline_of(L, prof, plan, opt, g, n64, n32, fmm64):
    counts = L.lbf_plan_counts(plan)
    bcounts = L.lbf_border_counts(plan)
    info = plan.info()
    P, P32 = info["p"] + 1, opt.p32 + 1
    cand = [k for k in prof if k in ("up", "down", "leaf", "esum", "up32", "down32", "leaf32", "esum32")]
    if not cand:
        return None, counts, bcounts, info
    dom = max(cand, key=lambda k: prof[k]["ms"])
    work, unit = kernel_work(dom, counts, bcounts, P, P32, g.N)
    if work is None:
        return None, counts, bcounts, info
    per_launch_ms = prof[dom]["ms"] / prof[dom]["launches"]
    f32 = dom.endswith("32")
    # leaf, up and down run once per application; esum once per FULL/PRECONDITIONED one
    rate = work / (per_launch_ms / 1e3)
    if f32:
        peak, src_p = FP32_PEAK_TFLOPS, "FP32: 152 SMs x 128 lanes x 2 flops x 2.07 GHz"
    else:
        peak = FP64_PEAK_TFLOPS
        src_p = ("nominal FP64: 152 SMs x 2 double multiply-adds per clock x 2.07 GHz (no measured "
                 "FP64 peak is available)")
        if fmm64 and dom in ("up", "down", "leaf"):
            src_p += ("; this kernel runs double-float arithmetic on the FP32 pipes, whose own "
                      f"ceiling is {FP32_PEAK_TFLOPS / DF64_FLOPS_PER_FLOP:.2f} TFLOP/s of double flops")
    ach = rate / 1e12
    return ({"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak, "unit": unit,
             "frac": ach / peak,
             "traffic": traffic_for(dom + ("_df64" if fmm64 and not f32 else ""),
                                    opt.p32 if f32 else info["p"], opt.leaf_size),
             "peak_source": src_p, "work_per_launch": work, "ms_per_launch": per_launch_ms},
            counts, bcounts, info)


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
    import workloads as wl

    __graft_entry__.build()
    g, src, gam = make_geometry(args.workload)
    T = args.targets
    tg = wl.targets_off_islands(g, T, seed=17)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(dev)
    inputs = dict(x=t(g.x), dx=t(g.dx), d2x=t(g.d2x), cen=t(g.centres), tgt=t(tg))
    srcd, gamd = t(src), t(gam)
    inputs["data"] = torch.empty(g.N, dtype=torch.float64, device=dev)
    L.lbf_green_sum(inputs["x"], srcd, gamd, inputs["data"])
    uex = torch.empty(T, dtype=torch.float64, device=dev)
    L.lbf_green_sum(inputs["tgt"], srcd, gamd, uex)
    stream = torch.cuda.current_stream()

    tune = None

    def options(prec):
        kw = dict(tol=args.tol, **precision_options(L, prec))
        for k, v in (("p", args.p), ("p32", args.p32), ("leaf_size", args.leaf),
                     ("inner_tol", args.inner_tol)):
            if v:
                kw[k] = v
        o = L.lbf_default_options(**kw)
        if tune:
            o.p2p_warps = tune["p2p_warps"] if tune["p2p_warps"] != 4 else 0
        return o

    opt = options(args.precision)
    if not args.no_tune and args.p is None and args.leaf is None:
        # the library's autotuner on this geometry, before (and outside) the timed region
        t0 = time.perf_counter()
        best, table = L.lbf_autotune(g.island_ptr, inputs["x"], inputs["dx"], inputs["d2x"],
                                     inputs["cen"], args.tune_target, opt=opt)
        tune = {"p": best.p, "leaf_size": best.leaf_size, "p2p_warps": best.p2p_warps or 4,
                "target": args.tune_target, "wall_s": time.perf_counter() - t0,
                "trials": table["trials"]}
        args.p, args.leaf = best.p, best.leaf_size
        opt = options(args.precision)
        opt.p2p_warps = best.p2p_warps
    step = Step(L, g, inputs, opt)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    n0 = L.lbf_launch_count()
    with Clocks(local) as clk:
        ms, outs = timed(step, stream, args.steps)
    launches = L.lbf_launch_count() - n0
    clocks = clk.summary()
    rcs = [o[0] for o in outs]
    tot = {k: sum(o[3][k] for o in outs) for k in ("arnoldi", "fp64_applies", "fp32_applies",
                                                    "refine_steps")}
    n64, n32 = tot["fp64_applies"] / args.steps, tot["fp32_applies"] / args.steps
    ms, units = aggregate(ms, float(g.N * (tot["fp64_applies"] + tot["fp32_applies"])), world, dev)
    value = units / (ms / 1e3) / 1e6
    err = float((step.u - uex).abs().max() / uex.abs().max())
    u64, s64 = step.u.clone(), step.sig.clone()
    rr = outs[-1][2]

    # one untimed, traced step: per-kernel device time and launches
    prof = traced(L, step)
    roofline, counts, bcounts, info = roofline_of(L, prof, step.plan, opt, g, n64, n32, opt.fmm64)
    stage = {k: round(prof[k]["ms"], 3) for k in prof if k.startswith("plan_")}
    # the step's phases, untraced, on the last plan: the solve (GMRES to tol from zero)
    # and the evaluation, each with CUDA events
    solve_ms = timed(lambda: L.lbf_gmres_solve(step.plan, inputs["data"], step.sig, step.a), stream, 1)[0]
    eval_ms = timed(lambda: L.lbf_evaluate(step.plan, step.sig, step.a, inputs["tgt"], step.u),
                    stream, 1)[0]

    # pure operator throughput (density block, random density) in this step's arithmetic
    vin = torch.randn(g.N, dtype=torch.float64, device=dev,
                      generator=torch.Generator(device=dev).manual_seed(1))
    vout = torch.empty_like(vin)
    matvec = {}
    a_ms = apply_rate(L, step.plan, L.LBF_OP_K_ONLY, vin, vout, stream)
    ref_apply = vout.clone()
    matvec[args.precision if args.precision != "fp32r" else "fp64"] = {
        "ms": a_ms, "mpts": g.N / a_ms / 1e3}

    # the same step in the other arithmetics
    variants = {}
    if not args.no_extras and world == 1:
        for prec in ("fp64", "df64", "fp32r"):
            if prec == args.precision:
                continue
            o2 = options(prec)
            st2 = Step(L, g, inputs, o2)
            st2()
            vms, vouts = timed(st2, stream, 2)
            s = vouts[-1][3]
            e = float((st2.u - uex).abs().max() / uex.abs().max())
            variants[prec] = {
                "step_ms": vms / 2, "status": [o[0] for o in vouts],
                "fp64_applies": s["fp64_applies"], "fp32_applies": s["fp32_applies"],
                "refine_steps": s["refine_steps"], "arnoldi": s["arnoldi"],
                "value_mpts": g.N * (s["fp64_applies"] + s["fp32_applies"]) / (vms / 2 / 1e3) / 1e6,
                "solution_max_rel_err": e,
                "u_max_rel_diff_vs_fp64": float((st2.u - u64).abs().max() / u64.abs().max()),
                "sigma_rel_l2_vs_fp64": float((st2.sig - s64).norm() / s64.norm()),
                "speedup_vs_fp64_step": (ms / args.steps) / (vms / 2)}
            if prec == "df64":
                m_ = apply_rate(L, st2.plan, L.LBF_OP_K_ONLY, vin, vout, stream)
                matvec["df64"] = {"ms": m_, "mpts": g.N / m_ / 1e3,
                                  "rel_l2_vs_fp64": float((vout - ref_apply).norm() / ref_apply.norm())}
            if prec == "fp32r":
                m_ = apply_rate(L, st2.plan, L.LBF_OP_K_ONLY | L.LBF_OP_FP32, vin, vout, stream)
                matvec["fp32"] = {"ms": m_, "mpts": g.N / m_ / 1e3,
                                  "rel_l2_vs_fp64": float((vout - ref_apply).norm() / ref_apply.norm())}
            del st2
            torch.cuda.empty_cache()

    # end to end through the public API, host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        pin = lambda a_: torch.from_numpy(np.ascontiguousarray(a_, dtype=np.float64).reshape(-1)).pin_memory()
        hx, hdx, hd2x, hc, ht = pin(g.x), pin(g.dx), pin(g.d2x), pin(g.centres), pin(tg)
        hg = inputs["data"].cpu().pin_memory()
        hu = torch.empty(T, dtype=torch.float64).pin_memory()
        bi = 8 * (hx.numel() + hdx.numel() + hd2x.numel() + hc.numel() + ht.numel() + hg.numel())
        bo = 8 * T
        holder = {}

        def e2e_step():
            holder.clear()
            d = dict(x=hx.to(dev, non_blocking=True), dx=hdx.to(dev, non_blocking=True),
                     d2x=hd2x.to(dev, non_blocking=True), cen=hc.to(dev, non_blocking=True),
                     tgt=ht.to(dev, non_blocking=True), data=hg.to(dev, non_blocking=True))
            st = Step(L, g, d, opt)
            holder["s"] = st
            out = st()
            hu.copy_(st.u, non_blocking=True)
            return out[3]["fp64_applies"] + out[3]["fp32_applies"]

        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ne = max(1, min(args.e2e_steps, args.steps))
        ems, aps = timed(e2e_step, stream, ne)
        holder.clear()
        ems, units_e = aggregate(ems, float(g.N * sum(aps)), world, dev)
        e2e = {"value": units_e / (ems / 1e3) / 1e6, "unit": "Mpts/s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": ems / ne, "steps": ne}

    extras = {}
    if not args.no_extras and world == 1:
        extras = run_extras(args, L, dev, stream)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        v, dt, cores, rows = oracle_rate(g, 4 * reference_rows(g))
        cpu = {"value": v, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
               "sample": f"{rows} rows of the N={g.N} density block (I+K), {dt:.1f} s wall"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "df64": "f64 (double-float FMM)", "fp32r": "f32+f64"}[args.precision],
                "data": "synthetic",
                "config": workload_config(args.workload, g, T, args.tol, args.precision),
                "solve": {"status": rcs, "step_ms": ms / args.steps, "solve_ms": solve_ms,
                          "evaluate_ms": eval_ms, "plan_ms": ms / args.steps - solve_ms - eval_ms,
                          "plan_stages_ms_traced": stage, "applies_per_step": n64 + n32,
                          "fp64_applies": n64, "fp32_applies": n32,
                          "refine_steps": tot["refine_steps"] / args.steps,
                          "arnoldi": tot["arnoldi"] / args.steps, "rel_residual": rr,
                          "solution_max_rel_err": err, "tree": info, "counts": counts,
                          "border_counts": bcounts},
                "matvec": matvec, "variants": variants, "workloads": extras, "autotune": tune,
                "kernels_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
                "kernel_launches": {k: v["launches"] for k, v in prof.items()},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks}
        if args.precision == "fp64":
            line["peak_fractions"] = peak_fractions(line)
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_extras(args, L, dev, stream):
    """The other workloads, each measured briefly: solve latency on one island (direct
    matvec), matvec and solve latency on 16 islands, the gradient at 256 islands x 512
    nodes, and batched uneven solves against the plain FP64 loop (a fixed stratified
    subset of the instances; bench.py --workload C4 runs all of them)."""
    import numpy as np
    import torch
    import workloads as wl

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(dev)
    out = {}

    def exact_case(g, src, gam, T, seed):
        tg = wl.targets_off_islands(g, T, seed=seed)
        d = dict(x=t(g.x), dx=t(g.dx), d2x=t(g.d2x), cen=t(g.centres), tgt=t(tg))
        d["data"] = torch.empty(g.N, dtype=torch.float64, device=dev)
        L.lbf_green_sum(d["x"], t(src), t(gam), d["data"])
        uex = torch.empty(T, dtype=torch.float64, device=dev)
        L.lbf_green_sum(d["tgt"], t(src), t(gam), uex)
        return d, uex

    # C1: one cap, N = 256, direct matvec, tol 1e-12
    g = wl.config_geometry("C1")
    src, gam, _ = wl.pair_sources(g, 0)
    d, uex = exact_case(g, src, gam, 256, 5)
    st = Step(L, g, d, L.lbf_default_options(matvec=L.LBF_MATVEC_DIRECT, tol=1e-12, fmm64=0))
    st()
    cms, co = timed(st, stream, 5)
    out["C1"] = {"what": "one island, N=256, direct matvec, GMRES tol 1e-12, 256 targets, FP64",
                 "step_ms": cms / 5, "iterations": co[-1][1],
                 "solution_max_rel_err": float((st.u - uex).abs().max() / uex.abs().max())}

    # C2: 16 islands x 512 nodes, FMM, tol 1e-12
    g = wl.config_geometry("C2")
    src, gam, _ = wl.pair_sources(g, 0, 1)
    d, uex = exact_case(g, src, gam, 256, 5)
    o2 = L.lbf_default_options(tol=1e-12, fmm64=0)
    st = Step(L, g, d, o2)
    st()
    cms, co = timed(st, stream, 5)
    vin = torch.randn(g.N + g.M, dtype=torch.float64, device=dev,
                      generator=torch.Generator(device=dev).manual_seed(2))
    vout = torch.empty_like(vin)
    am = apply_rate(L, st.plan, L.LBF_OP_FULL, vin, vout, stream)
    sms = timed(lambda: L.lbf_gmres_solve(st.plan, d["data"], st.sig, st.a), stream, 5)[0] / 5
    out["C2"] = {"what": "16 islands x 512 nodes (N=8192), FMM, GMRES tol 1e-12, FP64",
                 "step_ms": cms / 5, "solve_ms": sms, "matvec_ms": am, "iterations": co[-1][1],
                 "solution_max_rel_err": float((st.u - uex).abs().max() / uex.abs().max())}

    # C5: gradient of mean u^2 at 4096 targets, 256 islands x 512 nodes (N = 131072)
    from paper_1306_0612_gb300 import autograd as AG
    g = wl.config_geometry("C5")
    X, D1, D2 = g.x, g.dx, g.d2x
    z, z1, z2 = (A[:, 0] + 1j * A[:, 1] for A in (X, D1, D2))
    w, w1, w2 = 1 - X[:, 2], -D1[:, 2], -D2[:, 2]
    xi, xi1 = z / w, z1 / w - z * w1 / w ** 2
    xi2 = z2 / w - 2 * z1 * w1 / w ** 2 - z * w2 / w ** 2 + 2 * z * w1 ** 2 / w ** 3
    pl = lambda c: t(np.stack([c.real, c.imag], axis=1))
    tg = t(wl.targets_off_islands(g, 4096, seed=6))
    src, gam, _ = wl.pair_sources(g, 0, 1)
    data = torch.empty(g.N, dtype=torch.float64, device=dev)
    L.lbf_green_sum(t(g.x), t(src), t(gam), data)
    o5 = L.lbf_default_options(tol=1e-10, fmm64=0)
    cen, d1t, d2t = t(g.centres), pl(xi1), pl(xi2)

    def grad_step():
        gt = data.clone().requires_grad_(True)
        xt = pl(xi).reshape(g.N, 2).requires_grad_(True)
        u = AG.solve_evaluate(gt, xt, d1t, d2t, cen, tg, g.island_ptr, o5)
        loss = (u ** 2).mean()
        loss.backward()
        return float(loss.detach())

    grad_step()
    gms = timed(grad_step, stream, 3)[0] / 3
    out["C5"] = {"what": "gradient of mean u^2 at 4096 targets w.r.t. Dirichlet data and planar "
                         "node positions, 256 islands x 512 nodes (N=131072), FP64, tol 1e-10",
                 "forward_backward_ms": gms}

    # the paper's table shapes on elliptical islands (Sec. 6, Examples 1 and 3): GMRES
    # iterations, plan ("CPU Prec") and solve time, and the error at 75 points against the
    # exact data (1/2) sum Re 1/(xi - xi_k), for growing nodes per island
    def ellipse_row(M, n, precond):
        g = wl.ellipse_islands(1 if M == 15 else M, M, n)
        x = t(g.x)
        data = torch.empty(g.N, dtype=torch.float64, device=dev)
        L.lbf_dipole_sum(x, t(g.centres[1:]), data)
        tg = t(wl.targets_off_islands(g, 75, seed=2))
        ue = torch.empty(75, dtype=torch.float64, device=dev)
        L.lbf_dipole_sum(tg, t(g.centres[1:]), ue)
        opt = L.lbf_default_options(tol=1e-11, fmm64=0, precond=precond)
        t0 = time.perf_counter()
        plan = L.lbf_plan_create(g.island_ptr, x, t(g.dx), t(g.d2x), t(g.centres), opt=opt)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sig = torch.empty(g.N, dtype=torch.float64, device=dev)
        a = torch.empty(g.M, dtype=torch.float64, device=dev)
        rc, its, rr = L.lbf_gmres_solve(plan, data, sig, a)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        u = torch.empty(75, dtype=torch.float64, device=dev)
        L.lbf_evaluate(plan, sig, a, tg, u)
        err = float((u - ue).abs().max() / ue.abs().max())
        return {"N": n, "iterations": its, "status": rc, "plan_ms": 1e3 * (t1 - t0),
                "solve_ms": 1e3 * (t2 - t1), "error": err}

    ex1 = {"preconditioned": [ellipse_row(15, n, 1) for n in (32, 64, 128, 256, 512)],
           "unpreconditioned": [ellipse_row(15, n, 0) for n in (32, 64, 128, 256, 512)]}
    ex3 = {str(M): [ellipse_row(M, n, 1) for n in (128, 256, 512, 1024, 2048)] for M in (98, 200, 407)}
    out["ellipse_tables"] = {"what": "elliptical islands on a Fibonacci lattice with random axes, "
                                     "exact data (1/2) sum Re 1/(xi - xi_k), GMRES tol 1e-11, FP64, "
                                     "error at 75 points",
                             "example1_M15": ex1, "example3": ex3}

    # C4: batched uneven solves against the plain FP64 loop, every 16th instance
    insts = wl.batch_instances(seed=4, count=512, nrhs=16)[::16]
    T4 = 32
    inst = []
    for gg, pairs in insts:
        x = t(gg.x)
        data4 = torch.empty((len(pairs), gg.N), dtype=torch.float64, device=dev)
        tg4 = t(wl.targets_off_islands(gg, T4, seed=5))
        ue = torch.empty((len(pairs), T4), dtype=torch.float64, device=dev)
        for k, (pp, gm) in enumerate(pairs):
            L.lbf_green_sum(x, t(pp), t(gm), data4[k])
            L.lbf_green_sum(tg4, t(pp), t(gm), ue[k])
        inst.append(dict(island_ptr=gg.island_ptr, x=x, dx=t(gg.dx), d2x=t(gg.d2x),
                         centres=t(gg.centres), g=data4, targets=tg4, uex=ue, N=gg.N, M=gg.M))
    nsolve = sum(i["g"].shape[0] for i in inst)

    def errs(res):
        e = []
        for ins, r in zip(inst, res):
            e.extend(((r["u"] - ins["uex"]).abs().amax(dim=1) / ins["uex"].abs().amax(dim=1)).tolist())
        return float(np.max(e))

    ob = L.lbf_default_options(tol=args.tol, precision=L.LBF_PRECISION_FP32_REFINE, fmm64=0,
                               inner_tol=C4_INNER_TOL)
    L.lbf_batch_run(inst[:4], opt=ob, nworkers=args.workers)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = L.lbf_batch_run(inst, opt=ob, nworkers=args.workers)
    torch.cuda.synchronize()
    dtb = time.perf_counter() - t0
    eb = errs(res)
    t0 = time.perf_counter()
    L.lbf_batch_run(inst, opt=ob, nworkers=args.workers, lockstep=False)
    torch.cuda.synchronize()
    dts = time.perf_counter() - t0
    ol = L.lbf_default_options(tol=args.tol, fmm64=0)
    # the FP64 operator with each instance's right-hand sides in lockstep
    L.lbf_batch_run(inst[:4], opt=ol, nworkers=args.workers, lockstep=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    resk = L.lbf_batch_run(inst, opt=ol, nworkers=args.workers, lockstep=True)
    torch.cuda.synchronize()
    dtk = time.perf_counter() - t0
    ek = errs(resk)
    t0 = time.perf_counter()
    le = []
    for ins in inst:
        plan = L.lbf_plan_create(ins["island_ptr"], ins["x"], ins["dx"], ins["d2x"], ins["centres"], opt=ol)
        sig = torch.empty(ins["N"], dtype=torch.float64, device=dev)
        a = torch.empty(ins["M"], dtype=torch.float64, device=dev)
        u = torch.empty(T4, dtype=torch.float64, device=dev)
        for k in range(ins["g"].shape[0]):
            L.lbf_gmres_solve(plan, ins["g"][k], sig, a)
            L.lbf_evaluate(plan, sig, a, ins["targets"], u)
            le.append(float((u - ins["uex"][k]).abs().max() / ins["uex"][k].abs().max()))
        del plan
    torch.cuda.synchronize()
    dtl = time.perf_counter() - t0
    out["C4"] = {"what": f"{len(inst)} of the 512 uneven geometries (every 16th: 1-64 islands, "
                         f"64-1024 nodes per island) x 16 right-hand sides = {nsolve} solves to "
                         f"tol {args.tol:g}, {T4} targets each",
                 "batched_fp32r_solves_per_s": nsolve / dtb, "batched_fp32r_s": dtb,
                 "batched_fp32r_one_after_another_solves_per_s": nsolve / dts,
                 "batched_solution_err_max": eb,
                 "batched_fp64_lockstep_solves_per_s": nsolve / dtk, "batched_fp64_lockstep_s": dtk,
                 "batched_fp64_lockstep_err_max": ek,
                 "loop_fp64_solves_per_s": nsolve / dtl, "loop_fp64_s": dtl,
                 "loop_solution_err_max": float(np.max(le)),
                 "speedup": dtl / dtb}
    return out


def run_batch(args):
    """C4: independent geometries of uneven size (1-64 islands, 64-1024 nodes per
    island, log-uniform), 16 Green's-pair right-hand sides each, solved to 1e-10 and
    evaluated at off-curve targets.  Batched arms: the native scheduler (worker streams),
    FP32 FMM with FP64 refinement or FP64, each instance's right-hand sides in lockstep
    (lbf_gmres_solve_many) or one after another.  Baseline arm: the plain FP64 loop over
    all instances on one stream (plan, 16 solves, evaluations).  --arms picks a subset."""
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

    def batched(precision, sub, lockstep=False):
        kw = dict(inner_tol=args.inner_tol or C4_INNER_TOL)
        opt = L.lbf_default_options(tol=args.tol, precision=precision, fmm64=0, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = L.lbf_batch_run(sub, opt=opt, nworkers=args.workers, lockstep=lockstep)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = [r["status"] for r in res]
        return dt, res, st

    arms = set(args.arms.split(",")) if args.arms != "all" else {"fp32r", "fp32r_seq", "fp64",
                                                                  "fp64_lockstep", "loop"}
    line = {"metric": "batched uneven solves: solves per second (plan + GMRES to 1e-10 + evaluation)",
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"C4: {len(inst)} star-cap geometries, 1-64 islands, 64-1024 nodes "
                                   f"per island (log-uniform), 16 Green's-pair right-hand sides each, "
                                   f"{T} targets", "instances": len(inst), "solves": nsolve,
                       "nodes": nodes, "workers": args.workers, "tol": args.tol}}
    arm_defs = [("fp32r", "batched_fp32r", L.LBF_PRECISION_FP32_REFINE, True,
                 "each instance's 16 right-hand sides in lockstep (lbf_gmres_solve_many)"),
                ("fp32r_seq", "batched_fp32r_one_after_another", L.LBF_PRECISION_FP32_REFINE, False,
                 "each instance's right-hand sides one after another"),
                ("fp64", "batched_fp64", L.LBF_PRECISION_FP64, False,
                 "each instance's right-hand sides one after another"),
                ("fp64_lockstep", "batched_fp64_lockstep", L.LBF_PRECISION_FP64, True,
                 "each instance's 16 right-hand sides in lockstep (lbf_gmres_solve_many)")]
    for key, name, prec, lock, note in arm_defs:
        if key not in arms:
            continue
        batched(prec, inst[:args.workers], lockstep=lock)  # warm-up
        dt, res, st = batched(prec, inst, lockstep=lock)
        e = err(res, inst)
        line[name] = {"wall_s": dt, "solves_per_s": nsolve / dt, "statuses_ok": st.count(0),
                      "solution_err_max": e[0], "solution_err_median": e[1],
                      "fp32_applies": sum(r["fp32_applies"] for r in res),
                      "fp64_applies": sum(r["fp64_applies"] for r in res), "note": note}
        if "value" not in line:
            line["value"] = nsolve / dt
    if "loop" in arms:
        opt64 = L.lbf_default_options(tol=args.tol, fmm64=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nloop = 0
        loop_err = []
        for ins in inst:
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
        line["loop_fp64"] = {"instances": len(inst), "solves": nloop, "wall_s": dtl,
                             "solves_per_s": nloop / dtl, "solution_err_max": float(np.max(loop_err)),
                             "note": "plain FP64 loop over every instance on one stream"}
        if "value" in line:
            line["speedup_vs_loop_fp64"] = line["value"] / (nloop / dtl)
    print(json.dumps(line))
    return 0


def run_sweep(args):
    """C3 sweep: the density operator (I + 2K) sigma, sigma ~ N(0, 1), on 2^k islands x
    1024 nodes; native double, double-float and float FMM applies (median of 5 after 3
    warm-ups, CUDA events), per-kernel algorithmic rates, the errors against native
    double, and (N <= 262144) the FMM against the GPU's tiled direct sum."""
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

    for M in [int(v) for v in args.sweep_m.split(",")]:
        g = wl.star_caps(3, M, 1024)
        x, dx, d2x, cen = t(g.x), t(g.dx), t(g.d2x), t(g.centres)
        vin = t(wl.random_density(g.N, seed=1))
        line = {"sweep": "C3", "islands": M, "N": g.N}
        outs = {}
        for nm, kw, op in (("fp64", dict(fmm64=0), L.LBF_OP_K_ONLY),
                           ("df64", dict(fmm64=1), L.LBF_OP_K_ONLY),
                           ("fp32", dict(fmm64=1, precision=L.LBF_PRECISION_FP32_REFINE),
                            L.LBF_OP_K_ONLY | L.LBF_OP_FP32)):
            plan = L.lbf_plan_create(g.island_ptr, x, dx, d2x, cen,
                                     opt=L.lbf_default_options(border=0, **kw))
            o = torch.empty_like(vin)
            ms = apply_rate(L, plan, op, vin, o, stream)
            counts = L.lbf_plan_counts(plan)
            info = plan.info()
            P, P32 = info["p"] + 1, L.lbf_default_options().p32 + 1
            prof = traced(L, lambda: L.lbf_apply(plan, op, vin, o))
            kern = {}
            for name, v in prof.items():
                work, _ = kernel_work(name, counts, None, P, P32, g.N)
                if work:
                    peak = FP32_PEAK_TFLOPS if name.endswith("32") else FP64_PEAK_TFLOPS
                    ach = work / (v["ms"] / 1e3) / 1e12
                    kern[name] = {"ms": round(v["ms"], 3), "tflops": ach, "frac": ach / peak}
            outs[nm] = o
            line[nm] = {"apply_ms": ms, "mpts": g.N / ms / 1e3, "kernels": kern}
            line["tree"] = info
            del plan
        for nm in ("df64", "fp32"):
            line[nm]["rel_l2_vs_fp64"] = float((outs[nm] - outs["fp64"]).norm() / outs["fp64"].norm())
        if g.N <= 262144:
            od = torch.empty_like(vin)
            pd = L.lbf_plan_create(g.island_ptr, x, dx, d2x, cen,
                                   opt=L.lbf_default_options(border=0, matvec=L.LBF_MATVEC_DIRECT))
            msd = apply_rate(L, pd, L.LBF_OP_K_ONLY, vin, od, stream, reps=3)
            line["direct"] = {"apply_ms": msd, "mpts": g.N / msd / 1e3,
                              "pairs_per_s": g.N * (g.N - 1) / (msd / 1e3)}
            for nm in outs:
                line[nm]["rel_l2_vs_direct"] = float((outs[nm] - od).norm() / od.norm())
            del pd
        print(json.dumps(line), flush=True)
        del outs
        torch.cuda.empty_cache()
    return 0


def run_apply(args):
    """One application of the density operator (I + 2K) sigma, sigma ~ N(0, 1), on the
    workload's plan (border included, as in a solve: the float forward rows then take the
    far field by the per-node ancestor walk), in the precision's FMM arithmetic: the
    launches a kernel profile captures."""
    import numpy as np
    import torch
    import workloads as wl
    from paper_1306_0612_gb300 import lbfmm as L
    import __graft_entry__

    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    g, _, _ = make_geometry(args.workload)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(dev)
    kw = dict(**precision_options(L, args.precision))
    for k, v in (("p", args.p), ("p32", args.p32), ("leaf_size", args.leaf), ("p2p_warps", args.warps)):
        if v:
            kw[k] = v
    plan = L.lbf_plan_create(g.island_ptr, t(g.x), t(g.dx), t(g.d2x), t(g.centres),
                             opt=L.lbf_default_options(**kw))
    v = t(wl.random_density(g.N, 1))
    o = torch.empty_like(v)
    op = L.LBF_OP_K_ONLY | (L.LBF_OP_FP32 if args.precision == "fp32r" else 0)
    L.lbf_apply(plan, op, v, o)
    torch.cuda.synchronize()
    print(json.dumps({"apply": args.workload, "precision": args.precision, "tree": plan.info(),
                      "counts": L.lbf_plan_counts(plan), "norm": float(o.norm())}))
    return 0


def main():
    args = parse()
    if args.apply:
        return run_apply(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.workload == "C4":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
