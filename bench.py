"""Benchmark of the SEIRD backward-Euler Newton-Krylov-Schwarz step on GB300.

Metric: implicit DOF*steps/s at a 1e-8 relative Newton residual (DOF = 5 x
nodes).  Headline workload: the paper-scale Southern-Ontario-like mesh, a
seeded 24-gon meshed to 18.4M P1 nodes (92M unknowns, the size of the paper's
Section 4.2 scalability run), urban-Gaussian density, 5 infection seeds,
dt = 0.5 day, RAS with 4096 uneven subdomains, overlap 2, block ILU(2)
subdomain factors (ILU(3) on the mixed-precision path), the paper's
multiplicative two-grid with the constant coarse space, FGMRES(30) with CGS2.
A "step" is one backward-Euler time step (assembly, preconditioner set-up,
GMRES, line search) of that whole mesh.  The same line carries the
mixed-precision path on that workload, the 2.0M-node workload (10M unknowns,
512 subdomains, block ILU(1)), a 64-sample ensemble and the discrete adjoint
(256^2 mesh, block ILU(0)) and the oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --cpu-ladder      (the oracle on a ladder of square meshes)
  python bench.py --fp64-probe      (FP64 FMA and DGEMM rates of this GPU)

--impl reference times the CPU oracle (test infrastructure, not the product)
on the host cores, on a bounded sample of the same workload.  Under torchrun
(N > 1) every rank runs an independent replica of the workload (the path is one
coupled solve; it is not sharded across GPUs) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SEIRD implicit DOF·steps/s at 1e-8 Newton resid (FP64 vs mixed); BSR SpMV GB/s"
UNIT = "DOF·steps/s"
FALLBACK_HBM_GBS = 6800.0

# dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed ncu
# capture of each kernel class, as (bytes per launch there, units processed there,
# seird_get_info key of those units); scaled to a launch by the units it processes
# (traffic grows in proportion).  The SpMV was captured on the 200k-node case of the
# same generator, the subdomain solve at full size (18.4M nodes, 4096 subdomains,
# block ILU(2) factors in FP64 and ILU(3) in FP32, the autotuned variants).  Entries are removed when the kernel
# changes and restored by the next capture.
NCU_TRAFFIC = {
    ("spmv", "fp64"): (307.414e6, 1400635, "nnzb"),  # k_bsr_spmv<double>, 1.4M blocks
    ("ilu_solve", "fp64"): (60.66e9, 264544907, "subdomain_blocks"),  # k_ilu_solve<double, double, 4, 3, 118>, ILU(2)
    ("ilu_solve", "mixed"): (42.39e9, 344245751, "subdomain_blocks"),  # k_ilu_solve<float, float, 4, 3, 236>, ILU(3)
}

# kernel classes with one kernel launch per timed call
SINGLE_KERNEL = ("spmv", "ilu_solve")

PAPER_SCALE_NODES = 18_400_000
PAPER_SCALE_SUBDOMAINS = 4096


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nodes", type=int, default=PAPER_SCALE_NODES)
    ap.add_argument("--subdomains", type=int, default=PAPER_SCALE_SUBDOMAINS)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--forcing", choices=["fixed", "ew"], default="ew")
    ap.add_argument("--pc-lag", type=int, default=20)
    ap.add_argument("--pc-keep", type=int, default=3, help="steps a preconditioner may be carried over")
    ap.add_argument("--predictor", type=int, choices=[0, 1, 2, 3, 4, 5, 6], default=5,
                    help="Newton's first iterate: 0 u^n, p = 1-6 the degree-p extrapolation through u^n and the "
                         "p previous states")
    ap.add_argument("--coarse", type=int, choices=[1, 2, 3], default=2,
                    help="1 additive coarse correction, 2 the paper's multiplicative two-grid (Eq. RAS_2L), "
                         "3 coarse correction then RAS")
    ap.add_argument("--coarse-group", type=int, default=0, help="subdomains per coarse unit (0: automatic)")
    ap.add_argument("--ilu-fill", type=int, default=2, choices=range(0, 9),
                    help="levels of fill k of the block ILU(k) subdomain factors (headline workload)")
    ap.add_argument("--ilu-fill-mixed", type=int, default=3, choices=range(0, 9),
                    help="levels of fill of the headline workload's mixed-precision subdomain factors")
    ap.add_argument("--ilu-fill-2m", type=int, default=1, choices=range(0, 9),
                    help="levels of fill of the 2.0M-node object's subdomain factors (both precisions)")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--one-pass", action="store_true",
                    help="one classical Gram-Schmidt pass (PETSc's default) instead of CGS2")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-2m", action="store_true", help="skip the 2.0M-node (10M-unknown) object")
    ap.add_argument("--ensemble", type=int, default=64, help="samples of the ensemble line (0: skip it)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing line")
    ap.add_argument("--no-autotune", action="store_true", help="fixed launch shapes instead of the autotuner's")
    ap.add_argument("--cpu-ladder", action="store_true", help="time the oracle on the square-mesh ladder and exit")
    ap.add_argument("--fp64-probe", action="store_true", help="measure the FP64 FMA and DGEMM rates and exit")
    ap.add_argument("--oracle-sample", type=str, default=None, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def solver_options(args, precision, subdomains, ilu_fill=None):
    """Options of one measured context; ilu_fill defaults to the headline workload's for the precision."""
    if ilu_fill is None:
        ilu_fill = args.ilu_fill_mixed if precision == "mixed" else args.ilu_fill
    return dict(n_subdomains=subdomains, overlap=2, coarse=args.coarse, coarse_group=args.coarse_group,
                pc_keep_steps=args.pc_keep, predictor=args.predictor, newton_rtol=1e-8, gmres_rtol=1e-5,
                gmres_restart=30, gmres_maxit=200, precision=1 if precision == "mixed" else 0, seed=args.seed,
                gmres_forcing=1 if args.forcing == "ew" else 0, pc_lag=args.pc_lag,
                gmres_one_pass=1 if args.one_pass else 0,
                ilu_fill=ilu_fill)


def workload_config(wl, args, subdomains):
    return {
        "workload": "%s (Southern-Ontario-like 24-gon, %d P1 nodes, %d unknowns)" % (wl.name, wl.n, 5 * wl.n),
        "n_nodes": wl.n, "n_tris": int(len(wl.tri)), "dof": 5 * wl.n, "dt_days": wl.dt,
        "subdomains": subdomains, "overlap": 2,
        "coarse": {1: "additive", 2: "multiplicative two-grid (Eq. RAS_2L)",
                   3: "coarse correction, then RAS"}[args.coarse] + ", constant per subdomain and compartment",
        "subdomain_solver": "block ILU(%d)" % args.ilu_fill,
        "krylov": "FGMRES(30) right-preconditioned, %s, rtol 1e-5" % (
            "classical Gram-Schmidt single pass (PETSc default)" if args.one_pass else "CGS2"),
        "forcing": "Eisenstat-Walker" if args.forcing == "ew" else "fixed rtol 1e-5",
        "pc_lag": args.pc_lag, "pc_keep_steps": args.pc_keep, "predictor": args.predictor,
        "newton_rtol": 1e-8, "quadrature": "degree-5 seven-point", "seed": args.seed,
        "l2": "inputs larger than L2 (the FP64 Jacobian alone is > 2.7 GB)",
    }


# ---------------------------------------------------------------------------
# CPU oracle (run in a child process with one BLAS thread)
# ---------------------------------------------------------------------------

CPU_BASELINE_NODES = 20_000   # one step: about 20-25 s of one core
REFERENCE_NODES = 5_000       # per step about 3 s: a --steps 20 --warmup 5 run ends in a few minutes


def oracle_sample_child(spec):
    """Times the oracle (as it stands) on the workload generator named in spec."""
    from oracle import seird_oracle as O
    from paper_2208_01839_gb300 import inputs as I
    d = json.loads(spec)
    if d.get("nside"):
        wl = I.ontario_workload(d["nside"] ** 2, seed=d["seed"], structured=True, nside=d["nside"])
    elif d.get("square"):
        wl = I.square_workload(d["square"])
    else:
        wl = I.ontario_workload(d["nodes"], seed=d["seed"])
    U = wl.U0
    times = []
    for k in range(d["warmup"] + d["steps"]):
        t0 = time.perf_counter()
        U, info = O.newton_step(wl.xy, wl.tri, wl.params, wl.dt, U, rtol=1e-8)
        if k >= d["warmup"]:
            times.append(time.perf_counter() - t0)
    print(json.dumps({"n": wl.n, "dof": 5 * wl.n, "times": times, "name": wl.name}))


def run_oracle(spec):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", json.dumps(spec)], env=env,
                       capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: %s" % r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_sample(nodes, steps, warmup, seed):
    out = run_oracle({"nodes": nodes, "steps": steps, "warmup": warmup, "seed": seed})
    tot = sum(out["times"])
    return {"value": out["dof"] * len(out["times"]) / tot, "unit": UNIT, "cores": 1,
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d step(s) of the same generator at %d nodes (%d DOF), Newton to 1e-8 with a SuperLU "
                      "direct solve, one thread of the host's %d" % (len(out["times"]), out["n"], out["dof"],
                                                                     os.cpu_count() or 0),
            "s_per_step": tot / len(out["times"])}


def run_cpu_ladder(args):
    """The oracle on the 33x33 square (config 1) and on the urban-square ladder
    65^2, 129^2, 257^2 (steps bounded so that each rung takes minutes), then a
    power-law fit of seconds per step against nodes, extrapolated (and labelled
    so) to the 2.0M-node and 18.4M-node workloads."""
    rungs = [({"square": 33}, 10), ({"nside": 65}, 10), ({"nside": 129}, 3), ({"nside": 257}, 1)]
    out = []
    for spec, steps in rungs:
        d = run_oracle(dict(spec, steps=steps, warmup=0, seed=args.seed))
        sps = sum(d["times"]) / len(d["times"])
        out.append({"workload": d["name"], "nodes": d["n"], "steps": len(d["times"]), "s_per_step": sps,
                    "dof_steps_per_s": d["dof"] / sps})
    # fit log(s) = a + b log(n) on the urban-square rungs (same generator family as the workloads)
    pts = [(math.log(r["nodes"]), math.log(r["s_per_step"])) for r in out[1:]]
    mx = sum(p[0] for p in pts) / len(pts)
    my = sum(p[1] for p in pts) / len(pts)
    b = sum((x - mx) * (y - my) for x, y in pts) / sum((x - mx) ** 2 for x, _ in pts)
    a = my - b * mx
    extra = {}
    for name, n in (("ontario_like_2001k", 2_001_952), ("ontario_like_18408k", 18_408_616)):
        s = math.exp(a + b * math.log(n))
        extra[name] = {"nodes": n, "s_per_step": s, "dof_steps_per_s": 5 * n / s, "kind": "extrapolated",
                       "s_per_180_steps": 180 * s}
    print(json.dumps({"cpu_ladder": out, "fit": {"exponent": b, "s_per_step_at_1e5_nodes": math.exp(a + b * math.log(1e5))},
                      "extrapolated": extra, "cores": 1, "host_cores": os.cpu_count(),
                      "note": "oracle (NumPy assembly, SuperLU), one thread"}))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "seird_clocks_%d_%d.csv" % (os.getpid(), index))

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, world, device="cuda"):
    """Max of a per-rank scalar (elapsed time) over all ranks; identity at N = 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(dof, steps, seconds, world):
    """Whole-job DOF*steps/s: every rank advances its own replica by `steps` steps."""
    return world * dof * steps / seconds


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (profiling recipe)"


# GB300's FP64 peak from its unit counts and clock: 152 SMs x 2 FP64 FMA per clock x 2 flop x
# 2.070 GHz = 1.259 TFLOP/s (the part's nominal 1.25).  --fp64-probe measures 1.234 TFLOP/s with
# an FMA loop at 2070 MHz (98%) and 1.10 with cuBLAS DGEMM.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP64_PEAK_KIND = "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz (an FMA loop measures 1.234)"


def algorithmic_fma(cls, info):
    """FP64 FMAs one launch must perform: 25 per 5x5 block product."""
    if cls == "spmv":
        return 25 * info["nnzb"]
    if cls == "ilu_solve":  # forward L blocks + backward U blocks + the inverted pivots = every local block
        return 25 * info["subdomain_blocks"]
    return None


def class_sums(S, stats):
    """Per kernel class over the timed steps: device ms, launches, algorithmic bytes (library counts)."""
    kms = {k: sum(s["kernel_ms"][k] for s in stats) for k in S.KERNEL_CLASSES}
    kcalls = {k: sum(s["kernel_calls"][k] for s in stats) for k in S.KERNEL_CLASSES}
    kbytes = {k: sum(s["alg_bytes"][k] for s in stats) for k in S.KERNEL_CLASSES}
    return kms, kcalls, kbytes


def roofline(S, res, precision):
    """Dominant single-kernel class against its roofline, the SpMV, and the whole step.

    achieved = the library's algorithmic bytes (or, for FP64 work, 2 x its FMAs) / CUDA-event time on
    the context's stream.  The bound is whichever of the HBM time (bytes / HBM peak) and the FP64
    time (FMAs / FP64 peak) is longer: an FP64 5x5 block product moves 204 bytes per 25 FMAs, more
    work per byte than GB300's FP64 pipe keeps up with at full bandwidth, so the FP64 SpMV and
    subdomain solve are bound by the pipe ("alu"), their FP32 forms by HBM."""
    kms, kcalls, kbytes = class_sums(S, res["stats"])
    info = res["info"]
    peak, peak_kind = peaks()
    dom = max(SINGLE_KERNEL, key=lambda k: kms[k])
    ab = kbytes[dom] / max(kcalls[dom], 1)
    avg_ms = kms[dom] / max(kcalls[dom], 1)
    achieved = ab / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    traffic = None
    tr = NCU_TRAFFIC.get((dom, precision))
    if tr is not None:
        bytes_small, units_small, unit_key = tr
        traffic = bytes_small * info[unit_key] / units_small
    sp_ms = kms["spmv"] / max(kcalls["spmv"], 1)
    sp_ab = kbytes["spmv"] / max(kcalls["spmv"], 1)
    sp_gbs = sp_ab / (sp_ms * 1e-3) / 1e9 if kcalls["spmv"] and sp_ms > 0 else None
    fma = algorithmic_fma(dom, info) if precision == "fp64" else None
    alu = None
    if fma is not None and avg_ms > 0:
        tf = 2.0 * fma / (avg_ms * 1e-3) / 1e12
        alu = {"achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
               "peak_kind": FP64_PEAK_KIND, "fma_per_launch": fma}
    sp_fma = algorithmic_fma("spmv", info) if precision == "fp64" else None
    sp_alu = (2.0 * sp_fma / (sp_ms * 1e-3) / 1e12) / FP64_PEAK_TFLOPS if sp_fma and sp_ms > 0 else None
    step_s = res["ms_per_step"] * len(res["stats"]) * 1e-3
    total = sum(kbytes.values())
    step = {"bytes_per_step": total / max(len(res["stats"]), 1), "achieved": total / step_s / 1e9 if step_s else None,
            "peak": peak, "unit": "GB/s", "frac": (total / step_s / 1e9) / peak if step_s else None,
            "peak_kind": peak_kind,
            "bytes_by_class": {k: v / max(len(res["stats"]), 1) for k, v in kbytes.items()},
            "note": "sum of the library's algorithmic bytes over the timed steps / their device time"}
    hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind}
    common = {"kernel": dom, "traffic": traffic, "algorithmic_bytes_per_launch": ab, "avg_launch_ms": avg_ms,
              "launches": kcalls[dom]}
    if alu is not None and 2.0 * fma / (FP64_PEAK_TFLOPS * 1e12) > ab / (peak * 1e9):
        roof = dict({"bound": "alu"}, **{k: alu[k] for k in ("achieved", "peak", "unit", "frac", "peak_kind")},
                    **common, fma_per_launch=fma, hbm=hbm)
    else:
        roof = dict({"bound": "hbm"}, **hbm, **common, fp64_alu=alu)
    return (roof,
            {"gbs": sp_gbs, "frac_of_hbm": (sp_gbs / peak) if sp_gbs else None, "frac_of_fp64": sp_alu,
             "avg_launch_ms": sp_ms, "launches": kcalls["spmv"], "algorithmic_bytes": sp_ab},
            step, kms, kcalls)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def measure(S, wl, args, stream, precision, subdomains, world, local, e2e=True):
    """Warm-up, then K device-timed steps (and K end-to-end steps) of one variant."""
    import torch
    import torch.distributed as dist
    t_create = time.perf_counter()
    sv = S.Solver(wl.xy, wl.tri, wl.params, stream=stream, dt=wl.dt, timing=1,
                  autotune=0 if args.no_autotune else 1, **solver_options(args, precision, subdomains))
    info = sv.info()
    t_create = time.perf_counter() - t_create  # partition, patterns, level schedules, upload
    sv.set_state(torch.tensor(wl.U0, device="cuda"))
    for _ in range(args.warmup):
        sv.step()
    if e2e:  # where the timed steps start: the e2e loop replays the same steps from here
        hstart = torch.empty((wl.n, 5), dtype=torch.float64, pin_memory=True)
        sv.get_state(hstart.numpy())
        t_start = sv.t
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = S.launch_count()
    stats = []
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(sv.step())
        e1.record(stream)
        torch.cuda.synchronize()
    launches = S.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    info = sv.info()  # after the first solve: the autotuner's launch shapes
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms, world)
    dof = 5 * wl.n
    out = {"value": aggregate_value(dof, args.steps, ms * 1e-3, world), "ms_per_step": ms / args.steps,
           "launches": launches, "create_s": t_create, "clocks": clk.summary(), "info": info, "stats": stats}
    if e2e:
        # The same K steps again, from the state the timed steps started from, through the C ABI with host
        # buffers: every step copies its input in and its result out.  The first set_state is a new state
        # (the step history is dropped, so that step runs without the predictor); later ones hand back the
        # state the context holds, which keeps the history.
        hbuf = hstart
        sv.t = t_start
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sv.set_state(hbuf.numpy(), t=sv.t)  # the step's input, at the context's time
            sv.step()
            sv.get_state(hbuf.numpy())
        torch.cuda.synchronize()
        wall = max_over_ranks(time.perf_counter() - t0, world)
        out["e2e"] = {"value": aggregate_value(dof, args.steps, wall, world), "unit": UNIT,
                      "h2d_bytes_per_step": dof * 8, "d2h_bytes_per_step": dof * 8}
    sv.close()
    return out


def summarize(S, res, precision, wl=None, args=None, subdomains=None):
    roof, spmv, step, kms, kcalls = roofline(S, res, precision)
    nits = [s["newton_its"] for s in res["stats"]]
    gits = [s["gmres_its"] for s in res["stats"]]
    out = {"value": res["value"], "unit": UNIT, "ms_per_step": res["ms_per_step"],
           "dtype": "f64" if precision == "fp64" else "f64+f32", "roofline": roof, "spmv": spmv,
           "step_roofline": step, "kernel_ms": {k: round(v, 3) for k, v in kms.items()}, "kernel_calls": kcalls,
           "newton_its_per_step": sum(nits) / len(nits), "gmres_its_per_step": sum(gits) / len(gits),
           "pc_setups": sum(s["pc_setups"] for s in res["stats"]), "gpu_launches": res["launches"],
           "clocks": res["clocks"], "create_s": round(res["create_s"], 2),
           "launch_shapes": {k: res["info"][k] for k in ("spmv_threads", "cgs_ctas", "cgs_tile", "ilu_batch", "ilu_warps", "ilu_ring")},
           "device_bytes": res["info"]["device_bytes"], "coarse_units": res["info"]["coarse_units"]}
    if wl is not None:
        out["config"] = workload_config(wl, args, subdomains)
    return out


def measure_ensemble(S, I, args, stream, world, local):
    """An ensemble of args.ensemble rate samples (each of the ten calibrated rates log-uniform within
    +-50% of the base) on the 256x256 urban square, 16 subdomains per sample: one context, one
    block-diagonal system, every kernel launch covers all samples.  The GMRES restart cycles run as
    replays of a captured CUDA graph (options.graph); the eager loop is timed beside it."""
    import numpy as np
    import torch
    import torch.distributed as dist
    wl = I.ontario_workload(256 * 256, seed=args.seed, structured=True, nside=256)
    samples = I.rate_samples(wl.params, args.ensemble, args.seed)
    u0 = torch.tensor(np.concatenate([wl.U0] * len(samples)), device="cuda")
    res = {}
    for mode in ("eager", "graph"):
        sv = S.Solver(wl.xy, wl.tri, samples, stream=stream, dt=wl.dt, graph=1 if mode == "graph" else 0,
                      **solver_options(args, "fp64", 16, ilu_fill=0))
        sv.set_state(u0)
        for _ in range(args.warmup):
            sv.step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        launches0 = S.launch_count()
        e0.record(stream)
        stats = [sv.step() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        res[mode] = (max_over_ranks(e0.elapsed_time(e1), world), S.launch_count() - launches0, stats)
        sv.close()
    ms, launches, stats = res["graph"]
    dof = 5 * wl.n * len(samples)
    return {"workload": "ensemble of %d rate samples on the 256x256 urban square (%d unknowns)" % (len(samples), dof),
            "value": aggregate_value(dof, args.steps, ms * 1e-3, world), "unit": UNIT, "graph": True,
            "ms_per_step": ms / args.steps, "eager_ms_per_step": res["eager"][0] / args.steps,
            "n_samples": len(samples), "dtype": "f64", "gpu_launches": launches,
            "newton_its_per_step": sum(s["newton_its"] for s in stats) / len(stats),
            "gmres_its_per_step": sum(s["gmres_its"] for s in stats) / len(stats)}


def measure_adjoint(S, I, args, stream):
    """Discrete adjoint of a 30-day run (60 steps of half a day) on the 256x256 urban square, checkpoints every 5
    steps, misfit of I and D at 50 seeded nodes observed daily, gradient w.r.t. the 10 rates and the per-node
    transmission field; timed against the same 60 forward steps."""
    import numpy as np
    import torch
    wl = I.ontario_workload(256 * 256, seed=args.seed, structured=True, nside=256)
    rng = np.random.default_rng(args.seed)
    nodes = np.sort(rng.choice(wl.n, 50, replace=False)).astype(np.int32)
    steps = np.arange(2, 61, 2, dtype=np.int32)
    field = np.ones(wl.n)
    opts = solver_options(args, "fp64", 16, ilu_fill=0)
    opts.update(pc_keep_steps=0, predictor=0)
    sv = S.Solver(wl.xy, wl.tri, wl.params, beta_field=field, stream=stream, dt=wl.dt, **opts)
    u0 = torch.tensor(wl.U0, device="cuda")
    sv.set_state(u0)
    obs = []
    for k in range(1, 61):
        sv.step()
        if k % 2 == 0:
            obs.append(sv.get_state()[nodes])
    obs = np.array(obs)
    I_hat, D_hat = 1.1 * obs[:, :, 2], 0.9 * obs[:, :, 4]  # misfit of a perturbed observation
    sv.set_state(u0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sv.run(60)
    torch.cuda.synchronize()
    fwd = time.perf_counter() - t0
    sv.set_state(u0)
    t0 = time.perf_counter()
    j, g, gb = sv.adjoint(60, nodes, steps, I_hat, D_hat, checkpoint_every=5)
    torch.cuda.synchronize()
    adj = time.perf_counter() - t0
    sv.close()
    return {"workload": "30-day discrete adjoint on the 256x256 urban square (327680 unknowns), checkpoints every 5 "
                        "steps, 50 observed nodes", "seconds": adj, "forward_seconds": fwd, "ratio_to_forward": adj / fwd,
            "misfit": j, "gradient_entries": int(g.size + gb.size)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2208_01839_gb300 import build as B
    B.build()
    from paper_2208_01839_gb300 import inputs as I
    from paper_2208_01839_gb300 import seird as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()

    t_setup = time.perf_counter()
    wl = I.ontario_workload(args.nodes, seed=args.seed, n_subdomains=args.subdomains)
    t_gen = time.perf_counter() - t_setup
    cfg_main = workload_config(wl, args, args.subdomains)

    res = measure(S, wl, args, stream, args.precision, args.subdomains, world, local, e2e=not args.no_e2e)
    other = None
    if not args.no_mixed and args.precision == "fp64":
        other = measure(S, wl, args, stream, "mixed", args.subdomains, world, local, e2e=False)
    del wl

    two = None
    if not args.no_2m and args.nodes != 2_000_000:
        wl2 = I.ontario_workload(2_000_000, seed=args.seed, n_subdomains=512)
        args2 = argparse.Namespace(**vars(args))
        args2.ilu_fill = args2.ilu_fill_mixed = args.ilu_fill_2m
        r64 = measure(S, wl2, args2, stream, "fp64", 512, world, local, e2e=False)
        r32 = measure(S, wl2, args2, stream, "mixed", 512, world, local, e2e=False)
        two = summarize(S, r64, "fp64", wl2, args2, 512)
        two["mixed"] = summarize(S, r32, "mixed")
        two["mixed"]["speedup_vs_fp64"] = r32["value"] / r64["value"]
        del wl2

    ens = None
    if args.ensemble > 0:
        ens = measure_ensemble(S, I, args, stream, world, local)
    adj = None
    if not args.no_adjoint and rank == 0:
        adj = measure_adjoint(S, I, args, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = run_oracle_sample(CPU_BASELINE_NODES, 1, 0, args.seed)
        except Exception as ex:  # reported, never fatal
            cpu = {"error": str(ex)[:300]}

    if rank == 0:
        main = summarize(S, res, args.precision)
        line = {
            "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": main["dtype"],
            "data": "synthetic (seeded Southern-Ontario-like mesh, density and infection seeds)",
            "config": dict(cfg_main, precision=args.precision,
                           parallelism="replicas" if world > 1 else "single GPU"),
            "roofline": main["roofline"], "spmv": main["spmv"], "step_roofline": main["step_roofline"],
            "cpu_baseline": cpu, "e2e": res.get("e2e"), "gpu_launches": res["launches"], "clocks": res["clocks"],
            "kernel_ms": main["kernel_ms"], "kernel_calls": main["kernel_calls"],
            "newton_its_per_step": main["newton_its_per_step"], "gmres_its_per_step": main["gmres_its_per_step"],
            "pc_setups": main["pc_setups"],
            "setup_s": {"generate": round(t_gen, 2), "create": round(res["create_s"], 2)},
            "launch_shapes": main["launch_shapes"], "device_bytes": main["device_bytes"],
            "coarse_units": main["coarse_units"],
            "paper_context": "the paper's 92.57M-unknown Southern Ontario forecast: three months in under seven "
                             "hours on 1780 processes (its estimate from scaling runs; Section 4.2)",
        }
        if other is not None:
            m = summarize(S, other, "mixed")
            m["speedup_vs_fp64"] = other["value"] / res["value"]
            m["subdomain_solver"] = "block ILU(%d)" % args.ilu_fill_mixed
            line["mixed"] = m
        if two is not None:
            line["ontario_2m"] = two
        if ens is not None:
            line["ensemble"] = ens
        if adj is not None:
            line["adjoint"] = adj
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = run_oracle_sample(REFERENCE_NODES, args.steps, args.warmup, args.seed)
    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * res["s_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "Southern-Ontario-like 24-gon, %d P1 nodes (timed on a %d-node sample)"
                               % (args.nodes, REFERENCE_NODES), "dt_days": 0.5, "newton_rtol": 1e-8},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "host_cores": os.cpu_count(), "sample": res["sample"],
                         "value": res["value"], "unit": UNIT},
        "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# FP64 rates of the GPU (the measurement behind the no-tensor-core decision)
# ---------------------------------------------------------------------------

def run_fp64_probe(args):
    """FP64 FMA rate (an elementwise kernel of 1024 dependent-chain-free FMA groups per
    element, compiled at run time by torch's jiterator) and torch.matmul float64
    (cuBLAS DGEMM) TFLOP/s, best of 5, CUDA events, clocks sampled meanwhile."""
    import torch
    torch.cuda.set_device(0)
    out = {}
    with ClockSampler(0) as clk:
        # DGEMM
        n = 8192
        a = torch.randn(n, n, dtype=torch.float64, device="cuda")
        b = torch.randn(n, n, dtype=torch.float64, device="cuda")
        torch.matmul(a, b)
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out["dgemm"] = {"n": n, "ms": best, "tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12}
        del a, b
        # FMA loop: eight independent chains per element, 128 FMAs each
        code = """
        template <typename T> T fma_probe(T x, T y) {
          T a0 = x, a1 = x + 1, a2 = x + 2, a3 = x + 3, a4 = x + 4, a5 = x + 5, a6 = x + 6, a7 = x + 7;
          for (int i = 0; i < 128; ++i) {
            a0 = a0 * y + x; a1 = a1 * y + x; a2 = a2 * y + x; a3 = a3 * y + x;
            a4 = a4 * y + x; a5 = a5 * y + x; a6 = a6 * y + x; a7 = a7 * y + x;
          }
          return a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
        }"""
        fn = torch.cuda.jiterator._create_jit_fn(code)
        m = 1 << 26
        x = torch.rand(m, dtype=torch.float64, device="cuda")
        y = torch.full((m,), 0.999, dtype=torch.float64, device="cuda")
        fn(x, y)
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(x, y)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        fmas = m * 8 * 128
        out["fma_loop"] = {"elements": m, "fma_per_element": 1024, "ms": best,
                           "tflops": 2.0 * fmas / (best * 1e-3) / 1e12}
    out["clocks"] = clk.summary()
    out["gpu"] = torch.cuda.get_device_name(0)
    print(json.dumps({"fp64_probe": out}))


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample_child(args.oracle_sample)
        return
    if args.cpu_ladder:
        run_cpu_ladder(args)
        return
    if args.fp64_probe:
        run_fp64_probe(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
