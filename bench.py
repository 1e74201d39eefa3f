"""Benchmark of the SEIRD backward-Euler Newton-Krylov-Schwarz step on GB300.

Metric: implicit DOF*steps/s at a 1e-8 relative Newton residual (DOF = 5 x
nodes), on the Southern-Ontario-like workload: a seeded 24-gon meshed to 2.0M
P1 nodes (10M unknowns), urban-Gaussian density, 5 infection seeds, dt = 0.5
day, RAS with 512 uneven subdomains, overlap 2, plus the constant coarse space.
A "step" is one backward-Euler time step (assembly, preconditioner set-up,
GMRES, line search) of that whole mesh.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (test infrastructure, not the product)
on the host cores, on a bounded sample of the same workload.  Under torchrun
(N > 1) every rank runs an independent replica of the workload (the path is one
coupled solve; it is not sharded across GPUs) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
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
# capture of each kernel class at this workload (profiles/); None until captured
# or after the kernel changed.
# (kernel class, precision) -> (bytes per launch at the captured small case,
# units processed there, seird_get_info key of those units); scaled to the
# full launch by the units it processes (traffic grows in proportion).
NCU_TRAFFIC = {
    ("spmv", "fp64"): (307.414e6, 1400635, "nnzb"),  # profiles/k_bsr_spmv_ontario200k.md
    ("ilu_solve", "fp64"): (373.090e6, 1577927, "subdomain_blocks"),  # profiles/k_ilu_solve_ontario200k.md (v9)
    ("ilu_solve", "mixed"): (202.650e6, 1577927, "subdomain_blocks"),  # same file, FP32 instantiation (v9)
}

# kernel classes with one kernel launch per timed call, and their algorithmic
# bytes per launch
SINGLE_KERNEL = ("spmv", "ilu_solve", "ilu_factor")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nodes", type=int, default=2_000_000)
    ap.add_argument("--subdomains", type=int, default=512)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--forcing", choices=["fixed", "ew"], default="ew")
    ap.add_argument("--pc-lag", type=int, default=20)
    ap.add_argument("--pc-keep", type=int, default=3, help="steps a preconditioner may be carried over")
    ap.add_argument("--predictor", type=int, choices=[0, 1], default=1,
                    help="Newton's first iterate: 0 u^n, 1 the extrapolation 2 u^n - u^{n-1}")
    ap.add_argument("--coarse", type=int, choices=[1, 2, 3], default=2,
                    help="1 additive coarse correction, 2 the paper's multiplicative two-grid (Eq. RAS_2L), "
                         "3 coarse correction then RAS")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--cgs2", action="store_true", help="re-orthogonalise (CGS2) instead of PETSc's single pass")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ensemble", type=int, default=64, help="samples of the ensemble line (0: skip it)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing line")
    ap.add_argument("--no-autotune", action="store_true", help="fixed launch shapes instead of the autotuner's")
    ap.add_argument("--oracle-sample", type=str, default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def workload_config(wl, args):
    return {
        "workload": "%s (Southern-Ontario-like 24-gon, %d P1 nodes, %d unknowns)" % (wl.name, wl.n, 5 * wl.n),
        "n_nodes": wl.n, "n_tris": int(len(wl.tri)), "dof": 5 * wl.n, "dt_days": wl.dt,
        "subdomains": args.subdomains, "overlap": 2,
        "coarse": {1: "additive", 2: "multiplicative two-grid (Eq. RAS_2L)",
                   3: "coarse correction, then RAS"}[args.coarse] + ", constant per subdomain and compartment",
        "subdomain_solver": "block ILU(0)",
        "krylov": "FGMRES(30) right-preconditioned, %s, rtol 1e-5" % (
            "CGS2" if args.cgs2 else "classical Gram-Schmidt single pass (PETSc default)"),
        "newton_rtol": 1e-8, "quadrature": "degree-5 seven-point", "seed": args.seed,
        "l2": "inputs larger than L2 (the FP64 Jacobian alone is > 2.7 GB)",
    }


# ---------------------------------------------------------------------------
# CPU oracle sample (run in a child process with one BLAS thread)
# ---------------------------------------------------------------------------

SAMPLE_NODES = 20_000


def oracle_sample_child(spec):
    """Times the oracle (as it stands) on the same generator at SAMPLE_NODES."""
    from oracle import seird_oracle as O
    from paper_2208_01839_gb300 import inputs as I
    d = json.loads(spec)
    wl = I.ontario_workload(d["nodes"], seed=d["seed"])
    U = wl.U0
    times = []
    for k in range(d["warmup"] + d["steps"]):
        t0 = time.perf_counter()
        U, info = O.newton_step(wl.xy, wl.tri, wl.params, wl.dt, U, rtol=1e-8)
        if k >= d["warmup"]:
            times.append(time.perf_counter() - t0)
    print(json.dumps({"n": wl.n, "dof": 5 * wl.n, "times": times}))


def run_oracle_sample(nodes, steps, warmup, seed):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    spec = json.dumps({"nodes": nodes, "steps": steps, "warmup": warmup, "seed": seed})
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", spec], env=env,
                       capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: %s" % r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    tot = sum(out["times"])
    return {"value": out["dof"] * len(out["times"]) / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d steps of the same generator at %d nodes (%d DOF), Newton to 1e-8 with a SuperLU "
                      "direct solve, one thread" % (len(out["times"]), out["n"], out["dof"]),
            "s_per_step": tot / len(out["times"])}


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


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes(cls, info, precision="fp64"):
    """Bytes each launch of a kernel class must move at least (each array the
    kernel needs, read or written once); the mixed path stores matrix values,
    factors and the preconditioned basis in FP32."""
    n, nnzb = info["n_nodes"], info["nnzb"]
    nl, nlb = info["subdomain_rows"], info["subdomain_blocks"]
    w = 4 if precision == "mixed" else 8
    if cls == "spmv":  # values + column indices + row pointers + x once + y once (FP64)
        return nnzb * (25 * w + 4) + (n + 1) * 4 + 5 * n * w + 5 * n * 8
    if cls == "ilu_solve":  # factor blocks + columns + inverse diagonals + r gathered + z written
        return nlb * (25 * w + 4) + nl * (25 * w + 8 + 16) + nl * 5 * 8 + 5 * n * w
    if cls == "ilu_factor":  # J blocks gathered (FP64), factor blocks written, inverse diagonals written
        return nlb * (25 * 8 + 25 * w + 4 + 4) + nl * 25 * w
    return None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def measure(S, wl, args, stream, precision, forcing, pc_lag, world, local, e2e=True):
    """Warm-up, then K device-timed steps (and K end-to-end steps) of one variant."""
    import torch
    import torch.distributed as dist
    t_create = time.perf_counter()
    sv = S.Solver(wl.xy, wl.tri, wl.params, stream=stream, dt=wl.dt, n_subdomains=args.subdomains, overlap=2,
                  coarse=args.coarse, pc_keep_steps=args.pc_keep, predictor=args.predictor, newton_rtol=1e-8,
                  gmres_rtol=1e-5,
                  gmres_restart=30, gmres_maxit=200,
                  precision=1 if precision == "mixed" else 0, seed=args.seed, timing=1,
                  gmres_forcing=1 if forcing == "ew" else 0, pc_lag=pc_lag, gmres_one_pass=0 if args.cgs2 else 1,
                  autotune=0 if args.no_autotune else 1)
    info = sv.info()
    t_create = time.perf_counter() - t_create  # partition, patterns, level schedules, upload
    sv.set_state(torch.tensor(wl.U0, device="cuda"))
    for _ in range(args.warmup):
        sv.step()
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
           "launches": launches, "create_s": t_create,
           "clocks": clk.summary(), "info": info, "stats": stats}
    if e2e:
        hbuf = torch.empty((wl.n, 5), dtype=torch.float64, pin_memory=True)
        sv.get_state(hbuf.numpy())
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sv.set_state(hbuf.numpy())
            sv.step()
            sv.get_state(hbuf.numpy())
        torch.cuda.synchronize()
        wall = max_over_ranks(time.perf_counter() - t0, world)
        out["e2e"] = {"value": aggregate_value(dof, args.steps, wall, world), "unit": UNIT,
                      "h2d_bytes_per_step": dof * 8,
                      "d2h_bytes_per_step": dof * 8}
    sv.close()
    return out


def measure_ensemble(S, I, args, stream, world, local):
    """An ensemble of args.ensemble rate samples (each of the ten calibrated rates log-uniform within
    +-50% of the base) on the 256x256 urban square, 16 subdomains per sample: one context, one
    block-diagonal system, every kernel launch covers all samples.  Device-timed like the main line."""
    import numpy as np
    import torch
    import torch.distributed as dist
    wl = I.ontario_workload(256 * 256, seed=args.seed, structured=True, nside=256)
    samples = I.rate_samples(wl.params, args.ensemble, args.seed)
    sv = S.Solver(wl.xy, wl.tri, samples, stream=stream, dt=wl.dt, n_subdomains=16, overlap=2, coarse=args.coarse,
                  pc_keep_steps=args.pc_keep, predictor=args.predictor, newton_rtol=1e-8, gmres_rtol=1e-5,
                  gmres_restart=30, gmres_maxit=200,
                  seed=args.seed, gmres_forcing=1, pc_lag=args.pc_lag, gmres_one_pass=0 if args.cgs2 else 1)
    sv.set_state(torch.tensor(np.concatenate([wl.U0] * len(samples)), device="cuda"))
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
    launches = S.launch_count() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    sv.close()
    dof = 5 * wl.n * len(samples)
    return {"workload": "ensemble of %d rate samples on the 256x256 urban square (%d unknowns)" % (len(samples), dof),
            "value": aggregate_value(dof, args.steps, ms * 1e-3, world), "unit": UNIT,
            "ms_per_step": ms / args.steps, "n_samples": len(samples), "dtype": "f64", "gpu_launches": launches,
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
    sv = S.Solver(wl.xy, wl.tri, wl.params, beta_field=field, stream=stream, dt=wl.dt, n_subdomains=16, overlap=2,
                  coarse=args.coarse, newton_rtol=1e-8, gmres_rtol=1e-5, gmres_restart=30, gmres_maxit=200,
                  seed=args.seed, gmres_forcing=1, pc_lag=args.pc_lag, gmres_one_pass=0 if args.cgs2 else 1)
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


def kernel_summary(S, res):
    stats, info = res["stats"], res["info"]
    kms = {k: sum(s["kernel_ms"][k] for s in stats) for k in S.KERNEL_CLASSES}
    kcalls = {k: sum(s["kernel_calls"][k] for s in stats) for k in S.KERNEL_CLASSES}
    return kms, kcalls


# GB300's nominal FP64 rate (no FP64 tensor path beyond the FP64 pipe's 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 1.25


def algorithmic_fma(cls, info):
    """FP64 FMAs one launch must perform: 25 per 5x5 block product."""
    if cls == "spmv":
        return 25 * info["nnzb"]
    if cls == "ilu_solve":  # forward L blocks + backward U blocks + the inverted pivots = every local block
        return 25 * info["subdomain_blocks"]
    return None


def roofline(S, res, precision, coarse=2):
    kms, kcalls = kernel_summary(S, res)
    info = res["info"]
    peak, peak_kind = hbm_peak()
    dom = max(SINGLE_KERNEL, key=lambda k: kms[k])
    ab = algorithmic_bytes(dom, info, precision)
    avg_ms = kms[dom] / max(kcalls[dom], 1)
    achieved = ab / (avg_ms * 1e-3) / 1e9
    traffic = None
    tr = NCU_TRAFFIC.get((dom, precision))
    if tr is not None:
        bytes_small, units_small, unit_key = tr
        traffic = bytes_small * info[unit_key] / units_small
    sp_ab = algorithmic_bytes("spmv", info, precision)
    # with the multiplicative two-grid every coarse application follows an SpMV that also
    # reads r (it computes r - J z): those launches move 5n FP64 values more
    fused = kcalls["coarse_apply"] if coarse == 2 else 0
    if kcalls["spmv"]:
        sp_ab = sp_ab + min(fused, kcalls["spmv"]) / kcalls["spmv"] * 5 * info["n_nodes"] * 8
    sp_ms = kms["spmv"] / max(kcalls["spmv"], 1)
    sp_gbs = sp_ab / (sp_ms * 1e-3) / 1e9 if kcalls["spmv"] else None
    fma = algorithmic_fma(dom, info) if precision == "fp64" else None
    alu = None
    if fma is not None:
        tf = 2.0 * fma / (avg_ms * 1e-3) / 1e12
        alu = {"achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
               "peak_kind": "nominal FP64 (profiling recipe)", "fma_per_launch": fma}
    return ({"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
             "frac": achieved / peak, "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind ==
             "measured" else peak_kind, "traffic": traffic, "algorithmic_bytes_per_launch": ab,
             "avg_launch_ms": avg_ms, "launches": kcalls[dom], "fp64_alu": alu},
            {"gbs": sp_gbs, "frac_of_hbm": (sp_gbs / peak) if sp_gbs else None, "avg_launch_ms": sp_ms,
             "launches": kcalls["spmv"], "algorithmic_bytes": sp_ab},
            kms, kcalls)


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

    res = measure(S, wl, args, stream, args.precision, args.forcing, args.pc_lag, world, local,
                  e2e=not args.no_e2e)
    other = None
    if not args.no_mixed and args.precision == "fp64":
        other = measure(S, wl, args, stream, "mixed", args.forcing, args.pc_lag, world, local, e2e=False)

    ens = None
    if args.ensemble > 0:
        ens = measure_ensemble(S, I, args, stream, world, local)
    adj = None
    if not args.no_adjoint and rank == 0:
        adj = measure_adjoint(S, I, args, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = run_oracle_sample(SAMPLE_NODES, 2, 0, args.seed)
        except Exception as ex:  # reported, never fatal
            cpu = {"error": str(ex)[:300]}

    if rank == 0:
        roof, spmv, kms, kcalls = roofline(S, res, args.precision, args.coarse)
        nits = [s["newton_its"] for s in res["stats"]]
        gits = [s["gmres_its"] for s in res["stats"]]
        line = {
            "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic (seeded Southern-Ontario-like mesh, density and infection seeds)",
            "config": dict(workload_config(wl, args), precision=args.precision,
                           forcing="Eisenstat-Walker" if args.forcing == "ew" else "fixed rtol 1e-5",
                           pc_lag=args.pc_lag, pc_keep_steps=args.pc_keep, predictor=args.predictor,
                           parallelism="replicas" if world > 1 else "single GPU"),
            "roofline": roof, "spmv": spmv, "cpu_baseline": cpu, "e2e": res.get("e2e"),
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "kernel_ms": {k: round(v, 3) for k, v in kms.items()}, "kernel_calls": kcalls,
            "newton_its_per_step": sum(nits) / len(nits), "gmres_its_per_step": sum(gits) / len(gits),
            "setup_s": {"generate": round(t_gen, 2), "create": round(res["create_s"], 2)},
            "launch_shapes": {k: res["info"][k] for k in ("spmv_threads", "cgs_ctas", "cgs_tile")},
            "device_bytes": res["info"]["device_bytes"],
        }
        if other is not None:
            r2, s2, k2, c2 = roofline(S, other, "mixed", args.coarse)
            g2 = [s["gmres_its"] for s in other["stats"]]
            line["mixed"] = {"value": other["value"], "ms_per_step": other["ms_per_step"],
                             "speedup_vs_fp64": other["value"] / res["value"], "dtype": "f64+f32",
                             "roofline": r2, "spmv": s2, "kernel_ms": {k: round(v, 3) for k, v in k2.items()},
                             "gmres_its_per_step": sum(g2) / len(g2), "gpu_launches": other["launches"],
                             "clocks": other["clocks"]}
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
    res = run_oracle_sample(SAMPLE_NODES, args.steps, args.warmup, args.seed)
    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * res["s_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "Southern-Ontario-like 24-gon, %d P1 nodes (timed on a %d-node sample)"
                               % (args.nodes, SAMPLE_NODES), "dt_days": 0.5, "newton_rtol": 1e-8},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": res["sample"], "value": res["value"], "unit": UNIT},
        "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample_child(args.oracle_sample)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
