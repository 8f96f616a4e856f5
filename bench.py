#!/usr/bin/env python
"""Benchmark of the hot path on one GB300 per rank.

One step = set the cell fields, assemble the Newton system (Sec. 2.2,
Eq. AXR), build the block preconditioner (S~_T of Eq. Se plus one AMG
hierarchy each for A_pp and S~_T) and solve with FGMRES(30) to relative
residual 1e-8 (Sec. 3.2, Sec. 4 settings), all through the C-ABI library.

Workload: the 64x64x32 five-spot recipe (131,072 cells, 262,144 unknowns,
Gaussian-random-field log-permeability, 10-day step). Metric: unknowns per
second of the whole step (higher is better); time-to-1e-8 is ms_per_step.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU: the path does not shard here (replicas only): each rank solves its
own copy of the workload, value = total unknowns of all ranks / max time.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

# the CPU-baseline / reference legs time the single-threaded oracle
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import RECIPE_SHAPES, make_problem  # noqa: E402

METRIC = "unknowns/s (assemble + preconditioner setup + FGMRES to rel-res 1e-8)"
CPU_SAMPLE = "grf32"  # the 64x64x32 recipe at 32x32x16 (1/8 of the cells)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="grf64", choices=sorted(RECIPE_SHAPES),
                    help="workload recipe (default: the 64x64x32 five-spot)")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=600)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-sample", default=CPU_SAMPLE,
                    help="recipe the reference arm times per step (default: the 64x64x32 "
                         "recipe at 32x32x16)")
    ap.add_argument("--no-variant", action="store_true",
                    help="skip the FP32-hierarchy + learned-Schur variant")
    ap.add_argument("--train-problems", type=int, default=16)
    ap.add_argument("--nu", type=int, default=3, help="l1-Jacobi sweeps before and after")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--sequence", type=int, default=0,
                    help="run this many backward-Euler steps with Newton (e.g. on "
                         "layered256) instead of the single-system benchmark")
    ap.add_argument("--max-newton", type=int, default=4,
                    help="Newton iterations per time step in --sequence mode")
    ap.add_argument("--max-cuts", type=int, default=3,
                    help="--sequence: a step whose Newton iteration fails is repeated as two "
                         "halves, at most this many times")
    ap.add_argument("--scaling2d", action="store_true",
                    help="run the problem-size scaling study (2D Cases I-V) instead")
    ap.add_argument("--scaling-sizes", default="20,40,80,160,320")
    ap.add_argument("--sequence-variant", action="store_true",
                    help="--sequence with FP32 hierarchies + learned S~ (trained untimed)")
    ap.add_argument("--probe", type=int, default=0,
                    help="kernel timed for the roofline: 0 finest A_pp sweep, "
                         "1 finest S~ sweep, 2 block SpMV")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


PROBE_NAMES = {0: "k_jacobi_ell (finest A_pp level, l1-Jacobi sweep, ELL)",
               1: "k_jacobi_ell (finest S~ level, l1-Jacobi sweep, ELL)",
               2: "k_block_spmv (2x2 block-CSR SpMV, FP64)"}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the probed
# kernel, keyed by (recipe, probe, precision); None until a capture of the
# current kernel
TRAFFIC = {("grf64", 0, 0): 14.16e6,  # profiles/k_jacobi_ell_grf64_64x64x32_fp64.md
           ("channel128", 0, 0): 118.4e6}  # profiles/k_jacobi_ell_channel128_128x128x64_fp64.md


def cpu_baseline(seconds_target=20.0):
    """The oracle (as it stands) on a bounded sample of the same recipe."""
    from oracle import krylov as okry
    prob = make_problem(CPU_SAMPLE)
    N = prob["nx"] * prob["ny"] * prob["nz"]
    t0 = time.perf_counter()
    out = okry.solve(prob, rtol=1e-8)
    t = time.perf_counter() - t0
    return {"value": 2 * N / t, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
            "sample": f"one assemble+setup+solve of the 64x64x32 recipe at 32x32x16 "
                      f"({2 * N} unknowns, {out['iters']} FGMRES its, {t:.1f} s, single thread)",
            "host_cores": os.cpu_count()}


def arm_config(args, world):
    """The workload description both arms print (the reference arm times a
    bounded sample of it, described in its cpu_baseline)."""
    nx, ny, nz = RECIPE_SHAPES[args.config]
    n2 = 2 * nx * ny * nz
    return {"workload": f"{args.config}: {WORKLOAD[args.config]}, {n2} unknowns, "
                        f"one Newton system",
            "grid": [nx, ny, nz], "unknowns": n2,
            "rtol": args.rtol, "precision": "fp64" if args.precision == 0 else "fp32 hierarchy",
            "l2": "flushed (512 MB write) before every timed step",
            "parallelism": f"replicas{world}"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    if rank != 0:
        return
    from oracle import krylov as okry
    prob = make_problem(args.ref_sample)
    N = prob["nx"] * prob["ny"] * prob["nz"]
    for _ in range(args.warmup):
        okry.solve(prob, rtol=args.rtol)
    t0 = time.perf_counter()
    its = []
    for _ in range(args.steps):
        out = okry.solve(prob, rtol=args.rtol)
        its.append(out["iters"])
    dt = (time.perf_counter() - t0) / args.steps
    value = 2 * N / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(args, world),
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                         "sample": f"one assemble+setup+solve per step of the same recipe on a "
                                   f"{prob['nx']}x{prob['ny']}x{prob['nz']} grid ({2 * N} "
                                   f"unknowns), single thread; value in unknowns of the "
                                   f"sample per second"},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "fgmres_iters": int(np.median(its)),
    }
    print(json.dumps(line), flush=True)


def train_schur_model(args, after_step=False):
    """Train the learned Schur correction on the GPU (untimed): exact Schur
    columns probed on --train-problems seeded 32x32x16 problems of the
    64x64x32 recipe, 128 columns each, 40 epochs of Adam; with after_step the
    systems are those at the start of a second time step (behind a
    temperature front), as in a time-step sequence."""
    from paper_1902_00095_gb300 import learned as L
    from paper_1902_00095_gb300 import thermo
    from synthetic.mlp import flatten, initial_params
    t0 = time.perf_counter()
    rng = np.random.Generator(np.random.PCG64(12345))
    parts = []
    ts = None
    for q in range(args.train_problems):
        tp = make_problem("grf32", seed=1000 + q)
        if ts is None:
            ts = thermo.Solver.from_problem(tp)
        else:
            ts.set_fields(tp["Kx"], tp["Ky"], tp["Kz"], tp["phi"], tp["kTr"])
            ts.set_wells(tp["wells"])
        if after_step:
            tp = L.advance_one_step(ts, tp)
        parts.append(L.collect_samples(ts, tp, 128, rng))
    ts.close()
    mlp, hist = L.train(L.concat(parts), flatten(initial_params(0)), epochs=40)
    return mlp, hist, time.perf_counter() - t0


WORKLOAD = {
    "iid16": "16x16x8 i.i.d. log-normal permeability, two wells, 1-day step",
    "grf64": "64x64x32 Gaussian-random-field permeability, five-spot, 10-day step",
    "grf32": "32x32x16 Gaussian-random-field permeability, five-spot, 10-day step",
    "grf96": "96x96x48 Gaussian-random-field permeability, five-spot, 10-day step",
    "channel128": "128x128x64 channelised permeability, five-spot, 10-day step",
    "layered256": "256x256x64 layered permeability, five-spot, 30-day steps",
}


def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_1902_00095_gb300 import thermo

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = make_problem(args.config)
    N = prob["nx"] * prob["ny"] * prob["nz"]
    stream = torch.cuda.Stream(device=dev)
    s = thermo.Solver(prob["nx"], prob["ny"], prob["nz"], prob["fluid"], prob["dx"], prob["dy"],
                      prob["dz"], prob["g"], stream=stream.cuda_stream)
    s.set_wells(prob["wells"])
    d = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()
    fields = [d(prob[k]) for k in ("Kx", "Ky", "Kz", "phi", "kTr")]
    state = [d(prob[k]) for k in ("p_k", "T_k", "p_n", "T_n")]
    Rm = torch.empty(N, dtype=torch.float64, device=dev)
    Re = torch.empty(N, dtype=torch.float64, device=dev)
    xp = torch.empty(N, dtype=torch.float64, device=dev)
    xT = torch.empty(N, dtype=torch.float64, device=dev)
    opts = thermo.default_opts(precision=args.precision, nu_pre=args.nu, nu_post=args.nu)
    s.probe_enable(args.probe)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    def step():
        s.set_fields(*fields)
        s.assemble(*state, prob["dt"], R_m=Rm, R_e=Re)
        s.build(opts)
        return s.solve(rtol=args.rtol, maxit=args.maxit, restart=args.restart, out=(xp, xT))[2]

    # the clock sampler starts during the warm-up (nvidia-smi's own start-up
    # then falls outside the timed region) and samples until it ends
    clk = ClockSampler(local)
    torch.cuda.synchronize()
    for w in range(args.warmup):
        if w == args.warmup - 1:
            clk.start()
        info = step()
    if args.warmup == 0:
        clk.start()
    # timed region: K steps, L2 flushed before each (flush not timed)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    s.probe_read(reset=True)
    l0 = thermo.kernel_launches()
    t0 = time.perf_counter()
    infos = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        evs[k][0].record(stream)
        infos.append(step())
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = thermo.kernel_launches() - l0
    pr = s.probe_read(reset=True)
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    peak, peak_kind = measured_peak()
    achieved = pr["bytes"] / (pr["ms"] * 1e-3) / 1e9 if pr["ms"] > 0 else None
    roofline = {"bound": "hbm", "kernel": PROBE_NAMES[args.probe],
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst copy)",
                "traffic": TRAFFIC.get((args.config, args.probe, args.precision)),
                "launches_timed": pr["launches"],
                "avg_launch_us": pr["ms"] * 1e3 / max(1, pr["launches"]),
                "algorithmic_bytes_per_launch": pr["bytes"] / max(1, pr["launches"])}
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 2 * N / (ms * 1e-3)

    # end to end through the C-ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.as_tensor(a, dtype=torch.float64).contiguous().pin_memory()
        hf = [pin(prob[k]) for k in ("Kx", "Ky", "Kz", "phi", "kTr")]
        hs = [pin(prob[k]) for k in ("p_k", "T_k", "p_n", "T_n")]
        hx = (torch.empty(N, dtype=torch.float64).pin_memory(),
              torch.empty(N, dtype=torch.float64).pin_memory())

        def step_host():
            s.set_fields(*hf)
            s.assemble(*hs, prob["dt"])
            s.build(opts)
            return s.solve(rtol=args.rtol, maxit=args.maxit, restart=args.restart, out=hx)[2]

        step_host()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / args.steps
        if world > 1:
            t = torch.tensor([te], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        e2e = {"value": world * 2 * N / te, "unit": "unknowns/s",
               "h2d_bytes_per_step": 9 * N * 8, "d2h_bytes_per_step": 2 * N * 8 + 2 * N * 8,
               "ms_per_step": te * 1e3}

    # variant: FP32 hierarchy + learned Schur correction (network trained on
    # probed exact Schur columns of the 32x32x16 recipe before timing)
    variant = None
    if not args.no_variant:
        mlp, hist, t_train = train_schur_model(args)
        s.set_schur_model(mlp)
        # the same smoothing and restart as the FP64 run
        vopts = thermo.default_opts(precision=1, schur=1, nu_pre=args.nu, nu_post=args.nu)
        s.probe_enable(args.probe)

        def step_variant():
            s.set_fields(*fields)
            s.assemble(*state, prob["dt"], R_m=Rm, R_e=Re)
            s.build(vopts)
            return s.solve(rtol=args.rtol, maxit=args.maxit, restart=args.restart,
                           out=(xp, xT))[2]

        for _ in range(args.warmup):
            step_variant()
        torch.cuda.synchronize()
        s.probe_read(reset=True)
        vev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        vinfo = None
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            vev[k][0].record(stream)
            vinfo = step_variant()
            vev[k][1].record(stream)
        torch.cuda.synchronize()
        vms = sum(a.elapsed_time(b) for a, b in vev) / args.steps
        vpr = s.probe_read(reset=True)
        fb_rows, fb_all = s.learned_status()
        variant = {"name": "fp32 hierarchy + learned S~ (FP64 FGMRES)", "ms_per_step": vms,
                   "value": world * 2 * N / (vms * 1e-3), "unit": "unknowns/s",
                   "speedup_vs_fp64_plain": ms / vms, "iters": vinfo["iters"],
                   "rel_res": vinfo["rel_res"], "rel_res_unscaled": vinfo["rel_res_unscaled"],
                   "t_solve_ms": vinfo["t_solve_ms"],
                   "finest_sweep_gbs": (vpr["bytes"] / (vpr["ms"] * 1e-3) / 1e9) if vpr["ms"] > 0 else None,
                   "learned_fallback_rows": fb_rows, "learned_global_fallback": fb_all,
                   "training": {"problems": args.train_problems, "columns_per_problem": 128,
                                "loss_first": hist[0], "loss_last": hist[-1],
                                "val_loss_identity": mlp.val_losses[0],
                                "val_loss_selected": mlp.val_losses[mlp.selected_epoch],
                                "selected_epoch": mlp.selected_epoch,
                                "seconds_untimed": t_train}}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f64+f32",
        "data": "synthetic",
        "config": arm_config(args, world),
        "e2e": e2e,
        "variant": variant,
        "roofline": roofline,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed": wall,
        "solver": {k: infos[-1][k] for k in ("iters", "restarts", "rel_res", "rel_res_unscaled",
                                              "levels_pp", "levels_S", "opc_pp", "opc_S",
                                              "t_solve_ms")},
        "setup_ms": {"A_pp": s.setup_timings(0), "S": s.setup_timings(1)},
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def run_sequence(args, rank, world, local):
    """Backward-Euler time steps, each solved by Newton with line search (at
    most --max-newton linear solves, AMG structure reused between Newton
    iterations, a failed step repeated as two halves up to --max-cuts times)
    on one GPU; with --sequence-variant the hierarchies run in FP32 with the
    learned Schur correction."""
    import torch
    from paper_1902_00095_gb300 import thermo
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = make_problem(args.config)
    N = prob["nx"] * prob["ny"] * prob["nz"]
    s = thermo.Solver.from_problem(prob)
    train = None
    if args.sequence_variant:
        mlp, hist, t_train = train_schur_model(args, after_step=True)
        s.set_schur_model(mlp)
        opts = thermo.default_opts(precision=1, schur=1, nu_pre=args.nu, nu_post=args.nu)
        train = {"problems": args.train_problems, "loss_first": hist[0], "loss_last": hist[-1],
                 "selected_epoch": mlp.selected_epoch, "seconds_untimed": t_train}
    else:
        opts = thermo.default_opts(precision=args.precision, nu_pre=args.nu, nu_post=args.nu)
    d = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()
    p, T = d(prob["p_n"]), d(prob["T_n"])
    from paper_1902_00095_gb300.timestep import advance
    steps = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.sequence):
        p, T, rec = advance(s, p, T, prob["dt"], max_cuts=args.max_cuts,
                            max_newton=args.max_newton, tol_f=1e-8, tol_dx=1e-8, rtol=args.rtol,
                            maxit=args.maxit, restart=args.restart, reuse=True, opts=opts)
        acc = [r for r in rec if r["accepted"]]
        steps.append({"substeps": len(acc), "solves": len(rec),
                      "converged": all(r["status"] == 0 for r in acc),
                      "newton_iters": sum(r.get("newton_iters", 0) for r in rec),
                      "linear_iters": sum(r.get("linear_iters", 0) for r in rec),
                      "line_search_halvings": sum(r.get("line_search_halvings", 0) for r in rec),
                      "t_ms": sum(r.get("t_ms", 0.0) for r in rec),
                      "substep_days": [r["dt"] / 86400.0 for r in acc]})
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if rank != 0:
        return
    print(json.dumps({
        "metric": "backward-Euler steps (Newton + block-preconditioned FGMRES) per second",
        "value": args.sequence / wall, "unit": "steps/s", "n_gpus": world, "steps": args.sequence,
        "ms_per_step": wall * 1e3 / args.sequence, "higher_is_better": True,
        "dtype": "f64+f32" if (args.sequence_variant or args.precision) else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.config}: {WORKLOAD[args.config]}, {args.sequence} steps",
                   "unknowns": 2 * N, "nu": args.nu, "restart": args.restart,
                   "max_newton": args.max_newton, "max_cuts": args.max_cuts,
                   "solver": "fp32 hierarchy + learned S~" if args.sequence_variant else
                             ("fp32 hierarchy" if args.precision else "fp64 plain")},
        "steps_detail": steps,
        "learned": (dict(train, fallback=s.learned_status()) if train else None),
        "final_T_range": [float(T.min()), float(T.max())],
        "final_p_range": [float(p.min()), float(p.max())],
    }), flush=True)


# coarsest AMG grid of the scaling study: at most 64 rows at every size, so
# that even the 400-cell grid runs multi-level V-cycles, as the paper's hypre
# setup (coarsening down to a few rows) did; the library default (256) would
# solve the smallest grids' blocks exactly
SCALING_COARSE_SIZE = 64


def run_scaling2d(args, rank, world, local):
    """Sec. 4.3 problem-size scaling: Cases I-V on n x n grids of the 20 m
    square (n = 20..320), two time steps each, Newton with line search and
    FGMRES(30) to the paper's 1e-5, for the Schur approximations S~_T, S~_ATT
    and S~_diag; reports the average FGMRES iterations per Newton iteration
    (the quantity of the paper's Tables 7-11) and the wall time."""
    import torch
    from paper_1902_00095_gb300 import thermo
    from synthetic import scaling_case
    torch.cuda.set_device(local)
    sizes = [int(v) for v in args.scaling_sizes.split(",")]
    schurs = {"S_T": 0, "S_ATT": 2, "S_diag": 3}
    table = {}
    t0 = time.perf_counter()
    for case in (1, 2, 3, 4, 5):
        for name, sc in schurs.items():
            row = []
            for n in sizes:
                prob = scaling_case(case, n)
                s = thermo.Solver.from_problem(prob)
                p, T = prob["p_n"], prob["T_n"]
                newton = lin = 0
                ok = True
                for step in range(2):
                    try:
                        p, T, info = s.newton_step(p, T, prob["dt"], max_newton=10, tol_f=1e-8,
                                                   tol_dx=1e-8, rtol=1e-5, maxit=200,
                                                   restart=30, reuse=True, schur=sc,
                                                   coarse_size=SCALING_COARSE_SIZE)
                    except thermo.ThermoError:
                        ok = False
                        break
                    newton += info["newton_iters"]
                    lin += info["linear_iters"]
                    ok = ok and info["status"] == 0 and info["last_linear_status"] == 0
                s.close()
                row.append({"n": n, "newton": newton, "linear": lin,
                            "per_newton": (lin / newton) if newton else None, "converged": ok})
            table[f"case{case}/{name}"] = row
    wall = time.perf_counter() - t0
    if rank != 0:
        return
    print(json.dumps({"metric": "FGMRES iterations per Newton iteration (Sec. 4.3 scaling study)",
                      "sizes": sizes, "rtol": 1e-5, "wall_s": wall, "table": table}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if args.impl != "reference":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.sequence > 0:
        run_sequence(args, rank, world, local)
    elif args.scaling2d:
        run_scaling2d(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
