#!/usr/bin/env python
"""Benchmark of the hot path on one GB300 per rank.

One step = set the cell fields, assemble the Newton system (Sec. 2.2,
Eq. AXR), build the block preconditioner (S~_T of Eq. Se plus one AMG
hierarchy each for A_pp and S~_T) and solve with FGMRES(30) to relative
residual 1e-8 (Sec. 3.2, Sec. 4 settings), all through the C-ABI library.

Workload (default): the first Newton system of the 256x256x64 layered
time-step recipe (4,194,304 cells, 8,388,608 unknowns, eight layers of
log-permeability, five-spot, 30-day step). Metric: unknowns per second of
the whole step with the plain S~_T and FP64 hierarchies (higher is better;
ms_per_step is the time to relative residual 1e-8 in both the
equation-scaled and the unscaled 2-norm). The variant line carries the same
for FP32 hierarchies with the learned S~ correction; both carry an
end-to-end figure through host buffers. V-cycle bandwidth (algorithmic
bytes of one V-cycle over its event time) and the CUDA-event roofline of
the largest kernel class are measured after the timed regions.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--config RECIPE] [--shape NX,NY,NZ]

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

METRIC = ("unknowns/s (assemble + preconditioner setup + FGMRES to relative residual 1e-8 "
          "in the scaled and the unscaled 2-norm)")
# the oracle's bounded sample of the workload: the same recipe at 32x32x16
CPU_SAMPLE_SHAPE = (32, 32, 16)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="layered256", choices=sorted(RECIPE_SHAPES),
                    help="workload recipe (default: the 256x256x64 layered recipe)")
    ap.add_argument("--shape", default=None,
                    help="run the recipe at another grid shape nx,ny,nz (profiling cuts)")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=600)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-shape", default="32,32,16",
                    help="grid shape of the bounded sample of the workload recipe that the "
                         "reference arm times per step")
    ap.add_argument("--no-variant", action="store_true",
                    help="skip the FP32-hierarchy + learned-Schur variant")
    ap.add_argument("--train-problems", type=int, default=16)
    ap.add_argument("--train-shape", default="32,32,16",
                    help="grid of the training problems (the workload recipe, seeds 1000..)")
    ap.add_argument("--nu", type=int, default=None,
                    help="l1-Jacobi sweeps of A_pp's hierarchy before and after (default: the "
                         "library's 3 and 4)")
    ap.add_argument("--sell-rows", type=int, default=None,
                    help="minimum rows of a level's sliced-ELL copy (default: the library's "
                         "half a wave of resident threads; -1 never, 1 every level between the "
                         "finest and the coarsest)")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--sequence", type=int, default=0,
                    help="run this many backward-Euler steps with Newton (e.g. on "
                         "layered256) instead of the single-system benchmark")
    ap.add_argument("--adaptive-days", type=float, default=0.0,
                    help="--sequence mode with adaptive steps instead: simulate this many days, "
                         "steps sized for about 4 Newton iterations (Sec. 4), at most the "
                         "recipe's step, starting from it")
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
    ap.add_argument("--probe", type=int, default=3,
                    help="kernel class timed for the roofline: 0 finest A_pp sweep, "
                         "1 finest S~ line step, 2 block SpMV, 3 A_pp level-1 CSR sweep "
                         "(default: the largest class of the layered step)")
    ap.add_argument("--vcycle-reps", type=int, default=20)
    ap.add_argument("--single", action="store_true",
                    help="one untimed assemble + build + solve of the workload with the default "
                         "options (no clock sampler, no measurement passes): the command the "
                         "launch lists and kernel profiles are captured on")
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
               1: "k_line_sweep (finest S~ level, vertical-line step)",
               2: "k_block_spmv (2x2 block-CSR SpMV, FP64)",
               3: "k_jacobi (A_pp level 1, l1-Jacobi sweep, CSR)"}
# class 3 when level 1 keeps a sliced-ELL copy (levels of a full wave of
# resident threads or more)
PROBE_NAME_SLICED = "k_sell_jacobi (A_pp level 1, l1-Jacobi sweep, sliced ELL)"


def nu_kw(args):
    """A_pp's sweep counts (--nu overrides both) and the sliced-ELL threshold
    (--sell-rows): the library defaults unless given."""
    kw = {} if args.nu is None else {"nu_pre": args.nu, "nu_post": args.nu}
    if args.sell_rows is not None:
        kw["sell_rows"] = args.sell_rows
    return kw


def shape_of(text):
    return tuple(int(v) for v in text.split(",")) if text else None


# FP64 FMA peak of the GB300 (a bound of the FP64 sparse kernels next to
# HBM: ncu shows the FP64 pipe 85 % busy where DRAM is 39 % in the CSR sweep
# with lanes per row, 69 % and 54 % in the sliced-ELL sweep): 2 DFMA per clock per SM
# (ncu sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained) x 152
# SMs x 2 flops x 2.07 GHz maximum SM clock
FP64_TFLOPS = 2 * 152 * 2 * 2.07e9 / 1e12

# probe classes that run in FP64 with the FP64 pipe as a bound next to HBM,
# and the algorithmic FP64 flops of one launch from the probed level's size:
# 2 per matrix entry (multiply-add) + 3 per row (b - Ax, scaling, update)
ALU_PROBES = {3: (0, 1)}  # probe -> (hierarchy, level)


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the probed
# kernel class of the current kernels, keyed by (recipe, shape, probe,
# level 1 sliced, precision); absent until captured. The 256x256x64 figures
# are scaled from a capture of the same kernel on the recipe at 160x160x64
# (one pass over the level's stored slots and rows, so the traffic grows in
# proportion).
TRAFFIC = {
    # sliced-ELL sweep at 160x160x64 (15,413,760 stored slots): FP64 198.73 +
    # 4.77 MB, FP32 131.21 + 3.66 MB per launch; scaled by the stored slots of
    # the 256x256x64 level (39,624,512; rows scale by 2.562, slots by 2.571)
    ("layered256", (256, 256, 64), 3, True, 0): 203.50e6 * 39624512 / 15413760,
    ("layered256", (256, 256, 64), 3, True, 1): 134.87e6 * 39624512 / 15413760,
}


def cpu_baseline(recipe, seconds_target=10.0):
    """The oracle (as it stands) on a bounded sample of the same recipe: one
    or more assemble + setup + solve passes at 32x32x16, single thread."""
    from oracle import krylov as okry
    prob = make_problem(recipe, shape=CPU_SAMPLE_SHAPE)
    N = prob["nx"] * prob["ny"] * prob["nz"]
    t0 = time.perf_counter()
    runs = 0
    while True:
        out = okry.solve(prob, rtol=1e-8)
        runs += 1
        if time.perf_counter() - t0 >= seconds_target:
            break
    t = (time.perf_counter() - t0) / runs
    nx, ny, nz = CPU_SAMPLE_SHAPE
    return {"value": 2 * N / t, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
            "sample": f"{runs} assemble+setup+solve passes of the {recipe} recipe at "
                      f"{nx}x{ny}x{nz} ({2 * N} unknowns, {out['iters']} FGMRES its, "
                      f"{t:.1f} s each, single thread)",
            "host_cores": os.cpu_count()}


def arm_config(recipe, shape, args, world, precision="fp64 plain S~_T"):
    """The workload description of a line: the recipe and the grid timed."""
    nx, ny, nz = shape
    n2 = 2 * nx * ny * nz
    full = tuple(RECIPE_SHAPES[recipe]) == tuple(shape)
    where = "" if full else f" at {nx}x{ny}x{nz}"
    return {"workload": f"{recipe}: {WORKLOAD[recipe]}{where}, {n2} unknowns, "
                        f"first Newton system",
            "grid": [nx, ny, nz], "unknowns": n2,
            "rtol": args.rtol, "solver": precision,
            "nu": args.nu if args.nu is not None else [3, 4], "restart": args.restart,
            "sell_rows": args.sell_rows if args.sell_rows is not None else "half a wave",
            "l2": "flushed (512 MB write) before every timed step; inputs > L2",
            "parallelism": f"replicas{world}"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle timed on the host cores, each step
    one assemble + setup + solve of a bounded sample (--ref-shape) of the
    workload recipe."""
    if rank != 0:
        return
    from oracle import krylov as okry
    shape = shape_of(args.ref_shape)
    prob = make_problem(args.config, shape=shape)
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
        "config": arm_config(args.config, shape, args, world),
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                         "sample": f"one assemble+setup+solve per step of the {args.config} "
                                   f"recipe on a {prob['nx']}x{prob['ny']}x{prob['nz']} grid "
                                   f"({2 * N} unknowns), single thread; value in unknowns of "
                                   f"the sample per second"},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "fgmres_iters": int(np.median(its)),
    }
    print(json.dumps(line), flush=True)


def train_schur_model(args, after_step=False, recipe="grf32"):
    """Train the learned Schur correction on the GPU (untimed): exact Schur
    columns probed on --train-problems seeded problems of `recipe` at
    --train-shape (seeds 1000..), 128 columns each, 40 epochs of Adam; with
    after_step the systems are those at the start of a second time step
    (behind a temperature front), as in a time-step sequence."""
    from paper_1902_00095_gb300 import learned as L
    from paper_1902_00095_gb300 import thermo
    from synthetic.mlp import flatten, initial_params
    t0 = time.perf_counter()
    rng = np.random.Generator(np.random.PCG64(12345))
    shape = shape_of(args.train_shape)
    parts = []
    ts = None
    for q in range(args.train_problems):
        tp = make_problem(recipe, seed=1000 + q, shape=shape)
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
    shape = shape_of(args.shape) or tuple(RECIPE_SHAPES[args.config])
    prob = make_problem(args.config, shape=shape)
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
    pin = lambda a: torch.as_tensor(a, dtype=torch.float64).contiguous().pin_memory()
    hf = [pin(prob[k]) for k in ("Kx", "Ky", "Kz", "phi", "kTr")]
    hs = [pin(prob[k]) for k in ("p_k", "T_k", "p_n", "T_n")]
    hx = (torch.empty(N, dtype=torch.float64).pin_memory(),
          torch.empty(N, dtype=torch.float64).pin_memory())
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    plain = thermo.default_opts(precision=args.precision, **nu_kw(args))

    def step(opts, rtol):
        s.set_fields(*fields)
        s.assemble(*state, prob["dt"], R_m=Rm, R_e=Re)
        s.build(opts)
        return s.solve(rtol=rtol, maxit=args.maxit, restart=args.restart, out=(xp, xT))[2]

    def step_host(opts, rtol):
        # end to end: inputs from pinned host memory, solution back to it
        s.set_fields(*hf)
        s.assemble(*hs, prob["dt"])
        s.build(opts)
        return s.solve(rtol=rtol, maxit=args.maxit, restart=args.restart, out=hx)[2]

    def warm(opts):
        """W untimed warm-up steps; the FGMRES tolerance (a bound on the
        equation-scaled residual) is halved until the solution also meets
        the target in the unscaled 2-norm."""
        rtol = args.rtol
        w = 0
        while True:
            info = step(opts, rtol)
            w += 1
            if info["rel_res_unscaled"] > args.rtol and rtol > args.rtol / 1024:
                rtol *= 0.5
                continue
            if w >= max(1, args.warmup):
                return rtol

    def timed(opts, rtol):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = thermo.kernel_launches()
        t0 = time.perf_counter()
        infos = []
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            evs[k][0].record(stream)
            infos.append(step(opts, rtol))
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        launches = thermo.kernel_launches() - l0
        if world > 1:
            dist.barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, infos, launches, wall

    def e2e_run(opts, rtol):
        if args.no_e2e:
            return None
        step_host(opts, rtol)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host(opts, rtol)
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / args.steps
        if world > 1:
            t = torch.tensor([te], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        # per step: five fields and four states in, x_p and x_T out
        return {"value": world * 2 * N / te, "unit": "unknowns/s",
                "h2d_bytes_per_step": 9 * N * 8, "d2h_bytes_per_step": 2 * N * 8,
                "ms_per_step": te * 1e3}

    def solver_summary(infos, rtol):
        last = infos[-1]
        out = {k: last[k] for k in ("iters", "restarts", "levels_pp", "levels_S", "opc_pp",
                                    "opc_S", "t_solve_ms")}
        out.update(rtol_scaled_stop=rtol,
                   max_rel_res=max(i["rel_res"] for i in infos),
                   max_rel_res_unscaled=max(i["rel_res_unscaled"] for i in infos),
                   max_rel_res_p=max(i["rel_res_p"] for i in infos),
                   max_rel_res_T=max(i["rel_res_T"] for i in infos))
        return out

    peak, peak_kind = measured_peak()

    def vcycles(opts):
        """Untimed: each hierarchy's V-cycle replayed as a graph (the timed
        build's hierarchies), algorithmic bytes / event time."""
        out = {}
        for which, name in ((0, "A_pp"), (1, "S")):
            m = s.vcycle_measure(which, args.vcycle_reps)
            m["frac"] = m["gbs"] / peak if m["gbs"] else None
            out[name] = m
        return out

    clk = ClockSampler(local)
    clk.start()
    # ---- FP64 plain
    rtol64 = warm(plain)
    ms, infos, launches, wall = timed(plain, rtol64)
    value = world * 2 * N / (ms * 1e-3)
    e2e = e2e_run(plain, rtol64)
    step(plain, rtol64)
    vc64 = vcycles(plain)
    setup64 = {"A_pp": s.setup_timings(0), "S": s.setup_timings(1)}
    # ---- variant: FP32 hierarchies + learned Schur correction (network
    # trained untimed on probed exact Schur columns of the same recipe)
    variant = None
    if not args.no_variant:
        mlp, hist, t_train = train_schur_model(args, recipe=args.config)
        s.set_schur_model(mlp)
        vopts = thermo.default_opts(precision=1, schur=1, **nu_kw(args))
        rtol32 = warm(vopts)
        vms, vinfos, vlaunches, _ = timed(vopts, rtol32)
        ve2e = e2e_run(vopts, rtol32)
        step(vopts, rtol32)
        fb_rows, fb_all = s.learned_status()
        variant = {"name": "fp32 hierarchy + learned S~ (FP64 FGMRES)", "ms_per_step": vms,
                   "value": world * 2 * N / (vms * 1e-3), "unit": "unknowns/s",
                   "speedup_vs_fp64_plain": ms / vms, "e2e": ve2e,
                   "solver": solver_summary(vinfos, rtol32),
                   "vcycle": vcycles(vopts),
                   "gpu_launches": int(vlaunches),
                   "learned_fallback_rows": fb_rows, "learned_global_fallback": fb_all,
                   "training": {"recipe": args.config, "shape": args.train_shape,
                                "problems": args.train_problems, "columns_per_problem": 128,
                                "loss_first": hist[0], "loss_last": hist[-1],
                                "val_loss_identity": mlp.val_losses[0],
                                "val_loss_selected": mlp.val_losses[mlp.selected_epoch],
                                "selected_epoch": mlp.selected_epoch,
                                "seconds_untimed": t_train}}
    clocks = clk.stop()
    # ---- roofline of the probed kernel class (untimed FP64 pass: the probe's
    # events sit between the kernels of the captured preconditioner graph)
    def probe_pass(opts, rtol, precision):
        s.probe_enable(args.probe)
        step(opts, rtol)
        pr = s.probe_read(reset=True)
        levels = s.hierarchy_info(0)  # before the probe is switched off (that unbuilds)
        sliced = args.probe == 3 and s.level_storage(0, 1)[0] == 2
        s.probe_enable(-1)
        nl = max(1, pr["launches"])
        gbs = pr["bytes"] / (pr["ms"] * 1e-3) / 1e9 if pr["ms"] > 0 else None
        hbm = {"achieved": gbs, "peak": peak, "unit": "GB/s",
               "frac": gbs / peak if gbs else None,
               "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst copy)"}
        name = PROBE_NAME_SLICED if sliced else PROBE_NAMES[args.probe]
        out = {"kernel": name + (" FP32" if precision else " FP64"),
               "traffic": TRAFFIC.get((args.config, shape, args.probe, sliced, precision)),
               "launches_timed": pr["launches"], "avg_launch_us": pr["ms"] * 1e3 / nl,
               "algorithmic_bytes_per_launch": pr["bytes"] / nl}
        if precision == 0 and args.probe in ALU_PROBES and pr["ms"] > 0:
            # the FP64 sweep has two bounds: the FP64 FMA pipe and HBM; the
            # one it reaches the larger fraction of is reported as the bound
            # (CSR with lanes per row: the pipe, 85 % busy in ncu; sliced
            # ELL: HBM, the pipe 66 % busy), the other nested beside it
            which, level = ALU_PROBES[args.probe]
            n_l, nnz_l = levels if which == 0 else s.hierarchy_info(which)
            flops = 2.0 * float(nnz_l[level]) + 3.0 * float(n_l[level])
            tf = flops / (pr["ms"] * 1e-3 / nl) / 1e12
            alu = {"achieved": tf, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                   "frac": tf / FP64_TFLOPS,
                   "peak_kind": "FP64 FMA pipe: 2 DFMA/clock/SM x 152 SMs x 2 flops x 2.07 GHz "
                                "(unit counts and clock)",
                   "algorithmic_flops_per_launch": flops}
            if hbm["frac"] is not None and hbm["frac"] >= alu["frac"]:
                out.update({"bound": "hbm", **{k: hbm[k] for k in ("achieved", "peak", "unit",
                                                                   "frac", "peak_kind")},
                            "alu": alu})
            else:
                out.update({"bound": "alu", **alu, "hbm": hbm})
        else:
            out.update({"bound": "hbm", **{k: hbm[k] for k in ("achieved", "peak", "unit",
                                                               "frac", "peak_kind")}})
        return out

    roofline = probe_pass(plain, rtol64, args.precision)
    if variant is not None:
        s.set_schur_model(mlp)
        variant["roofline"] = probe_pass(vopts, rtol32, 1)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f64+f32",
        "data": "synthetic",
        "config": arm_config(args.config, shape, args, world),
        "e2e": e2e,
        "variant": variant,
        "vcycle": vc64,
        "roofline": roofline,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed": wall,
        "solver": solver_summary(infos, rtol64),
        "setup_ms": setup64,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.config)
    print(json.dumps(line), flush=True)


def run_single(args, rank, world, local):
    """One assemble + preconditioner build + FGMRES solve, nothing else."""
    import torch
    from paper_1902_00095_gb300 import thermo
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shape = shape_of(args.shape) or tuple(RECIPE_SHAPES[args.config])
    prob = make_problem(args.config, shape=shape)
    N = prob["nx"] * prob["ny"] * prob["nz"]
    s = thermo.Solver.from_problem(prob)
    d = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()
    st = [d(prob[k]) for k in ("p_k", "T_k", "p_n", "T_n")]
    xp = torch.empty(N, dtype=torch.float64, device=dev)
    xT = torch.empty(N, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.assemble(*st, prob["dt"])
    s.build(thermo.default_opts(precision=args.precision, **nu_kw(args)))
    info = s.solve(rtol=args.rtol, maxit=args.maxit, restart=args.restart, out=(xp, xT))[2]
    torch.cuda.synchronize()
    if rank == 0:
        # per level: rows, entries, storage format (0 CSR, 1 ELL, 2 sliced
        # ELL) and stored entries (padding included)
        levels = {name: [[int(a), int(b), *s.level_storage(w, l)]
                         for l, (a, b) in enumerate(zip(*s.hierarchy_info(w)))]
                  for w, name in ((0, "A_pp"), (1, "S"))}
        print(json.dumps({"single_step": f"{args.config} {shape}", "precision": args.precision,
                          "iters": info["iters"], "status": info["status"],
                          "ms": (time.perf_counter() - t0) * 1e3,
                          "launches": thermo.kernel_launches(),
                          "levels_rows_nnz": levels}), flush=True)


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
        opts = thermo.default_opts(precision=1, schur=1, **nu_kw(args))
        train = {"problems": args.train_problems, "loss_first": hist[0], "loss_last": hist[-1],
                 "selected_epoch": mlp.selected_epoch, "seconds_untimed": t_train}
    else:
        opts = thermo.default_opts(precision=args.precision, **nu_kw(args))
    d = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()
    p, T = d(prob["p_n"]), d(prob["T_n"])
    from paper_1902_00095_gb300.timestep import advance, simulate
    steps = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.adaptive_days > 0:
        p, T, rec = simulate(s, p, T, args.adaptive_days * 86400.0, prob["dt"], dt_max=prob["dt"],
                             target=4, max_cuts=args.max_cuts, max_newton=args.max_newton,
                             tol_f=1e-8, tol_dx=1e-8, rtol=args.rtol, maxit=args.maxit,
                             restart=args.restart, reuse=True, opts=opts)
        for r in rec:
            steps.append({"t_days": r["t"] / 86400.0, "dt_days": r["dt"] / 86400.0,
                          "accepted": r["accepted"], "status": r["status"],
                          "newton_iters": r.get("newton_iters", 0),
                          "linear_iters": r.get("linear_iters", 0),
                          "line_search_halvings": r.get("line_search_halvings", 0),
                          "t_ms": r.get("t_ms", 0.0)})
    for k in range(0 if args.adaptive_days > 0 else args.sequence):
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
    if args.adaptive_days > 0:
        acc = [r for r in steps if r["accepted"]]
        nacc = max(1, len(acc))
        print(json.dumps({
            "metric": "simulated days per second (adaptive backward-Euler steps, Newton + "
                      "block-preconditioned FGMRES)",
            "value": args.adaptive_days / wall, "unit": "days/s", "n_gpus": world,
            "higher_is_better": True,
            "dtype": "f64+f32" if (args.sequence_variant or args.precision) else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.config}: {WORKLOAD[args.config]}, "
                                   f"{args.adaptive_days:g} days, adaptive steps",
                       "unknowns": 2 * N, "max_newton": args.max_newton,
                       "max_cuts": args.max_cuts, "dt_max_days": prob["dt"] / 86400.0,
                       "solver": "fp32 hierarchy + learned S~" if args.sequence_variant else
                                 ("fp32 hierarchy" if args.precision else "fp64 plain")},
            "wall_s": wall, "steps_accepted": len(acc), "solves": len(steps),
            "all_converged": all(r["status"] == 0 for r in acc),
            "newton_per_step": sum(r["newton_iters"] for r in steps) / nacc,
            "linear_per_newton": sum(r["linear_iters"] for r in steps) /
                                 max(1, sum(r["newton_iters"] for r in steps)),
            "steps_detail": steps,
            "learned": (dict(train, fallback=s.learned_status()) if train else None),
            "final_T_range": [float(T.min()), float(T.max())],
            "final_p_range": [float(p.min()), float(p.max())],
        }), flush=True)
        return
    print(json.dumps({
        "metric": "backward-Euler steps (Newton + block-preconditioned FGMRES) per second",
        "value": args.sequence / wall, "unit": "steps/s", "n_gpus": world, "steps": args.sequence,
        "ms_per_step": wall * 1e3 / args.sequence, "higher_is_better": True,
        "dtype": "f64+f32" if (args.sequence_variant or args.precision) else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.config}: {WORKLOAD[args.config]}, {args.sequence} steps",
                   "unknowns": 2 * N, "nu": args.nu if args.nu is not None else [3, 4],
                   "restart": args.restart,
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
    elif args.single:
        run_single(args, rank, world, local)
    elif args.sequence > 0 or args.adaptive_days > 0:
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
