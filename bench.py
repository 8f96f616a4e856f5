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

from synthetic import make_problem  # noqa: E402

METRIC = "unknowns/s (assemble + preconditioner setup + FGMRES to rel-res 1e-8)"
CPU_SAMPLE = "4train"  # the 64x64x32 recipe at 32x32x16 (1/8 of the cells)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="2")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=600)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--probe", type=int, default=0,
                    help="kernel timed for the roofline: 0 finest A_pp sweep, "
                         "1 finest S~ sweep, 2 block SpMV")
    a = ap.parse_args()
    a.config = int(a.config) if a.config.isdigit() else a.config
    return a


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
# kernel, keyed by (config, probe); None until a capture of the current kernel
TRAFFIC = {("2", 0, 0): 14.16e6,   # profiles/k_jacobi_ell_config2_64x64x32_fp64.md
           ("3", 0, 0): 118.3e6}  # profiles/k_jacobi_ell_config3_128x128x64_fp64.md


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


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    if rank != 0:
        return
    from oracle import krylov as okry
    prob = make_problem(CPU_SAMPLE)
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
        "config": {"workload": "64x64x32 five-spot recipe, bounded sample 32x32x16",
                   "grid": [32, 32, 16], "unknowns": 2 * N, "rtol": args.rtol},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                         "sample": "32x32x16 grid of the 64x64x32 recipe per step, single thread"},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "fgmres_iters": int(np.median(its)),
    }
    print(json.dumps(line), flush=True)


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
    opts = thermo.default_opts(precision=args.precision)
    s.probe_enable(args.probe)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    def step():
        s.set_fields(*fields)
        s.assemble(*state, prob["dt"], R_m=Rm, R_e=Re)
        s.build(opts)
        return s.solve(rtol=args.rtol, maxit=args.maxit, out=(xp, xT))[2]

    torch.cuda.synchronize()
    for _ in range(args.warmup):
        info = step()
    # timed region: K steps, L2 flushed before each (flush not timed)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clk = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
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
                "traffic": TRAFFIC.get((str(args.config), args.probe, args.precision)),
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
            return s.solve(rtol=args.rtol, maxit=args.maxit, out=hx)[2]

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

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f64+f32",
        "data": "synthetic",
        "config": {"workload": f"config {args.config}: {prob['nx']}x{prob['ny']}x{prob['nz']} five-spot, "
                               f"{2 * N} unknowns, one Newton system",
                   "grid": [prob["nx"], prob["ny"], prob["nz"]], "unknowns": 2 * N,
                   "rtol": args.rtol, "precision": "fp64" if args.precision == 0 else "fp32 hierarchy",
                   "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": f"replicas{world}"},
        "e2e": e2e,
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
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
