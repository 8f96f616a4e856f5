"""Training driver of the learned Schur correction.

Orchestration only: assembling, probing exact Schur columns, features, the
MLP's forward/backward and Adam all run in the CUDA library; this module
picks problems and columns, gathers the samples and loops over epochs.

    python -m paper_1902_00095_gb300.learned --problems 200 --cols 256

trains on the 32x32x16 recipe (seeds 1000..) and evaluates FGMRES
iterations with and without the correction on the 96x96x48 recipe
(seeds 5000..).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

from . import thermo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def direction_slots(rowptr, col, nx, ny):
    """0 for the diagonal entry of a row, 1..6 for the face direction
    (z-, y-, x-, x+, y+, z+) of the column."""
    N = rowptr.size - 1
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    d = col - rows
    slot = np.zeros(col.size, np.int32)
    for k, off in enumerate((-nx * ny, -nx, -1, 1, nx, nx * ny)):
        slot[d == off] = k + 1
    return rows, slot


def collect_samples(solver, prob, ncols, rng, rtol=1e-10):
    """Assemble prob, build the plain preconditioner and probe ncols exact
    Schur columns; returns the training samples of their pattern entries."""
    solver.assemble(prob["p_k"], prob["T_k"], prob["p_n"], prob["T_n"], prob["dt"])
    solver.build()
    X = solver.learned_features()
    rp, col, val, S, _ = solver.export_system()
    rows, slot = direction_slots(rp, col, prob["nx"], prob["ny"])
    dpos = np.array([rp[i] + np.searchsorted(col[rp[i]:rp[i + 1]], i) for i in range(solver.N)])
    cols = rng.choice(solver.N, size=min(ncols, solver.N), replace=False)
    entry, value, its, st = solver.probe_schur_columns(cols, rtol)
    ok = entry >= 0
    e = entry[ok]
    r = rows[e]
    return dict(X=X[r], slot=slot[e], St=S[e], Sd=S[dpos[r]], target=value[ok], probe_iters=its,
                probe_status=st)


def concat(parts):
    return {k: np.concatenate([p[k] for p in parts]) for k in ("X", "slot", "St", "Sd", "target")}


def train(data, params0, epochs=40, batch=4096, lr=2e-3, seed=0):
    """Mini-batch Adam on the GPU; returns (mlp, per-epoch mean loss)."""
    mlp = thermo.MLP(params0)
    rng = np.random.Generator(np.random.PCG64(seed))
    n = data["target"].size
    hist = []
    for ep in range(epochs):
        perm = rng.permutation(n)
        losses = []
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            losses.append(mlp.train_step(data["X"][idx], data["slot"][idx], data["St"][idx],
                                         data["Sd"][idx], data["target"][idx], lr=lr))
        hist.append(float(np.mean(losses)))
    return mlp, hist


def evaluate(mlp, prob, rtol=1e-8, maxit=600, **opts):
    """FGMRES iterations and true residual with plain and learned S~."""
    s = thermo.Solver.from_problem(prob)
    s.assemble(prob["p_k"], prob["T_k"], prob["p_n"], prob["T_n"], prob["dt"])
    s.build(schur=0, **opts)
    _, _, plain = s.solve(rtol=rtol, maxit=maxit)
    s.set_schur_model(mlp)
    s.build(schur=1, **opts)
    _, _, learned = s.solve(rtol=rtol, maxit=maxit)
    fb_rows, fb_all = s.learned_status()
    s.close()
    return dict(plain_iters=plain["iters"], plain_rel_res=plain["rel_res"],
                learned_iters=learned["iters"], learned_rel_res=learned["rel_res"],
                fallback_rows=fb_rows, global_fallback=fb_all)


def main():
    from synthetic import make_problem
    from synthetic.mlp import flatten, initial_params
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=200)
    ap.add_argument("--cols", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--eval", type=int, default=5)
    ap.add_argument("--eval-shape", default="96,96,48")
    ap.add_argument("--out", default=None, help="write trained parameters (.npy)")
    a = ap.parse_args()
    t0 = time.time()
    rng = np.random.Generator(np.random.PCG64(12345))
    parts = []
    s = None
    for q in range(a.problems):
        prob = make_problem("grf32", seed=1000 + q)
        if s is None:
            s = thermo.Solver.from_problem(prob)
        else:
            s.set_fields(prob["Kx"], prob["Ky"], prob["Kz"], prob["phi"], prob["kTr"])
            s.set_wells(prob["wells"])
        parts.append(collect_samples(s, prob, a.cols, rng))
    data = concat(parts)
    t1 = time.time()
    mlp, hist = train(data, flatten(initial_params(0)), epochs=a.epochs)
    t2 = time.time()
    shape = tuple(int(v) for v in a.eval_shape.split(","))
    evals = [evaluate(mlp, make_problem("grf96", seed=5000 + q, shape=shape)) for q in range(a.eval)]
    if a.out:
        np.save(a.out, mlp.params())
    print(json.dumps(dict(samples=int(data["target"].size), probe_s=t1 - t0, train_s=t2 - t1,
                          loss_first=hist[0], loss_last=hist[-1], eval=evals)))


if __name__ == "__main__":
    main()
