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
    (z-, y-, x-, x+, y+, z+) of the column, from the cells' grid
    coordinates (the one coordinate in which row and column cell differ)."""
    N = rowptr.size - 1
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    coord = lambda c: (c % nx, (c // nx) % ny, c // (nx * ny))
    xi, yi, zi = coord(rows)
    xj, yj, zj = coord(col)
    slot = np.zeros(col.size, np.int32)
    for k, m in enumerate((zj < zi, yj < yi, xj < xi, xj > xi, yj > yi, zj > zi)):
        slot[m] = k + 1
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


def advance_one_step(solver, prob, max_newton=8):
    """The problem one backward-Euler step later: Newton on the GPU from
    (p_n, T_n), and the result as both the previous time level and the
    first iterate of the next step. Within time stepping the temperature
    front makes S~_T differ from the exact Schur complement by about a per
    cent, where at a uniform first step it is exact to about 1e-7."""
    p, T, info = solver.newton_step(prob["p_n"], prob["T_n"], prob["dt"], max_newton=max_newton)
    nxt = dict(prob)
    nxt.update(p_n=p, T_n=T, p_k=p.copy(), T_k=T.copy())
    return nxt


def concat(parts):
    return {k: np.concatenate([p[k] for p in parts]) for k in ("X", "slot", "St", "Sd", "target")}


def train(data, params0, epochs=40, batch=4096, lr=2e-3, seed=0, val_frac=0.1):
    """Mini-batch Adam on the GPU with model selection: a held-out share
    `val_frac` of the samples scores the parameters after every epoch, and
    the network ends with the best-scoring ones, the untrained identity
    correction (epoch 0) included, so training never returns a correction
    that is worse than plain S~ on held-out entries. Returns (mlp, per-epoch
    mean training loss); mlp.val_losses and mlp.selected_epoch record the
    selection."""
    mlp = thermo.MLP(params0)
    rng = np.random.Generator(np.random.PCG64(seed))
    n = data["target"].size
    perm0 = rng.permutation(n)
    nval = int(round(val_frac * n)) if n >= 20 else 0
    vidx, tidx = perm0[:nval], perm0[nval:]
    pick = lambda idx: [data[k][idx] for k in ("X", "slot", "St", "Sd", "target")]
    val = pick(vidx) if nval else None
    score = (lambda: mlp.gradient(*val)[0]) if val else (lambda: 0.0)
    best, best_ep = mlp.params(), 0
    vl = [score()]
    hist = []
    for ep in range(epochs):
        perm = tidx[rng.permutation(tidx.size)]
        losses = []
        for b0 in range(0, perm.size, batch):
            idx = perm[b0:b0 + batch]
            losses.append(mlp.train_step(*pick(idx), lr=lr))
        hist.append(float(np.mean(losses)))
        vl.append(score())
        if vl[-1] < vl[best_ep]:
            best, best_ep = mlp.params(), ep + 1
    mlp.set_params(best)
    mlp.val_losses = vl
    mlp.selected_epoch = best_ep
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
                plain_rel_res_unscaled=plain["rel_res_unscaled"],
                learned_iters=learned["iters"], learned_rel_res=learned["rel_res"],
                learned_rel_res_unscaled=learned["rel_res_unscaled"],
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
    ap.add_argument("--after-step", action="store_true",
                    help="train and evaluate at the start of a second time step (behind "
                         "the temperature front of the first), where S~_T is not exact")
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
        if a.after_step:
            prob = advance_one_step(s, prob)
        parts.append(collect_samples(s, prob, a.cols, rng))
    data = concat(parts)
    t1 = time.time()
    mlp, hist = train(data, flatten(initial_params(0)), epochs=a.epochs)
    t2 = time.time()
    shape = tuple(int(v) for v in a.eval_shape.split(","))
    evals = []
    for q in range(a.eval):
        prob = make_problem("grf96", seed=5000 + q, shape=shape)
        if a.after_step:
            es = thermo.Solver.from_problem(prob)
            prob = advance_one_step(es, prob)
            es.close()
        evals.append(evaluate(mlp, prob))
    if a.out:
        np.save(a.out, mlp.params())
    print(json.dumps(dict(samples=int(data["target"].size), probe_s=t1 - t0, train_s=t2 - t1,
                          loss_first=hist[0], loss_last=hist[-1],
                          val_loss_identity=mlp.val_losses[0],
                          val_loss_selected=mlp.val_losses[mlp.selected_epoch],
                          selected_epoch=mlp.selected_epoch, after_step=a.after_step,
                          eval=evals)))


if __name__ == "__main__":
    main()
