"""Write the stored oracle references of the full-size parity tests.

Calls only oracle/ (and the seeded input recipes of synthetic/):

  ref_<name>.npz   the oracle's solution x* = (x_p, x_T) of the first Newton
                   system of a workload recipe, by the oracle's FGMRES to a
                   scaled relative residual of 1e-13 (a tighter truth than
                   the 1e-8 solutions it checks), stored as float32 (its
                   rounding, 6e-8 relative, is far below the 1e-6 bound
                   checked against it), with the oracle's iteration count
                   and residuals;
  amg_<name>.json  SHA-256 digests of every level of the oracle's AMG
                   hierarchies of that system's A_pp (extended+i) and S~_T
                   (classical), truncation to 4 weights, theta 0.25, seed 0,
                   coarsening down to 256 rows: C/F split, strength mask,
                   interpolation pattern and values, and the level's
                   operator (pattern and values), each hashed in a fixed
                   byte layout (int8 flags, int32 indices, float64 values,
                   little endian); the patterns alone are hashed as well
                   ("A_pattern", "P_pattern").

    python tests/golden/make_references.py [grf64] [layered64] [--amg-only]

grf64 is the 64x64x32 recipe; layered64 the 256x256x64 layered recipe cut to
64x64x64 (all eight layers of eight cells, a sixteenth of the columns).
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import amg, krylov  # noqa: E402
from synthetic import make_problem  # noqa: E402

CASES = {
    "grf64": lambda: make_problem("grf64"),
    "layered64": lambda: make_problem("layered256", shape=(64, 64, 64)),
}
AMG_OPTS = {"App": dict(interp="ext+i"), "S": dict(interp="classical")}


def digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def level_digests(hier):
    out = []
    levels = hier["levels"]
    for l, lev in enumerate(levels):
        A = lev["A"]
        rec = {"n": int(lev["n"]), "nnz": int(A[1].size),
               "A": digest(A[0].astype("<i4"), A[1].astype("<i4"), A[2].astype("<f8")),
               "A_pattern": digest(A[0].astype("<i4"), A[1].astype("<i4"))}
        if "cf" in lev:
            P = lev["P"]
            rec["cf"] = digest(lev["cf"].astype("<i1"))
            rec["strong"] = digest(lev["S"].astype("<i1"))
            rec["P"] = digest(P[0].astype("<i4"), P[1].astype("<i4"), P[2].astype("<f8"))
            rec["P_pattern"] = digest(P[0].astype("<i4"), P[1].astype("<i4"))
        out.append(rec)
    return out


def make(name, solve=True):
    prob = CASES[name]()
    t0 = time.time()
    if solve:
        out = krylov.solve(prob, rtol=1e-13, maxit=600, restart=30)
        N = out["sys"].N
        x = out["x"]
        np.savez_compressed(os.path.join(HERE, f"ref_{name}.npz"),
                            x_p=x[:N].astype(np.float32), x_T=x[N:].astype(np.float32),
                            iters=out["iters"], rel_res=out["rel_res"],
                            rel_res_unscaled=out["rel_res_unscaled"])
        print(f"{name}: FGMRES {out['iters']} its, scaled {out['rel_res']:.2e}, unscaled "
              f"{out['rel_res_unscaled']:.2e} ({time.time() - t0:.0f} s)", flush=True)
        sys_, S = out["sys"], out["S"]
    else:
        sys_, _, _, S = krylov.assemble(prob)
    rec = {"seed": 0, "theta": 0.25, "coarse_size": 256, "pmax": 4, "hierarchies": {}}
    for which, A in (("App", sys_.App), ("S", S)):
        h = amg.setup(A, theta=0.25, seed=0, coarse_size=256, pmax=4, **AMG_OPTS[which])
        rec["hierarchies"][which] = {"interp": AMG_OPTS[which]["interp"],
                                     "levels": level_digests(h)}
    with open(os.path.join(HERE, f"amg_{name}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(f"{name}: hierarchies written ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    names = [a for a in sys.argv[1:] if not a.startswith("--")] or list(CASES)
    for name in names:
        make(name, solve="--amg-only" not in sys.argv)
