"""Oracle: Newton iteration of one backward-Euler step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3: at each Newton iterate x_k solve dG/dx|_{x_k} (x_{k+1} - x_k) =
-G(x_k) (Eq. AXR); Sec. 4 stops on relative function norm and relative step
1e-8. Full steps (no line search, a reading: the paper's line search is not
specified). The function norm is measured in the equation scaling D of the
first linearisation (see krylov.py).
"""
import numpy as np

from . import krylov, physics


def newton_step(prob, max_newton=3, tol_f=1e-8, tol_dx=1e-8, linear="direct", rtol=1e-10):
    """Returns (p, T, history) where history lists (rel_f, rel_dx) per
    iteration; `linear` is "direct" (sparse LU of the scaled system) or
    "fgmres" (the block-preconditioned FGMRES of krylov.solve)."""
    p = prob["p_n"].copy()
    T = prob["T_n"].copy()
    hist = []
    G0 = None
    D = None
    for k in range(max_newton + 1):
        sysb, bp, bT, S = krylov.assemble(prob, p, T)
        if D is None:
            D = (sysb.s_m, sysb.s_e)
        G = np.sqrt(np.sum((D[0] * bp) ** 2) + np.sum((D[1] * bT) ** 2))
        if G0 is None:
            G0 = G
        relf = G / G0 if G0 > 0 else 0.0
        if G == 0.0 or (k > 0 and relf <= tol_f) or k == max_newton:
            hist.append((relf, None))
            break
        if linear == "direct":
            dp, dT = krylov.direct_solution(sysb, bp, bT)
        else:
            out = krylov.solve(prob, rtol=rtol, p=p, T=T)
            dp, dT = out["x"][:p.size], out["x"][p.size:]
        p = p + dp
        T = T + dT
        reldx = np.sqrt(np.sum(dp ** 2) + np.sum(dT ** 2)) / np.sqrt(np.sum(p ** 2) + np.sum(T ** 2))
        hist.append((relf, reldx))
        if reldx <= tol_dx:
            break
    return p, T, hist
