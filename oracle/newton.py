"""Oracle: Newton iteration of one backward-Euler step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3: at each Newton iterate x_k solve dG/dx|_{x_k} dx = -G(x_k)
(Eq. AXR); Sec. 4: Newton's method with line search, stopped on relative
function norm and relative step 1e-8. The paper does not give the line
search; the reading here is backtracking on the function norm: take
x_k + alpha dx with alpha = 1, 1/2, 1/4, ... the first time
||G(x_k + alpha dx)|| <= (1 - 1e-4 alpha) ||G(x_k)||, accepting the sixth
halving whatever its norm. The function norm is measured in the equation
scaling D of the first linearisation (see krylov.py).
"""
import numpy as np

from . import krylov, physics


MAX_HALVINGS = 6
ARMIJO = 1e-4


def _norm(D, bp, bT):
    return np.sqrt(np.sum((D[0] * bp) ** 2) + np.sum((D[1] * bT) ** 2))


def newton_step(prob, max_newton=3, tol_f=1e-8, tol_dx=1e-8, linear="direct", rtol=1e-10,
                line_search=True):
    """Returns (p, T, history) where history lists (rel_f, rel_dx, alpha)
    per iteration (the last entry (rel_f, None, None) when the loop stops on
    the function norm or the iteration limit); `linear` is "direct" (sparse
    LU of the scaled system) or "fgmres" (the block-preconditioned FGMRES of
    krylov.solve); line_search=False takes full steps. A non-finite
    accepted iterate raises FloatingPointError."""
    p = prob["p_n"].copy()
    T = prob["T_n"].copy()
    hist = []
    sysb, bp, bT, S = krylov.assemble(prob, p, T)
    D = (sysb.s_m, sysb.s_e)
    G = G0 = _norm(D, bp, bT)
    for k in range(max_newton + 1):
        relf = G / G0 if G0 > 0 else 0.0
        if G == 0.0 or (k > 0 and relf <= tol_f) or k == max_newton:
            hist.append((relf, None, None))
            break
        if linear == "direct":
            dp, dT = krylov.direct_solution(sysb, bp, bT)
        else:
            out = krylov.solve(prob, rtol=rtol, p=p, T=T)
            dp, dT = out["x"][:p.size], out["x"][p.size:]
        alpha = 1.0
        for h in range(MAX_HALVINGS + 1 if line_search else 1):
            pt, Tt = p + alpha * dp, T + alpha * dT
            with np.errstate(all="ignore"):
                try:
                    sysb, bp, bT, S = krylov.assemble(prob, pt, Tt)
                    Gt = _norm(D, bp, bT)
                except (FloatingPointError, ValueError):
                    Gt = np.inf
            last = not line_search or h == MAX_HALVINGS
            if (np.isfinite(Gt) and Gt <= (1.0 - ARMIJO * alpha) * G) or last:
                if not np.isfinite(Gt):
                    raise FloatingPointError("non-finite Newton iterate")
                break
            alpha *= 0.5
        p, T, G = pt, Tt, Gt
        reldx = alpha * np.sqrt(np.sum(dp ** 2) + np.sum(dT ** 2)) / np.sqrt(np.sum(p ** 2) + np.sum(T ** 2))
        hist.append((relf, reldx, alpha))
        if reldx <= tol_dx:
            break
    return p, T, hist
