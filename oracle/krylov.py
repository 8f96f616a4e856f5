"""Oracle: block preconditioner (Sec. 3.2) and flexible GMRES (Sec. 4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Vectors of the coupled system are kept split as (p part, T part), each [N].

Equation scaling (a reading): the mass and energy rows differ by about ten
orders of magnitude in SI units, so the Krylov solve works on D A x = D b
with D = diag(s_m I, s_e I), s_m = N / sum_i |A_pp,ii|, s_e = N / sum_i
|A_TT,ii|. Because every V-cycle here is linear and homogeneous in the
matrix scale, the preconditioner for D A is M^{-1} D^{-1}; the solution x is
unchanged. The stopping test is ||D (b - A x)|| <= rtol ||D b||; the
unscaled relative residual is reported as well.
"""
import numpy as np
import scipy.sparse
import scipy.sparse.linalg

from . import amg, physics


# ------------------------------------------------------------ block algebra
class BlockSystem:
    """Block-CSR A with its four scalar blocks sharing one pattern."""

    def __init__(self, rowptr, col, val):
        self.rowptr, self.col, self.val = rowptr, col, val
        self.N = rowptr.size - 1
        App, ApT, ATp, ATT = physics.extract_blocks(val)
        self.App = (rowptr, col, App)
        self.ApT = (rowptr, col, ApT)
        self.ATp = (rowptr, col, ATp)
        self.ATT = (rowptr, col, ATT)
        d = amg.diag_positions(self.App)
        self.s_m = self.N / np.sum(np.abs(App[d]))
        self.s_e = self.N / np.sum(np.abs(ATT[d]))

    def matvec(self, xp, xT):
        """Eq. AXR: [A_pp A_pT; A_Tp A_TT] [x_p; x_T]."""
        return (amg.spmv(self.App, xp) + amg.spmv(self.ApT, xT),
                amg.spmv(self.ATp, xp) + amg.spmv(self.ATT, xT))

    def scipy(self):
        """The 2N x 2N matrix in interleaved ordering (2i = p_i, 2i+1 = T_i)."""
        N = self.N
        rows = np.repeat(np.arange(N), np.diff(self.rowptr))
        R, Cc, V = [], [], []
        for a in range(2):
            for b in range(2):
                R.append(2 * rows + a)
                Cc.append(2 * self.col + b)
                V.append(self.val[:, a, b])
        return scipy.sparse.csr_matrix(
            (np.concatenate(V), (np.concatenate(R), np.concatenate(Cc))), shape=(2 * N, 2 * N))


def block_preconditioner(sys, inv_pp, inv_S, variant="full"):
    """The five steps of Sec. 3.2 for y = M^{-1} b:
      1. x_p = A_pp^{-1} b_p
      2. bt_T = b_T - A_Tp x_p
      3. d_T = S~^{-1} bt_T
      4. bt_p = b_p - A_pT d_T       (the print reads x_p - A_pT d_T; b_p
                                      is the reading that reproduces
                                      Eq. Ainv with exact inverses)
      5. d_p = A_pp^{-1} bt_p
    variant "lower" stops after step 3 with d_p = x_p (block lower
    triangular preconditioner). inv_pp / inv_S are callables."""
    def apply(bp, bT):
        xp = inv_pp(bp)
        btT = bT - amg.spmv(sys.ATp, xp)
        dT = inv_S(btT)
        if variant == "lower":
            return xp, dT
        btp = bp - amg.spmv(sys.ApT, dT)
        return inv_pp(btp), dT
    return apply


# -------------------------------------------------------------------- FGMRES
def fgmres(matvec, precond, bp, bT, rtol=1e-8, maxit=300, restart=30):
    """Right-preconditioned flexible GMRES with restarts (Saad 1993), modified
    Gram-Schmidt Arnoldi and Givens rotations, zero initial guess. `matvec`
    and `precond` act on split (p, T) pairs. Stops when the Givens residual
    estimate reaches rtol ||b|| and the recomputed true residual confirms it,
    or after maxit iterations. Returns a dict with x, iterations, restarts,
    the true relative residual and the estimate history."""
    N = bp.size
    b = np.concatenate([bp, bT])
    bnorm = np.linalg.norm(b)
    x = np.zeros(2 * N)
    hist = []
    its = 0
    restarts = 0
    status = "not_converged"
    if bnorm == 0.0:
        return dict(x=x, iters=0, restarts=0, rel_res=0.0, hist=hist, status="converged")
    while True:
        yp, yT = matvec(x[:N], x[N:])
        r = b - np.concatenate([yp, yT])
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm:
            status = "converged"
            break
        if its >= maxit:
            break
        V = np.zeros((restart + 1, 2 * N))
        Z = np.zeros((restart, 2 * N))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        m = 0
        for j in range(restart):
            zp, zT = precond(V[j, :N], V[j, N:])
            Z[j] = np.concatenate([zp, zT])
            wp, wT = matvec(zp, zT)
            w = np.concatenate([wp, wT])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            m = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or its >= maxit:
                break
            hn = np.linalg.norm(w)
            if hn == 0.0:
                break
            V[j + 1] = w / hn
        y = np.zeros(m)
        for i in range(m - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:m] @ y[i + 1:m]) / H[i, i]
        x = x + Z[:m].T @ y
        restarts += 1
    yp, yT = matvec(x[:N], x[N:])
    rel = np.linalg.norm(b - np.concatenate([yp, yT])) / bnorm
    return dict(x=x, iters=its, restarts=restarts, rel_res=rel, hist=hist, status=status)


# ------------------------------------------------------------ whole solve
def assemble(prob, p=None, T=None):
    """Newton system at the iterate (p, T): A (block-CSR), b = -G(x_k) and
    the plain Schur approximation S~_T values on the same pattern."""
    p = prob["p_k"] if p is None else p
    T = prob["T_k"] if T is None else T
    rowptr, col, val = physics.jacobian(prob, p, T)
    Rm, Re = physics.residual(prob, p, T)
    _, _, Sv = physics.schur_approx(prob, p, T)
    return BlockSystem(rowptr, col, val), -Rm, -Re, (rowptr, col, Sv)


def solve(prob, rtol=1e-8, maxit=300, restart=30, theta=0.25, seed=0,
          variant="full", smoother="l1jacobi", nu_pre=3, nu_post=4,
          coarse_size=256, p=None, T=None, schur="plain", interp="ext+i",
          interp_S="classical", cheb_degree=2, pmax=4, smoother_S="line", nu_line=1,
          nu_S=1):
    """Assemble, build the block preconditioner with one V-cycle per
    approximate inverse, and solve with FGMRES(restart) in the scaled
    system. A_pp's hierarchy uses `interp` (extended+i by default: the
    elliptic pressure block), S~_T's uses `interp_S` (classical by default:
    under the gravity-driven upwind advection of S~_T extended+i produces
    weights above one and indefinite coarse operators). `smoother` is A_pp's
    smoother, `smoother_S` S~_T's: "line" (default) smooths the finest
    level of S~'s hierarchy by nu_line vertical-line Jacobi steps
    (amg.line_factor; grids with nz = 1 keep l1-Jacobi there) and the
    coarser levels by l1-Jacobi; "l1jacobi" everywhere; or "chebyshev"
    (on D^{-1} S~_T, whose spectrum is not real for the advective S~_T, it
    can amplify). S~'s hierarchy smooths its coarser levels (all levels
    without the line steps) with nu_S sweeps before and after (None: nu_pre
    and nu_post). Returns the FGMRES dict plus the pieces it used."""
    sys, bp, bT, S = assemble(prob, p, T)
    if schur == "att":
        S = sys.ATT
    elif schur == "diag":
        S = physics.schur_diag_sparse(sys.rowptr, sys.col, sys.val)
    h_pp = amg.setup(sys.App, theta, seed, coarse_size, smoother=smoother,
                     interp=interp, cheb_degree=cheb_degree, pmax=pmax)
    line = (prob["nx"] * prob["ny"], prob["nz"]) if smoother_S == "line" else None
    h_S = amg.setup(S, theta, seed, coarse_size,
                    smoother="l1jacobi" if smoother_S == "line" else smoother_S,
                    interp=interp_S, cheb_degree=cheb_degree, pmax=pmax, line=line,
                    nu_line=nu_line)
    sm, se = sys.s_m, sys.s_e
    V_pp = lambda r: amg.vcycle(h_pp, r, 0, nu_pre, nu_post)
    nS_pre, nS_post = (nu_pre, nu_post) if nu_S is None else (nu_S, nu_S)
    V_S = lambda r: amg.vcycle(h_S, r, 0, nS_pre, nS_post)
    M = block_preconditioner(sys, V_pp, V_S, variant)

    def matvec(xp, xT):
        yp, yT = sys.matvec(xp, xT)
        return sm * yp, se * yT

    def precond(vp, vT):
        return M(vp / sm, vT / se)

    out = fgmres(matvec, precond, sm * bp, se * bT, rtol, maxit, restart)
    N = sys.N
    x = out["x"]
    yp, yT = sys.matvec(x[:N], x[N:])
    b = np.concatenate([bp, bT])
    out["rel_res_unscaled"] = np.linalg.norm(b - np.concatenate([yp, yT])) / np.linalg.norm(b)
    out.update(sys=sys, bp=bp, bT=bT, S=S, h_pp=h_pp, h_S=h_S)
    return out


def direct_solution(sys, bp, bT):
    """Reference solution of A x = b by sparse LU (SuperLU) of the
    equation-scaled system D A x = D b (without the scaling the ten orders
    of magnitude between mass and energy rows cost SuperLU's pivoting about
    six digits); returns the split (x_p, x_T)."""
    N = sys.N
    b = np.empty(2 * N)
    d = np.empty(2 * N)
    b[0::2], b[1::2] = bp, bT
    d[0::2], d[1::2] = sys.s_m, sys.s_e
    A = scipy.sparse.diags(d) @ sys.scipy()
    x = scipy.sparse.linalg.spsolve(A.tocsc(), d * b)
    return x[0::2].copy(), x[1::2].copy()


def schur_condition_numbers(prob, p, T):
    """Sec. 4.2 (Table 4): 2-norm condition numbers of S~^{-1} S for the
    three Schur approximations (S~_diag, S~_ATT, S~_T) and of A_TT and the
    exact Schur complement S = A_TT - A_Tp A_pp^{-1} A_pT, all dense (small
    grids only)."""
    sys, bp, bT, S = assemble(prob, p, T)
    dense = lambda A: amg.to_dense(A)
    App, ApT, ATp, ATT = (dense(x) for x in (sys.App, sys.ApT, sys.ATp, sys.ATT))
    Sx = ATT - ATp @ np.linalg.solve(App, ApT)
    St = dense(S)
    Sd = physics.schur_diag(sys.rowptr, sys.col, sys.val)
    c = np.linalg.cond
    return dict(diag=c(np.linalg.solve(Sd, Sx)), att=c(np.linalg.solve(ATT, Sx)),
                T=c(np.linalg.solve(St, Sx)), ATT=c(ATT), S=c(Sx))
