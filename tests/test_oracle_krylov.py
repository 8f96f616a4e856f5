"""Pins of the oracle's block preconditioner and FGMRES.

With exact inner solves the five-step preconditioner of Sec. 3.2 is A^{-1}
(Eq. Afact / Eq. Ainv), so preconditioned GMRES converges in one iteration;
the block lower-triangular variant has a preconditioned operator with
minimal polynomial of degree 2, so two iterations suffice. FGMRES is pinned
to a least-squares minimisation over an explicit Krylov basis and to a
dense direct solve."""
import numpy as np
import pytest

from oracle import amg, krylov, physics
from synthetic import make_problem
from synthetic.recipes import perturbed_state


def small_system(shape=(5, 4, 3), seed=1):
    prob = make_problem("tiny", shape=shape, seed=seed)
    p, T = perturbed_state(prob, seed=seed + 10)
    sys, bp, bT, S = krylov.assemble(prob, p, T)
    return prob, sys, bp, bT, S


def dense(A):
    return amg.to_dense(A)


def exact_parts(sys):
    App, ApT, ATp, ATT = (dense(m) for m in (sys.App, sys.ApT, sys.ATp, sys.ATT))
    Sx = ATT - ATp @ np.linalg.solve(App, ApT)
    return App, Sx


def run(sys, bp, bT, inv_pp, inv_S, variant, rtol=1e-12, maxit=20):
    M = krylov.block_preconditioner(sys, inv_pp, inv_S, variant)
    sm, se = sys.s_m, sys.s_e
    mv = lambda xp, xT: tuple(s * y for s, y in zip((sm, se), sys.matvec(xp, xT)))
    pc = lambda vp, vT: M(vp / sm, vT / se)
    return krylov.fgmres(mv, pc, sm * bp, se * bT, rtol, maxit, 30)


def test_exact_block_factorisation_converges_in_one_iteration():
    prob, sys, bp, bT, S = small_system()
    App, Sx = exact_parts(sys)
    out = run(sys, bp, bT, lambda r: np.linalg.solve(App, r), lambda r: np.linalg.solve(Sx, r), "full")
    assert out["iters"] == 1
    assert out["rel_res"] < 1e-10


def test_exact_lower_triangular_converges_in_two_iterations():
    prob, sys, bp, bT, S = small_system((4, 4, 3), seed=2)
    App, Sx = exact_parts(sys)
    out = run(sys, bp, bT, lambda r: np.linalg.solve(App, r), lambda r: np.linalg.solve(Sx, r), "lower")
    assert out["iters"] <= 2
    assert out["rel_res"] < 1e-9


def test_preconditioner_equals_inverse_with_exact_solves():
    prob, sys, bp, bT, S = small_system((3, 3, 3), seed=3)
    App, Sx = exact_parts(sys)
    M = krylov.block_preconditioner(sys, lambda r: np.linalg.solve(App, r),
                                    lambda r: np.linalg.solve(Sx, r), "full")
    rng = np.random.default_rng(0)
    vp, vT = rng.standard_normal(sys.N), rng.standard_normal(sys.N)
    zp, zT = M(vp, vT)
    yp, yT = sys.matvec(zp, zT)
    assert np.max(np.abs(yp - vp)) <= 1e-6 * np.max(np.abs(vp))
    assert np.max(np.abs(yT - vT)) <= 1e-6 * np.max(np.abs(vT))


def test_fgmres_residuals_are_krylov_least_squares_minima():
    """Without preconditioning, |g_{m}| after m steps equals
    min_y ||b - A K_m y|| over the Krylov space K_m(A, b)."""
    rng = np.random.default_rng(4)
    n = 40
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.5
    b = rng.standard_normal(n)
    h = n // 2
    mv = lambda xp, xT: ((A @ np.concatenate([xp, xT]))[:h], (A @ np.concatenate([xp, xT]))[h:])
    pc = lambda vp, vT: (vp, vT)
    out = krylov.fgmres(mv, pc, b[:h], b[h:], rtol=1e-14, maxit=12, restart=30)
    K = np.zeros((n, 12))
    v = b.copy()
    for m in range(12):
        K[:, m] = v / np.linalg.norm(v)
        v = A @ K[:, m]
    for m in range(1, 13):
        Q, _ = np.linalg.qr(A @ K[:, :m])
        r = b - Q @ (Q.T @ b)
        assert abs(out["hist"][m - 1] - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-9


def test_amg_preconditioned_solve_matches_direct_solve():
    prob = make_problem("iid16")
    out = krylov.solve(prob, rtol=1e-10)
    assert out["status"] == "converged"
    xp, xT = krylov.direct_solution(out["sys"], out["bp"], out["bT"])
    N = out["sys"].N
    x = out["x"]
    assert np.linalg.norm(x[:N] - xp) <= 1e-7 * np.linalg.norm(xp)
    assert np.linalg.norm(x[N:] - xT) <= 1e-6 * np.linalg.norm(xT)
    assert out["iters"] < 40


@pytest.mark.parametrize("variant", ["full", "lower"])
def test_schur_approximation_beats_ATT_in_condition_number(variant):
    """Trend of Table 4: on a heterogeneous grid with wells, S~_T^{-1} S is
    better conditioned than A_TT^{-1} S (the paper's SPE10 numbers are not
    reproduced, only the ordering)."""
    prob = make_problem("tiny", shape=(6, 6, 2), seed=8, dt_days=100.0)
    prob["wells"][0]["value"] = 1e-2
    p, T = perturbed_state(prob, seed=3, dp=1e5, dT=20.0)
    sys, bp, bT, S = krylov.assemble(prob, p, T)
    App, Sx = exact_parts(sys)
    St = dense(S)
    ATT = dense(sys.ATT)
    k_t = np.linalg.cond(np.linalg.solve(St, Sx))
    k_a = np.linalg.cond(np.linalg.solve(ATT, Sx))
    assert k_t < k_a


def test_newton_converges_quadratically_to_a_root():
    """Newton on the discrete residual with the analytic Jacobian (Sec. 3):
    the scaled function norm falls quadratically and the final state is a
    root of G to rounding."""
    from oracle import newton
    prob = make_problem("tiny", shape=(6, 5, 3), seed=5, dt_days=0.5)
    prob["wells"][0]["value"] = 2e-4
    prob["wells"][1]["value"] = 14.8e6
    p, T, hist = newton.newton_step(prob, max_newton=8, tol_f=1e-13, tol_dx=0.0)
    relf = [h[0] for h in hist]
    assert relf[-1] < 1e-12
    # e_{k+1} <= C e_k^2 over the last two steps (quadratic convergence)
    for a, b in zip(relf[-3:-1], relf[-2:]):
        assert b <= 1e3 * a * a, relf
    sysb, bp, bT, _ = krylov.assemble(prob, p, T)
    sys0, bp0, bT0, _ = krylov.assemble(prob)
    g = np.hypot(np.linalg.norm(sys0.s_m * bp), np.linalg.norm(sys0.s_e * bT))
    g0 = np.hypot(np.linalg.norm(sys0.s_m * bp0), np.linalg.norm(sys0.s_e * bT0))
    assert g <= 1e-12 * g0


def test_line_search_keeps_full_steps_on_a_mild_step():
    """Where full Newton steps already decrease the function norm enough,
    the line search (Sec. 4) accepts alpha = 1 every time and the iterates
    are those of plain Newton."""
    from oracle import newton
    prob = make_problem("tiny", shape=(6, 5, 3), seed=5, dt_days=0.5)
    prob["wells"][0]["value"] = 2e-4
    prob["wells"][1]["value"] = 14.8e6
    p, T, hist = newton.newton_step(prob, max_newton=8, tol_f=1e-13, tol_dx=0.0)
    pf, Tf, histf = newton.newton_step(prob, max_newton=8, tol_f=1e-13, tol_dx=0.0,
                                       line_search=False)
    assert all(h[2] == 1.0 for h in hist[:-1])
    assert np.array_equal(p, pf) and np.array_equal(T, Tf)


def test_line_search_rescues_a_step_where_full_newton_diverges():
    """30-day step with a 10x injection rate: full Newton steps leave the
    physical range (non-finite or growing function norm) while the
    backtracking line search converges quadratically to a root; every
    accepted step meets the sufficient-decrease test with alpha a power of
    1/2 no smaller than 2^-6."""
    from oracle import newton
    prob = make_problem("tiny", shape=(6, 5, 3), seed=5, dt_days=30)
    prob["wells"][0]["value"] = 2e-3
    prob["wells"][1]["value"] = 14.8e6
    try:
        _, _, hf = newton.newton_step(prob, max_newton=12, tol_f=1e-12, tol_dx=0.0,
                                      line_search=False)
        assert not hf[-1][0] <= 1e-12
    except FloatingPointError:
        pass
    p, T, hist = newton.newton_step(prob, max_newton=12, tol_f=1e-12, tol_dx=0.0)
    relf = [h[0] for h in hist]
    alphas = [h[2] for h in hist[:-1]]
    assert relf[-1] <= 1e-12
    assert min(alphas) < 1.0
    for a in alphas:
        assert a >= 2.0 ** -6 and np.log2(a) == np.round(np.log2(a))
    for k, a in enumerate(alphas):
        assert relf[k + 1] <= (1.0 - 1e-4 * a) * relf[k]
    assert relf[-1] <= 1e3 * relf[-2] ** 2


@pytest.mark.parametrize("case", [1, 2, 3, 4, 5])
def test_scaling_cases_are_well_posed(case):
    """The problem-size scaling Cases I-V (Sec. 4.3) at n = 20: sources
    inside the square, heaters or 3 + 3 rate wells as stated, and a
    backward-Euler step that the oracle's Newton with line search solves to
    the paper's 1e-8 tolerances."""
    from oracle import newton
    from synthetic import scaling_case
    prob = scaling_case(case, 20)
    kinds = sorted(w["kind"] for w in prob["wells"])
    assert kinds == ([2] * 6 if case in (1, 4) else [0, 0, 0, 3, 3, 3])
    assert all(0 <= w["i"] < 20 and 0 <= w["j"] < 20 for w in prob["wells"])
    assert abs(prob["dx"] * prob["nx"] - 20.0) < 1e-12
    p, T, hist = newton.newton_step(prob, max_newton=10, tol_f=1e-8, tol_dx=1e-8)
    assert len(hist) <= 10
    assert hist[-1][0] <= 1e-8 or hist[-1][1] is not None and hist[-1][1] <= 1e-8


def _table4_case(kind, high_perm, shape=(8, 8, 3)):
    """Heater (H), well (W) or both on a small heterogeneous grid of the
    paper's heavy oil, permeability x1000 for the high-permeability cases,
    evaluated at the state after one backward-Euler step."""
    from oracle import newton
    from synthetic import bennison_oil
    nx, ny, nz = shape
    prob = make_problem("tiny", shape=shape, seed=8, fluid=bennison_oil(), dt_days=10.0)
    if high_perm:
        for k in ("Kx", "Ky", "Kz"):
            prob[k] = prob[k] * 1000.0
    wells = []
    if "W" in kind:
        wells += [dict(i=0, j=0, k0=0, k1=nz - 1, kind=0, value=1e-3, T_inj=422.039, U=0.0),
                  dict(i=nx - 1, j=ny - 1, k0=0, k1=nz - 1, kind=3, value=1e-3, T_inj=0.0, U=0.0)]
    if "H" in kind:
        wells += [dict(i=nx // 2, j=ny // 2, k0=0, k1=nz - 1, kind=2, value=0.0, T_inj=422.039,
                       U=5e3)]
    prob["wells"] = wells
    p, T, _ = newton.newton_step(prob, max_newton=8)
    return krylov.schur_condition_numbers(prob, p, T)


@pytest.mark.parametrize("kind,high_perm", [("H", False), ("W", False), ("WH", False),
                                            ("W", True), ("WH", True)])
def test_table4_ordering_of_schur_approximations(kind, high_perm):
    """Sec. 4.2 / Table 4, in kind: S~_T^{-1} S stays close to the identity
    (condition number below 2 here, at most 6 in the paper) in every case,
    while S~_ATT and S~_diag degrade once wells drive advection (the paper's
    W and high-permeability columns)."""
    k = _table4_case(kind, high_perm)
    assert k["T"] < 2.0, k
    assert k["T"] <= k["att"] and k["T"] <= k["diag"], k
    if "W" in kind:
        assert k["att"] > 5 * k["T"] and k["diag"] > 5 * k["T"], k
