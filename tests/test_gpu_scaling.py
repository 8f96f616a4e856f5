"""The problem-size scaling claim of Sec. 4.3 on the GPU: for Case II
(isotropic medium, 3 + 3 rate wells) the block preconditioner's FGMRES
iterations per Newton iteration grow slowly as the mesh is refined, and the
Schur approximation S~_T needs fewer of them than S~_ATT and S~_diag (the
ordering of the paper's Table 8). The coarsest AMG grids have at most 64
rows, so every size runs multi-level V-cycles."""
import pytest

from synthetic import scaling_case

pytestmark = pytest.mark.gpu

thermo = pytest.importorskip("paper_1902_00095_gb300.thermo")


def per_newton(case, n, schur):
    prob = scaling_case(case, n)
    s = thermo.Solver.from_problem(prob)
    p, T = prob["p_n"], prob["T_n"]
    newton = lin = 0
    for _ in range(2):
        p, T, info = s.newton_step(p, T, prob["dt"], max_newton=10, tol_f=1e-8, tol_dx=1e-8,
                                   rtol=1e-5, maxit=200, restart=30, schur=schur,
                                   coarse_size=64)
        assert info["status"] == 0 and info["last_linear_status"] == 0
        newton += info["newton_iters"]
        lin += info["linear_iters"]
    s.close()
    return lin / newton


def test_case_two_iterations_grow_slowly_and_S_T_is_best():
    its = {sc: [per_newton(2, n, sc) for n in (20, 40, 80)] for sc in (0, 2, 3)}
    # Table 8 puts S~_T below both others at every size (and S~_diag below
    # S~_ATT, an order between the two weaker ones that is not asserted)
    for k in range(3):
        assert its[0][k] <= min(its[2][k], its[3][k]), its
    # 16x more cells: at most 1.6x more iterations per Newton iteration with S~_T
    assert its[0][2] <= 1.6 * its[0][0], its
