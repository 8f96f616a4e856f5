"""Pins of the oracle's TPFA residual, Jacobian and Schur approximation.

Each test checks the oracle against something other than itself: finite
differences, exact cancellation of interior fluxes (Sec. 2.2, the
conservative form of Eq. Fm / Eq. Fe), hydrostatic equilibrium of Darcy's
law (Eq. darcy), Peaceman's closed form for square cells, and the
decoupled case in which S~_T must equal A_TT (Sec. 3.3).
"""
import numpy as np
import pytest

from oracle import physics
from synthetic import make_problem, default_fluid, bennison_oil
from synthetic.recipes import perturbed_state


def tiny(shape=(4, 3, 3), seed=11, fluid=None, wells=True):
    prob = make_problem("tiny", seed=seed, shape=shape, fluid=fluid)
    nx, ny, nz = shape
    if not wells:
        prob["wells"] = []
    return prob


def dense_blocks(rowptr, col, val):
    N = rowptr.size - 1
    J = np.zeros((2 * N, 2 * N))
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    for a in range(2):
        for b in range(2):
            J[2 * rows + a, 2 * col + b] = val[:, a, b]
    return J


@pytest.mark.parametrize("shape,oil", [((4, 3, 3), False), ((3, 5, 2), False), ((4, 3, 3), True)])
def test_jacobian_matches_central_differences(shape, oil):
    prob = tiny(shape, fluid=bennison_oil() if oil else None)
    # make the producer active and the injector present; perturb the state
    p, T = perturbed_state(prob, seed=5)
    prob["p_n"] = prob["p_n"] + 1.0e5
    rowptr, col, val = physics.jacobian(prob, p, T)
    J = dense_blocks(rowptr, col, val)
    N = p.size
    Jfd = np.zeros_like(J)
    for j in range(N):
        for which, h in ((0, 1.0), (1, 1.0e-4)):
            xp, xm = p.copy(), p.copy()
            tp_, tm = T.copy(), T.copy()
            if which == 0:
                xp[j] += h
                xm[j] -= h
            else:
                tp_[j] += h
                tm[j] -= h
            gp = physics.residual_interleaved(prob, xp, tp_)
            gm = physics.residual_interleaved(prob, xm, tm)
            Jfd[:, 2 * j + which] = (gp - gm) / (2 * h)
    for c in range(2 * N):
        scale = np.max(np.abs(J[:, c]))
        assert np.max(np.abs(J[:, c] - Jfd[:, c])) <= 1e-6 * scale, c


def test_interior_fluxes_cancel_in_the_sum_of_residuals():
    prob = tiny((5, 4, 3))
    p, T = perturbed_state(prob, seed=3)
    fl = prob["fluid"]
    Rm, Re = physics.residual(prob, p, T)
    V = prob["dx"] * prob["dy"] * prob["dz"]
    rho = physics.density(p, T, fl)
    rho_n = physics.density(prob["p_n"], prob["T_n"], fl)
    acc_m = np.sum(V * prob["phi"] * (rho - rho_n) / prob["dt"])
    src_m = 0.0
    src_e = 0.0
    for (c, kind, q, val, Tinj, U) in physics.well_cells(prob):
        if kind == 0:
            r = physics.density(p[c], Tinj, fl)
            src_m += q * r
            src_e += q * r * fl["cv"] * Tinj
        elif kind == 1 and p[c] > val:
            lam = rho[c] / physics.viscosity(T[c], fl)
            src_m -= q * (p[c] - val) * lam
            src_e -= q * (p[c] - val) * lam * fl["cv"] * T[c]
    ft = physics._face_terms(prob, p, T)
    flux_m = np.sum(np.abs(ft["F"]))
    flux_e = np.sum(np.abs(ft["E"]))
    assert flux_m > 0.5 * abs(acc_m - src_m)  # fluxes are not negligible: a real check
    assert abs(np.sum(Rm) - (acc_m - src_m)) <= 1e-13 * flux_m
    acc_e = np.sum(V * (prob["phi"] * fl["cv"] * (rho * T - rho_n * prob["T_n"])
                        + (1 - prob["phi"]) * fl["rho_r"] * fl["cr"] * (T - prob["T_n"])) / prob["dt"])
    assert abs(np.sum(Re) - (acc_e - src_e)) <= 1e-13 * flux_e


def test_column_sums_of_flux_parts_vanish():
    """Every interior flux enters two rows with opposite signs, so the column
    sums of the Jacobian blocks keep only accumulation and well terms (the
    observation behind the True-IMPES operator in Sec. 3.1)."""
    prob = tiny((4, 4, 2), wells=False)
    p, T = perturbed_state(prob, seed=9)
    fl = prob["fluid"]
    rowptr, col, val = physics.jacobian(prob, p, T)
    N = p.size
    V = prob["dx"] * prob["dy"] * prob["dz"]
    dt, phi, cv = prob["dt"], prob["phi"], fl["cv"]
    rho = physics.density(p, T, fl)
    rho_p, rho_T = fl["c"] * rho, fl["beta"] * rho
    expect = {
        (0, 0): V * phi * rho_p / dt,
        (0, 1): V * phi * rho_T / dt,
        (1, 0): V * phi * cv * rho_p * T / dt,
        (1, 1): V * (phi * cv * (rho_T * T + rho) + (1 - phi) * fl["rho_r"] * fl["cr"]) / dt,
    }
    for (a, b), e in expect.items():
        cs = np.zeros(N)
        np.add.at(cs, col, val[:, a, b])
        scale = np.max(np.abs(val[:, a, b]))
        assert np.max(np.abs(cs - e)) <= 1e-11 * scale, (a, b)


def test_schur_column_sums_are_the_accumulation_and_source_terms():
    prob = tiny((4, 4, 3))
    p, T = perturbed_state(prob, seed=2)
    fl = prob["fluid"]
    rowptr, col, S = physics.schur_approx(prob, p, T)
    N = p.size
    V = prob["dx"] * prob["dy"] * prob["dz"]
    rho = physics.density(p, T, fl)
    e = V * (prob["phi"] * fl["cv"] * rho + (1 - prob["phi"]) * fl["rho_r"] * fl["cr"]) / prob["dt"]
    for (c, kind, q, val, Tinj, U) in physics.well_cells(prob):
        if kind == 1 and p[c] > val:
            e[c] += fl["cv"] * q * (p[c] - val) * rho[c] / physics.viscosity(T[c], fl)
    cs = np.zeros(N)
    np.add.at(cs, col, S)
    assert np.max(np.abs(cs - e)) <= 1e-11 * np.max(np.abs(S))


def test_hydrostatic_column_has_zero_mass_residual():
    """p = p_top + rho g (z_top - z) with incompressible fluid, uniform T and no
    wells is Darcy equilibrium (Eq. darcy): every face potential difference and
    hence every mass residual vanishes. A flipped gravity sign would leave
    2 rho g dz on every vertical face."""
    fl = default_fluid(c=0.0)
    prob = tiny((3, 3, 6), fluid=fl, wells=False)
    N = prob["nx"] * prob["ny"] * prob["nz"]
    k = np.arange(N) // (prob["nx"] * prob["ny"])
    T = np.full(N, 330.0)
    rho = physics.density(np.zeros(N), T, fl)[0]
    p = 2.0e7 - rho * prob["g"] * (k * prob["dz"])
    prob["p_n"], prob["T_n"] = p.copy(), T.copy()
    Rm, Re = physics.residual(prob, p, T)
    lo, hi, Tf, Tcf, dz = physics.faces(prob)
    lam = rho / physics.viscosity(330.0, fl)
    scale = np.max(Tf) * lam * rho * prob["g"] * prob["dz"]
    assert np.max(np.abs(Rm)) <= 1e-9 * scale
    assert np.max(np.abs(Re)) <= 1e-9 * scale * fl["cv"] * 330.0
    # wrong-sign control: reversing gravity must produce a clear residual
    prob2 = dict(prob, g=-prob["g"])
    Rm2, _ = physics.residual(prob2, p, T)
    assert np.max(np.abs(Rm2)) > 0.5 * scale


def test_schur_equals_ATT_when_pressure_and_temperature_decouple():
    """beta = 0 and a T-independent viscosity make A_pT = 0, so the exact Schur
    complement is A_TT; the approximation of Eq. Se then reproduces A_TT
    (the dropped terms all carry rho_T or mu_T)."""
    fl = default_fluid(beta=0.0, mu_coef=0.0)
    prob = tiny((4, 3, 3), fluid=fl)
    p, T = perturbed_state(prob, seed=4)
    rowptr, col, val = physics.jacobian(prob, p, T)
    assert np.max(np.abs(val[:, 0, 1])) == 0.0
    _, _, S = physics.schur_approx(prob, p, T)
    ATT = val[:, 1, 1]
    assert np.max(np.abs(S - ATT)) <= 1e-12 * np.max(np.abs(ATT))


def test_peaceman_square_cell_radius_is_0198_dx():
    """For isotropic K and square cells Peaceman's equivalent radius reduces
    to 0.14 sqrt(2) Dx ~= 0.198 Dx (Sec. 2.1.5)."""
    K = 2.0e-13
    wi = physics.peaceman_wi(np.array(K), np.array(K))
    re = 0.14 * np.sqrt(2.0) * 5.0
    assert abs(wi - 2 * np.pi * 5.0 * K / np.log(re / 0.1)) <= 1e-15 * abs(wi) * 10
    assert abs(re - 0.19799 * 5.0) < 1e-4


def test_density_and_viscosity_reference_values():
    fl = default_fluid()
    assert physics.density(np.array(fl["p0"]), np.array(fl["T0"]), fl) == fl["rho0"]
    assert physics.viscosity(np.array(fl["T_mu0"]), fl) == fl["mu0"]
    # one bar above p0 scales density by exp(5.5e-5)
    r = physics.density(np.array(fl["p0"] + 1.0e5), np.array(fl["T0"]), fl)
    assert abs(r / fl["rho0"] - np.exp(5.5e-5)) < 1e-15


def test_block_pattern_is_seven_point_and_sorted():
    prob = tiny((5, 4, 3))
    rowptr, col = physics.block_pattern(prob)
    N = 60
    F = (4 * 4 * 3) + (5 * 3 * 3) + (5 * 4 * 2)
    assert rowptr[-1] == N + 2 * F
    for i in range(N):
        c = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c


def test_sparse_schur_diag_equals_the_dense_formula():
    """S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3): the sparse
    evaluation on the 25-point pattern equals the dense matrix product, and
    its pattern is the product pattern of two 7-point stencils (offsets
    with |dx| + |dy| + |dz| <= 2)."""
    prob = tiny((5, 4, 3))
    p, T = perturbed_state(prob, seed=2)
    rowptr, col, val = physics.jacobian(prob, p, T)
    rp, c, v = physics.schur_diag_sparse(rowptr, col, val)
    D = physics.schur_diag(rowptr, col, val)
    N = rowptr.size - 1
    S = np.zeros((N, N))
    rows = np.repeat(np.arange(N), np.diff(rp))
    S[rows, c] = v
    assert np.max(np.abs(S - D)) <= 1e-13 * np.max(np.abs(D))
    nx, ny = prob["nx"], prob["ny"]
    xyz = lambda i: np.array([i % nx, (i // nx) % ny, i // (nx * ny)])
    for i in range(N):
        want = [j for j in range(N) if np.abs(xyz(i) - xyz(j)).sum() <= 2]
        assert list(c[rp[i]:rp[i + 1]]) == want


def test_bennison_viscosity_behaves_as_the_correlation_states():
    """Eq. bennison is a power law in the Fahrenheit temperature: the ratio
    of two viscosities is the temperature ratio to the power A3 API + A4
    (Table 1), here checked between 100 F and 350 F given in kelvin; a
    heavier oil (lower API) is more viscous at the same temperature; and the
    result is in Pa s (1 cp = 1e-3 Pa s): a 12-API oil at 60 F is a few tens
    of Pa s, far above water's 1e-3."""
    to_k = lambda f: (f - 32.0) * 5.0 / 9.0 + 273.15
    for api in (8.0, 12.0, 20.0):
        fl = bennison_oil(api)
        m = physics.viscosity(np.array([to_k(100.0), to_k(350.0)]), fl)
        assert abs(m[1] / m[0] - 3.5 ** (0.31458 * api - 9.21592)) <= 1e-12 * (m[1] / m[0])
    T = np.array([to_k(150.0)])
    assert physics.viscosity(T, bennison_oil(10.0)) > physics.viscosity(T, bennison_oil(15.0))
    assert 10.0 < physics.viscosity(np.array([to_k(60.0)]), bennison_oil(12.0))[0] < 100.0
    fl = bennison_oil(12.0)
    assert abs(fl["rho0"] / 999.0 - 141.5 / 143.5) < 1e-15
