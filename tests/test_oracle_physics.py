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


# --------------------------------------------------- hand-computed values
def two_cells(shape=(2, 1, 1), dxyz=(10.0, 10.0, 10.0), K=(1e-13, 3e-13), kTr=(2.0, 3.0),
              p=(15.1e6, 15.0e6), T=(320.0, 330.0), g=0.0, kT_mix=0):
    """Two cells along the axis of `shape`, incompressible water (c = beta =
    0, rho = 999 kg/m^3) with mu = 1e-3 exp(-0.02 (T - 320)) Pa s,
    porosity 0.2, fluid conductivity 0.6 W/m/K, no wells, one day step from
    the same state."""
    fl = default_fluid(c=0.0, beta=0.0, mu_coef=0.02, T_mu0=320.0, kT_mix=kT_mix)
    K = np.array(K)
    pa, Ta = np.array(p), np.array(T)
    return dict(nx=shape[0], ny=shape[1], nz=shape[2], dx=dxyz[0], dy=dxyz[1], dz=dxyz[2],
                g=g, fluid=fl, Kx=K.copy(), Ky=K.copy(), Kz=K.copy(), phi=np.full(2, 0.2),
                kTr=np.array(kTr), wells=[], p_n=pa.copy(), T_n=Ta.copy(), p_k=pa.copy(),
                T_k=Ta.copy(), dt=86400.0)


@pytest.mark.parametrize("shape,dxyz,area,dist", [
    ((2, 1, 1), (10.0, 10.0, 10.0), 100.0, 10.0),
    ((2, 1, 1), (4.0, 5.0, 10.0), 50.0, 4.0),    # x-face: dy dz over dx
    ((1, 2, 1), (4.0, 5.0, 10.0), 40.0, 5.0),    # y-face: dx dz over dy
    ((1, 1, 2), (4.0, 5.0, 10.0), 20.0, 10.0)])  # z-face: dx dy over dz
def test_transmissibilities_by_hand(shape, dxyz, area, dist):
    """Sec. 2.2 (TPFA, harmonic face averages): K = 1e-13 and 3e-13 m^2 give
    the harmonic mean 2 K1 K2 / (K1 + K2) = 1.5e-13 m^2; k_T = 0.2 k_T,r +
    0.8 * 0.6 (Sec. 2.1.2 as printed) = 0.88 and 1.08 W/m/K, harmonic mean
    2 * 0.88 * 1.08 / 1.96 = 0.969795918... W/m/K; each times face area
    over centre distance."""
    prob = two_cells(shape, dxyz)
    lo, hi, Tf, Tcf, dz = physics.faces(prob)
    assert lo.tolist() == [0] and hi.tolist() == [1]
    assert Tf[0] == pytest.approx(area / dist * 1.5e-13, rel=1e-14)
    assert Tcf[0] == pytest.approx(area / dist * 0.9697959183673469, rel=1e-14)
    assert dz[0] == (dxyz[2] if shape[2] == 2 else 0.0)


def test_thermal_conductivity_mixing_by_hand():
    """Sec. 2.1.2: k_T = phi k_T,r + (1 - phi) k_T,f as printed (kT_mix 0)
    and the swapped weights (kT_mix 1): phi = 0.2, k_T,f = 0.6, k_T,r = 2, 3
    -> 0.88, 1.08 and 1.72, 2.52 W/m/K."""
    np.testing.assert_allclose(physics.thermal_conductivity(two_cells(kT_mix=0)),
                               [0.88, 1.08], rtol=1e-15)
    np.testing.assert_allclose(physics.thermal_conductivity(two_cells(kT_mix=1)),
                               [1.72, 2.52], rtol=1e-15)


def test_schur_approximation_entries_by_hand():
    """Eq. Se on the two cells (flow from cell 0 to cell 1, dPhi = 1e5 Pa):
    T_f = 1.5e-12 m^3, lambda_0 = 999 / 1e-3 = 9.99e5, advective
    coefficient c_v T_f lambda_0 dPhi = 4184 * 0.14985 = 626.9724 W/K,
    Tc_f = 9.697959... W/K, accumulation V [phi c_v rho + (1 - phi) rho_r c_r]
    / dt = 1000 (0.2 * 4184 * 999 + 0.8 * 2650 * 920) / 86400 =
    32249.574074... W/K. Upwind cell 0: S_00 = acc + adv + Tc, S_01 = -Tc;
    downstream cell 1: S_11 = acc + Tc, S_10 = -Tc - adv."""
    prob = two_cells()
    rp, col, Sv = physics.schur_approx(prob, prob["p_k"], prob["T_k"])
    assert rp.tolist() == [0, 2, 4] and col.tolist() == [0, 1, 0, 1]
    want = [32886.24443325774, -9.69795918367347, -636.6703591836733, 32259.27203325775]
    np.testing.assert_allclose(Sv, want, rtol=1e-13)


def test_jacobian_diagonal_blocks_by_hand():
    """Eq. AXR on the two cells: A_pp,00 = T_f lambda_0 = 1.4985e-6 (c = 0,
    no accumulation term); A_pT,00 = T_f dlambda_0/dT dPhi with
    dlambda/dT = 0.02 lambda (viscosity law) = 2.997e-3; A_Tp,00 = c_v T_0
    T_f lambda_0 = 2.00631168; A_TT,00 = acc + c_v (T_0 T_f dlambda_0/dT dPhi
    + F) + Tc_f = 36898.8677932...; A_TT,11 = acc + Tc_f (its upwind cell is
    the other one)."""
    prob = two_cells()
    rp, col, val = physics.jacobian(prob, prob["p_k"], prob["T_k"])
    np.testing.assert_allclose(val[0].ravel(), [1.4985e-06, 0.002997, 2.00631168,
                                                36898.86779325774], rtol=1e-13)
    assert val[3, 0, 0] == pytest.approx(1.4985e-06, rel=1e-13)
    assert val[3, 1, 1] == pytest.approx(32259.27203325775, rel=1e-13)


def test_darcy_and_fourier_fluxes_in_a_column():
    """A 5 x 1 x 1 column without gravity, incompressible fluid of constant
    viscosity, uniform K = 2e-13 m^2, linear p falling by 1e5 Pa per 10 m
    cell and linear T rising by 20 K per cell, state = previous state (no
    accumulation). Darcy (Sec. 2.1): the mass flux through every face is
    rho K A |grad p| / mu = 999 * 2e-13 * 100 * 1e4 / 1e-3 = 0.1998 kg/s, so
    the residual is +0.1998 in the first cell, -0.1998 in the last and 0
    inside. Fourier: the conducted heat k_T A dT/dx = 0.88 * 100 * 2 = 176 W
    flows against the flow. Energy: each interior cell receives c_v T_up F
    from the upstream face and sends c_v T_i F downstream, so R_e,i =
    c_v F (T_i - T_{i-1}) = 4184 * 0.1998 * 20 = 16719.264 W; the end cells
    add -+176 W of conduction."""
    nx = 5
    fl = default_fluid(c=0.0, beta=0.0, mu_coef=0.0)
    x = 10.0 * np.arange(nx)
    p = 15e6 - 1e4 * x
    T = 300.0 + 2.0 * x
    prob = dict(nx=nx, ny=1, nz=1, dx=10.0, dy=10.0, dz=10.0, g=0.0, fluid=fl,
                Kx=np.full(nx, 2e-13), Ky=np.full(nx, 2e-13), Kz=np.full(nx, 2e-13),
                phi=np.full(nx, 0.2), kTr=np.full(nx, 2.0), wells=[], p_n=p.copy(),
                T_n=T.copy(), p_k=p.copy(), T_k=T.copy(), dt=86400.0)
    Rm, Re = physics.residual(prob, p, T)
    np.testing.assert_allclose(Rm, [0.1998, 0, 0, 0, -0.1998], atol=1e-12, rtol=0)
    F = 0.1998
    want = np.array([4184 * 300.0 * F + (-176.0), 16719.264, 16719.264, 16719.264,
                     -(4184 * 360.0 * F) + 176.0])
    np.testing.assert_allclose(Re, want, rtol=1e-12, atol=1e-9)


def test_source_terms_by_hand():
    """Eq. f / Eq. fT and the heater of Sec. 2.1.5 in one 10 m cell of an
    incompressible fluid (rho = 999) at p = 15 MPa, T = 320 K, state =
    previous state so only the source remains in the residual:
      rate injector 1e-3 m^3/s at 450 K: R_m = -0.999 kg/s,
        R_e = -0.999 * 4184 * 450 = -1880920.8 W;
      BHP producer at 10 MPa, K = 1e-13 m^2: Peaceman WI = 2 pi h K /
        ln(r_e / r_w), r_e = 0.14 sqrt(5^2 + 5^2) = 0.98994949 m, h = 5 m,
        r_w = 0.1 m -> WI = 1.370373e-12 m^3; q = WI / mu (p - p_bh), mass
        rate = rho WI / mu * 5e6 = 6.8450... kg/s leaving, energy rho q c_v T;
      heater U = 5e3 W/K towards 450 K: R_e = -5e3 * (450 - 320) = -650000 W;
      rate producer 1e-3 m^3/s: R_m = +0.999, R_e = 0.999 * 4184 * 320."""
    fl = default_fluid(c=0.0, beta=0.0, mu_coef=0.0)
    one = lambda a: np.full(1, a)
    base = dict(nx=1, ny=1, nz=1, dx=10.0, dy=10.0, dz=10.0, g=9.81, fluid=fl, Kx=one(1e-13),
                Ky=one(1e-13), Kz=one(1e-13), phi=one(0.2), kTr=one(2.0), p_n=one(15e6),
                T_n=one(320.0), p_k=one(15e6), T_k=one(320.0), dt=86400.0)
    well = lambda kind, value, T_inj=0.0, U=0.0: [dict(i=0, j=0, k0=0, k1=0, kind=kind,
                                                      value=value, T_inj=T_inj, U=U)]
    wi = 2 * np.pi * 5.0 * 1e-13 / np.log(0.14 * np.sqrt(50.0) / 0.1)
    assert wi == pytest.approx(1.370373e-12, rel=1e-6)
    m_prod = 999.0 / 1e-3 * wi * 5e6
    cases = [(well(0, 1e-3, 450.0), -0.999, -0.999 * 4184 * 450.0),
             (well(1, 10e6), m_prod, m_prod * 4184 * 320.0),
             (well(2, 0.0, 450.0, 5e3), 0.0, -650000.0),
             (well(3, 1e-3), 0.999, 0.999 * 4184 * 320.0)]
    for wells, rm, re in cases:
        prob = dict(base, wells=wells)
        Rm, Re = physics.residual(prob, prob["p_k"], prob["T_k"])
        assert Rm[0] == pytest.approx(rm, rel=1e-13, abs=1e-15), wells
        assert Re[0] == pytest.approx(re, rel=1e-13), wells
