"""Oracle: TPFA finite-volume residual, Jacobian and Schur approximation.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Discretisation (Sec. 2.2): DG0 == two-point flux on a Cartesian grid of
dx*dy*dz cells, harmonic face averages of K and k_T, arithmetic face average
of rho, upwinding of rho/mu and T by the sign of the face potential
difference (ties to the lower cell index, the "E1" side), backward Euler, and
delta sources integrated as 1/|E_i| (Eq. Fm, Eq. Fe).

Sign conventions (a reading; the paper writes them through [p] and n_e):
z points up, layer k = 0 at the bottom, and for the face between cells
lo < hi
    dPhi = p_lo - p_hi - rhobar * g * (z_hi - z_lo)
    F    = T_f * (rho/mu)_up * dPhi             (mass leaving lo towards hi)
    E    = c_v * T_up * F + Tc_f * (T_lo - T_hi) (energy leaving lo)
with up = lo if dPhi >= 0 else hi. Cell residuals (integrated over the cell):
    R_m,i = V phi (rho_i - rho_i^n)/dt + sum_faces(+-F) - Q_m,i
    R_e,i = V [phi c_v (rho_i T_i - rho^n T^n) + (1-phi) rho_r c_r (T_i - T^n)]/dt
            + sum_faces(+-E) - Q_e,i
Wells (Eq. f, Eq. fT, Peaceman model of Sec. 2.1.5 with Dx = Dy = 5 m,
h = 5 m, r_w = 0.1 m) and heaters (Sec. 2.1.5).

Unknown ordering: block-CSR with one 2x2 block per (cell, neighbour) pair,
block = [[dR_m/dp, dR_m/dT], [dR_e/dp, dR_e/dT]], columns sorted per row.
"""
import numpy as np


# ---------------------------------------------------------------- fluid laws
def density(p, T, fl):
    """rho(p,T) = rho0 exp(c (p - p0)) exp(beta (T - T0))  (Sec. 2.1.4)."""
    return fl["rho0"] * np.exp(fl["c"] * (p - fl["p0"])) * np.exp(fl["beta"] * (T - fl["T0"]))


BENNISON = (-0.8021, 23.8765, 0.31458, -9.21592)  # A1..A4 of Table 1


def fahrenheit(T):
    return (T - 273.15) * 9.0 / 5.0 + 32.0


def viscosity(T, fl):
    """mu_law 0: mu(T) = mu0 exp(-a (T - T_mu0)) (an exponential water law);
    mu_law 1: the Bennison heavy-oil correlation of Eq. bennison,
    mu = 10^(A1 API + A2) T_F^(A3 API + A4) centipoise with T_F in degrees
    Fahrenheit (A_i from Table 1), returned in Pa s."""
    if fl.get("mu_law", 0) == 1:
        A1, A2, A3, A4 = BENNISON
        api = fl["api"]
        return 1e-3 * 10.0 ** (A1 * api + A2) * fahrenheit(T) ** (A3 * api + A4)
    return fl["mu0"] * np.exp(-fl["mu_coef"] * (T - fl["T_mu0"]))


def dlog_viscosity_dT(T, fl):
    """d(ln mu)/dT of `viscosity`: -a for the exponential law,
    (A3 API + A4) (9/5) / T_F for Bennison."""
    if fl.get("mu_law", 0) == 1:
        A1, A2, A3, A4 = BENNISON
        return (A3 * fl["api"] + A4) * 9.0 / 5.0 / fahrenheit(T)
    return -fl["mu_coef"] * np.ones_like(T)


def cell_props(p, T, fl):
    """rho, its p/T derivatives, and the mobility lam = rho/mu with its p/T
    derivatives, all per cell."""
    rho = density(p, T, fl)
    mu = viscosity(T, fl)
    rho_p = fl["c"] * rho
    rho_T = fl["beta"] * rho
    lam = rho / mu
    lam_p = rho_p / mu
    # d(rho/mu)/dT = rho_T/mu - (rho/mu) d(ln mu)/dT
    lam_T = rho_T / mu - dlog_viscosity_dT(T, fl) * lam
    return dict(rho=rho, rho_p=rho_p, rho_T=rho_T, mu=mu, lam=lam, lam_p=lam_p, lam_T=lam_T)


def thermal_conductivity(prob):
    """k_T = phi k_T,r + (1 - phi) k_T,f as printed in Sec. 2.1.2 (kT_mix=0),
    or the swapped weights (kT_mix=1)."""
    fl, phi = prob["fluid"], prob["phi"]
    if fl.get("kT_mix", 0) == 0:
        return phi * prob["kTr"] + (1.0 - phi) * fl["kTf"]
    return (1.0 - phi) * prob["kTr"] + phi * fl["kTf"]


# ------------------------------------------------------------------ geometry
def faces(prob):
    """All interior faces as arrays (lo, hi, T_f, Tc_f, dz) with lo < hi.

    T_f = |e|/d * 2 K_lo K_hi / (K_lo + K_hi) (harmonic average of the K
    component normal to the face), Tc_f the same with k_T, and
    dz = z_hi - z_lo (0 for horizontal neighbours). Order: x-faces, then
    y-faces, then z-faces, each in cell order of lo.
    """
    nx, ny, nz = prob["nx"], prob["ny"], prob["nz"]
    dx, dy, dz = prob["dx"], prob["dy"], prob["dz"]
    kT = thermal_conductivity(prob)
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    out = []
    for axis, (Kc, area, dist, dzf) in enumerate((
            (prob["Kx"], dy * dz, dx, 0.0),
            (prob["Ky"], dx * dz, dy, 0.0),
            (prob["Kz"], dx * dy, dz, dz))):
        if axis == 0:
            lo, hi = idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()
        elif axis == 1:
            lo, hi = idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()
        else:
            lo, hi = idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()
        Tf = area / dist * (2.0 * Kc[lo] * Kc[hi] / (Kc[lo] + Kc[hi]))
        Tcf = area / dist * (2.0 * kT[lo] * kT[hi] / (kT[lo] + kT[hi]))
        out.append((lo, hi, Tf, Tcf, np.full(lo.size, dzf)))
    cat = lambda j: np.concatenate([o[j] for o in out])
    return cat(0), cat(1), cat(2), cat(3), cat(4)


def peaceman_wi(Kx, Ky, Dx=5.0, Dy=5.0, h=5.0, rw=0.1):
    """Peaceman well index 2 pi h K_e / ln(r_e / r_w) with K_e = sqrt(Kx Ky)
    and the anisotropic equivalent radius r_e (Sec. 2.1.5); the paper fixes
    Dx = Dy = 5 m, h = 5 m, r_w = 0.1 m so the model does not change with
    the mesh."""
    Ke = np.sqrt(Kx * Ky)
    ryx, rxy = np.sqrt(Ky / Kx), np.sqrt(Kx / Ky)
    re = 0.14 * np.sqrt(ryx * Dx ** 2 + rxy * Dy ** 2) / (0.5 * (np.sqrt(ryx) + np.sqrt(rxy)))
    return 2.0 * np.pi * h * Ke / np.log(re / rw)


def well_cells(prob):
    """Expand wells into per-cell completions: list of (cell, kind, q_or_WI,
    value, T_inj, U). Rates are split equally over the completed layers; BHP
    producers get one Peaceman WI per completed cell."""
    nx, ny = prob["nx"], prob["ny"]
    comps = []
    for w in prob["wells"]:
        ks = range(w["k0"], w["k1"] + 1)
        nl = len(ks)
        for k in ks:
            c = w["i"] + nx * (w["j"] + ny * k)
            if w["kind"] in (0, 3):
                comps.append((c, w["kind"], w["value"] / nl, w["value"], w["T_inj"], 0.0))
            elif w["kind"] == 1:
                wi = peaceman_wi(prob["Kx"][c], prob["Ky"][c])
                comps.append((c, 1, wi, w["value"], 0.0, 0.0))
            elif w["kind"] == 2:
                comps.append((c, 2, 0.0, 0.0, w["T_inj"], w["U"]))
            else:
                raise ValueError("unknown well kind")
    return comps


# -------------------------------------------------------------- block pattern
def block_pattern(prob):
    """7-point block-CSR pattern: rowptr [N+1], col [nnzb], columns ascending
    (z-1, y-1, x-1, self, x+1, y+1, z+1)."""
    nx, ny, nz = prob["nx"], prob["ny"], prob["nz"]
    N = nx * ny * nz
    i = np.arange(N)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    offs = [(-nx * ny, z > 0), (-nx, y > 0), (-1, x > 0), (0, np.ones(N, bool)),
            (1, x < nx - 1), (nx, y < ny - 1), (nx * ny, z < nz - 1)]
    valid = np.stack([m for _, m in offs], axis=1)
    cols = np.stack([i + o for o, _ in offs], axis=1)
    counts = valid.sum(axis=1)
    rowptr = np.zeros(N + 1, np.int64)
    rowptr[1:] = np.cumsum(counts)
    col = cols[valid]  # row-major order keeps rows contiguous and ascending
    return rowptr, col


def block_positions(rowptr, col, rows, cols):
    """Index into the (row-sorted, column-sorted) pattern of each (row, col)."""
    N = rowptr.size - 1
    key = np.repeat(np.arange(N), np.diff(rowptr)) * N + col
    pos = np.searchsorted(key, rows * N + cols)
    assert np.all(key[pos] == rows * N + cols), "entry outside the pattern"
    return pos


# ---------------------------------------------------------- face quantities
def _face_terms(prob, p, T):
    fl = prob["fluid"]
    lo, hi, Tf, Tcf, dzf = faces(prob)
    cp = cell_props(p, T, fl)
    g = prob["g"]
    rhobar = 0.5 * (cp["rho"][lo] + cp["rho"][hi])
    dphi = p[lo] - p[hi] - rhobar * g * dzf
    up_lo = dphi >= 0.0
    up = np.where(up_lo, lo, hi)
    F = Tf * cp["lam"][up] * dphi
    E = fl["cv"] * T[up] * F + Tcf * (T[lo] - T[hi])
    return dict(lo=lo, hi=hi, Tf=Tf, Tcf=Tcf, dz=dzf, cp=cp, rhobar=rhobar,
                dphi=dphi, up_lo=up_lo, up=up, F=F, E=E)


# ------------------------------------------------------------------ residual
def residual(prob, p, T):
    """G(x) split as (R_m, R_e), each [N] (Eq. Fm, Eq. Fe integrated per
    cell with q = r = indicator of the cell)."""
    fl = prob["fluid"]
    N = p.size
    V = prob["dx"] * prob["dy"] * prob["dz"]
    dt = prob["dt"]
    phi = prob["phi"]
    ft = _face_terms(prob, p, T)
    cp = ft["cp"]
    rho_n = density(prob["p_n"], prob["T_n"], fl)
    Rm = V * phi * (cp["rho"] - rho_n) / dt
    Re = V * (phi * fl["cv"] * (cp["rho"] * T - rho_n * prob["T_n"])
              + (1.0 - phi) * fl["rho_r"] * fl["cr"] * (T - prob["T_n"])) / dt
    np.add.at(Rm, ft["lo"], ft["F"])
    np.add.at(Rm, ft["hi"], -ft["F"])
    np.add.at(Re, ft["lo"], ft["E"])
    np.add.at(Re, ft["hi"], -ft["E"])
    for (c, kind, q, val, Tinj, U) in well_cells(prob):
        if kind == 0:
            rho_inj = density(p[c], Tinj, fl)
            Rm[c] -= q * rho_inj
            Re[c] -= q * rho_inj * fl["cv"] * Tinj
        elif kind == 1:
            dp = p[c] - val
            if dp > 0.0:
                Rm[c] += q * dp * cp["lam"][c]
                Re[c] += q * dp * cp["lam"][c] * fl["cv"] * T[c]
        elif kind == 2:
            Re[c] -= U * (Tinj - T[c])
        elif kind == 3:
            Rm[c] += q * cp["rho"][c]
            Re[c] += q * cp["rho"][c] * fl["cv"] * T[c]
    return Rm, Re


def residual_interleaved(prob, p, T):
    Rm, Re = residual(prob, p, T)
    out = np.empty(2 * p.size)
    out[0::2], out[1::2] = Rm, Re
    return out


# ------------------------------------------------------------------ Jacobian
def jacobian(prob, p, T):
    """Analytic Jacobian dG/dx at (p, T) as block-CSR (rowptr, col, val)
    with val [nnzb, 2, 2] (Eq. AXR; blocks Eq. App .. Eq. rhouT written out
    for the discrete residual). Only the derivative of the selected upwind
    branch is taken; rhobar depends on both cells (1/2 rho_p each)."""
    fl = prob["fluid"]
    N = p.size
    V = prob["dx"] * prob["dy"] * prob["dz"]
    dt = prob["dt"]
    phi = prob["phi"]
    cv = fl["cv"]
    g = prob["g"]
    rowptr, col = block_pattern(prob)
    val = np.zeros((col.size, 2, 2))
    ft = _face_terms(prob, p, T)
    cp = ft["cp"]
    lo, hi, Tf, Tcf, dzf = ft["lo"], ft["hi"], ft["Tf"], ft["Tcf"], ft["dz"]
    dphi, up_lo, up, F = ft["dphi"], ft["up_lo"], ft["up"], ft["F"]
    lam_u = cp["lam"][up]
    # d dPhi / d(p_lo, T_lo, p_hi, T_hi)
    dPhi = [1.0 - 0.5 * cp["rho_p"][lo] * g * dzf,
            -0.5 * cp["rho_T"][lo] * g * dzf,
            -1.0 - 0.5 * cp["rho_p"][hi] * g * dzf,
            -0.5 * cp["rho_T"][hi] * g * dzf]
    # d lam_up / d(...) : nonzero only for the upwind cell's variables
    dLam = [np.where(up_lo, cp["lam_p"][lo], 0.0),
            np.where(up_lo, cp["lam_T"][lo], 0.0),
            np.where(up_lo, 0.0, cp["lam_p"][hi]),
            np.where(up_lo, 0.0, cp["lam_T"][hi])]
    dTup = [0.0, np.where(up_lo, 1.0, 0.0), 0.0, np.where(up_lo, 0.0, 1.0)]
    dTdiff = [0.0, 1.0, 0.0, -1.0]
    dF = [Tf * (dLam[a] * dphi + lam_u * dPhi[a]) for a in range(4)]
    Tu = T[up]
    dE = [cv * (Tu * dF[a] + F * dTup[a]) + Tcf * dTdiff[a] for a in range(4)]
    pos_ll = block_positions(rowptr, col, lo, lo)
    pos_lh = block_positions(rowptr, col, lo, hi)
    pos_hl = block_positions(rowptr, col, hi, lo)
    pos_hh = block_positions(rowptr, col, hi, hi)
    for (pos, sign, a0) in ((pos_ll, 1.0, 0), (pos_lh, 1.0, 2),
                            (pos_hl, -1.0, 0), (pos_hh, -1.0, 2)):
        np.add.at(val[:, 0, 0], pos, sign * dF[a0])
        np.add.at(val[:, 0, 1], pos, sign * dF[a0 + 1])
        np.add.at(val[:, 1, 0], pos, sign * dE[a0])
        np.add.at(val[:, 1, 1], pos, sign * dE[a0 + 1])
    # accumulation
    dpos = block_positions(rowptr, col, np.arange(N), np.arange(N))
    val[dpos, 0, 0] += V * phi * cp["rho_p"] / dt
    val[dpos, 0, 1] += V * phi * cp["rho_T"] / dt
    val[dpos, 1, 0] += V * phi * cv * cp["rho_p"] * T / dt
    val[dpos, 1, 1] += V * (phi * cv * (cp["rho_T"] * T + cp["rho"])
                            + (1.0 - phi) * fl["rho_r"] * fl["cr"]) / dt
    # wells and heaters
    for (c, kind, q, wval, Tinj, U) in well_cells(prob):
        d = dpos[c]
        if kind == 0:
            rho_inj_p = fl["c"] * density(p[c], Tinj, fl)
            val[d, 0, 0] -= q * rho_inj_p
            val[d, 1, 0] -= q * rho_inj_p * cv * Tinj
        elif kind == 1:
            dp = p[c] - wval
            if dp > 0.0:
                lam, lp, lT = cp["lam"][c], cp["lam_p"][c], cp["lam_T"][c]
                val[d, 0, 0] += q * (lam + dp * lp)
                val[d, 0, 1] += q * dp * lT
                val[d, 1, 0] += q * cv * T[c] * (lam + dp * lp)
                val[d, 1, 1] += q * dp * cv * (lT * T[c] + lam)
        elif kind == 2:
            val[d, 1, 1] += U
        elif kind == 3:
            val[d, 0, 0] += q * cp["rho_p"][c]
            val[d, 0, 1] += q * cp["rho_T"][c]
            val[d, 1, 0] += q * cv * cp["rho_p"][c] * T[c]
            val[d, 1, 1] += q * cv * (cp["rho_T"][c] * T[c] + cp["rho"][c])
    return rowptr, col, val


def extract_blocks(val):
    """Scalar value arrays A_pp, A_pT, A_Tp, A_TT sharing the block pattern
    (the four blocks of Eq. AXR)."""
    return val[:, 0, 0].copy(), val[:, 0, 1].copy(), val[:, 1, 0].copy(), val[:, 1, 1].copy()


# ------------------------------------------------------ Schur approximation
def schur_approx(prob, p, T):
    """S~_T of Eq. Se (final form of Eq. schurapproxfull) on the 7-point
    pattern, frozen at the Newton iterate (p, T):

      diag  V[phi c_v rho_i + (1-phi) rho_r c_r]/dt
            + sum over faces where i is upwind of c_v T_f lam_i |dPhi|
            + sum of Tc_f + c_v rho_i q_prod,i + U_i
      (i,j) -Tc_f + (c_v T_f lam_j dPhi_ij if j is upwind else 0)

    The advection term carries c_v as in the semidiscrete form (the fully
    discrete print omits it). The injector and the rho_T accumulation terms
    are dropped, as the derivation assumes.
    """
    fl = prob["fluid"]
    N = p.size
    V = prob["dx"] * prob["dy"] * prob["dz"]
    dt = prob["dt"]
    phi = prob["phi"]
    cv = fl["cv"]
    rowptr, col = block_pattern(prob)
    S = np.zeros(col.size)
    ft = _face_terms(prob, p, T)
    cp = ft["cp"]
    lo, hi, Tf, Tcf = ft["lo"], ft["hi"], ft["Tf"], ft["Tcf"]
    dphi, up_lo = ft["dphi"], ft["up_lo"]
    adv = cv * Tf * cp["lam"][ft["up"]] * dphi  # c_v T_f lam_up dPhi (lo -> hi)
    pos_ll = block_positions(rowptr, col, lo, lo)
    pos_lh = block_positions(rowptr, col, lo, hi)
    pos_hl = block_positions(rowptr, col, hi, lo)
    pos_hh = block_positions(rowptr, col, hi, hi)
    # upwind advection of delta T: lo-row gets +adv on the upwind column,
    # hi-row gets -adv on the same column
    np.add.at(S, pos_ll, np.where(up_lo, adv, 0.0))
    np.add.at(S, pos_hl, np.where(up_lo, -adv, 0.0))
    np.add.at(S, pos_lh, np.where(up_lo, 0.0, adv))
    np.add.at(S, pos_hh, np.where(up_lo, 0.0, -adv))
    # conduction
    np.add.at(S, pos_ll, Tcf)
    np.add.at(S, pos_hh, Tcf)
    np.add.at(S, pos_lh, -Tcf)
    np.add.at(S, pos_hl, -Tcf)
    dpos = block_positions(rowptr, col, np.arange(N), np.arange(N))
    S[dpos] += V * (phi * cv * cp["rho"] + (1.0 - phi) * fl["rho_r"] * fl["cr"]) / dt
    for (c, kind, q, wval, Tinj, U) in well_cells(prob):
        if kind == 1:
            dp = p[c] - wval
            if dp > 0.0:
                S[dpos[c]] += cv * q * dp * cp["lam"][c]   # c_v rho q_prod
        elif kind == 3:
            S[dpos[c]] += cv * q * cp["rho"][c]
        elif kind == 2:
            S[dpos[c]] += U
    return rowptr, col, S


def schur_att(val):
    """S~_ATT = A_TT (Sec. 3.3)."""
    return val[:, 1, 1].copy()


def schur_diag_sparse(rowptr, col, val):
    """S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3) as CSR on the
    structural pattern of A_Tp A_pT (the 25-point stencil, which contains
    A_TT's 7 points). Evaluation order: b_kj = (A_pT)_kj / (A_pp)_kk, one
    division per entry; (A_Tp B)_ij = 0.0 + sum over k ascending of
    (A_Tp)_ik b_kj, one rounded product and one rounded sum at a time;
    S_ij = (A_TT)_ij - (A_Tp B)_ij, or -(A_Tp B)_ij off A_TT's pattern.
    Returns (rowptr, col, values)."""
    N = rowptr.size - 1
    dpos = block_positions(rowptr, col, np.arange(N), np.arange(N))
    App = val[dpos, 0, 0]
    B = val[:, 0, 1].copy()
    for k in range(N):
        for e in range(rowptr[k], rowptr[k + 1]):
            B[e] = val[e, 0, 1] / App[k]
    rows = []
    for i in range(N):
        acc = {}
        for e in range(rowptr[i], rowptr[i + 1]):
            k = col[e]
            a = val[e, 1, 0]
            for f in range(rowptr[k], rowptr[k + 1]):
                j = int(col[f])
                acc[j] = acc.get(j, 0.0) + a * B[f]
        att = {int(col[e]): val[e, 1, 1] for e in range(rowptr[i], rowptr[i + 1])}
        rows.append([(j, att[j] - c if j in att else -c) for j, c in sorted(acc.items())])
    S_rp = np.zeros(N + 1, np.int64)
    S_rp[1:] = np.cumsum([len(r) for r in rows])
    S_c = np.array([j for r in rows for (j, _) in r], dtype=np.int64)
    S_v = np.array([v for r in rows for (_, v) in r], dtype=np.float64)
    return S_rp, S_c, S_v


def schur_diag(rowptr, col, val):
    """S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3). With a 7-point
    A_Tp and A_pT the product has a wider pattern; it is returned as a dense
    matrix (small grids only)."""
    N = rowptr.size - 1
    App, ApT, ATp, ATT = (np.zeros((N, N)) for _ in range(4))
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    App[rows, col], ApT[rows, col] = val[:, 0, 0], val[:, 0, 1]
    ATp[rows, col], ATT[rows, col] = val[:, 1, 0], val[:, 1, 1]
    return ATT - ATp @ np.diag(1.0 / np.diag(App)) @ ApT
