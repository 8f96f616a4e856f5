"""Oracle: learned correction of the Schur approximation (spec growth
direction; the paper has no learned component).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A per-cell MLP 24 -> 64 -> 64 -> 8 (GELU, tanh form) maps local features of
cell i to output o; row i of S~_T (Eq. Se) becomes
    S_ii <- S~_ii exp(o_0) + o_7 S~_ii,
    S_ij <- S~_ij exp(o_d)     (d = 1..6 the face direction of j),
and is trained on exact Schur complement entries S = A_TT - A_Tp A_pp^{-1}
A_pT (Sec. 3.2, Eq. Afact) restricted to the 7-point pattern, obtained one
column at a time: z = A_pp^{-1} A_pT e_j, S e_j = A_TT e_j - A_Tp z.
Loss: mean over sampled entries of ((S_learned,ij - S_ij) / S_ii)^2.
Everything here is float64.
"""
import numpy as np
import scipy.sparse
import scipy.sparse.linalg

from synthetic import mlp as _mlp_init

from . import physics

NF, NH, NO = 24, 64, 8
# face directions in block-pattern column order; slot 3 is the diagonal
DIRS = ("z-", "y-", "x-", "x+", "y+", "z+")


def direction_slots(prob):
    """For every pattern entry e = (i, j): 0 for the diagonal, 1..6 for the
    face direction of j seen from i (z-, y-, x-, x+, y+, z+), read from the
    cells' grid coordinates (the one coordinate in which i and j differ), so
    that grids with nx = 1 or ny = 1, where index offsets coincide, still
    name the face's true direction."""
    nx, ny = prob["nx"], prob["ny"]
    rowptr, col = physics.block_pattern(prob)
    N = rowptr.size - 1
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    coord = lambda c: (c % nx, (c // nx) % ny, c // (nx * ny))
    xi, yi, zi = coord(rows)
    xj, yj, zj = coord(col)
    slot = np.zeros(col.size, np.int64)
    for k, m in enumerate((zj < zi, yj < yi, xj < xi, xj > xi, yj > yi, zj > zi)):
        slot[m] = k + 1
    return rowptr, col, slot


# ------------------------------------------------------------------ features
def features(prob, p, T, val, S):
    """24 features per cell (float64 [N, 24]):
      0-5   log10(T_f / 1e-12 m^3) per face direction (0 where no face)
      6-11  log10(Tc_f / 1 W/K) per face direction (0 where no face)
      12    log10(lam_i / 1e6)
      13-18 advective face coefficient c_v T_f lam_up dPhi (out of cell i)
            divided by S~_ii, per face direction
      19    A_pT,ii A_Tp,ii / (A_pp,ii A_TT,ii)
      20    log10(A_pp,ii s_m),  21  log10(A_TT,ii s_e)
      22    (A_TT,ii - S~_ii) / S~_ii
      23    V [phi c_v rho + (1 - phi) rho_r c_r] / dt / S~_ii
    with s_m = N / sum|A_pp,ii|, s_e = N / sum|A_TT,ii|."""
    fl = prob["fluid"]
    N = p.size
    rowptr, col, slot = direction_slots(prob)
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    ft = physics._face_terms(prob, p, T)
    lo, hi = ft["lo"], ft["hi"]
    adv = fl["cv"] * ft["Tf"] * ft["cp"]["lam"][ft["up"]] * ft["dphi"]
    dpos = physics.block_positions(rowptr, col, np.arange(N), np.arange(N))
    Sd = S[dpos]
    F = np.zeros((N, NF))
    pos_lh = physics.block_positions(rowptr, col, lo, hi)
    pos_hl = physics.block_positions(rowptr, col, hi, lo)
    for pos, r, sign in ((pos_lh, lo, 1.0), (pos_hl, hi, -1.0)):
        k = slot[pos] - 1  # 0..5
        F[r, k] = np.log10(ft["Tf"] / 1e-12)
        F[r, 6 + k] = np.log10(ft["Tcf"] / 1.0)
        F[r, 13 + k] = sign * adv / Sd[r]
    cp = ft["cp"]
    F[:, 12] = np.log10(cp["lam"] / 1e6)
    App, ApT, ATp, ATT = (val[dpos, a, b] for a, b in ((0, 0), (0, 1), (1, 0), (1, 1)))
    s_m = N / np.sum(np.abs(App))
    s_e = N / np.sum(np.abs(ATT))
    F[:, 19] = ApT * ATp / (App * ATT)
    F[:, 20] = np.log10(np.abs(App) * s_m)
    F[:, 21] = np.log10(np.abs(ATT) * s_e)
    F[:, 22] = (ATT - Sd) / Sd
    V = prob["dx"] * prob["dy"] * prob["dz"]
    acc = V * (prob["phi"] * fl["cv"] * cp["rho"] + (1 - prob["phi"]) * fl["rho_r"] * fl["cr"]) / prob["dt"]
    F[:, 23] = acc / Sd
    return F


# ------------------------------------------------------ exact Schur columns
def exact_schur_columns(rowptr, col, val, cols):
    """S restricted to the 7-point pattern on the given columns j: returns a
    dict j -> list of (pattern entry index e = (i, j), S_ij)."""
    N = rowptr.size - 1
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    mk = lambda v: scipy.sparse.csr_matrix((v, (rows, col)), shape=(N, N))
    App, ApT, ATp, ATT = (mk(val[:, a, b]) for a, b in ((0, 0), (0, 1), (1, 0), (1, 1)))
    lu = scipy.sparse.linalg.splu(App.tocsc())
    out = {}
    for j in cols:
        z = lu.solve(np.asarray(ApT[:, j].todense()).ravel())
        sj = np.asarray(ATT[:, j].todense()).ravel() - ATp @ z
        ents = []
        for i in col[rowptr[j]:rowptr[j + 1]]:  # pattern is symmetric: rows i of column j
            e = rowptr[i] + np.nonzero(col[rowptr[i]:rowptr[i + 1]] == j)[0][0]
            ents.append((int(e), float(sj[i])))
        out[int(j)] = ents
    return out


# ---------------------------------------------------------------------- MLP
def gelu(x):
    """GELU, tanh form: 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))."""
    c = np.sqrt(2.0 / np.pi)
    return 0.5 * x * (1.0 + np.tanh(c * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    c = np.sqrt(2.0 / np.pi)
    u = c * (x + 0.044715 * x ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * c * (1.0 + 3 * 0.044715 * x * x)


def init_params(seed):
    """Seeded initial weights (synthetic.mlp: W1, W2 uniform / sqrt(fan_in),
    W3 and biases zero, so the untrained network is the identity
    correction)."""
    return _mlp_init.initial_params(seed)


def forward(params, X):
    z1 = X @ params["W1"].T + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(z2)
    o = h2 @ params["W3"].T + params["b3"]
    return o, (X, z1, h1, z2, h2)


def learned_entries(o, slot, St, Sd):
    """Corrected values of sampled entries: slot 0 diagonal, 1..6 faces."""
    pick = np.where(slot == 0, 0, slot)
    val = St * np.exp(o[np.arange(o.shape[0]), pick])
    val = val + np.where(slot == 0, o[:, 7] * Sd, 0.0)
    return val


def loss_and_grads(params, X, slot, St, Sd, target):
    """Mean squared relative error and its gradients w.r.t. all parameters.
    Sample s: features X[s], entry slot, S~ value St, S~ diagonal Sd, exact
    S value target."""
    o, (X, z1, h1, z2, h2) = forward(params, X)
    B = X.shape[0]
    pick = np.where(slot == 0, 0, slot)
    e = np.exp(o[np.arange(B), pick])
    pred = St * e + np.where(slot == 0, o[:, 7] * Sd, 0.0)
    r = (pred - target) / Sd
    loss = np.mean(r * r)
    dpred = 2.0 * r / Sd / B
    do = np.zeros_like(o)
    do[np.arange(B), pick] = dpred * St * e
    do[:, 7] += np.where(slot == 0, dpred * Sd, 0.0)
    g = {}
    g["W3"] = do.T @ h2
    g["b3"] = do.sum(0)
    dh2 = do @ params["W3"]
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, g


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma and Ba 2015) with bias correction; state holds t, m, v."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = b1 * m + (1 - b1) * grads[k]
        v[...] = b2 * v + (1 - b2) * grads[k] ** 2
        mhat = m / (1 - b1 ** t)
        vhat = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return params


# ------------------------------------------------------ learned S~ + guard
def apply_correction(prob, S, O):
    """Learned S~ values on the pattern from per-cell outputs O [N, 8], with
    the per-row guard: a row falls back to plain S~ if its corrected diagonal
    is not positive or an off-diagonal changes sign or the row loses the
    diagonal dominance the plain row had, or any corrected value of the row
    is not finite (exp of a large output overflows to inf, which passes the
    sign and dominance tests). Returns (values, fallback rows)."""
    rowptr, col, slot = direction_slots(prob)
    N = rowptr.size - 1
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    dpos = physics.block_positions(rowptr, col, np.arange(N), np.arange(N))
    Sd = S[dpos]
    pick = np.where(slot == 0, 0, slot)
    with np.errstate(over="ignore", invalid="ignore"):
        new = S * np.exp(O[rows, pick]) + np.where(slot == 0, O[rows, 7] * Sd[rows], 0.0)
    off = slot != 0
    bad = np.zeros(N, bool)
    np.logical_or.at(bad, rows[~np.isfinite(new)], True)
    newd = new[dpos]
    bad |= ~(newd > 0)
    flip = off & (np.sign(new) != np.sign(S))
    np.logical_or.at(bad, rows[flip], True)
    offsum_old = np.zeros(N)
    offsum_new = np.zeros(N)
    np.add.at(offsum_old, rows[off], np.abs(S[off]))
    np.add.at(offsum_new, rows[off], np.abs(new[off]))
    bad |= (Sd >= offsum_old) & (newd < offsum_new)
    out = np.where(bad[rows], S, new)
    return out, bad
