"""Oracle: classical algebraic multigrid (setup and V-cycle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper inverts A_pp and S~_T approximately with one AMG V-cycle each
(Sec. 3.2) using BoomerAMG with classical Ruge-Stueben interpolation and
Gaussian elimination on the coarsest grid (Sec. 4 solver settings). This
oracle takes the parallel-friendly variant: PMIS coarsening with seeded
tie-breaks, modified classical interpolation, Galerkin R A P with R = P^T,
l1-Jacobi or Chebyshev smoothing, and dense LU with partial pivoting on the
coarsest level.

Matrices are CSR triples (rowptr, col, val) with ascending columns in every
row and the diagonal present. Everything that decides structure (strength,
C/F split, interpolation weights, Galerkin sums) is computed in one fixed
order with plain IEEE multiply/add/divide, so that an implementation
following the same order reproduces it bit for bit:
  * interpolation and Galerkin sums run over row entries in ascending column
    order; a sum starts at 0.0 (or at the stated first term) and adds one
    product at a time;
  * a product is one rounded multiply of the two stated factors.
"""
import numpy as np
import scipy.linalg

C_PT, F_PT, U_PT = 1, -1, 0
MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------- helpers
def row_of(A, i):
    rp, c, v = A
    return c[rp[i]:rp[i + 1]], v[rp[i]:rp[i + 1]]


def diag_positions(A):
    rp, c, _ = A
    n = rp.size - 1
    d = np.empty(n, np.int64)
    for i in range(n):
        hits = np.nonzero(c[rp[i]:rp[i + 1]] == i)[0]
        if hits.size != 1:
            raise ValueError(f"row {i} has no diagonal")
        d[i] = rp[i] + hits[0]
    return d


def transpose_positions(A):
    """For every entry e = (i, k), the index of entry (k, i); -1 if absent."""
    rp, c, _ = A
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    key = rows.astype(np.int64) * n + c
    tkey = c.astype(np.int64) * n + rows
    pos = np.searchsorted(key, tkey)
    pos = np.minimum(pos, key.size - 1)
    return np.where(key[pos] == tkey, pos, -1)


def to_dense(A, ncols=None):
    rp, c, v = A
    n = rp.size - 1
    D = np.zeros((n, n if ncols is None else ncols))
    rows = np.repeat(np.arange(n), np.diff(rp))
    np.add.at(D, (rows, c), v)
    return D


def spmv(A, x):
    rp, c, v = A
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    y = np.zeros(n)
    np.add.at(y, rows, v * x[c])
    return y


def splitmix64(x):
    """One output of the splitmix64 generator (Steele, Lea, Flood 2014) whose
    state is x: add the golden gamma, then the two xor-shift-multiply
    rounds and a final xor-shift, all modulo 2^64."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def pmis_hash(seed, i):
    """Tie-break h_i = upper 32 bits of splitmix64(seed xor i)."""
    return splitmix64((seed ^ i) & MASK64) >> 32


# ----------------------------------------------------------------- strength
def strength(A, theta):
    """Classical strength of connection: j != i is a strong dependence of i
    iff -a_ij >= theta * max_{k != i}(-a_ik); a row whose maximum is <= 0
    has no strong dependences. Returns a bool mask over the entries."""
    rp, c, v = A
    n = rp.size - 1
    S = np.zeros(c.size, bool)
    for i in range(n):
        lo, hi = rp[i], rp[i + 1]
        mx = -np.inf
        for e in range(lo, hi):
            if c[e] != i and -v[e] > mx:
                mx = -v[e]
        if not mx > 0.0:
            continue
        thr = theta * mx
        for e in range(lo, hi):
            if c[e] != i and -v[e] >= thr:
                S[e] = True
    return S


# --------------------------------------------------------------------- PMIS
def pmis(A, S, seed, max_rounds=64):
    """PMIS C/F splitting (parallel modified independent set).

    measure lambda_i = #{k : i is a strong dependence of k};
    points with lambda_i = 0 start as F; the rest are undecided. In each
    synchronous round an undecided point whose key (lambda_i, h_i, i) is
    lexicographically larger than the key of every undecided neighbour in
    the symmetrised strength graph S + S^T becomes C; then every still
    undecided point with a strong dependence on a C point becomes F.
    Returns (cf [n] with +1 = C, -1 = F, number of rounds)."""
    rp, c, _ = A
    n = rp.size - 1
    tpos = transpose_positions(A)
    if np.any(tpos < 0):
        raise ValueError("matrix pattern is not structurally symmetric")
    lam = np.zeros(n, np.int64)
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            if c[e] != i and S[tpos[e]]:
                lam[i] += 1
    h = np.array([pmis_hash(seed, i) for i in range(n)], dtype=np.uint64)
    key = lambda i: (int(lam[i]), int(h[i]), i)
    state = np.where(lam == 0, F_PT, U_PT)
    rounds = 0
    while np.any(state == U_PT):
        if rounds >= max_rounds:
            raise RuntimeError("PMIS did not finish within the round cap")
        rounds += 1
        new_c = []
        for i in np.nonzero(state == U_PT)[0]:
            is_max = True
            for e in range(rp[i], rp[i + 1]):
                k = c[e]
                if k == i or state[k] != U_PT:
                    continue
                if (S[e] or S[tpos[e]]) and key(k) > key(i):
                    is_max = False
                    break
            if is_max:
                new_c.append(i)
        state[np.array(new_c, dtype=np.int64)] = C_PT
        new_f = []
        for i in np.nonzero(state == U_PT)[0]:
            for e in range(rp[i], rp[i + 1]):
                if S[e] and state[c[e]] == C_PT:
                    new_f.append(i)
                    break
        state[np.array(new_f, dtype=np.int64)] = F_PT
    return state, rounds


# ------------------------------------------------------------ interpolation
def _opposite(a, d):
    return (d > 0.0 and a < 0.0) or (d < 0.0 and a > 0.0)


def interpolation(A, S, cf):
    """Modified classical (Ruge-Stueben) interpolation.

    C rows: identity. F row i with strong C set C_i^s (empty -> empty row):
      w_ij = -( a_ij + sum_{k in F_i^s} a_ik * ahat_kj / s_k ) / d_i ,
      s_k  = sum_{m in C_i^s} ahat_km,
      d_i  = a_ii + sum_{weak n} a_in + sum_{k in F_i^s, s_k = 0} a_ik,
    where ahat keeps entries whose sign is opposite to the diagonal of their
    row. Order: d_i accumulates over row i ascending; t_k = a_ik / s_k; the
    numerator of j starts at a_ij and adds t_k * ahat_kj over k ascending.
    Coarse columns are numbered by ascending fine index of the C points.
    Returns (P, cidx)."""
    rp, c, v = A
    n = rp.size - 1
    dpos = diag_positions(A)
    cidx = np.cumsum(cf == C_PT) - 1
    nc = int(np.sum(cf == C_PT))
    prow = [None] * n
    for i in range(n):
        if cf[i] == C_PT:
            prow[i] = ([int(cidx[i])], [1.0])
            continue
        ci = [int(c[e]) for e in range(rp[i], rp[i + 1])
              if S[e] and cf[c[e]] == C_PT]
        if not ci:
            prow[i] = ([], [])
            continue
        cset = set(ci)
        denom = v[dpos[i]]
        t = {}
        for e in range(rp[i], rp[i + 1]):
            k = int(c[e])
            if k == i:
                continue
            if not S[e]:
                denom = denom + v[e]
            elif cf[k] == C_PT:
                pass
            else:
                akk = v[dpos[k]]
                s = 0.0
                for f in range(rp[k], rp[k + 1]):
                    m = int(c[f])
                    if m in cset and _opposite(v[f], akk):
                        s = s + v[f]
                if s == 0.0:
                    denom = denom + v[e]
                else:
                    t[k] = v[e] / s
        num = {}
        for e in range(rp[i], rp[i + 1]):
            if int(c[e]) in cset:
                num[int(c[e])] = v[e]
        for k in sorted(t):
            akk = v[dpos[k]]
            for f in range(rp[k], rp[k + 1]):
                m = int(c[f])
                if m in cset and _opposite(v[f], akk):
                    num[m] = num[m] + t[k] * v[f]
        prow[i] = ([int(cidx[j]) for j in ci], [-num[j] / denom for j in ci])
    counts = np.array([len(r[0]) for r in prow])
    P_rp = np.zeros(n + 1, np.int64)
    P_rp[1:] = np.cumsum(counts)
    P_c = np.array([j for r in prow for j in r[0]], dtype=np.int64)
    P_v = np.array([w for r in prow for w in r[1]], dtype=np.float64)
    return (P_rp, P_c, P_v), nc


def interpolation_extpi(A, S, cf):
    """Extended+i (distance-two) interpolation of De Sterck, Falgout,
    Nolting and Yang (2008), the distance-two member of the classical
    interpolation family, used with PMIS because PMIS leaves F points whose
    strong F neighbours share no C point.

    For F row i the interpolatory set is C^_i = C_i^s plus the strong C
    dependences of every strong F neighbour k; with
      s_k = sum_{l in C^_i or l = i} ahat_kl   (row k ascending),
    an F neighbour with s_k = 0 is lumped into the diagonal, otherwise
    t_k = a_ik / s_k and
      d_i  = a_ii + sum_{weak n not in C^_i} a_in + sum_k t_k ahat_ki,
      w_ij = -( a_ij + sum_k t_k ahat_kj ) / d_i   (a_ij = 0 if not adjacent).
    d_i accumulates over row i ascending (the ahat_ki term of k at k's
    position); numerators start at a_ij (or 0.0) and add t_k * ahat_kj over
    k ascending. Empty C^_i gives an empty row. Returns (P, nc)."""
    rp, c, v = A
    n = rp.size - 1
    dpos = diag_positions(A)
    cidx = np.cumsum(cf == C_PT) - 1
    nc = int(np.sum(cf == C_PT))
    prow = [None] * n
    for i in range(n):
        if cf[i] == C_PT:
            prow[i] = ([int(cidx[i])], [1.0])
            continue
        cset = set()
        for e in range(rp[i], rp[i + 1]):
            k = int(c[e])
            if k == i or not S[e]:
                continue
            if cf[k] == C_PT:
                cset.add(k)
            else:
                for f in range(rp[k], rp[k + 1]):
                    if S[f] and cf[c[f]] == C_PT and int(c[f]) != k:
                        cset.add(int(c[f]))
        if not cset:
            prow[i] = ([], [])
            continue
        ci = sorted(cset)
        denom = v[dpos[i]]
        t = {}
        for e in range(rp[i], rp[i + 1]):
            k = int(c[e])
            if k == i:
                continue
            if S[e] and cf[k] != C_PT:
                akk = v[dpos[k]]
                s = 0.0
                aki = None
                for f in range(rp[k], rp[k + 1]):
                    m = int(c[f])
                    if (m in cset or m == i) and _opposite(v[f], akk):
                        s = s + v[f]
                    if m == i:
                        aki = v[f]
                if s == 0.0:
                    denom = denom + v[e]
                else:
                    t[k] = v[e] / s
                    if aki is not None and _opposite(aki, akk):
                        denom = denom + t[k] * aki
            elif k in cset:
                pass
            else:
                denom = denom + v[e]
        num = {j: 0.0 for j in ci}
        for e in range(rp[i], rp[i + 1]):
            if int(c[e]) in cset:
                num[int(c[e])] = v[e]
        for k in sorted(t):
            akk = v[dpos[k]]
            for f in range(rp[k], rp[k + 1]):
                m = int(c[f])
                if m in cset and _opposite(v[f], akk):
                    num[m] = num[m] + t[k] * v[f]
        prow[i] = ([int(cidx[j]) for j in ci], [-num[j] / denom for j in ci])
    counts = np.array([len(r[0]) for r in prow])
    P_rp = np.zeros(n + 1, np.int64)
    P_rp[1:] = np.cumsum(counts)
    P_c = np.array([j for r in prow for j in r[0]], dtype=np.int64)
    P_v = np.array([w for r in prow for w in r[1]], dtype=np.float64)
    return (P_rp, P_c, P_v), nc


def truncate(P, pmax):
    """Interpolation truncation: an F row with more than pmax entries keeps
    the pmax largest |w| (ties to the lower column), each kept weight scaled
    by (sum of all weights) / (sum of kept weights) so the row sum, and with
    it the interpolation of constants, is unchanged. Sums run over the row in
    ascending column order from 0.0; a zero kept sum leaves the kept weights
    unscaled. pmax <= 0 disables truncation."""
    if pmax <= 0:
        return P
    rp, c, v = P
    n = rp.size - 1
    rows = []
    for i in range(n):
        cols = c[rp[i]:rp[i + 1]]
        w = v[rp[i]:rp[i + 1]]
        if cols.size <= pmax:
            rows.append((list(cols), list(w)))
            continue
        order = sorted(range(cols.size), key=lambda q: (-abs(w[q]), cols[q]))
        keep = sorted(order[:pmax])
        s_all = 0.0
        for q in range(cols.size):
            s_all = s_all + w[q]
        s_keep = 0.0
        for q in keep:
            s_keep = s_keep + w[q]
        f = s_all / s_keep if s_keep != 0.0 else 1.0
        rows.append(([cols[q] for q in keep], [w[q] * f for q in keep]))
    P_rp = np.zeros(n + 1, np.int64)
    P_rp[1:] = np.cumsum([len(r[0]) for r in rows])
    P_c = np.array([j for r in rows for j in r[0]], dtype=np.int64)
    P_v = np.array([x for r in rows for x in r[1]], dtype=np.float64)
    return P_rp, P_c, P_v


def transpose(P, ncols):
    """R = P^T with ascending columns per row."""
    rp, c, v = P
    n = rp.size - 1
    rows = [[] for _ in range(ncols)]
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            rows[c[e]].append((i, v[e]))
    R_rp = np.zeros(ncols + 1, np.int64)
    R_rp[1:] = np.cumsum([len(r) for r in rows])
    R_c = np.array([i for r in rows for (i, _) in r], dtype=np.int64)
    R_v = np.array([w for r in rows for (_, w) in r], dtype=np.float64)
    return R_rp, R_c, R_v


def spgemm(A, B):
    """C = A B, keeping every structurally produced entry (no dropping of
    numerical zeros). C_ij = 0.0 + sum over k ascending (row i of A) of the
    product a_ik * b_kj."""
    rp, c, v = A
    brp, bc, bv = B
    n = rp.size - 1
    rows = []
    for i in range(n):
        acc = {}
        for e in range(rp[i], rp[i + 1]):
            k = c[e]
            for f in range(brp[k], brp[k + 1]):
                j = int(bc[f])
                acc[j] = acc.get(j, 0.0) + v[e] * bv[f]
        rows.append(sorted(acc.items()))
    C_rp = np.zeros(n + 1, np.int64)
    C_rp[1:] = np.cumsum([len(r) for r in rows])
    C_c = np.array([j for r in rows for (j, _) in r], dtype=np.int64)
    C_v = np.array([w for r in rows for (_, w) in r], dtype=np.float64)
    return C_rp, C_c, C_v


def galerkin(A, P, R):
    """A_c = R (A P) (Galerkin coarse operator, evaluated as two products)."""
    return spgemm(R, spgemm(A, P))


# -------------------------------------------------------------------- setup
def l1_diag(A):
    """l1-Jacobi scaling d_i = sign(a_ii) (|a_ii| + sum_{j != i} |a_ij|).

    Galerkin operators of the non-symmetric S~_T can carry a few negative
    diagonals on coarse levels; taking the row's l1 norm with the sign of
    its diagonal keeps every sweep a damped Jacobi step for that row (the
    sign convention hypre uses for l1 norms)."""
    rp, c, v = A
    n = rp.size - 1
    d = np.zeros(n)
    for i in range(n):
        diag = 0.0
        off = 0.0
        for e in range(rp[i], rp[i + 1]):
            if c[e] == i:
                diag = v[e]
            else:
                off += abs(v[e])
        d[i] = diag + off if diag >= 0.0 else diag - off
        if d[i] == 0.0:
            raise RuntimeError(f"row {i} is empty")
    return d


def line_factor(A, nxy, nz):
    """Vertical-line smoother of a grid operator (cells i = c + nxy k, column
    c, layer k): T is the tridiagonal part of A along each column, T_ii =
    a_ii and T_{i, i -+ nxy} = a_{i, i -+ nxy}. Factor every column's T by
    the Thomas algorithm (Gaussian elimination without pivoting on a
    tridiagonal matrix, Golub and Van Loan, Matrix Computations, Sec. 4.3):
    m_0 = d_0, m_k = d_k - l_k u_{k-1} / m_{k-1}, with l_k the coefficient
    of the cell below and u_k of the cell above. Returns (l, 1/m, u/m) per
    cell, each [n] in cell order. Needs n = nxy nz and both vertical
    neighbours in every row where they exist."""
    rp, c, v = A
    n = rp.size - 1
    if n != nxy * nz:
        raise ValueError("line smoother: the level is not the nxy x nz grid")
    lo, d, up = np.zeros(n), np.zeros(n), np.zeros(n)
    for i in range(n):
        found_lo = found_up = False
        for e in range(rp[i], rp[i + 1]):
            if c[e] == i:
                d[i] = v[e]
            elif c[e] == i - nxy:
                lo[i], found_lo = v[e], True
            elif c[e] == i + nxy:
                up[i], found_up = v[e], True
        k = i // nxy
        if (k > 0) != found_lo or (k < nz - 1) != found_up:
            raise ValueError("line smoother: a vertical neighbour is missing")
    minv, cp = np.zeros(n), np.zeros(n)
    for col in range(nxy):
        cprev = 0.0
        for k in range(nz):
            i = col + nxy * k
            m = d[i] - lo[i] * cprev
            if m == 0.0 or not np.isfinite(m):
                raise RuntimeError("line smoother: zero pivot")
            minv[i] = 1.0 / m
            cp[i] = up[i] / m
            cprev = cp[i]
    return dict(nxy=nxy, nz=nz, lo=lo, minv=minv, cp=cp)


def line_solve(lf, r):
    """e = T^{-1} r for every column: forward elimination g_k = (r_k - l_k
    g_{k-1}) / m_k, then back substitution e_k = g_k - (u_k / m_k) e_{k+1}."""
    nxy, nz = lf["nxy"], lf["nz"]
    lo, minv, cp = (lf[k].reshape(nz, nxy) for k in ("lo", "minv", "cp"))
    rr = r.reshape(nz, nxy)
    g = np.zeros((nz, nxy))
    for k in range(nz):
        prev = g[k - 1] if k > 0 else np.zeros(nxy)
        g[k] = (rr[k] - lo[k] * prev) * minv[k]
    e = np.zeros((nz, nxy))
    for k in range(nz - 1, -1, -1):
        nxt = e[k + 1] if k < nz - 1 else np.zeros(nxy)
        e[k] = g[k] - cp[k] * nxt
    return e.ravel()


def line_sweep(lf, A, b, x):
    """One vertical-line Jacobi step x <- x + T^{-1} (b - A x); from a zero
    guess (x None) x = T^{-1} b."""
    if x is None:
        return line_solve(lf, b)
    return x + line_solve(lf, b - spmv(A, x))


def setup(A, theta=0.25, seed=0, coarse_size=256, max_levels=25,
          max_coarse_dense=4096, smoother="l1jacobi", cheb_degree=2,
          interp="ext+i", pmax=4, line=None, nu_line=1):
    """Build the hierarchy. Coarsening stops when the level has at most
    coarse_size rows, when max_levels is reached, or when a split keeps
    more than 90% of the points (or none); the coarsest matrix is factored
    by dense LU with partial pivoting (Gaussian elimination, Sec. 4).

    line = (nxy, nz) with nz > 1 smooths the finest level by nu_line
    vertical-line Jacobi steps before and after the coarse correction
    (line_factor) instead of `smoother`; the coarser levels keep
    `smoother`. The paper smooths with hybrid symmetric Gauss-Seidel
    (Sec. 4 solver settings), which carries transport along its sweep
    direction; the line step carries the vertical (gravity-driven) part of
    it exactly and in parallel over columns."""
    levels = []
    cur = A
    while True:
        n = cur[0].size - 1
        lev = dict(A=cur, n=n)
        levels.append(lev)
        if n <= coarse_size or len(levels) >= max_levels:
            break
        S = strength(cur, theta)
        cf, rounds = pmis(cur, S, seed)
        nc = int(np.sum(cf == C_PT))
        if nc == 0 or nc > 0.9 * n:
            break
        if interp == "classical":
            P, nc = interpolation(cur, S, cf)
        else:
            P, nc = interpolation_extpi(cur, S, cf)
        P = truncate(P, pmax)
        R = transpose(P, nc)
        lev.update(S=S, cf=cf, rounds=rounds, P=P, R=R)
        cur = galerkin(cur, P, R)
    for lev in levels:
        lev["dl1"] = l1_diag(lev["A"])
        if smoother == "chebyshev":
            lev["cheb"] = chebyshev_bounds(lev["A"], seed)
    coarse = levels[-1]
    if coarse["n"] > max_coarse_dense:
        raise RuntimeError("coarsest level too large for the dense solve")
    coarse["lu"] = scipy.linalg.lu_factor(to_dense(coarse["A"]))
    if line is not None and line[1] > 1 and len(levels) > 1:
        levels[0]["line"] = line_factor(levels[0]["A"], line[0], line[1])
    return dict(levels=levels, smoother=smoother, cheb_degree=cheb_degree, nu_line=nu_line)


def operator_complexity(h):
    return sum(l["A"][1].size for l in h["levels"]) / h["levels"][0]["A"][1].size


# ---------------------------------------------------------------- smoothing
def chebyshev_bounds(A, seed, iters=10):
    """lambda_max of D^{-1} A by 10 power iterations from a seeded start
    vector (entries h_i / 2^32 + 0.5 with h_i the PMIS hash of the row);
    Chebyshev works on [lambda_max / 30, 1.1 lambda_max]."""
    n = A[0].size - 1
    d = A[2][diag_positions(A)]
    x = np.array([pmis_hash(seed + 1, i) for i in range(n)], float) / 2.0 ** 32 + 0.5
    lam = 0.0
    for _ in range(iters):
        y = spmv(A, x) / d
        lam = np.linalg.norm(y) / np.linalg.norm(x)
        x = y / np.linalg.norm(y)
    return (lam / 30.0, 1.1 * lam, d)


def smooth(lev, b, x, sweeps, kind, degree=2):
    """`sweeps` smoothing steps on A x = b starting from x (None = zero)."""
    A = lev["A"]
    for _ in range(sweeps):
        if kind == "l1jacobi":
            if x is None:
                x = b / lev["dl1"]
            else:
                x = x + (b - spmv(A, x)) / lev["dl1"]
        else:
            lo, hi, d = lev["cheb"]
            x = chebyshev(A, d, b, x, lo, hi, degree)
    return x


def chebyshev(A, d, b, x, lo, hi, degree):
    """Chebyshev polynomial smoother on D^{-1} A over [lo, hi] (three-term
    recurrence of Saad, Iterative Methods, Alg. 12.1)."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x is None:
        x = np.zeros_like(b)
    r = (b - spmv(A, x)) / d
    dk = r / theta
    for k in range(degree):
        x = x + dk
        if k == degree - 1:
            break
        r = r - spmv(A, dk) / d
        rho_new = 1.0 / (2.0 * sigma - rho)
        dk = rho_new * rho * dk + 2.0 * rho_new / delta * r
        rho = rho_new
    return x


def vcycle(h, b, level=0, nu_pre=1, nu_post=1):
    """One V-cycle for A_level x = b from a zero initial guess."""
    levels = h["levels"]
    lev = levels[level]
    if level == len(levels) - 1:
        return scipy.linalg.lu_solve(lev["lu"], b)
    kind, deg = h["smoother"], h["cheb_degree"]
    lf = lev.get("line")
    if lf is not None:
        x = None
        for _ in range(h["nu_line"]):
            x = line_sweep(lf, lev["A"], b, x)
    else:
        x = smooth(lev, b, None, nu_pre, kind, deg)
    if x is None:
        x = np.zeros_like(b)
    r = b - spmv(lev["A"], x)
    bc = spmv(lev["R"], r)
    ec = vcycle(h, bc, level + 1, nu_pre, nu_post)
    x = x + spmv(lev["P"], ec)
    if lf is not None:
        for _ in range(h["nu_line"]):
            x = line_sweep(lf, lev["A"], b, x)
    else:
        x = smooth(lev, b, x, nu_post, kind, deg)
    return x
