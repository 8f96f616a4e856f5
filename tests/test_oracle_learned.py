"""Pins of the oracle's learned Schur correction: finite-difference
gradients, Adam's first step, exact Schur columns against the dense Schur
complement (Sec. 3.2), the identity of an untrained network, and the guard."""
import numpy as np
import pytest

from oracle import krylov, learned, physics
from synthetic import make_problem, default_fluid
from synthetic.recipes import perturbed_state


def small(shape=(5, 4, 3), seed=3, fluid=None):
    prob = make_problem("tiny", shape=shape, seed=seed, fluid=fluid)
    p, T = perturbed_state(prob, seed=seed)
    rowptr, col, val = physics.jacobian(prob, p, T)
    _, _, S = physics.schur_approx(prob, p, T)
    return prob, p, T, rowptr, col, val, S


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    params = learned.init_params(1)
    params["W3"] = rng.normal(0, 0.3, params["W3"].shape)
    params["b3"] = rng.normal(0, 0.1, 8)
    params["b1"] = rng.normal(0, 0.1, 64)
    B = 12
    X = rng.normal(0, 1, (B, 24))
    slot = rng.integers(0, 7, B)
    Sd = rng.uniform(1, 2, B)
    St = np.where(slot == 0, Sd, -rng.uniform(0.1, 0.3, B))
    target = St * rng.uniform(0.8, 1.2, B)
    loss, g = learned.loss_and_grads(params, X, slot, St, Sd, target)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = params[k].reshape(-1)
        for idx in rng.choice(flat.size, min(8, flat.size), replace=False):
            h = 1e-6
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = learned.loss_and_grads(params, X, slot, St, Sd, target)
            flat[idx] = old - h
            lm, _ = learned.loss_and_grads(params, X, slot, St, Sd, target)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx)


def test_adam_first_step_moves_by_lr_times_sign():
    """With zero moments, bias correction makes the first Adam step
    -lr g / (|g| + eps) (Kingma and Ba 2015, Alg. 1)."""
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    out = learned.adam_step(dict(p), g, {}, lr=0.01)
    assert np.allclose(out["w"], p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=0, atol=1e-15)


def test_exact_schur_columns_match_dense_schur_complement():
    prob, p, T, rowptr, col, val, S = small()
    N = rowptr.size - 1
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    D = lambda a, b: np.asarray(__import__("scipy").sparse.csr_matrix(
        (val[:, a, b], (rows, col)), shape=(N, N)).todense())
    Sx = D(1, 1) - D(1, 0) @ np.linalg.solve(D(0, 0), D(0, 1))
    cols = [0, 7, N - 1, N // 2]
    out = learned.exact_schur_columns(rowptr, col, val, cols)
    for j in cols:
        for e, v in out[j]:
            i = rows[e]
            assert col[e] == j
            assert abs(v - Sx[i, j]) <= 1e-9 * np.abs(Sx[i]).max()


def test_untrained_network_is_the_identity_correction():
    prob, p, T, rowptr, col, val, S = small()
    params = learned.init_params(7)
    X = learned.features(prob, p, T, val, S)
    o, _ = learned.forward(params, X)
    assert np.all(o == 0.0)
    new, bad = learned.apply_correction(prob, S, o)
    assert np.array_equal(new, S) and not bad.any()


def test_guard_falls_back_on_indefinite_rows():
    prob, p, T, rowptr, col, val, S = small()
    N = rowptr.size - 1
    O = np.zeros((N, 8))
    O[3, 7] = -2.0          # diagonal -> S_ii (1 - 2) < 0
    O[5, 1:7] = 3.0         # off-diagonals grow e^3 times: loses dominance
    new, bad = learned.apply_correction(prob, S, O)
    assert bad[3] and bad[5] and bad.sum() == 2
    r = slice(rowptr[3], rowptr[4])
    assert np.array_equal(new[r], S[r])


def test_decoupled_features_vanish():
    """With A_pT = 0 and S~ = A_TT (beta = 0, T-independent viscosity) the
    coupling feature and the A_TT - S~ feature are zero."""
    fl = default_fluid(beta=0.0, mu_coef=0.0)
    prob, p, T, rowptr, col, val, S = small(fluid=fl)
    X = learned.features(prob, p, T, val, S)
    assert np.all(X[:, 19] == 0.0)
    assert np.max(np.abs(X[:, 22])) < 1e-12
    assert X.shape == (rowptr.size - 1, 24)


def test_training_reduces_the_loss():
    prob, p, T, rowptr, col, val, S = small((6, 5, 4), seed=5)
    X = learned.features(prob, p, T, val, S)
    N = rowptr.size - 1
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    _, _, slot = learned.direction_slots(prob)
    dpos = physics.block_positions(rowptr, col, np.arange(N), np.arange(N))
    cols = list(range(0, N, 3))
    ex = learned.exact_schur_columns(rowptr, col, val, cols)
    ents = [e for j in cols for e in ex[j]]
    e = np.array([a for a, _ in ents])
    tgt = np.array([b for _, b in ents])
    Xs, sl, St, Sd = X[rows[e]], slot[e], S[e], S[dpos[rows[e]]]
    params = learned.init_params(2)
    state = {}
    l0, _ = learned.loss_and_grads(params, Xs, sl, St, Sd, tgt)
    for _ in range(200):
        loss, g = learned.loss_and_grads(params, Xs, sl, St, Sd, tgt)
        params = learned.adam_step(params, g, state, lr=3e-3)
    assert loss < 0.5 * l0


def test_features_by_hand_on_two_cells():
    """All 24 features of a 2 x 1 x 1 grid evaluated by hand (see
    tests/test_oracle_physics.py::two_cells: flow from cell 0 to cell 1,
    dPhi = 1e5 Pa, T_f = 1.5e-12 m^3, Tc_f = 9.6979592 W/K, lambda =
    9.99e5 and 999 / (1e-3 exp(-0.2)), advective coefficient 626.9724 W/K,
    accumulation 32249.574 W/K, S~ diagonals 32886.244 and 32259.272, A_pp
    diagonals 1.4985e-6, A_pT,00 = 2.997e-3, A_Tp,00 = 2.00631168, A_TT
    diagonals 36898.868 and 32259.272): cell 0 sees its neighbour through
    x+ (slot 3), cell 1 through x- (slot 2); 19 is A_pT A_Tp / (A_pp A_TT),
    20/21 the log10 of the diagonals times s_m = 2 / sum|A_pp,ii| and s_e,
    22 (A_TT - S~)/S~, 23 the accumulation over S~_ii; the outward advective
    coefficient is +626.97 out of cell 0 and -626.97 out of cell 1."""
    from test_oracle_physics import two_cells
    prob = two_cells()
    p, T = prob["p_k"], prob["T_k"]
    rowptr, col, val = physics.jacobian(prob, p, T)
    _, _, S = physics.schur_approx(prob, p, T)
    F = learned.features(prob, p, T, val, S)
    f0 = np.zeros(24)
    f1 = np.zeros(24)
    f0[3] = f1[2] = 0.17609125905568124           # log10(1.5)
    f0[9] = f1[8] = 0.9866803519446234            # log10(9.6979592)
    f0[12], f1[12] = -0.0004345117740176917, 0.08642438460663264
    f0[16], f1[15] = 0.019064882926125334, -0.019435416873437864
    f0[19] = 0.10874651716910394
    f0[21], f1[21] = 0.0281997327426756, -0.030158744886521743
    f0[22] = 0.1220152507272021
    f0[23], f1[23] = 0.9806402229821107, 0.999699374518629
    np.testing.assert_allclose(F[0], f0, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(F[1], f1, rtol=1e-12, atol=1e-15)


def test_guard_falls_back_on_non_finite_values():
    """An output of 1e3 overflows exp to +inf; inf passes the sign test and a
    diagonal of +inf passes the positivity test, so the guard must reject
    the row for not being finite; the other rows keep their corrections."""
    prob, p, T, rowptr, col, val, S = small()
    N = p.size
    O = np.full((N, 8), 0.01)
    O[5, 0] = 1e3      # diagonal of row 5 -> +inf
    O[7, 4] = 1e3      # the x+ off-diagonal of row 7 -> -inf
    out, bad = learned.apply_correction(prob, S, O)
    assert bad[5] and bad[7]
    assert bad.sum() == 2
    assert np.all(np.isfinite(out))


def test_direction_slots_on_degenerate_grids():
    """With nx = 1 the neighbour at index offset -1 is the cell below in y
    (slot 2, y-) and +1 the one above in y (slot 5, y+); with ny = 1 the
    offset -nx is the cell below in z (slot 1, z-): the slot names the grid
    coordinate in which the two cells differ."""
    prob = make_problem("tiny", shape=(1, 4, 3), seed=1)
    rowptr, col, slot = learned.direction_slots(prob)
    i = 5    # (x, y, z) = (0, 1, 1)
    got = {int(c) - i: int(s) for c, s in zip(col[rowptr[i]:rowptr[i + 1]],
                                              slot[rowptr[i]:rowptr[i + 1]])}
    assert got == {-4: 1, -1: 2, 0: 0, 1: 5, 4: 6}
    prob = make_problem("tiny", shape=(3, 1, 4), seed=1)
    rowptr, col, slot = learned.direction_slots(prob)
    i = 4    # (1, 0, 1)
    got = {int(c) - i: int(s) for c, s in zip(col[rowptr[i]:rowptr[i + 1]],
                                              slot[rowptr[i]:rowptr[i + 1]])}
    assert got == {-3: 1, -1: 3, 0: 0, 1: 4, 3: 6}
