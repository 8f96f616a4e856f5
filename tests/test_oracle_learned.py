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
