"""Parity of the GPU learned Schur correction with the FP64 oracle.

Tolerances: features are computed in FP64 and stored as FP32 (1e-5
relative); the MLP runs on BF16 tensor cores with FP32 accumulation, so its
outputs and gradients are compared at 2e-2 of their scale; exact Schur
columns come from FGMRES solves at rtol 1e-12 (1e-7 relative)."""
import numpy as np
import pytest

from oracle import krylov as okry
from oracle import learned as olearn
from oracle import physics as ophys
from synthetic import make_problem
from synthetic.recipes import perturbed_state
from synthetic.mlp import flatten, initial_params, unflatten

pytestmark = pytest.mark.gpu

thermo = pytest.importorskip("paper_1902_00095_gb300.thermo")


def problem(shape=(12, 10, 6), seed=4):
    prob = make_problem("tiny", shape=shape, seed=seed)
    p, T = perturbed_state(prob, seed=seed)
    prob["p_n"] = prob["p_n"] + 3e4
    return prob, p, T


def random_params(seed):
    rng = np.random.default_rng(seed)
    P = initial_params(seed)
    P["W3"] = rng.normal(0, 0.2, P["W3"].shape)
    P["b1"] = rng.normal(0, 0.1, P["b1"].shape)
    P["b2"] = rng.normal(0, 0.1, P["b2"].shape)
    P["b3"] = rng.normal(0, 0.05, P["b3"].shape)
    return P


@pytest.mark.parametrize("shape,seed", [((12, 10, 6), 4), ((1, 9, 6), 4), ((8, 1, 5), 5)])
def test_features_match_oracle(shape, seed):
    """Also on grids with nx = 1 or ny = 1, where index offsets of different
    face directions coincide: both sides name a face by the grid coordinate
    in which its two cells differ."""
    prob, p, T = problem(shape, seed)
    s = thermo.Solver.from_problem(prob)
    s.assemble(p, T, prob["p_n"], prob["T_n"], prob["dt"])
    X = s.learned_features().astype(np.float64)
    rowptr, col, val = ophys.jacobian(prob, p, T)
    _, _, S = ophys.schur_approx(prob, p, T)
    Xo = olearn.features(prob, p, T, val, S)
    scale = np.maximum(np.abs(Xo).max(axis=0), 1e-30)
    assert np.all(np.abs(X - Xo) <= 1e-5 * scale + 1e-6 * np.abs(Xo))


def test_mlp_forward_matches_oracle():
    P = random_params(3)
    mlp = thermo.MLP(flatten(P))
    X = np.random.default_rng(1).normal(0, 1, (1000, 24))
    O = mlp.forward(X).astype(np.float64)
    Oo, _ = olearn.forward(P, X)
    assert np.max(np.abs(O - Oo)) <= 2e-2 * np.max(np.abs(Oo))
    # the parameters round-trip through FP32
    assert np.allclose(mlp.params(), flatten(P), rtol=1e-6, atol=1e-7)


def _batch(seed, B=777):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (B, 24))
    slot = rng.integers(0, 7, B)
    Sd = rng.uniform(1, 2, B)
    St = np.where(slot == 0, Sd, -rng.uniform(0.05, 0.3, B))
    target = St * rng.uniform(0.7, 1.3, B)
    return X, slot, St, Sd, target


def test_mlp_gradients_match_oracle():
    P = random_params(5)
    mlp = thermo.MLP(flatten(P))
    X, slot, St, Sd, target = _batch(2)
    loss, g = mlp.gradient(X, slot, St, Sd, target)
    lo, go = olearn.loss_and_grads(P, X, slot, St, Sd, target)
    assert abs(loss - lo) <= 2e-2 * lo
    G = unflatten(g)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        ref = go[k]
        assert np.linalg.norm(G[k] - ref) <= 2e-2 * np.linalg.norm(ref), k


def test_adam_step_matches_oracle_on_the_gpu_gradient():
    P = random_params(6)
    mlp = thermo.MLP(flatten(P))
    X, slot, St, Sd, target = _batch(3)
    _, g = mlp.gradient(X, slot, St, Sd, target)
    mlp.train_step(X, slot, St, Sd, target, lr=1e-3)
    new = mlp.params()
    ref = flatten(olearn.adam_step(dict(P), unflatten(g), {}, lr=1e-3))
    assert np.max(np.abs(new - ref)) <= 2e-6


def test_probed_schur_columns_are_exact():
    prob, p, T = problem((10, 9, 5), seed=7)
    s = thermo.Solver.from_problem(prob)
    s.assemble(p, T, prob["p_n"], prob["T_n"], prob["dt"])
    s.build()
    cols = np.array([0, 17, 123, s.N - 1])
    entry, value, its, st = s.probe_schur_columns(cols, rtol=1e-12)
    assert st == 0 and its > 0
    rowptr, col, val = ophys.jacobian(prob, p, T)
    ex = olearn.exact_schur_columns(rowptr, col, val, cols)
    for q, j in enumerate(cols):
        ref = dict(ex[int(j)])
        got = {int(e): v for e, v in zip(entry[q], value[q]) if e >= 0}
        assert set(got) == set(ref)
        scale = max(abs(v) for v in ref.values())
        for e in ref:
            assert abs(got[e] - ref[e]) <= 1e-7 * scale


def test_identity_network_reproduces_the_plain_solve():
    """W3 = 0, b3 = 0: every output is 0, the corrected S~ equals S~ and the
    solve is the plain one."""
    prob, p, T = problem()
    s = thermo.Solver.from_problem(prob)
    s.assemble(p, T, prob["p_n"], prob["T_n"], prob["dt"])
    s.build(schur=0)
    _, _, plain = s.solve(rtol=1e-8)
    mlp = thermo.MLP(flatten(initial_params(0)))
    s.set_schur_model(mlp)
    s.build(schur=1)
    _, _, learned = s.solve(rtol=1e-8)
    assert s.learned_status() == (0, False)
    assert learned["iters"] == plain["iters"]
    assert abs(learned["rel_res"] - plain["rel_res"]) <= 1e-12


def test_guard_rejects_a_destructive_network():
    """A network whose o_7 = -3 makes every corrected diagonal negative: all
    rows fall back, the whole matrix reverts to plain S~ and the solve still
    converges."""
    prob, p, T = problem()
    P = initial_params(0)
    P["b3"][7] = -3.0
    s = thermo.Solver.from_problem(prob)
    s.assemble(p, T, prob["p_n"], prob["T_n"], prob["dt"])
    mlp = thermo.MLP(flatten(P))
    s.set_schur_model(mlp)
    s.build(schur=1)
    rows, glob = s.learned_status()
    assert rows == s.N and glob
    _, _, info = s.solve(rtol=1e-8)
    assert info["status"] == 0


def test_training_on_probed_columns_reduces_the_loss_and_solves():
    from paper_1902_00095_gb300 import learned as L
    rng = np.random.Generator(np.random.PCG64(0))
    parts = []
    for q in range(3):
        prob = make_problem("tiny", shape=(16, 16, 8), seed=100 + q)
        s = thermo.Solver.from_problem(prob)
        parts.append(L.collect_samples(s, prob, 96, rng))
        s.close()
    data = L.concat(parts)
    mlp, hist = L.train(data, flatten(initial_params(0)), epochs=30, batch=512, lr=3e-3)
    assert hist[-1] < 0.7 * hist[0]
    ev = L.evaluate(mlp, make_problem("tiny", shape=(16, 16, 8), seed=777))
    assert ev["learned_rel_res"] <= 1e-8


def test_trained_network_never_loses_to_the_plain_approximation():
    """What the learned correction gains, measured on an unseen problem: the
    RMS error of the corrected S~ against exact Schur-complement entries
    (probed columns, relative to the row's diagonal) and the FGMRES count,
    each against plain S~_T. At a Newton iterate equal to the previous time
    level S~_T of Eq. Se already matches the Schur complement to about 1e-7,
    below what a BF16 network can resolve; training then selects the
    untrained identity correction on held-out samples, so the gain is nil
    and nothing is lost. The bounds asserted are those guarantees."""
    from paper_1902_00095_gb300 import learned as L
    rng = np.random.Generator(np.random.PCG64(1))
    parts = []
    for q in range(4):
        prob = make_problem("grf32", shape=(16, 16, 8), seed=1000 + q)
        s = thermo.Solver.from_problem(prob)
        parts.append(L.collect_samples(s, prob, 128, rng))
        s.close()
    mlp, hist = L.train(L.concat(parts), flatten(initial_params(0)), epochs=40, batch=512,
                        lr=2e-3)
    assert mlp.val_losses[mlp.selected_epoch] == min(mlp.val_losses)
    prob = make_problem("grf32", shape=(16, 16, 8), seed=1999)
    s = thermo.Solver.from_problem(prob)
    s.assemble(prob["p_k"], prob["T_k"], prob["p_n"], prob["T_n"], prob["dt"])
    s.build(schur=0)
    _, _, plain = s.solve(rtol=1e-8)
    rp, col, val, S, _ = s.export_system()
    cols = rng.choice(s.N, 64, replace=False)
    entry, value, its, st = s.probe_schur_columns(cols, 1e-11)
    assert st == 0
    s.set_schur_model(mlp)
    s.build(schur=1)
    _, _, learned = s.solve(rtol=1e-8)
    assert s.learned_status()[1] is False
    SL = s.export_level(1, 0)["A"][2]
    ok = entry >= 0
    e = entry[ok]
    tgt = value[ok]
    rows = np.repeat(np.arange(s.N), np.diff(rp))[e]
    dpos = np.array([rp[i] + np.searchsorted(col[rp[i]:rp[i + 1]], i) for i in range(s.N)])
    Sd = S[dpos[rows]]
    err_plain = np.sqrt(np.mean(((S[e] - tgt) / Sd) ** 2))
    err_learned = np.sqrt(np.mean(((SL[e] - tgt) / Sd) ** 2))
    assert err_plain < 1e-5
    assert err_learned <= 1.05 * err_plain + 1e-7, (err_learned, err_plain, mlp.selected_epoch)
    assert learned["iters"] <= plain["iters"] + 2
    assert learned["rel_res"] <= 1e-8


def test_learned_correction_gains_at_time_stepping_states():
    """What the learned correction gains where S~_T is not exact: at the
    start of a second 30-day step (behind a temperature front) S~_T of
    Eq. Se differs from the exact Schur complement by under a per cent; a
    network trained on probed exact entries of eight such problems lowers
    that error on an unseen problem by a tenth or more, and FGMRES needs at
    most one iteration more than with plain S~_T."""
    from paper_1902_00095_gb300 import learned as L
    rng = np.random.Generator(np.random.PCG64(3))
    shape = (12, 12, 8)
    parts = []
    for q in range(8):
        prob = make_problem("grf32", shape=shape, seed=1000 + q, dt_days=30.0)
        s = thermo.Solver.from_problem(prob)
        parts.append(L.collect_samples(s, L.advance_one_step(s, prob), 256, rng))
        s.close()
    mlp, hist = L.train(L.concat(parts), flatten(initial_params(0)), epochs=80, batch=512,
                        lr=1e-3)
    assert mlp.selected_epoch > 0, mlp.val_losses[:3]
    prob = make_problem("grf32", shape=shape, seed=1999, dt_days=30.0)
    s = thermo.Solver.from_problem(prob)
    nxt = L.advance_one_step(s, prob)
    s.assemble(nxt["p_k"], nxt["T_k"], nxt["p_n"], nxt["T_n"], nxt["dt"])
    s.build(schur=0)
    _, _, plain = s.solve(rtol=1e-8)
    rp, col, val, S, _ = s.export_system()
    cols = rng.choice(s.N, 96, replace=False)
    entry, value, its, st = s.probe_schur_columns(cols, 1e-11)
    assert st == 0
    s.set_schur_model(mlp)
    s.build(schur=1)
    _, _, learned = s.solve(rtol=1e-8)
    assert s.learned_status()[1] is False
    SL = s.export_level(1, 0)["A"][2]
    ok = entry >= 0
    e = entry[ok]
    tgt = value[ok]
    rows = np.repeat(np.arange(s.N), np.diff(rp))[e]
    dpos = np.array([rp[i] + np.searchsorted(col[rp[i]:rp[i + 1]], i) for i in range(s.N)])
    Sd = S[dpos[rows]]
    err_plain = np.sqrt(np.mean(((S[e] - tgt) / Sd) ** 2))
    err_learned = np.sqrt(np.mean(((SL[e] - tgt) / Sd) ** 2))
    report = (err_learned, err_plain, learned["iters"], plain["iters"], mlp.selected_epoch)
    assert 1e-4 < err_plain < 5e-2, report
    assert err_learned < 0.9 * err_plain, report
    assert learned["iters"] <= plain["iters"] + 1, report
    assert learned["rel_res"] <= 1e-8


def partial_fallback_params(seed=42):
    """A network that changes every entry (outputs of order one) and whose
    diagonal term o_7 is negative enough on some rows to make the corrected
    diagonal non-positive there: the guard rejects about 7-14 % of the rows,
    below the 25 % global fallback."""
    P = initial_params(0)
    rng = np.random.default_rng(seed)
    P["W3"] = rng.normal(0, 0.5, P["W3"].shape)
    P["b3"] = rng.normal(0, 0.2, 8)
    P["W3"][7] = rng.normal(0, 1.0, 64)
    P["b3"][7] = -0.5
    return P


@pytest.mark.parametrize("shape,seed", [((7, 6, 5), 3), ((1, 9, 6), 4), ((8, 1, 5), 5)])
def test_learned_schur_matches_oracle_correction(shape, seed):
    """The corrected S~ of a learned build equals the oracle's correction
    (oracle.learned.apply_correction) of the same plain S~ with the same
    network outputs, entry by entry, and the rows that fall back are the
    same; some rows fall back, fewer than a quarter (no global fallback).
    The outputs are the GPU network's (BF16 tensor cores) evaluated on the
    GPU features through tp_mlp_forward, the kernel the build runs."""
    prob, p, T = problem(shape, seed)
    s = thermo.Solver.from_problem(prob)
    s.assemble(p, T, prob["p_n"], prob["T_n"], prob["dt"])
    mlp = thermo.MLP(flatten(partial_fallback_params()))
    s.set_schur_model(mlp)
    s.build(schur=1)
    rows, glob = s.learned_status()
    _, _, _, S_plain, _ = s.export_system()
    S_learned = s.export_level(1, 0)["A"][2]
    O = mlp.forward(s.learned_features()).astype(np.float64)
    want, bad = olearn.apply_correction(prob, S_plain, O)
    assert 0 < rows == int(bad.sum()) < s.N / 4 and not glob, (rows, int(bad.sum()), s.N)
    rp, _ = ophys.block_pattern(prob)
    r = np.repeat(np.arange(s.N), np.diff(rp))
    scale = np.zeros(s.N)
    np.maximum.at(scale, r, np.abs(want))
    assert np.all(np.abs(S_learned - want) <= 1e-12 * scale[r]), np.max(np.abs(S_learned - want))
    # changed entries outside the fallback rows
    assert np.any(np.abs(S_learned - S_plain) > 1e-3 * scale[r])


def test_overflowing_network_output_falls_back():
    """An output of 800 for the z- direction overflows exp to +inf: every
    row with a cell below falls back (not finite), as in the oracle, and with
    more than a quarter of the rows rejected the build uses plain S~."""
    prob, p, T = problem((7, 6, 5), 3)
    P = initial_params(0)
    P["b3"][1] = 800.0
    s = thermo.Solver.from_problem(prob)
    s.assemble(p, T, prob["p_n"], prob["T_n"], prob["dt"])
    mlp = thermo.MLP(flatten(P))
    s.set_schur_model(mlp)
    s.build(schur=1)
    rows, glob = s.learned_status()
    _, _, _, S_plain, _ = s.export_system()
    O = mlp.forward(s.learned_features()).astype(np.float64)
    _, bad = olearn.apply_correction(prob, S_plain, O)
    assert rows == int(bad.sum()) == 7 * 6 * 4 and glob
    assert np.array_equal(s.export_level(1, 0)["A"][2], S_plain)
    _, _, info = s.solve(rtol=1e-8)
    assert info["status"] == 0
