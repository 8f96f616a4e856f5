"""Host logic of the step-cutting time-step driver, against a stand-in
solver whose Newton iteration converges only for steps up to a limit."""
import numpy as np

from paper_1902_00095_gb300 import thermo
from paper_1902_00095_gb300.timestep import advance


class FakeSolver:
    """Newton 'converges' iff dt <= limit; the state advances by dt."""

    def __init__(self, limit):
        self.limit = limit
        self.calls = []

    def newton_step(self, p, T, dt, **kw):
        self.calls.append(dt)
        ok = dt <= self.limit
        return p + dt, T + dt, {"status": 0 if ok else 1, "newton_iters": 3}


def test_accepted_step_is_taken_whole():
    s = FakeSolver(limit=30.0)
    p, T, rec = advance(s, np.zeros(2), np.zeros(2), 30.0)
    assert s.calls == [30.0] and len(rec) == 1 and rec[0]["accepted"]
    assert np.all(p == 30.0)


def test_failed_step_is_repeated_as_halves_recursively():
    s = FakeSolver(limit=8.0)
    p, T, rec = advance(s, np.zeros(2), np.zeros(2), 30.0, max_cuts=3)
    # 30 fails, 15 fails, 7.5 twice succeeds, then 15 fails again, 7.5 twice
    assert s.calls == [30.0, 15.0, 7.5, 7.5, 15.0, 7.5, 7.5]
    assert [r["accepted"] for r in rec] == [False, False, True, True, False, True, True]
    assert np.all(p == 30.0)  # the halves add up to the whole step


def test_cut_limit_accepts_the_last_attempt():
    s = FakeSolver(limit=1.0)
    p, T, rec = advance(s, np.zeros(1), np.zeros(1), 8.0, max_cuts=1)
    assert s.calls == [8.0, 4.0, 4.0]
    assert [r["accepted"] for r in rec] == [False, True, True]
    assert all(r["status"] == 1 for r in rec)


def test_nonfinite_trial_counts_as_a_failure():
    class Blowup(FakeSolver):
        def newton_step(self, p, T, dt, **kw):
            self.calls.append(dt)
            if dt > 10.0:
                e = thermo.ThermoError.__new__(thermo.ThermoError)
                e.status = -4
                raise e
            return p + dt, T + dt, {"status": 0}

    s = Blowup(limit=None)
    p, T, rec = advance(s, np.zeros(1), np.zeros(1), 20.0)
    assert s.calls == [20.0, 10.0, 10.0] and np.all(p == 20.0)
    assert rec[0]["status"] == -4 and not rec[0]["accepted"]


class CountingSolver:
    """Newton converges iff dt <= limit, in iterations that grow with dt
    (ceil(8 dt / limit)); the state advances by dt."""

    def __init__(self, limit):
        self.limit = limit
        self.calls = []

    def newton_step(self, p, T, dt, **kw):
        self.calls.append(dt)
        if dt > self.limit:
            return p + dt, T + dt, {"status": 1, "newton_iters": 6}
        return p + dt, T + dt, {"status": 0, "newton_iters": int(np.ceil(8 * dt / self.limit))}


def test_next_step_scales_by_the_target_iteration_count():
    from paper_1902_00095_gb300.timestep import next_step
    assert next_step(10.0, 4) == 10.0
    assert next_step(10.0, 2) == 20.0
    assert next_step(10.0, 1) == 20.0    # grow capped at 2x
    assert next_step(10.0, 8) == 5.0
    assert next_step(10.0, 20) == 5.0    # shrink capped at 1/2
    assert next_step(10.0, 5) == 8.0
    assert next_step(10.0, 0) == 20.0


def test_simulate_reaches_the_end_time_exactly():
    from paper_1902_00095_gb300.timestep import simulate
    s = CountingSolver(limit=100.0)
    p, T, rec = simulate(s, np.zeros(1), np.zeros(1), t_end=600.0, dt0=30.0)
    acc = [r for r in rec if r["accepted"]]
    assert abs(sum(r["dt"] for r in acc) - 600.0) < 1e-9
    assert abs(p[0] - 600.0) < 1e-9
    # the accepted steps start where the previous ones ended
    t = 0.0
    for r in acc:
        assert abs(r["t"] - t) < 1e-9
        t += r["dt"]


def test_simulate_adapts_towards_the_target():
    """With iterations ceil(8 dt / limit) the target of 4 iterations is met
    by steps of limit / 2: the lengths settle there from above and below."""
    from paper_1902_00095_gb300.timestep import simulate
    for dt0 in (5.0, 45.0):
        s = CountingSolver(limit=100.0)
        p, T, rec = simulate(s, np.zeros(1), np.zeros(1), t_end=1000.0, dt0=dt0)
        acc = [r for r in rec if r["accepted"]]
        assert all(r["status"] == 0 for r in acc)
        mid = [r["dt"] for r in acc[3:-1]]
        assert mid and all(37.5 <= d <= 50.0 for d in mid), mid


def test_simulate_halves_a_failed_step_and_respects_dt_max():
    from paper_1902_00095_gb300.timestep import simulate
    s = CountingSolver(limit=20.0)
    p, T, rec = simulate(s, np.zeros(1), np.zeros(1), t_end=100.0, dt0=60.0, dt_max=50.0)
    # 50 (capped) fails, 25 fails, 12.5 converges in 5 iterations
    assert s.calls[:3] == [50.0, 25.0, 12.5]
    assert [r["accepted"] for r in rec[:3]] == [False, False, True]
    assert all(r["dt"] <= 50.0 for r in rec)
    assert abs(p[0] - 100.0) < 1e-9


def test_simulate_raises_when_a_step_never_converges():
    import pytest
    from paper_1902_00095_gb300.timestep import simulate

    class Blowup(CountingSolver):
        def newton_step(self, p, T, dt, **kw):
            self.calls.append(dt)
            e = thermo.ThermoError.__new__(thermo.ThermoError)
            e.status = -4
            raise e

    s = Blowup(limit=1.0)
    with pytest.raises(thermo.ThermoError):
        simulate(s, np.zeros(1), np.zeros(1), t_end=10.0, dt0=8.0, max_cuts=2)
    assert s.calls == [8.0, 4.0, 2.0]
