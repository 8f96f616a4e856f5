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
