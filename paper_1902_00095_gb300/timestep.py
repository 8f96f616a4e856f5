"""Time-step driver with step cutting.

Sec. 4 chooses time steps so that Newton's method converges in a few
iterations. This driver keeps the requested step length when Newton
converges and otherwise repeats the step as two halves, recursively (at most
`max_cuts` halvings), from the same starting state. Orchestration only: every
Newton iteration runs in the CUDA library (`Solver.newton_step`).
"""
from . import thermo


def advance(solver, p, T, dt, max_cuts=3, **newton_kw):
    """One backward-Euler step of length dt from (p, T) (host or device
    arrays, not modified). Returns (p_new, T_new, record): record lists every
    Newton solve in order as dicts with the step length `dt`, `accepted`
    and the Newton info; a rejected solve is followed by the records of its
    two half steps. A step that still fails after max_cuts halvings is
    accepted as it is (its record says so through `status`)."""
    try:
        p1, T1, info = solver.newton_step(p, T, dt, **newton_kw)
        ok = info["status"] == 0
    except thermo.ThermoError as e:
        # a trial state outside the physical range (non-finite residual)
        p1, T1, info, ok = None, None, {"status": e.status}, False
    if ok or max_cuts == 0:
        if p1 is None:
            raise thermo.ThermoError(info["status"], "advance")
        return p1, T1, [dict(info, dt=dt, accepted=True)]
    rec = [dict(info, dt=dt, accepted=False)]
    pa, Ta, ra = advance(solver, p, T, 0.5 * dt, max_cuts - 1, **newton_kw)
    pb, Tb, rb = advance(solver, pa, Ta, 0.5 * dt, max_cuts - 1, **newton_kw)
    return pb, Tb, rec + ra + rb
