"""Time-step drivers.

Sec. 4 chooses time steps so that Newton's method converges in about four
iterations. `advance` keeps a requested step length when Newton converges and
otherwise repeats the step as two halves, recursively (at most `max_cuts`
halvings), from the same starting state. `simulate` runs to an end time
with step lengths adapted to the Newton iteration count. Orchestration only:
every Newton iteration runs in the CUDA library (`Solver.newton_step`).
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


def next_step(dt, newton_iters, target=4, grow=2.0, shrink=0.5):
    """Step length after a step that converged in `newton_iters` Newton
    iterations: dt scaled by target / newton_iters, kept within
    [shrink, grow] times dt (a step that needed no iteration grows by
    `grow`)."""
    if newton_iters <= 0:
        return dt * grow
    return dt * min(grow, max(shrink, target / newton_iters))


def simulate(solver, p, T, t_end, dt0, dt_max=None, target=4, max_cuts=6, **newton_kw):
    """Backward-Euler steps from time 0 to t_end with adaptive step lengths
    (Sec. 4: steps sized so that Newton converges in about `target`
    iterations). The first step has length dt0. After a converged step of n
    Newton iterations the next length is next_step(dt, n), capped at dt_max
    and at the time left. A step whose Newton iteration fails (or leaves the
    physical range) is retried from the same state with half the length, at
    most max_cuts times in a row; a step that still fails is accepted as it
    is, its record saying so through `status`.

    Returns (p, T, records): one dict per Newton solve in order, with the
    step length `dt`, the time `t` at its start, `accepted` and the Newton
    info. Orchestration only: every Newton iteration runs in the CUDA
    library (`Solver.newton_step`)."""
    t, dt, rec = 0.0, dt0, []
    eps = 1e-9 * t_end
    while t < t_end - eps:
        dt = min(dt, t_end - t)
        if dt_max is not None:
            dt = min(dt, dt_max)
        cuts = 0
        while True:
            try:
                p1, T1, info = solver.newton_step(p, T, dt, **newton_kw)
                ok = info["status"] == 0
            except thermo.ThermoError as e:
                p1, T1, info, ok = None, None, {"status": e.status}, False
            if ok or (cuts == max_cuts and p1 is not None):
                rec.append(dict(info, dt=dt, t=t, accepted=True))
                break
            if cuts == max_cuts:
                raise thermo.ThermoError(info["status"], "simulate")
            rec.append(dict(info, dt=dt, t=t, accepted=False))
            dt *= 0.5
            cuts += 1
        p, T, t = p1, T1, t + dt
        dt = next_step(dt, info.get("newton_iters", target), target) if ok else dt
    return p, T, rec
