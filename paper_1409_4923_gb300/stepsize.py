"""Step size of a run from Sec. 4's local-error indicator chi.

The paper notes that chi = (predictor) - (corrector) measures the local error
of Algorithm 1 and could steer a dynamic step size.  Within one run the steps
stay uniform (the jump countdowns count whole steps and the random streams
are addressed by step index), so the control acts per run: two short probes
at dt and dt / 2 over the same stretch of time measure chi's order p, and the
step that brings the RMS of chi to the tolerance follows from
chi(dt') = chi(dt) (dt' / dt)^p.  The result is rounded to a whole number of
steps per drive period, so that the drive phase stays exact per period.
"""
import math


def suggest_dt(engine, dt0, tol, omega=None, paths=4096, probe_time=None, component="rms_x"):
    """dt for rms chi = tol (component rms_x or rms_v), from probes at dt0 and
    dt0 / 2 over probe_time (default: one drive period, or 100 dt0).  Returns
    dict(dt, steps_per_period (or None), order, chi_dt0, chi_half)."""
    if not (tol > 0.0 and dt0 > 0.0):
        raise ValueError("tol and dt0 must be > 0")
    period = 2.0 * math.pi / omega if omega else None
    span = probe_time or (period if period else 100.0 * dt0)
    n0 = max(2, int(round(span / dt0)))
    a = engine.local_error(paths, dt0, n0)[component]
    b = engine.local_error(paths, dt0 / 2.0, 2 * n0)[component]
    if not (a > 0.0 and b > 0.0):
        raise ValueError("chi vanishes: any step size meets the tolerance")
    order = math.log(a / b, 2.0)
    order = min(max(order, 1.0), 4.0)
    dt = dt0 * (tol / a) ** (1.0 / order)
    spp = None
    if period:
        spp = max(1, int(math.ceil(period / dt)))
        dt = period / spp
    return {"dt": dt, "steps_per_period": spp, "order": order, "chi_dt0": a, "chi_half": b}
