"""Charging-rate correlation of Sec. 4 and the tools to hold a simulation
against it (host code; the simulation itself runs in libtribo.so).

The paper fits, by symbolic regression over its DNS/LES runs, the early-time
charging rate d<q>_rel/dt+ (<q>_rel = <q>/q_sat) as a function of Re_tau and
the particle diameter: a compact form (Eq. pysr-result-simple)
  log10 rate = -5.89 - 9070 / (d_rel (Re_tau - 42.5))
and a more accurate one (Eq. pysr-result)
  log10 rate = -2.18e-5 Re_tau d_rel - 4.64 - 30360 / (Re_tau (d_rel + 4.92) + 2668).
Readings: d_rel is the diameter in micrometres (the printed d_p / (50 delta)
is garbled; micrometres reproduce the Re_tau of the largest rate the paper
quotes for 25, 50 and 100 um), and the rate is dimensionless (its "C" unit
is a slip).  Rates are fitted over t+ < 4000, where the paper finds them
constant.
"""
from __future__ import annotations

import math

import numpy as np

Q_SAT = 1.26e-13            # condenser-model saturation charge of Sec. 3.1 [C]
T_PLUS_MAX = 4000.0         # fitting window of the charging rate (Sec. 4)

_A2, _B2, _C2, _D2, _E2 = -2.18e-5, -4.64, 30360.0, 4.92, 2668.0


def rate_simple(re_tau, d_um):
    """d<q>_rel/dt+ by the compact correlation (Eq. pysr-result-simple)."""
    re_tau = np.asarray(re_tau, np.float64)
    d_um = np.asarray(d_um, np.float64)
    return 10.0 ** (-5.89 - 9070.0 / (d_um * (re_tau - 42.5)))


def rate(re_tau, d_um):
    """d<q>_rel/dt+ by the accurate correlation (Eq. pysr-result)."""
    re_tau = np.asarray(re_tau, np.float64)
    d_um = np.asarray(d_um, np.float64)
    return 10.0 ** (_A2 * re_tau * d_um + _B2 - _C2 / (re_tau * (d_um + _D2) + _E2))


def peak_re_tau(d_um):
    """Re_tau of the largest rate of Eq. pysr-result at a given diameter:
    d/dRe of the exponent vanishes where
    (Re (d + 4.92) + 2668)^2 = 30360 (d + 4.92) / (2.18e-5 d)."""
    d_um = np.asarray(d_um, np.float64)
    s = d_um + _D2
    return (np.sqrt(_C2 * s / (-_A2 * d_um)) - _E2) / s


def fit_rate(t_plus, q_rel, t_plus_max: float = T_PLUS_MAX) -> float:
    """Least-squares slope of <q>_rel over t+ on the samples with t+ < t_plus_max."""
    t = np.asarray(t_plus, np.float64)
    q = np.asarray(q_rel, np.float64)
    m = t < t_plus_max
    if m.sum() < 2:
        raise ValueError("need at least two samples with t+ below the fitting window")
    t, q = t[m], q[m]
    tc = t - t.mean()
    return float(np.dot(tc, q - q.mean()) / np.dot(tc, tc))


def t_plus(t, u_tau: float, nu: float):
    """Time in wall units, t+ = t u_tau^2 / nu."""
    return np.asarray(t, np.float64) * u_tau * u_tau / nu


def charging_history(channel, particles, dt: float, nsteps: int, every: int, u_tau: float, nu: float,
                     q_sat: float = Q_SAT):
    """Advance `particles` nsteps in `channel`, sampling <q>_rel every `every`
    steps (the mean of the device charges, read through tribo_stats).
    Returns (t+, <q>_rel) including the start."""
    st = channel.stats(particles)
    ts, qs = [0.0], [st["sum_q"] / max(particles.n, 1) / q_sat]
    done = 0
    while done < nsteps:
        k = min(every, nsteps - done)
        channel.step(particles, dt, k)
        done += k
        st = channel.stats(particles)
        ts.append(done * dt)
        qs.append(st["sum_q"] / max(particles.n, 1) / q_sat)
    return t_plus(np.array(ts), u_tau, nu), np.array(qs)


def calibrate(channel, make_particles, dt: float, nsteps: int, target: float, param: str = "U_c",
              iters: int = 6, rtol: float = 1e-10, ckpt_every: int = 50):
    """Newton iteration on one parameter (U_c or kappa_A) so that the mean
    charge after nsteps, J, equals `target`; dJ/dparam comes from the
    reverse-mode pass of tribo_adjoint.  make_particles() returns a fresh
    particle set (the adjoint advances the one it is given).  Returns
    (value, [(value, J), ...])."""
    if param not in ("U_c", "kappa_A"):
        raise ValueError("param must be 'U_c' or 'kappa_A'")
    params = channel.params
    theta = float(getattr(params, param))
    hist = []
    for _ in range(iters):
        channel.set_params(params.with_(**{param: theta}))
        J, dU, dK, _ = channel.adjoint(make_particles(), dt, nsteps, ckpt_every, want_dd=False)
        hist.append((theta, J))
        g = dU if param == "U_c" else dK
        if abs(J - target) <= rtol * abs(target):
            break
        if g == 0.0 or not math.isfinite(g):
            raise ArithmeticError(f"dJ/d{param} = {g}: the mean charge does not depend on {param}")
        theta = theta - (J - target) / g
    channel.set_params(params.with_(**{param: theta}))
    return theta, hist
