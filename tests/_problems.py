"""Shared set-up of parity problems: one seeded input feeds both the oracle
and the CUDA path; comparison helpers state the tolerances."""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth

TOL_FP64 = 1e-12      # FP64 mode, 10-step horizons (per-particle, relative)
TOL_MIXED = 1e-5      # FP32 particle state, 10-step horizons


def problem(nx=64, ny=64, nz=64, n=2000, re_tau=180.0, dplus=(1.0, 1.0), density_ratio=1000.0,
            q_scale=0.0, vy_scale=0.0, near_wall=0.0, seed=7, gamma=2.0, lx=None, lz=None,
            time_varying=False):
    """Grid faces, gas lattice (nz, ny+2, nx, 3) and a particle dict (FP64)."""
    c = synth.case("re180_64").with_(
        nx=nx, ny=ny, nz=nz, n_particles=n, re_tau=re_tau, dplus=dplus,
        density_ratio=density_ratio, gamma=gamma, field_seed=1000 + seed, particle_seed=2000 + seed,
        lx=lx if lx is not None else 2 * math.pi * 0.02, lz=lz if lz is not None else math.pi * 0.02,
        time_varying=time_varying)
    faces = synth.y_faces(ny, c.delta, c.gamma)
    lat = synth.fluid_lattice(c, faces=faces)
    P = synth.draw_particles(c, n)
    rng = np.random.default_rng(seed)
    parts = dict(x=P.x, y=P.y.copy(), z=P.z, vx=P.vx, vy=P.vy + rng.standard_normal(n) * vy_scale,
                 vz=P.vz.copy(), d=P.d, q=rng.standard_normal(n) * q_scale)
    if near_wall > 0 and n > 0:
        m = rng.random(n) < near_wall
        r = 0.5 * P.d[m]
        top = rng.random(m.sum()) < 0.5
        gap = rng.uniform(0.0, 3e-4, m.sum()) * (c.u_tau * 20.0 * c.dt)
        parts["y"][m] = np.where(top, c.ly - r - gap, r + gap)
        speed = np.abs(rng.standard_normal(m.sum())) * 0.5 + 0.05
        parts["vy"][m] = np.where(top, speed, -speed)
    return c, faces, lat, parts


def round_inputs(lat, parts, real):
    """Inputs as the CUDA path stores them (FP32 in mixed mode)."""
    lat = lat.astype(real).astype(np.float64)
    out = {}
    for k, v in parts.items():
        out[k] = v if k == "q" else np.asarray(v).astype(real).astype(np.float64)
    return lat, out


def oracle_params(c, **kw):
    return oracle.Params(rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, **kw)


def oracle_state(parts):
    return oracle.State.from_arrays(parts["x"], parts["y"], parts["z"], parts["vx"], parts["vy"],
                                    parts["vz"], parts["q"], parts["d"])


def periodic_err(a, b, L):
    return np.abs(np.mod(a - b + 0.5 * L, L) - 0.5 * L)


def compare_states(g, got: dict, ref: oracle.State, tol: float, ids=None, label=""):
    """Per-particle comparison under the tolerance reading of the parity bar
    ("per-particle position, velocity and charge ... relative error"):
    * position: each coordinate's distance (periodic in x, z) over the box
      extent in that direction;
    * velocity: |v - v_ref| / |v_ref| of each particle's velocity vector;
    * charge: the charge q and the received wall charge q_wall, each against
      the particle's charge scale max(|q_ref|, |q_wall_ref|, |q_ref -
      q_wall_ref|) (its final, received and initial charge: a particle whose
      received charges cancel, or cancel its initial charge, is measured
      against the charges it carried).  A particle whose reference charges
      are all zero must match exactly.
    Returns a dict of the worst relative errors, and under "component_max" the
    worst errors of each velocity component and the charge against the
    largest magnitude of that quantity over all particles (reported, not
    asserted)."""
    if ids is None:
        ids = np.arange(ref.n)
    ex = periodic_err(got["x"], ref.x[ids], g.lx) / g.lx
    ey = np.abs(got["y"] - ref.y[ids]) / g.ly
    ez = periodic_err(got["z"], ref.z[ids], g.lz) / g.lz
    out = dict(x=ex.max(initial=0), y=ey.max(initial=0), z=ez.max(initial=0))
    dv = np.sqrt(sum((np.asarray(got[k], np.float64) - getattr(ref, k)[ids]) ** 2 for k in ("vx", "vy", "vz")))
    sp = np.sqrt(sum(getattr(ref, k)[ids] ** 2 for k in ("vx", "vy", "vz")))
    out["v"] = _rel_max(dv, sp)
    qr, qw = ref.q[ids], ref.q_wall[ids]
    qs = np.maximum(np.maximum(np.abs(qr), np.abs(qw)), np.abs(qr - qw))
    out["q"] = _rel_max(np.abs(got["q"] - qr), qs)
    out["q_wall"] = _rel_max(np.abs(got["q_wall"] - qw), qs)
    cm = {}
    for k in ("vx", "vy", "vz", "q"):
        r = getattr(ref, k)[ids]
        cm[k] = float((np.abs(got[k] - r)).max(initial=0) / max(np.abs(r).max(initial=0), 1e-300))
    bad = {k: v for k, v in out.items() if not v <= tol}
    assert not bad, f"{label} relative errors above {tol}: {bad}"
    out["component_max"] = cm
    return out


def _rel_max(err, scale):
    """Largest err / scale; entries with scale 0 count as 0 when err is 0 and
    as infinite otherwise."""
    err = np.asarray(err, np.float64)
    scale = np.asarray(scale, np.float64)
    if not err.size:
        return 0.0
    zero = scale == 0
    if np.any(zero & (err != 0)):
        return float("inf")
    r = np.where(zero, 0.0, err / np.where(zero, 1.0, scale))
    return float(r.max())
