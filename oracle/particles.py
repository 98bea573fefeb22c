"""Particle forces, time integration, wall impacts, condenser charging (FP64).

Part of the FP64 CPU oracle: test infrastructure only.

Sec. 2.2, Eq. (particle-motion): du_p/dt = f_ad + f_coll + f_g + f_el.  The hot
path keeps drag (Schiller-Naumann, Sec. 2.2), the mesh (Gauss) electrostatic
force q E / m_p with m_p = pi d^3 rho_p / 6, and hard-sphere particle-wall
collisions (wall-normal velocity flips, tangential unchanged).  Gravity is zero
in all of the paper's runs (Sec. 3.1).

Sec. 2.3.1, condenser model for particle-wall impacts (after John et al.):
  dq_w = dq_c + dq_t                             Eq. (particle-wall charge sum)
  dq_c = -C U_c (1 - exp(-dt_w / T_w))           Eq. particle-wall-exchange
  C = eps A_iw / h                               Eq. capacity-capacitor
  A_iw = pi (d/2) alpha_iw                       Eq. charge-contact-area
  alpha_iw = (d/2) (5/8 pi rho_p (1+k_e) |u_i|^2
              ((1-mu_p^2)/E_p + (1-mu_w^2)/E_w))^(2/5)   Eq. charge-contact-area-alpha2
  dt_w = 2.94 alpha_iw / |u_i|,  T_w = eps_w eps0 phi_p
  dq_t: Eq. precharge-surface.

Readings (the paper is silent or inconsistent):
* integrator: exponential (exact for gas velocity and field frozen over the
  step); Re_p from the relative speed at the start of the step.
* drag: the source formula drops the (u - u_p) factor; the specific drag is
  f_ad = (u - u_p) / tau with 1/tau = (3/4) rho nu C_D Re_p / (rho_p d^2).
* order within a step: locate, deposit, Poisson and E from the state at the
  start of the step, then push.
* collision is elastic (e = 1, "fully elastic", Sec. 2.2); k_e only enters
  alpha_iw.
* contact: the centre comes closer than r = d/2 to a wall; the position is
  mirrored about the contact plane y = r (or Ly - r) and v_y flips.
* |u_i|: full particle speed after the push (literal reading); the switch
  IMPACT_NORMAL uses the wall-normal speed instead.
* dq_t = -(1/4) alpha_iw q is dimensionally inconsistent (alpha is a length);
  with the pre-charge spread uniformly over the surface, the transferred
  fraction is the contact area over the sphere area, dq_t = -A_iw/(pi d^2) q,
  which equals -(1/4)(alpha_iw / r) q.
* 1 - exp(-x) is evaluated as -expm1(-x) (x ~ 1e-8 here).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .constants import (DRAG_OFF, DRAG_SCHILLER_NAUMANN, DRAG_STOKES,
                        IMPACT_NORMAL, Params)
from .grid import Grid, locate, trilinear
from .poisson import deposit, efield, poisson


@dataclasses.dataclass
class State:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    q: np.ndarray
    d: np.ndarray
    n_imp: np.ndarray
    q_wall: np.ndarray
    id: np.ndarray = None       # particle identities (random-number counters of the SSM)
    site: np.ndarray = None     # SSM charging-site density c / c_0 (None: not tracked, held at 1)

    def __post_init__(self):
        if self.id is None:
            self.id = np.arange(self.x.shape[0], dtype=np.int64)

    @staticmethod
    def from_arrays(x, y, z, vx, vy, vz, q, d, n_imp=None, q_wall=None, ids=None, site=None) -> "State":
        n = np.asarray(x).shape[0]
        f = lambda a: np.array(a, dtype=np.float64)
        return State(f(x), f(y), f(z), f(vx), f(vy), f(vz), f(q), f(d),
                     np.zeros(n, np.int64) if n_imp is None else np.array(n_imp, np.int64),
                     np.zeros(n) if q_wall is None else f(q_wall),
                     np.arange(n, dtype=np.int64) if ids is None else np.array(ids, np.int64),
                     None if site is None else f(site))

    def copy(self) -> "State":
        return State(*(None if getattr(self, f.name) is None else np.array(getattr(self, f.name))
                       for f in dataclasses.fields(self)))

    @property
    def n(self) -> int:
        return self.x.shape[0]


def particle_mass(p: Params, d):
    """m_p = (1/6) pi d^3 rho_p (Sec. 2.2)."""
    return math.pi * np.asarray(d, np.float64) ** 3 * p.rho_p / 6.0


def relaxation_time(p: Params, d, rel_speed):
    """Drag relaxation time tau with f_ad = (u - u_p) / tau (Sec. 2.2).

    Stokes: tau_p = rho_p d^2 / (18 rho nu).  Schiller-Naumann:
    C_D = 24/Re_p (1 + Re_p^(2/3)/6) for Re_p <= 1000, 0.424 above, with
    1/tau = (3/4) rho nu C_D Re_p / (rho_p d^2).  DRAG_OFF returns inf.
    """
    d = np.asarray(d, np.float64)
    rel_speed = np.asarray(rel_speed, np.float64)
    if p.drag_law == DRAG_OFF:
        return np.full(np.broadcast(d, rel_speed).shape, np.inf)
    tau_p = p.rho_p * d ** 2 / (18.0 * p.rho * p.nu)
    if p.drag_law == DRAG_STOKES:
        return np.broadcast_to(tau_p, np.broadcast(d, rel_speed).shape).copy()
    re_p = rel_speed * d / p.nu
    cd = np.where(re_p <= 1000.0,
                  24.0 / np.where(re_p > 0, re_p, 1.0) * (1.0 + re_p ** (2.0 / 3.0) / 6.0),
                  0.424)
    inv_tau = 0.75 * p.rho * p.nu * cd * re_p / (p.rho_p * d ** 2)
    # Re_p -> 0 limit of the Schiller-Naumann branch is the Stokes time
    return np.where(re_p > 0, 1.0 / np.where(inv_tau > 0, inv_tau, 1.0), tau_p)


def _phi12(s):
    """phi1 = 1 - e^-s and phi2 = s - phi1 = e^-s - 1 + s (series for small s)."""
    s = np.asarray(s, np.float64)
    phi1 = -np.expm1(-s)
    small = s < 0.5
    ss = np.where(small, s, 0.0)
    # sum_{n=2}^{22} (-1)^n s^n / n!  (truncation below 1e-16 relative for s < 0.5)
    acc = np.zeros_like(ss)
    pw = ss * ss
    for n in range(2, 23):
        acc = acc + ((-1.0) ** n) * pw / math.factorial(n)
        pw = pw * ss
    phi2 = np.where(small, acc, s - phi1)
    return phi1, phi2


def coulomb_near(g: Grid, p: Params, st: "State") -> np.ndarray:
    """Near-field acceleration of the hybrid electrostatics (Sec. 2.2).

    Coulomb's law between every pair of particles that share a grid cell,
    F_i = q_i q_j / (4 pi eps) (s_i - s_j) / |s_i - s_j|^3 (like charges repel,
    Newton's third law F_j = -F_i), divided by m_p as a specific force like
    the other terms of Eq. (particle-motion).  Readings: the printed unit
    vector and magnitude are read as the textbook Coulomb law; the far field
    is the mesh field of all charges, unchanged; coincident centres exert no
    force.  Returns (n, 3).
    """
    i, j, k = locate(g, st.x, st.y, st.z)
    key = g.cell_key(i, j, k)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    starts = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    ends = np.r_[starts[1:], ks.shape[0]]
    X = np.stack([st.x, st.y, st.z], axis=1)
    coef = 1.0 / (4.0 * math.pi * p.eps)
    mass = particle_mass(p, st.d)
    acc = np.zeros((st.n, 3))
    for s, e in zip(starts, ends):
        if e - s < 2:
            continue
        idx = order[s:e]
        r = X[idx][:, None, :] - X[idx][None, :, :]          # s_a - s_b
        dist = np.linalg.norm(r, axis=2)
        dist = np.where(dist > 0, dist, np.inf)          # self and coincident centres: no force
        f = coef * (st.q[idx][:, None] * st.q[idx][None, :])[:, :, None] * r / dist[:, :, None] ** 3
        acc[idx] += f.sum(axis=1) / mass[idx][:, None]
    return acc


def pp_charge(p: Params, di, dj, qi, qj, speed):
    """Charge gained by particle i in a contact with particle j (condenser
    model, Sec. 2.3.1):
      dq_ij = C_i C_j / (C_i + C_j) (q_j / C_j - q_i / C_i) (1 - exp(-dt_12 / T_12)),
      C = 4 pi eps d / 2,  T_12 = C_i C_j / (C_i + C_j) (d_i + d_j) / (2 A_12) phi_p,
      A_12 = pi d_i d_j / (2 (d_i + d_j)) alpha_12,  dt_12 = 2.94 alpha_12 / |u_12|,
      alpha_12 = (d_i d_j / 2) (5/8 pi rho_p (1 + k_e) |u_12|^2 sqrt(d_i + d_j) / (d_i^3 + d_j^3) el)^(2/5).
    Reading: the elastic factor el is 2 (1 - mu_p^2) / E_p (the wall formula's sum
    of the two bodies' (1 - mu^2) / E for one material); with it and k_e = 1,
    alpha_12 is the Hertz maximum compression of the two spheres.
    Returns (dq_i, details); dq_j = -dq_i.  A zero speed transfers nothing.
    """
    di, dj = np.asarray(di, np.float64), np.asarray(dj, np.float64)
    qi, qj = np.asarray(qi, np.float64), np.asarray(qj, np.float64)
    speed = np.asarray(speed, np.float64)
    Ci = 2.0 * math.pi * p.eps * di
    Cj = 2.0 * math.pi * p.eps * dj
    el = 2.0 * (1.0 - p.mu_p ** 2) / p.E_p
    alpha = (di * dj / 2.0) * (0.625 * math.pi * p.rho_p * (1.0 + p.k_e) * speed ** 2
                               * np.sqrt(di + dj) / (di ** 3 + dj ** 3) * el) ** 0.4
    A = math.pi * di * dj / (2.0 * (di + dj)) * alpha
    pos = speed > 0
    dt = np.where(pos, 2.94 * alpha / np.where(pos, speed, 1.0), 0.0)
    Cs = Ci * Cj / (Ci + Cj)
    T = Cs * (di + dj) / (2.0 * np.where(A > 0, A, 1.0)) * p.phi_p
    dq = np.where(pos, Cs * (qj / Cj - qi / Ci) * (-np.expm1(-dt / T)), 0.0)
    return dq, dict(alpha=alpha, A=A, dt=dt, T=T, Cs=Cs)


def pp_collisions(g: Grid, p: Params, x, y, z, v, q, d):
    """Hard-sphere particle-particle collisions (4-way coupling, Sec. 2.2) with
    the condenser charge exchange, applied to the end-of-step state.

    Readings: candidates are particles of the same cell; a pair collides when
    the spheres overlap, approach each other ((v_i - v_j).(s_i - s_j) < 0) and
    each is the other's nearest such partner (ties to the lower index); the
    collision is elastic along the line of centres with the particle masses
    (for equal masses the normal components are exchanged); the charge uses
    the relative speed before the collision.  Returns (v', q', pairs).
    """
    v = np.array(v, np.float64)
    q = np.array(q, np.float64)
    n = x.shape[0]
    i, j, k = locate(g, x, y, z)
    key = g.cell_key(i, j, k)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    starts = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]]) if n else np.zeros(0, np.int64)
    ends = np.r_[starts[1:], n] if n else np.zeros(0, np.int64)
    S = np.stack([x, y, z], axis=1)
    partner = np.full(n, -1, np.int64)
    for s_, e_ in zip(starts, ends):
        if e_ - s_ < 2:
            continue
        idx = np.sort(order[s_:e_])
        r = S[idx][:, None, :] - S[idx][None, :, :]
        dist2 = np.sum(r * r, axis=2)
        rel = v[idx][:, None, :] - v[idx][None, :, :]
        appr = np.sum(rel * r, axis=2) < 0
        reach = 0.5 * (d[idx][:, None] + d[idx][None, :])
        ok = (dist2 < reach ** 2) & appr
        np.fill_diagonal(ok, False)
        for a in range(idx.shape[0]):
            if ok[a].any():
                cand = np.flatnonzero(ok[a])
                partner[idx[a]] = idx[cand[np.argmin(dist2[a, cand])]]
    pairs = [(a, b) for a, b in enumerate(partner) if b > a and partner[b] == a]
    mass = particle_mass(p, d)
    v_new, q_new = v.copy(), q.copy()
    for a, b in pairs:
        nrm = S[a] - S[b]
        nrm = nrm / np.linalg.norm(nrm)
        vn = np.dot(v[a] - v[b], nrm)
        ma, mb = mass[a], mass[b]
        v_new[a] = v[a] - (2.0 * mb / (ma + mb)) * vn * nrm
        v_new[b] = v[b] + (2.0 * ma / (ma + mb)) * vn * nrm
        dq, _ = pp_charge(p, d[a], d[b], q[a], q[b], np.linalg.norm(v[b] - v[a]))
        q_new[a] = q[a] + dq
        q_new[b] = q[b] - dq
    return v_new, q_new, pairs


def push(p: Params, x, v, uf, acc, d, dt):
    """Advance position and velocity over dt with u, a frozen (exponential).

    dv/dt = (u - v)/tau + a  gives
      v' = v + (u + a tau - v) phi1,  x' = x + tau (v phi1 + (u + a tau) phi2),
    phi1 = 1 - e^-s, phi2 = s - phi1, s = dt / tau.  With drag off:
      v' = v + a dt, x' = x + v dt + a dt^2 / 2.
    x, v, uf, acc: (n, 3).  Returns x', v', tau.
    """
    rel = np.linalg.norm(v - uf, axis=1)
    tau = relaxation_time(p, d, rel)
    if p.drag_law == DRAG_OFF:
        return x + v * dt + 0.5 * acc * dt * dt, v + acc * dt, tau
    s = dt / tau
    phi1, phi2 = _phi12(s)
    term = uf + acc * tau[:, None]
    vn = v + (term - v) * phi1[:, None]
    xn = x + tau[:, None] * (v * phi1[:, None] + term * phi2[:, None])
    return xn, vn, tau


def momentum_source(g: Grid, p: Params, st: "State", uf, acc, tau, dt):
    """F_s of the gas momentum equation (Eq. ns): the particles' aerodynamic
    forces summed over each control volume, per unit gas mass.

    Reading: the drag force of a particle over the step is its drag impulse
    under the integrator of push() divided by dt; with u, a and tau frozen,
    dv/dt = (u - v)/tau + a integrates to a drag impulse
      dv_drag = (u - v) phi1 - a tau phi2,
    and F_s[c] = -(1 / (rho V_c)) sum_{p in c} m_p dv_drag,p / dt over the
    particles whose start position lies in cell c (where u was gathered).
    Returns planes (3, nz, ny, nx).
    """
    fs = np.zeros((3, g.nz, g.ny, g.nx))
    if p.drag_law == DRAG_OFF or st.n == 0:
        return fs
    V = np.stack([st.vx, st.vy, st.vz], axis=1)
    phi1, phi2 = _phi12(dt / tau)
    dv = (uf - V) * phi1[:, None] - acc * (tau * phi2)[:, None]
    i, j, k = locate(g, st.x, st.y, st.z)
    w = -particle_mass(p, st.d) / (p.rho * dt)
    for c in range(3):
        np.add.at(fs[c], (k, j, i), w * dv[:, c])
    return fs / g.vol_y[None, None, :, None]


def wrap(s, length):
    """Periodic wrap into [0, L); a result equal to L (rounding) becomes 0."""
    w = s - length * np.floor(s / length)
    return np.where(w >= length, w - length, w)


def condenser_wall(p: Params, d, speed, q):
    """Charge gained by a particle in one wall impact (condenser model).

    Returns (dq_c, dq_t, details) with details = dict(alpha, A, C, dt_w, T_w).
    A zero impact speed transfers nothing.
    """
    d = np.asarray(d, np.float64)
    speed = np.asarray(speed, np.float64)
    q = np.asarray(q, np.float64)
    r = 0.5 * d
    elastic = (1.0 - p.mu_p ** 2) / p.E_p + (1.0 - p.mu_w ** 2) / p.E_w
    alpha = r * (0.625 * math.pi * p.rho_p * (1.0 + p.k_e) * speed ** 2 * elastic) ** 0.4
    A = p.kappa_A * math.pi * r * alpha
    C = p.eps * A / p.h
    pos = speed > 0
    dt_w = np.where(pos, 2.94 * alpha / np.where(pos, speed, 1.0), 0.0)
    T_w = p.eps_w * p.eps0 * p.phi_p
    dq_c = -C * p.U_c * (-np.expm1(-dt_w / T_w))
    dq_t = -(A / (math.pi * d ** 2)) * q if p.dq_t else np.zeros_like(q)
    return dq_c, dq_t, dict(alpha=alpha, A=A, C=C, dt_w=dt_w, T_w=T_w)


def wall_impacts(p: Params, ly: float, y, vy, d):
    """Specular reflection at the walls (hard sphere, Sec. 2.2).

    Returns (y', vy', hit) with hit = -1 (bottom), +1 (top), 0 (none), and a
    flag array of particles still outside after one reflection.
    """
    r = 0.5 * np.asarray(d, np.float64)
    lo = y < r
    hi = y > ly - r
    yn = np.where(lo, 2.0 * r - y, np.where(hi, 2.0 * (ly - r) - y, y))
    vyn = np.where(lo | hi, -vy, vy)
    hit = np.where(lo, -1, np.where(hi, 1, 0))
    bad = (yn < r) | (yn > ly - r)
    return yn, vyn, hit, bad


def step(g: Grid, p: Params, st: State, u_lat: np.ndarray, dt: float,
         diag: dict | None = None, E_lat: np.ndarray | None = None) -> State:
    """One coupled particle step (deposit -> Poisson -> E -> gather -> push -> wall).

    u_lat: gas velocity on the wall-extended lattice (Nz, Ny+2, Nx, 3).
    E_lat: optional field lattice of the same layout to use instead of the
    field of st's own charges (replaying a subsample of a larger ensemble in
    the field of all its particles).
    """
    n = st.n
    X = np.stack([st.x, st.y, st.z], axis=1)
    V = np.stack([st.vx, st.vy, st.vz], axis=1)
    uf = trilinear(g, u_lat, st.x, st.y, st.z)
    if p.electrostatics and E_lat is not None:
        Ep = trilinear(g, E_lat, st.x, st.y, st.z)
        acc = (st.q / particle_mass(p, st.d))[:, None] * Ep
    elif p.electrostatics:
        i, j, k = locate(g, st.x, st.y, st.z)
        rho = deposit(g, st.q, i, j, k)
        phi = poisson(g, rho, p.eps)
        E = efield(g, phi)
        Ep = trilinear(g, E, st.x, st.y, st.z)
        acc = (st.q / particle_mass(p, st.d))[:, None] * Ep
        if diag is not None:
            diag.update(rho=rho, phi=phi, E=E, Ep=Ep)
    else:
        acc = np.zeros((n, 3))
    if p.electrostatics and p.coulomb:
        acc = acc + coulomb_near(g, p, st)
    Xn, Vn, tau = push(p, X, V, uf, acc, st.d, dt)
    xn = wrap(Xn[:, 0], g.lx)
    zn = wrap(Xn[:, 2], g.lz)
    yn, vyn, hit, bad = wall_impacts(p, g.ly, Xn[:, 1], Vn[:, 1], st.d)
    if np.any(bad):
        raise FloatingPointError("particle crossed both contact planes in one step")
    vxn, vzn = Vn[:, 0], Vn[:, 2]
    q = st.q.copy()
    n_imp = st.n_imp.copy()
    q_wall = st.q_wall.copy()
    site = None if st.site is None else st.site.copy()
    m = hit != 0
    if np.any(m):
        if p.impact_vel == IMPACT_NORMAL:
            speed = np.abs(Vn[m, 1])
        else:
            speed = np.linalg.norm(Vn[m], axis=1)
        if p.ssm is not None:
            from .ssm import ssm_wall_charge
            dq, det = ssm_wall_charge(p, p.ssm, st.d[m], speed, q[m], st.id[m], n_imp[m],
                                      site=None if site is None else site[m])
            if site is not None:
                site[m] = det["site"]
        else:
            dq_c, dq_t, _ = condenser_wall(p, st.d[m], speed, q[m])
            dq = dq_c + dq_t
        q[m] += dq
        q_wall[m] += dq
        n_imp[m] += 1
    if p.collisions:
        Vc, q, pairs = pp_collisions(g, p, xn, yn, zn, np.stack([vxn, vyn, vzn], axis=1), q, st.d)
        vxn, vyn, vzn = Vc[:, 0], Vc[:, 1], Vc[:, 2]
        if diag is not None:
            diag.update(pairs=pairs)
    if diag is not None:
        diag.update(uf=uf, hit=hit, tau=tau, acc=acc, F_s=momentum_source(g, p, st, uf, acc, tau, dt))
    return State(xn, yn, zn, vxn, vyn, vzn, q, st.d.copy(), n_imp, q_wall, st.id.copy(), site)


def run(g: Grid, p: Params, st: State, u_lat, dt: float, nsteps: int,
        hist: np.ndarray | None = None, fs: np.ndarray | None = None) -> State:
    """nsteps coupled steps; optionally accumulate the y-cell histogram and
    the mean momentum source over the steps (fs, planes (3, nz, ny, nx),
    overwritten).

    u_lat may be an array or a callable t -> lattice (time-varying gas field).
    """
    if fs is not None:
        fs[...] = 0.0
    for n in range(nsteps):
        lat = u_lat(n * dt) if callable(u_lat) else u_lat
        diag = {} if fs is not None else None
        st = step(g, p, st, lat, dt, diag=diag)
        if fs is not None:
            fs += diag["F_s"] / nsteps
        if hist is not None:
            hist += ystats(g, st)
    return st


def ystats(g: Grid, st: State) -> np.ndarray:
    """Particle count per wall-normal cell (the bins of C_rel, Sec. 4.1)."""
    _, j, _ = locate(g, st.x, st.y, st.z)
    return np.bincount(j, minlength=g.ny).astype(np.float64)


def c_rel(g: Grid, counts: np.ndarray) -> np.ndarray:
    """Relative concentration C_rel = C / C0 per y-cell (Sec. 4.1)."""
    conc = counts / (g.vol_y * g.nx * g.nz)
    c0 = counts.sum() / (g.lx * g.ly * g.lz)
    return conc / c0


# ---------------------------------------------------------------------------
# non-dimensional groups (Sec. 3.1, Table 2)

def dplus(d, re_tau, delta):
    """d_p+ = d_p u_tau / nu = d_p Re_tau / delta."""
    return np.asarray(d) * re_tau / delta


def stokes_number(p: Params, d, u_c, delta):
    """St = (1/18)(rho_p/rho) d^2/nu * u_c/delta (Sec. 3.1)."""
    return (1.0 / 18.0) * (p.rho_p / p.rho) * np.asarray(d) ** 2 / p.nu * u_c / delta


def volume_fraction_ppm(number_density, d):
    """omega = C pi d^3 / 6, in parts per million."""
    return number_density * math.pi * np.asarray(d) ** 3 / 6.0 * 1e6
