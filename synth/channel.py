"""Seeded synthetic channel-flow inputs (grid, gas-velocity lattice, particles).

Units are SI.  The channel half height is delta = 0.02 m (paper Sec. 3.1) and
the gas is air (Table 1: nu = 1.46e-5 m^2/s, rho = 1.2 kg/m^3).  Wall units
follow Sec. 3.1: u_tau = Re_tau nu / delta, y+ = y u_tau / nu,
t+ = t u_tau^2 / nu.

Recipe (the paper's DNS/LES gas fields are not available, so a synthetic
field of the same shape stands in for them):

* grid: periodic x, z with uniform cells; wall-normal faces tanh-stretched,
  y_f[j] = delta (1 - tanh(gamma (1 - 2 j / Ny)) / tanh(gamma)), j = 0..Ny.
* gather lattice: x, z nodes at cell centres, y nodes at [0, cell centres,
  2 delta] (Ny + 2 nodes); the gas velocity is zero on the wall nodes.
* gas velocity: Reichardt mean profile (mirrored about the centre line) along
  x, plus 256 random Fourier modes: |k| log-uniform in [2 pi / Lx, pi / dx],
  random direction with k_x, k_z quantised to the periodic box, amplitude
  vector perpendicular to k, Gaussian amplitudes weighted by a von Karman
  spectrum (k_e = 2 pi / delta), random phases; fluctuations normalised to a
  per-component rms of u_tau, then damped by y+ / (y+ + 10).  A time-varying
  field advects each mode's phase with the local mean velocity.
* particles: uniform in x, z and in y in [r, 2 delta - r]; initial velocity
  is the local mean gas velocity; charges zero or Gaussian with zero mean.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

DELTA = 0.02          # channel half height [m], Sec. 3.1
NU = 1.46e-5          # air kinematic viscosity [m^2/s], Table 1
RHO_F = 1.2           # air density [kg/m^3], Table 1
Q_SAT = 1.26e-13      # condenser-model saturation charge [C], Sec. 3.1
N_MODES = 256


@dataclasses.dataclass(frozen=True)
class Case:
    """One synthetic workload: grid, gas field, particle ensemble, schedule."""
    name: str
    re_tau: float
    nx: int
    ny: int
    nz: int
    lx: float
    lz: float
    n_particles: int
    dplus: Tuple[float, float]          # (lo, hi); lo == hi means monodisperse
    density_ratio: float                # rho_p / rho
    q0_sigma: float = 0.0               # std of the initial charge [C]
    steps: int = 200
    dt_plus: float = 0.05
    time_varying: bool = False
    field_seed: int = 1000
    particle_seed: int = 2000
    delta: float = DELTA
    gamma: float = 2.0
    nu: float = NU
    rho_f: float = RHO_F

    @property
    def ly(self) -> float:
        return 2.0 * self.delta

    @property
    def u_tau(self) -> float:
        return friction_velocity(self.re_tau, self.nu, self.delta)

    @property
    def dt(self) -> float:
        return self.dt_plus * self.nu / self.u_tau ** 2

    @property
    def rho_p(self) -> float:
        return self.density_ratio * self.rho_f

    def with_(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


def friction_velocity(re_tau: float, nu: float = NU, delta: float = DELTA) -> float:
    return re_tau * nu / delta


_TWO_PI = 2.0 * math.pi

CASES = {
    # plain FP64 parity case (Re_tau = 180, 64^3)
    "re180_64": Case("re180_64", 180.0, 64, 64, 64, _TWO_PI * DELTA, math.pi * DELTA,
                     2000, (1.0, 1.0), 1000.0, 0.0, 200, 0.05, False, 1001, 2001),
    # Re_tau = 180, 128^3, time-varying field, polydisperse, charged
    "re180_128": Case("re180_128", 180.0, 128, 128, 128, _TWO_PI * DELTA, math.pi * DELTA,
                      1_000_000, (0.5, 2.0), 1000.0, 0.01 * Q_SAT, 2000, 0.05, True, 1002, 2002),
    # headline: Re_tau = 550, 384 x 256 x 256, 8M particles
    "re550_384": Case("re550_384", 550.0, 384, 256, 256, _TWO_PI * DELTA, math.pi * DELTA,
                      8_000_000, (2.5, 2.5), 2000.0, 0.0, 1000, 0.05, False, 1003, 2003),
    # differentiation case: Re_tau = 180, 128^3, 1M particles
    "re180_128_adj": Case("re180_128_adj", 180.0, 128, 128, 128, _TWO_PI * DELTA, math.pi * DELTA,
                          1_000_000, (1.0, 1.0), 1000.0, 0.0, 500, 0.05, False, 1005, 2005),
}


def case(name: str) -> Case:
    return CASES[name]


def ensemble_cases(n_channels: int = 64, seed: int = 1004,
                   scale: float = 1.0) -> list:
    """Independent channels of uneven size for the batched ensemble.

    Re_tau in {180, 300, 395, 550}; grids between 64^3 and 192 x 128 x 128;
    particle counts uniform in [50k, 2M] (times `scale`); d+ in [0.5, 3].
    """
    rng = np.random.Generator(np.random.Philox(seed))
    grids = [(64, 64, 64), (96, 64, 64), (128, 96, 96), (128, 128, 128), (192, 128, 128)]
    out = []
    for c in range(n_channels):
        re = float(rng.choice([180.0, 300.0, 395.0, 550.0]))
        nx, ny, nz = grids[int(rng.integers(len(grids)))]
        npart = max(1, int(round(rng.uniform(50_000, 2_000_000) * scale)))
        dp = float(rng.uniform(0.5, 3.0))
        out.append(Case(f"ens{c:02d}", re, nx, ny, nz, _TWO_PI * DELTA, math.pi * DELTA,
                        npart, (dp, dp), 1000.0, 0.0, 500, 0.05, False,
                        10_000 + c, 20_000 + c))
    return out


# ----------------------------------------------------------------------------
# grid

def y_faces(ny: int, delta: float = DELTA, gamma: float = 2.0) -> np.ndarray:
    """tanh-stretched wall-normal cell faces, y_f[0] = 0, y_f[ny] = 2 delta."""
    j = np.arange(ny + 1, dtype=np.float64)
    f = delta * (1.0 - np.tanh(gamma * (1.0 - 2.0 * j / ny)) / math.tanh(gamma))
    f[0] = 0.0
    f[-1] = 2.0 * delta
    return f


def node_y(faces: np.ndarray) -> np.ndarray:
    """Wall-extended lattice coordinates [0, cell centres, 2 delta] (Ny+2)."""
    yc = 0.5 * (faces[1:] + faces[:-1])
    return np.concatenate(([faces[0]], yc, [faces[-1]]))


def reichardt_uplus(yplus: np.ndarray) -> np.ndarray:
    """Reichardt's composite law of the wall u+(y+)."""
    yp = np.asarray(yplus, dtype=np.float64)
    return (np.log1p(0.41 * yp) / 0.41
            + 7.8 * (1.0 - np.exp(-yp / 11.0) - (yp / 11.0) * np.exp(-yp / 3.0)))


def _wall_distance_plus(y: np.ndarray, c: Case) -> np.ndarray:
    yw = np.minimum(y, c.ly - y)
    return np.maximum(yw, 0.0) * c.u_tau / c.nu


def mean_velocity(y: np.ndarray, c: Case) -> np.ndarray:
    return c.u_tau * reichardt_uplus(_wall_distance_plus(np.asarray(y, np.float64), c))


def damping(y: np.ndarray, c: Case) -> np.ndarray:
    yp = _wall_distance_plus(np.asarray(y, np.float64), c)
    return yp / (yp + 10.0)


# ----------------------------------------------------------------------------
# random Fourier modes

@dataclasses.dataclass
class Modes:
    nxi: np.ndarray     # integer x wavenumber index (k_x = 2 pi nxi / Lx)
    nzi: np.ndarray     # integer z wavenumber index
    kx: np.ndarray
    ky: np.ndarray
    kz: np.ndarray
    amp: np.ndarray     # (n, 3) amplitude vectors [m/s], perpendicular to k
    phase: np.ndarray


def draw_modes(c: Case, n_modes: int = N_MODES) -> Modes:
    rng = np.random.Generator(np.random.Philox(c.field_seed))
    dx = c.lx / c.nx
    kmin, kmax = _TWO_PI / c.lx, math.pi / dx
    k = np.exp(rng.uniform(math.log(kmin), math.log(kmax), n_modes))
    # uniform direction on the sphere
    mu = rng.uniform(-1.0, 1.0, n_modes)
    ang = rng.uniform(0.0, _TWO_PI, n_modes)
    s = np.sqrt(1.0 - mu * mu)
    dirv = np.stack([s * np.cos(ang), mu, s * np.sin(ang)], axis=1)
    nxi = np.rint(k * dirv[:, 0] * c.lx / _TWO_PI).astype(np.int64)
    nzi = np.rint(k * dirv[:, 2] * c.lz / _TWO_PI).astype(np.int64)
    nxi = np.clip(nxi, -(c.nx // 2) + 1, c.nx // 2 - 1)
    nzi = np.clip(nzi, -(c.nz // 2) + 1, c.nz // 2 - 1)
    kx = _TWO_PI * nxi / c.lx
    kz = _TWO_PI * nzi / c.lz
    ky = k * dirv[:, 1]
    kvec = np.stack([kx, ky, kz], axis=1)
    kn = np.linalg.norm(kvec, axis=1)
    kn = np.where(kn > 0, kn, 1.0)
    khat = kvec / kn[:, None]
    g = rng.standard_normal((n_modes, 3))
    a_dir = g - np.sum(g * khat, axis=1)[:, None] * khat
    a_dir /= np.linalg.norm(a_dir, axis=1)[:, None]
    ke = _TWO_PI / c.delta
    kr = kn / ke
    spec = kr ** 4 / (1.0 + kr ** 2) ** (17.0 / 6.0)
    weight = np.sqrt(spec * kn)          # log-uniform sampling density ~ 1/k
    mag = rng.standard_normal(n_modes) * weight
    amp = a_dir * mag[:, None]
    # per-component rms of the undamped fluctuation = u_tau
    total = 0.5 * np.sum(amp ** 2)
    amp *= math.sqrt(3.0 * c.u_tau ** 2 / total)
    phase = rng.uniform(0.0, _TWO_PI, n_modes)
    return Modes(nxi, nzi, kx, ky, kz, amp, phase)


def fluid_lattice(c: Case, modes: Optional[Modes] = None, t: float = 0.0,
                  faces: Optional[np.ndarray] = None) -> np.ndarray:
    """Gas velocity on the wall-extended lattice, shape (Nz, Ny+2, Nx, 3), FP64.

    Node (k, jn, i) sits at x = (i + 1/2) dx, y = node_y[jn], z = (k + 1/2) dz.
    Each y-plane is a sparse sum of Fourier modes in x, z, evaluated exactly
    with an inverse 2-D DFT of the mode coefficients.
    """
    if modes is None:
        modes = draw_modes(c)
    if faces is None:
        faces = y_faces(c.ny, c.delta, c.gamma)
    Y = node_y(faces)
    ubar = mean_velocity(Y, c)
    damp = damping(Y, c)
    out = np.zeros((c.nz, c.ny + 2, c.nx, 3), dtype=np.float64)
    ix = np.mod(modes.nxi, c.nx)
    iz = np.mod(modes.nzi, c.nz)
    # half-cell offset of the nodes: exp(i pi (nxi / Nx + nzi / Nz))
    shift = np.exp(1j * math.pi * (modes.nxi / c.nx + modes.nzi / c.nz))
    for jn in range(c.ny + 2):
        if damp[jn] == 0.0:
            continue
        ph = modes.ky * Y[jn] + modes.phase - modes.kx * ubar[jn] * t
        coef = np.exp(1j * ph) * shift
        for comp in range(3):
            spec = np.zeros((c.nz, c.nx), dtype=np.complex128)
            np.add.at(spec, (iz, ix), coef * modes.amp[:, comp])
            plane = np.fft.ifft2(spec).real * (c.nx * c.nz)
            out[:, jn, :, comp] = damp[jn] * plane
    out[:, :, :, 0] += ubar[None, :, None]
    out[:, 0, :, :] = 0.0
    out[:, -1, :, :] = 0.0
    return out


# ----------------------------------------------------------------------------
# particles

@dataclasses.dataclass
class Particles:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    q: np.ndarray
    d: np.ndarray

    @property
    def n(self) -> int:
        return self.x.shape[0]

    def copy(self) -> "Particles":
        return Particles(*(np.array(getattr(self, f.name)) for f in dataclasses.fields(self)))


def draw_particles(c: Case, n: Optional[int] = None) -> Particles:
    n = c.n_particles if n is None else n
    rng = np.random.Generator(np.random.Philox(c.particle_seed))
    lo, hi = c.dplus
    if lo == hi:
        dplus = np.full(n, lo)
    else:
        dplus = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    d = dplus * c.nu / c.u_tau
    r = 0.5 * d
    x = rng.uniform(0.0, c.lx, n)
    z = rng.uniform(0.0, c.lz, n)
    y = r + rng.uniform(0.0, 1.0, n) * (c.ly - 2.0 * r)
    vx = mean_velocity(y, c)
    vy = np.zeros(n)
    vz = np.zeros(n)
    q = rng.standard_normal(n) * c.q0_sigma if c.q0_sigma > 0 else np.zeros(n)
    return Particles(x, y, z, vx, vy, vz, q, d)


def replay_state(c: Case, parts: dict, sample_every: int = 1000, wall_every: int = 2000,
                 seed: int = 77) -> dict:
    """A copy of a particle state (arrays indexed by particle id) prepared for
    a one-step replay against the oracle on a subsample: every particle gets a
    Gaussian charge (std 0.01 q_sat, so that the mesh field matters), and the
    particles whose id is a multiple of `wall_every` (half of the 1-in-
    `sample_every` subsample) are placed just inside their reach of a wall,
    moving towards it, so that the replayed step has wall impacts to compare.
    Positions and velocities keep the precision of the input arrays."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = {k: np.array(v) for k, v in parts.items()}
    n = out["x"].shape[0]
    out["q"] = rng.standard_normal(n) * 0.01 * Q_SAT
    m = np.arange(n) % wall_every == 0
    k = int(m.sum())
    d = np.asarray(out["d"][m], np.float64)
    r = 0.5 * d
    top = rng.random(k) < 0.5
    speed = np.abs(rng.standard_normal(k)) * 0.5 + 0.05
    gap = rng.uniform(0.0, 0.5, k) * speed * c.dt
    y = np.where(top, c.ly - r - gap, r + gap)
    dt = out["y"].dtype
    out["y"][m] = y.astype(dt)
    out["vy"][m] = np.where(top, speed, -speed).astype(dt)
    return out
