"""Stochastic scaling model (SSM) of particle-wall impact charging (FP64).

Part of the FP64 CPU oracle: test infrastructure only.

Sec. 2.3.2: the contact area holds charge-exchange sites.  The wall's active
sites give the particle a charge with mean mu_w = dq0_min N_w / N_w0; the
particle's own sites exchange charge stochastically, a sum of Bernoulli
variables approximated by a skew-normal distribution G(mu_i, sigma_i,
gamma_i) with
  mu_i = (dq0_min - mu_0) N_i / N_0,  sigma_i = sigma_0 sqrt(N_i / N_0),
  gamma_i = -gamma_0 N_0 / N_i,
  N_w / N_w0 = (A / A_0)(chi_w / chi_0),  N_i / N_0 = (A / A_0)(chi_i / chi_0)(c / c_0),
  chi_w / chi_0 = 1 - sgn(dq0_min) 4 q / (C_sat d^2),
  chi_i / chi_0 = 1 + sgn(dq0_min - mu_0) 4 q / (C_sat d^2),   both clipped to [0, 1],
with the Hertz contact area A of the impact and A_0 of the reference impact
(diameter 2 r_0, normal speed u_n0).  The reference parameters are those of
Sec. 3.1.

Readings:
* the charge of one impact is dq = mu_w - Y with Y ~ G(mu_i, sigma_i, gamma_i)
  (at the reference impact its mean is mu_0 and, Y being a sum of
  same-signed site transfers, its bound is dq0_min);
* gamma_i as printed (-gamma_0 N_0 / N_i), clipped to |gamma| <= 0.99, inside
  the skew-normal family's range (|gamma| < 0.99527), where the sample stays
  well conditioned;
* the charging-site density c / c_0 of a particle follows the printed sum
  over its earlier contacts m = 1 .. M-1,
    c / c_0 = 1 - sum_m (c_{m-1} / c_0)(A_m / A_p)(chi_m / chi_0)(q_m / q_max),
  read as: A_m the Hertz area of contact m, A_p = pi d^2 the particle's
  surface, chi_m the particle's own activity ratio chi_i at contact m, q_m
  its charge as the contact begins, and q_max = sgn(dq0_min) C_sat d^2 / 4
  the saturation charge the wall drives it towards (where chi_w reaches 0),
  so that q_m / q_max >= 0 while the particle charges towards saturation.
  Term by term the sum is the product c_M = c_{M-1} (1 - a_M) with
  a_M = (A_M / A_p)(chi_M / chi_0)(q_M / q_max); the result is clipped to
  [0, 1] as the paper bounds it.  Only wall contacts count (particle-particle
  contacts charge by the condenser model here).  A particle whose history is
  not tracked keeps c / c_0 = 1;
* A and A_0 are the Hertz contact areas pi (d/2) alpha without kappa_A;
* random numbers: Philox4x32-10 (Salmon et al., SC'11) with counter
  (particle id, impact count before this impact, 0, 0) and key (seed low
  32 bits, seed high 32 bits); the four 32-bit outputs give two uniforms
  (x + 0.5) 2^-32 each for two Box-Muller normals z0, z1; the skew-normal
  sample is xi + omega (delta |z0| + sqrt(1 - delta^2) z1) with delta, omega,
  xi from the mean, standard deviation and skewness (method of moments).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .constants import Params

# |skewness| is clipped below the skew-normal family's supremum 0.99527, where
# delta -> 1 and sqrt(1 - delta^2) would be the root of rounding noise
GAMMA_MAX = 0.99


@dataclasses.dataclass
class SSM:
    """Reference impact of the SSM (Sec. 3.1) and the generator seed."""
    r0: float = 2e-4          # reference particle radius [m]
    un0: float = 0.925        # reference normal impact speed [m/s]
    mu0: float = -4.12e-15    # mean impact charge [C]
    sigma0: float = 6.49e-15  # standard deviation [C]
    gamma0: float = -0.191    # skewness
    dq0_min: float = -2.19e-14   # minimum impact charge [C]
    c_sat: float = 500e-6     # C_sat [C/m^2]
    seed: int = 0


# ---------------------------------------------------------------- Philox4x32-10
_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on arrays of counters (4, n) and a key (2,)."""
    c = [np.asarray(x, np.uint64) & _MASK for x in ctr]
    k0, k1 = np.uint64(key[0] & _MASK), np.uint64(key[1] & _MASK)
    for r in range(10):
        p0 = np.uint64(_M0) * c[0]
        p1 = np.uint64(_M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + np.uint64(_W0)) & np.uint64(_MASK)
        k1 = (k1 + np.uint64(_W1)) & np.uint64(_MASK)
    return [x.astype(np.uint32) for x in c]


def normals(ids, counts, seed):
    """Two standard normals per (id, count) by Box-Muller from Philox words."""
    ids = np.asarray(ids, np.uint64)
    counts = np.asarray(counts, np.uint64)
    zero = np.zeros_like(ids)
    w = philox4x32_10([ids, counts, zero, zero], (seed & _MASK, (seed >> 32) & _MASK))
    u = [(x.astype(np.float64) + 0.5) * 2.0 ** -32 for x in w]
    rad = np.sqrt(-2.0 * np.log(u[0]))
    ang = 2.0 * math.pi * u[1]
    return rad * np.cos(ang), rad * np.sin(ang)


def skew_normal_params(mean, sd, skew):
    """(xi, omega, delta) of the skew-normal with the given first three moments."""
    g = np.clip(np.asarray(skew, np.float64), -GAMMA_MAX, GAMMA_MAX)
    b = math.sqrt(2.0 / math.pi)
    a = np.abs(g) ** (2.0 / 3.0)
    t = a / (((4.0 - math.pi) / 2.0) ** (2.0 / 3.0) + a)      # (delta b)^2
    delta = np.sign(g) * np.sqrt(t) / b
    omega = np.asarray(sd, np.float64) / np.sqrt(1.0 - 2.0 * delta ** 2 / math.pi)
    xi = np.asarray(mean, np.float64) - omega * delta * b
    return xi, omega, delta


def hertz_area(p: Params, d, speed):
    """Hertz contact area pi (d/2) alpha of a wall impact (Sec. 2.3.1)."""
    d = np.asarray(d, np.float64)
    elastic = (1.0 - p.mu_p ** 2) / p.E_p + (1.0 - p.mu_w ** 2) / p.E_w
    r = 0.5 * d
    alpha = r * (0.625 * math.pi * p.rho_p * (1.0 + p.k_e) * np.asarray(speed, np.float64) ** 2 * elastic) ** 0.4
    return math.pi * r * alpha


def saturation_charge(s: SSM, d):
    """q_sat = C_sat d^2 / 4, where the wall's active-site ratio reaches zero."""
    return s.c_sat * np.asarray(d, np.float64) ** 2 / 4.0


def site_depletion(p: Params, s: SSM, d, speed, q, chi_i):
    """a = (A / A_p)(chi_i / chi_0)(q / q_max) of one wall contact: the
    fraction of the particle's remaining charging sites the contact uses up
    (q_max = sgn(dq0_min) C_sat d^2 / 4, A_p = pi d^2)."""
    d = np.asarray(d, np.float64)
    q_max = np.sign(s.dq0_min) * saturation_charge(s, d)
    return hertz_area(p, d, speed) / (math.pi * d ** 2) * np.asarray(chi_i, np.float64) * np.asarray(q, np.float64) / q_max


def ssm_wall_charge(p: Params, s: SSM, d, speed, q, ids, counts, site=None):
    """Charge of one wall impact per particle; returns (dq, details).  site:
    the particles' charging-site density c / c_0 before the impact (None: 1,
    not tracked); details["site"] holds its value after the impact."""
    d = np.asarray(d, np.float64)
    q = np.asarray(q, np.float64)
    c = np.ones_like(d) if site is None else np.asarray(site, np.float64)
    area = hertz_area(p, d, speed) / float(hertz_area(p, 2.0 * s.r0, s.un0))
    x = 4.0 * q / (s.c_sat * d ** 2)
    chi_w = np.clip(1.0 - np.sign(s.dq0_min) * x, 0.0, 1.0)
    chi_i = np.clip(1.0 + np.sign(s.dq0_min - s.mu0) * x, 0.0, 1.0)
    nw = area * chi_w
    ni = area * chi_i * c
    mu_w = s.dq0_min * nw
    mu_i = (s.dq0_min - s.mu0) * ni
    sigma_i = s.sigma0 * np.sqrt(ni)
    gamma_i = np.where(ni > 0, -s.gamma0 / np.where(ni > 0, ni, 1.0), 0.0)
    xi, omega, delta = skew_normal_params(mu_i, sigma_i, gamma_i)
    z0, z1 = normals(ids, counts, s.seed)
    y = xi + omega * (delta * np.abs(z0) + np.sqrt(np.maximum(1.0 - delta ** 2, 0.0)) * z1)
    dq = mu_w - y
    c_new = np.clip(c * (1.0 - site_depletion(p, s, d, speed, q, chi_i)), 0.0, 1.0)
    return dq, dict(area_ratio=area, chi_w=chi_w, chi_i=chi_i, mu_w=mu_w, mu_i=mu_i, sigma_i=sigma_i,
                    gamma_i=gamma_i, site=c_new if site is not None else None)
