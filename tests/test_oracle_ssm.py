"""Pins of the oracle's stochastic scaling model of wall-impact charging
(Sec. 2.3.2, reference parameters of Sec. 3.1) and of its random numbers."""
import math
import os

import numpy as np

import oracle
from oracle.ssm import SSM, hertz_area, normals, philox4x32_10, saturation_charge, skew_normal_params, \
    ssm_wall_charge

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _moments(x):
    m = x.mean()
    s = x.std()
    return m, s, np.mean(((x - m) / s) ** 3)


def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(v, 16) for v in r]
        ctr = [np.array([v], np.uint64) for v in w[:4]]
        out = [int(x[0]) for x in philox4x32_10(ctr, (w[4], w[5]))]
        assert out == w[6:10]


def test_box_muller_normals():
    n = 400_000
    z0, z1 = normals(np.arange(n), np.zeros(n, np.int64), seed=12345)
    for z in (z0, z1):
        m, s, g = _moments(z)
        assert abs(m) < 0.01 and abs(s - 1) < 0.01 and abs(g) < 0.02
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 0.01
    # the counter decides the draw: another count gives independent normals
    y0, _ = normals(np.arange(n), np.ones(n, np.int64), seed=12345)
    assert abs(np.corrcoef(z0, y0)[0, 1]) < 0.01


def test_skew_normal_sampler_moments():
    n = 400_000
    z0, z1 = normals(np.arange(n), np.full(n, 7, np.int64), seed=3)
    for mean, sd, skew in ((1.0, 2.0, 0.5), (-3.0, 0.5, -0.8), (0.0, 1.0, 0.0), (2.0, 0.1, 0.99)):
        xi, om, de = skew_normal_params(mean, sd, skew)
        x = xi + om * (de * np.abs(z0) + np.sqrt(1 - de ** 2) * z1)
        m, s, g = _moments(x)
        assert abs(m - mean) < 0.01 * sd and abs(s / sd - 1) < 0.01 and abs(g - skew) < 0.03, (mean, sd, skew)


def test_reference_impact_reproduces_reference_statistics():
    p = oracle.Params(rho_p=1150.0)
    s = SSM(seed=99)
    n = 400_000
    d = np.full(n, 2 * s.r0)
    dq, det = ssm_wall_charge(p, s, d, np.full(n, s.un0), np.zeros(n), np.arange(n), np.zeros(n, np.int64))
    assert np.allclose(det["area_ratio"], 1.0, rtol=1e-14)
    m, sd, g = _moments(dq)
    assert abs(m - s.mu0) < 4 * s.sigma0 / math.sqrt(n)
    assert abs(sd / s.sigma0 - 1) < 0.01
    assert abs(g - s.gamma0) < 0.03


def test_saturation_charges_printed_in_the_paper():
    s = SSM()
    assert abs(saturation_charge(s, 50e-6) / 3.13e-13 - 1) < 2e-3          # Sec. 3.1
    assert abs(saturation_charge(s, 100e-6) / 1.25e-12 - 1) < 2e-3         # Sec. 3.1
    # the paper prints 7.81e-15 C for 25 um; the formula gives ten times that
    assert abs(saturation_charge(s, 25e-6) / 7.81e-14 - 1) < 2e-3
    # at q = -q_sat (dq0_min < 0) the wall's active sites are exhausted
    p = oracle.Params()
    d = np.array([50e-6])
    _, det = ssm_wall_charge(p, s, d, [0.3], -saturation_charge(s, d), [0], [0])
    assert det["chi_w"][0] == 0.0 and det["mu_w"][0] == 0.0


def test_deterministic_limit_scales_with_the_hertz_area():
    """sigma_0 = gamma_0 = 0, q = 0: dq = mu_0 A / A_0 = mu_0 (d/d_0)^2 (u/u_0)^(4/5)."""
    p = oracle.Params(rho_p=1150.0)
    s = SSM(sigma0=0.0, gamma0=0.0)
    d = np.array([50e-6, 91e-6, 400e-6])
    u = np.array([0.01, 0.3, 0.925])
    dq, _ = ssm_wall_charge(p, s, d, u, np.zeros(3), np.arange(3), np.zeros(3, np.int64))
    ref = s.mu0 * (d / (2 * s.r0)) ** 2 * (u / s.un0) ** 0.8
    assert np.allclose(dq, ref, rtol=1e-12, atol=0)


def test_deterministic_limit_matched_to_the_condenser_model():
    """Sec. 3.1: with sigma_0 = gamma_0 = 0 and mu_0 = dq0_min = mu_condenser the SSM
    stands in for the condenser model.  Matched at the reference impact, the two
    agree there; elsewhere their ratio is the closed form of the two scalings:
    the condenser charge C U_c dt_w / T_w (dt_w / T_w ~ 1e-8) goes as d^3 u^(3/5),
    the SSM's mu_0 A / A_0 as d^2 u^(4/5), so SSM / condenser = (d_0 / d)(u / u_0)^(1/5)."""
    p = oracle.Params(rho_p=1150.0, U_c=5.0)
    s0 = SSM()
    mu_c, _, _ = oracle.condenser_wall(p, np.array([2 * s0.r0]), np.array([s0.un0]), np.zeros(1))
    s = SSM(sigma0=0.0, gamma0=0.0, mu0=float(mu_c[0]), dq0_min=float(mu_c[0]))
    d = np.array([2 * s0.r0, 50e-6, 91e-6, 400e-6, 1e-3])
    u = np.array([s0.un0, 0.01, 0.3, 0.925, 2.0])
    dq, _ = ssm_wall_charge(p, s, d, u, np.zeros(5), np.arange(5), np.zeros(5, np.int64))
    cond, _, _ = oracle.condenser_wall(p, d, u, np.zeros(5))
    assert abs(dq[0] / cond[0] - 1) < 1e-13
    ratio = (2 * s0.r0 / d) * (u / s0.un0) ** 0.2
    assert np.allclose(dq / cond, ratio, rtol=1e-7, atol=0)


def test_step_uses_the_ssm_with_the_impact_counter():
    g = oracle.Grid(4, 4, 2 * math.pi * 0.02, math.pi * 0.02, np.linspace(0, 0.04, 5))
    lat = np.zeros((4, 6, 4, 3))
    n = 6
    d = np.full(n, 1e-4)
    st = oracle.State.from_arrays(np.linspace(0.001, 0.1, n), np.full(n, 0.5e-4 + 1e-6), np.full(n, 0.01),
                                  np.zeros(n), np.full(n, -0.5), np.zeros(n), np.zeros(n), d,
                                  n_imp=np.arange(n), ids=np.arange(n) + 100)
    p = oracle.Params(drag_law=2, electrostatics=False, ssm=SSM(seed=5))
    out = oracle.step(g, p, st, lat, 1e-5)
    assert np.all(out.n_imp == st.n_imp + 1)
    speed = np.abs(out.vy)
    dq, _ = ssm_wall_charge(p, p.ssm, d, speed, np.zeros(n), st.id, st.n_imp)
    assert np.array_equal(out.q, dq)
    assert np.array_equal(out.q_wall, dq)
    other = oracle.step(g, p.with_(ssm=SSM(seed=6)), st, lat, 1e-5)
    assert not np.array_equal(other.q, out.q)


# ---------------------------------------------------------------- charging-site history c / c_0

def _det(s):
    """The deterministic limit of the SSM (no scatter, no skew)."""
    return SSM(r0=s.r0, un0=s.un0, mu0=s.mu0, sigma0=0.0, gamma0=0.0, dq0_min=s.dq0_min, c_sat=s.c_sat,
               seed=s.seed)


def test_site_history_is_inert_for_an_uncharged_particle():
    """A first impact of an uncharged particle uses up no sites (q_m = 0 in
    the printed sum), so tracking the history changes neither its charge nor
    its site density."""
    p = oracle.Params(rho_p=1150.0)
    s = SSM(seed=5)
    n = 1000
    d = np.full(n, 80e-6)
    sp = np.linspace(0.1, 2.0, n)
    dq0, _ = ssm_wall_charge(p, s, d, sp, np.zeros(n), np.arange(n), np.zeros(n, np.int64))
    dq1, det = ssm_wall_charge(p, s, d, sp, np.zeros(n), np.arange(n), np.zeros(n, np.int64), site=np.ones(n))
    assert np.array_equal(dq0, dq1)
    assert np.array_equal(det["site"], np.ones(n))


def test_site_history_is_the_printed_sum_over_earlier_contacts():
    """Many impacts of one particle, its charge taken as each contact begins:
    the product form the oracle carries equals the printed sum
    1 - sum_m (c_{m-1}/c_0)(A_m/A_p)(chi_m/chi_0)(q_m/q_max) term by term, and
    with the charge and speed held fixed it is the closed form (1 - a)^M."""
    p = oracle.Params(rho_p=1150.0)
    s = _det(SSM(seed=1))
    d = np.array([60e-6])
    q_max = -saturation_charge(s, d)[0]          # dq0_min < 0: the wall charges the particle negative
    site = np.ones(1)
    q = np.zeros(1)
    hist_a, hist_c = [], [1.0]
    rng = np.random.default_rng(3)
    for m in range(60):
        sp = rng.uniform(0.2, 3.0, 1)
        dq, det = ssm_wall_charge(p, s, d, sp, q, np.zeros(1, np.int64), np.full(1, m), site=site)
        # the contact's share A_m / A_p (chi_m / chi_0)(q_m / q_max), with the Hertz area of Sec. 2.3.1
        a = hertz_area(p, d, sp)[0] / (math.pi * d[0] ** 2) * det["chi_i"][0] * q[0] / q_max
        hist_a.append(a)
        site = det["site"]
        hist_c.append(site[0])
        q = q + dq
        # the printed sum over the contacts so far
        printed = 1.0 - sum(hist_c[k] * hist_a[k] for k in range(len(hist_a)))
        assert abs(site[0] - printed) <= 1e-13, (m, site[0], printed)
    assert hist_c[-1] < 1.0 - 1e-6 and q[0] < 0
    # fixed charge and speed: (1 - a)^M
    qf = np.array([0.4 * q_max])
    site = np.ones(1)
    for m in range(200):
        _, det = ssm_wall_charge(p, s, d, np.array([1.5]), qf, np.zeros(1, np.int64), np.full(1, m), site=site)
        site = det["site"]
    a = hertz_area(p, d, 1.5)[0] / (math.pi * d[0] ** 2) * det["chi_i"][0] * 0.4
    assert abs(site[0] - (1.0 - a) ** 200) <= 1e-12


def test_site_density_scales_the_particle_sites_linearly():
    """N_i / N_0 carries c / c_0: in the deterministic limit the impact charge
    is affine in c (c = 1/2 lies halfway between c = 0 and c = 1), and c = 0
    leaves only the wall's share mu_w."""
    p = oracle.Params(rho_p=1150.0)
    s = _det(SSM(seed=2))
    n = 50
    d = np.full(n, 120e-6)
    sp = np.linspace(0.3, 2.5, n)
    q = -np.linspace(0.0, 0.8, n) * saturation_charge(s, d)
    args = (p, s, d, sp, q, np.arange(n), np.zeros(n, np.int64))
    dq = {c: ssm_wall_charge(*args, site=np.full(n, c))[0] for c in (0.0, 0.5, 1.0)}
    assert np.allclose(dq[0.5], 0.5 * (dq[0.0] + dq[1.0]), rtol=1e-13, atol=0)
    _, det = ssm_wall_charge(*args, site=np.zeros(n))
    assert np.allclose(dq[0.0], det["mu_w"], rtol=1e-15, atol=0)


def test_site_history_counts_the_charge_before_the_contact_and_stays_in_bounds():
    """The depletion of a contact is formed from the charge the particle
    brings to it (a first contact with q0 = 0 uses up nothing even though it
    leaves the particle charged); a particle charged against the wall's
    direction (q / q_max < 0) keeps c / c_0 = 1, and c / c_0 never leaves
    [0, 1]."""
    p = oracle.Params(rho_p=1150.0)
    s = SSM(seed=8)
    d = np.full(3, 90e-6)
    qs = saturation_charge(s, d)
    q = np.array([0.0, 0.5 * qs[1], -0.999 * qs[2]])     # uncharged, against, nearly saturated
    dq, det = ssm_wall_charge(p, s, d, np.full(3, 1.0), q, np.arange(3), np.zeros(3, np.int64),
                              site=np.array([1.0, 1.0, 1e-12]))
    assert det["site"][0] == 1.0 and dq[0] != 0.0
    assert det["site"][1] == 1.0
    assert 0.0 <= det["site"][2] < 1e-12
