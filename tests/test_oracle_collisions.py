"""Pins of the oracle's 4-way coupling: particle-particle hard-sphere
collisions (Sec. 2.2) with the condenser-model charge exchange (Sec. 2.3.1)."""
import math

import numpy as np

import oracle
import synth
from test_oracle_pins import _hertz_impact


def test_contact_parameters_match_two_sphere_hertz_ode():
    """With k_e = 1, alpha_12 is the Hertz maximum compression of two spheres
    (reduced mass, effective radius R* = R_i R_j / (R_i + R_j), 1/E* =
    2 (1 - mu_p^2) / E_p), dt_12 the contact time and A_12 = pi R* alpha_12."""
    p = oracle.Params(k_e=1.0, rho_p=1150.0)
    for di, dj, u in ((50e-6, 50e-6, 0.4), (30e-6, 90e-6, 0.15), (120e-6, 70e-6, 1.1)):
        mi, mj = (p.rho_p * math.pi * dd ** 3 / 6 for dd in (di, dj))
        mstar = mi * mj / (mi + mj)
        Rstar = (di / 2) * (dj / 2) / (di / 2 + dj / 2)
        Estar = 1.0 / (2 * (1 - p.mu_p ** 2) / p.E_p)
        dmax, tc = _hertz_impact(mstar, Rstar, Estar, u)
        _, det = oracle.pp_charge(p, di, dj, 0.0, 0.0, u)
        assert abs(float(det["alpha"]) / dmax - 1) < 1e-6
        assert abs(float(det["dt"]) / tc - 1) < 2e-3            # 2.94 vs 2.9432...
        assert abs(float(det["A"]) / (math.pi * Rstar * dmax) - 1) < 1e-6


def test_charge_exchange_is_rc_discharge_of_two_capacitors():
    """Two spheres (C = 4 pi eps d/2) joined through the contact resistance
    R = phi_p ((d_i + d_j)/2) / A_12 for dt_12: dq_i/dt = (q_j/C_j - q_i/C_i)/R."""
    p = oracle.Params(rho_p=1150.0, phi_p=3e3)
    di, dj, qi, qj, u = 60e-6, 110e-6, 4e-15, -9e-15, 0.5
    dq, det = oracle.pp_charge(p, di, dj, qi, qj, u)
    Ci, Cj = 2 * math.pi * p.eps * di, 2 * math.pi * p.eps * dj
    R = p.phi_p * ((di + dj) / 2) / float(det["A"])
    f = lambda a: ((qi + qj - a) / Cj - a / Ci) / R
    nst = 400
    h = float(det["dt"]) / nst
    a = qi
    for _ in range(nst):
        k1 = f(a); k2 = f(a + h / 2 * k1); k3 = f(a + h / 2 * k2); k4 = f(a + h * k3)
        a += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert 0.05 < abs(float(dq)) / abs(qi - (qi + qj) * Ci / (Ci + Cj)) < 0.95   # partial discharge
    assert abs(float(dq) / (a - qi) - 1) < 1e-9


def test_fast_contact_equalises_potentials_and_conserves_charge():
    p = oracle.Params(rho_p=1150.0, phi_p=1e-6)          # T_12 << dt_12
    di, dj, qi, qj = 40e-6, 80e-6, 5e-15, 1e-15
    dq, _ = oracle.pp_charge(p, di, dj, qi, qj, 0.3)
    Ci, Cj = 2 * math.pi * p.eps * di, 2 * math.pi * p.eps * dj
    assert abs((qi + dq) / Ci - (qj - dq) / Cj) < 1e-12 * abs(qi / Ci)
    # equal potentials exchange nothing
    dq0, _ = oracle.pp_charge(p, di, dj, qj * di / dj, qj, 0.3)
    assert abs(float(dq0)) < 1e-12 * abs(qj)


def _grid():
    return oracle.Grid(4, 4, 2 * math.pi * 0.02, math.pi * 0.02, synth.y_faces(4))


def test_elastic_update_conserves_momentum_and_energy():
    g = _grid()
    p = oracle.Params(rho_p=1000.0)
    x = np.array([0.010, 0.01008]); y = np.array([0.012, 0.01203]); z = np.array([0.003, 0.00302])
    d = np.array([1.2e-4, 0.8e-4])
    v = np.array([[0.5, -0.1, 0.2], [-0.4, 0.3, 0.0]])        # approaching
    q = np.array([2e-15, -3e-15])
    vn, qn, pairs = oracle.pp_collisions(g, p, x, y, z, v, q, d)
    assert pairs == [(0, 1)]
    m = math.pi * d ** 3 * p.rho_p / 6
    assert np.allclose((m[:, None] * vn).sum(0), (m[:, None] * v).sum(0), rtol=1e-13, atol=1e-25)
    assert abs((m * (vn ** 2).sum(1)).sum() / (m * (v ** 2).sum(1)).sum() - 1) < 1e-13
    assert abs(qn.sum() - q.sum()) < 1e-28
    assert qn[0] != q[0]
    # after the collision the pair separates
    assert np.dot(vn[0] - vn[1], [x[0] - x[1], y[0] - y[1], z[0] - z[1]]) > 0
    # equal masses, head-on: the normal components are exchanged
    d2 = np.array([1e-4, 1e-4])
    x2 = np.array([0.010, 0.0100 + 0.9e-4]); y2 = np.array([0.012, 0.012]); z2 = np.array([0.003, 0.003])
    v2 = np.array([[0.3, 0.1, 0.0], [-0.2, 0.0, 0.05]])
    vn2, _, _ = oracle.pp_collisions(g, p, x2, y2, z2, v2, np.zeros(2), d2)
    assert np.allclose(vn2[:, 0], [-0.2, 0.3], rtol=1e-13)
    assert np.allclose(vn2[:, 1:], v2[:, 1:], rtol=1e-13)
    # overlapping but separating: no collision
    _, _, none = oracle.pp_collisions(g, p, x2, y2, z2, -v2, np.zeros(2), d2)
    assert none == []


def test_pair_selection_brute_force():
    """Mutual nearest overlapping approaching partners of the same cell,
    checked by plain loops over all pairs."""
    g = _grid()
    p = oracle.Params(rho_p=1000.0)
    rng = np.random.default_rng(5)
    n = 300
    x = rng.uniform(0, 2 * g.dx, n); y = rng.uniform(g.yf[1], g.yf[2], n); z = rng.uniform(0, g.dz, n)
    d = rng.uniform(1.0e-3, 3.0e-3, n)                 # large spheres: many overlaps
    v = rng.standard_normal((n, 3))
    q = rng.standard_normal(n) * 1e-15
    vn, qn, pairs = oracle.pp_collisions(g, p, x, y, z, v, q, d)
    i, j, k = oracle.locate(g, x, y, z)
    best = {}
    for a in range(n):
        bd, bb = None, None
        for b in range(n):
            if a == b or (i[a], j[a], k[a]) != (i[b], j[b], k[b]):
                continue
            s = np.array([x[a] - x[b], y[a] - y[b], z[a] - z[b]])
            if np.dot(s, s) < (0.5 * (d[a] + d[b])) ** 2 and np.dot(v[a] - v[b], s) < 0:
                if bd is None or np.dot(s, s) < bd:
                    bd, bb = np.dot(s, s), b
        best[a] = bb
    ref = sorted((a, b) for a, b in best.items() if b is not None and a < b and best[b] == a)
    assert sorted(pairs) == ref
    assert len(ref) > 5
    untouched = np.ones(n, bool)
    for a, b in ref:
        untouched[[a, b]] = False
    assert np.array_equal(vn[untouched], v[untouched]) and np.array_equal(qn[untouched], q[untouched])
    assert abs(qn.sum() - q.sum()) <= 1e-12 * np.abs(q).sum()
