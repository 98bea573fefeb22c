"""Pins of the oracle's near field of the hybrid electrostatics
(Coulomb's law between particles that share a cell, Sec. 2.2)."""
import math

import numpy as np

import oracle
import synth

EPS = 8.854e-12


def _grid(nx=4, ny=4, nz=4):
    faces = synth.y_faces(ny)
    return oracle.Grid(nx, nz, 2 * math.pi * 0.02, math.pi * 0.02, faces)


def _state(x, y, z, q, d):
    n = len(x)
    return oracle.State.from_arrays(x, y, z, np.zeros(n), np.zeros(n), np.zeros(n), q, d)


def test_two_particles_closed_form_and_third_law():
    g = _grid()
    p = oracle.Params(rho_p=1000.0)
    x = np.array([0.010, 0.0112]); y = np.array([0.011, 0.0104]); z = np.array([0.005, 0.0061])
    q = np.array([3e-14, -5e-14]); d = np.array([1e-4, 2e-4])
    acc = oracle.coulomb_near(g, p, _state(x, y, z, q, d))
    r = np.array([x[0] - x[1], y[0] - y[1], z[0] - z[1]])
    m = math.pi * d ** 3 * p.rho_p / 6
    f0 = q[0] * q[1] / (4 * math.pi * EPS) * r / np.linalg.norm(r) ** 3
    assert np.allclose(acc[0], f0 / m[0], rtol=1e-13, atol=0)
    assert np.allclose(m[0] * acc[0], -m[1] * acc[1], rtol=1e-13, atol=0)
    # opposite charges attract: particle 0 is pulled towards particle 1
    assert np.dot(acc[0], -r) > 0


def test_brute_force_over_all_pairs():
    g = _grid(6, 5, 4)
    rng = np.random.default_rng(3)
    n = 80
    # clustered: many particles share cells
    x = rng.uniform(0, 2 * g.dx, n); y = rng.uniform(g.yf[1], g.yf[3], n); z = rng.uniform(0, 2 * g.dz, n)
    q = rng.standard_normal(n) * 1e-14
    d = rng.uniform(5e-5, 2e-4, n)
    p = oracle.Params(rho_p=1200.0)
    acc = oracle.coulomb_near(g, p, _state(x, y, z, q, d))
    i, j, k = oracle.locate(g, x, y, z)
    ref = np.zeros((n, 3))
    for a in range(n):
        for b in range(n):
            if a == b or (i[a], j[a], k[a]) != (i[b], j[b], k[b]):
                continue
            r = np.array([x[a] - x[b], y[a] - y[b], z[a] - z[b]])
            ref[a] += q[a] * q[b] / (4 * math.pi * EPS) * r / np.linalg.norm(r) ** 3
        ref[a] /= math.pi * d[a] ** 3 * p.rho_p / 6
    assert np.abs(acc - ref).max() <= 1e-12 * np.abs(ref).max()
    assert (np.abs(ref).sum(axis=1) > 0).sum() > n // 2
    # total momentum change of the pair forces vanishes
    m = math.pi * d ** 3 * p.rho_p / 6
    tot = (m[:, None] * acc).sum(axis=0)
    assert np.abs(tot).max() <= 1e-12 * (m[:, None] * np.abs(acc)).sum()


def test_no_interaction_across_a_face():
    g = _grid()
    p = oracle.Params()
    x = np.array([g.dx - 1e-7, g.dx + 1e-7]); y = np.array([0.02, 0.02]); z = np.array([0.003, 0.003])
    acc = oracle.coulomb_near(g, p, _state(x, y, z, np.array([1e-13, 1e-13]), np.array([1e-4, 1e-4])))
    assert np.all(acc == 0.0)


def test_step_applies_near_field_only_when_enabled():
    g = _grid()
    x = np.array([0.010, 0.0102]); y = np.array([0.011, 0.0109]); z = np.array([0.005, 0.0052])
    st = _state(x, y, z, np.array([2e-13, 2e-13]), np.array([1e-4, 1e-4]))
    lat = np.zeros((g.nz, g.ny + 2, g.nx, 3))
    p = oracle.Params(drag_law=2)
    a = oracle.step(g, p, st, lat, 1e-5)
    b = oracle.step(g, p.with_(coulomb=True), st, lat, 1e-5)
    acc = oracle.coulomb_near(g, p, st)
    # drag off: the near field adds acc dt to v and acc dt^2 / 2 to x
    assert np.allclose(b.vx - a.vx, acc[:, 0] * 1e-5, rtol=1e-9, atol=0)
    assert np.allclose(b.y - a.y, 0.5 * acc[:, 1] * 1e-10, rtol=1e-6, atol=1e-18)
    assert (b.vx - a.vx)[0] * (b.vx - a.vx)[1] < 0
