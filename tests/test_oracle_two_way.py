"""Pins of the oracle's momentum source of the particles on the gas, F_s of
the gas momentum equation (Eq. ns): the aerodynamic forces of the particles of
a control volume, per unit gas mass (oracle.momentum_source).

* momentum balance: rho V_c dt F_s summed over the cells equals minus the
  particles' own velocity change from the integrator less the field impulse,
  sum_p m_p (v' - v - a dt), with an applied field large enough that the
  field part of the integrator matters;
* small-step limit: F_s tends to the instantaneous aerodynamic force
  -(1/(rho V_c)) sum m_p (u - v)/tau of the drag laws of Sec. 2.2;
* one particle in a uniform gas flow: the closed-form relaxation
  v(t) = u + (v0 - u) e^(-t/tau_p), booked in its start cell although it
  crosses into the next cell during the step;
* drag off: no source.
"""
import math

import numpy as np
import pytest

import oracle
from _problems import oracle_params, oracle_state, problem


def _vel(st):
    return np.stack([st.vx, st.vy, st.vz], axis=1)


@pytest.mark.parametrize("drag", [0, 1])
def test_balance_with_the_particles_drag_impulse(drag):
    c, faces, lat, parts = problem(16, 12, 8, n=300, q_scale=1e-13, vy_scale=0.3, seed=31 + drag,
                                   dplus=(0.8, 2.5))
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    p = oracle_params(c, drag_law=drag)
    st = oracle_state(parts)
    dt = 40 * c.dt
    m = oracle.particle_mass(p, st.d)
    # a field whose force is as large as the drag
    d0 = {}
    oracle.step(g, p, st, lat, dt, diag=d0, E_lat=np.zeros_like(lat))
    drag_acc = np.linalg.norm(d0["uf"] - _vel(st), axis=1) / d0["tau"]
    e_scale = np.median(drag_acc * m / np.abs(st.q))
    E = np.random.default_rng(drag).standard_normal(lat.shape) * e_scale
    diag = {}
    oracle.step(g, p, st, lat, dt, diag=diag, E_lat=E)
    acc = diag["acc"]
    assert np.median(np.linalg.norm(acc, axis=1) / drag_acc) > 0.1
    X = np.stack([st.x, st.y, st.z], axis=1)
    _, Vn, _ = oracle.push(p, X, _vel(st), diag["uf"], acc, st.d, dt)
    particles = (m[:, None] * (Vn - _vel(st) - acc * dt)).sum(axis=0)
    gas = (p.rho * dt * g.vol_y[None, None, :, None] * diag["F_s"]).sum(axis=(1, 2, 3))
    scale = (m[:, None] * np.abs(Vn - _vel(st))).sum(axis=0)
    assert np.all(np.abs(gas + particles) <= 1e-9 * scale), (gas, particles)
    # the field's share of the integrator (a tau phi2) is far above that bar
    s = dt / diag["tau"]
    assert np.abs((m * (s - (1 - np.exp(-s))) * diag["tau"])[:, None] * acc).sum(axis=0).min() > 1e-6 * scale.max()


@pytest.mark.parametrize("drag", [0, 1])
def test_small_step_limit_is_the_instantaneous_drag(drag):
    c, faces, lat, parts = problem(16, 12, 8, n=400, vy_scale=0.5, seed=41 + drag, dplus=(0.8, 2.5))
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    p = oracle_params(c, drag_law=drag, electrostatics=False)
    st = oracle_state(parts)
    V = _vel(st)
    uf = oracle.trilinear(g, lat, st.x, st.y, st.z)
    tau = oracle.relaxation_time(p, st.d, np.linalg.norm(V - uf, axis=1))
    dt = 1e-7 * tau.min()
    diag = {}
    oracle.step(g, p, st, lat, dt, diag=diag)
    force = oracle.particle_mass(p, st.d)[:, None] * (uf - V) / tau[:, None]
    i, j, k = oracle.locate(g, st.x, st.y, st.z)
    key = g.cell_key(i, j, k)
    for comp in range(3):
        ref = -np.bincount(key, weights=force[:, comp], minlength=g.ncells).reshape(g.nz, g.ny, g.nx)
        ref /= p.rho * g.vol_y[None, :, None]
        bound = np.bincount(key, weights=np.abs(force[:, comp]), minlength=g.ncells).reshape(g.nz, g.ny, g.nx)
        bound /= p.rho * g.vol_y[None, :, None]
        assert np.all(np.abs(diag["F_s"][comp] - ref) <= 1e-6 * bound + 1e-300), comp
    assert np.count_nonzero(diag["F_s"][0]) == len(np.unique(key))


def test_single_particle_in_uniform_flow_closed_form():
    nx, ny, nz = 16, 12, 8
    lx, lz = 2 * math.pi * 0.02, math.pi * 0.02
    faces = np.linspace(0.0, 0.04, ny + 1)
    g = oracle.Grid(nx, nz, lx, lz, faces)
    U, v0, d = 1.0, 2.0, 1e-4
    lat = np.zeros((nz, ny + 2, nx, 3))
    lat[..., 0] = U
    p = oracle.Params(drag_law=0, electrostatics=False)
    x0 = 3 * g.dx - 1e-5
    st = oracle.State.from_arrays([x0], [0.0213], [0.3 * lz], [v0], [0.0], [0.0], [0.0], [d])
    dt = 1e-4
    diag = {}
    out = oracle.step(g, p, st, lat, dt, diag=diag)
    assert out.x[0] > 3 * g.dx                    # ends in the next cell
    tau_p = p.rho_p * d * d / (18.0 * p.rho * p.nu)
    m = math.pi * d ** 3 * p.rho_p / 6.0
    j = int(np.searchsorted(faces, 0.0213, side="right") - 1)
    vol = g.dx * (faces[j + 1] - faces[j]) * g.dz
    ref = -m * (U - v0) * (1.0 - math.exp(-dt / tau_p)) / (p.rho * vol * dt)
    k = int(0.3 * lz / g.dz)
    fs = diag["F_s"]
    assert abs(fs[0, k, j, 2] - ref) <= 1e-12 * abs(ref)
    fs0 = fs.copy()
    fs0[0, k, j, 2] = 0.0
    assert not np.any(fs0)
    # the particle's own velocity change agrees with the closed form too
    assert abs(out.vx[0] - (U + (v0 - U) * math.exp(-dt / tau_p))) <= 1e-14


def test_drag_off_gives_no_source():
    c, faces, lat, parts = problem(16, 12, 8, n=50, seed=3)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    diag = {}
    oracle.step(g, oracle_params(c, drag_law=2), oracle_state(parts), lat, c.dt, diag=diag)
    assert not np.any(diag["F_s"])


def test_run_returns_the_mean_over_its_steps():
    c, faces, lat, parts = problem(16, 12, 8, n=80, vy_scale=0.3, seed=5)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    p = oracle_params(c)
    fs = np.full((3, g.nz, g.ny, g.nx), 7.0)
    oracle.run(g, p, oracle_state(parts), lat, c.dt, 3, fs=fs)
    st = oracle_state(parts)
    acc = np.zeros_like(fs)
    for _ in range(3):
        diag = {}
        st = oracle.step(g, p, st, lat, c.dt, diag=diag)
        acc += diag["F_s"]
    assert np.allclose(fs, acc / 3, rtol=1e-14, atol=0)
