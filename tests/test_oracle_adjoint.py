"""Pins of the oracle's gradient of the mean charge (oracle/adjoint.py).

* its forward values equal the numpy oracle's step map;
* linearity: with electrostatics and dq_t off and zero initial charge, J is
  linear in U_c and in kappa_A, so dJ/dU_c = J/U_c and dJ/dkappa_A = J/kappa_A;
* central differences of the numpy oracle (no impact flips between +-h) for
  U_c, kappa_A and a random direction in the diameters;
* closed form: one ballistic impact, derivative of the condenser-model charge
  (Sec. 2.3.1) with respect to d, U_c and kappa_A by sympy.
"""
import math

import numpy as np
import pytest

import oracle
from _problems import oracle_params, oracle_state, problem

torch = pytest.importorskip("torch")
from oracle.adjoint import mean_charge_gradient  # noqa: E402


def _small(seed=4, n=150, drag=0, **kw):
    c, faces, lat, parts = problem(16, 12, 8, n=n, q_scale=2e-13, vy_scale=0.4, near_wall=0.3, seed=seed,
                                   dplus=(0.8, 2.5), **kw)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    return c, g, lat, parts


def _J(g, p, parts, lat, dt, nsteps):
    st = oracle.run(g, p, oracle_state(parts), lat, dt, nsteps)
    return st.q.mean(), st.n_imp


@pytest.mark.parametrize("drag", [0, 1, 2])
def test_forward_equals_numpy_oracle(drag):
    c, g, lat, parts = _small(seed=5 + drag)
    p = oracle_params(c, U_c=300.0, drag_law=drag)
    res = mean_charge_gradient(g, p, oracle_state(parts), lat, 2 * c.dt, 6)
    ref = oracle.run(g, p, oracle_state(parts), lat, 2 * c.dt, 6)
    f = res["final"]
    assert np.array_equal(f["n_imp"], ref.n_imp)
    assert ref.n_imp.sum() > 10
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        r = getattr(ref, k)
        assert np.abs(f[k] - r).max() <= 1e-13 * max(np.abs(r).max(), 1e-30), k
    assert np.abs(f["q"] - ref.q).max() <= 1e-13 * np.abs(ref.q).max()
    assert abs(res["J"] - ref.q.mean()) <= 1e-13 * np.abs(ref.q).max()


def test_linearity_in_U_c_and_kappa_A():
    c, g, lat, parts = _small(seed=9)
    parts["q"] = np.zeros_like(parts["q"])
    p = oracle_params(c, U_c=7.0, kappa_A=1.3, electrostatics=False, dq_t=False)
    res = mean_charge_gradient(g, p, oracle_state(parts), lat, c.dt, 5)
    assert res["J"] != 0.0
    assert abs(res["dU_c"] - res["J"] / 7.0) <= 1e-13 * abs(res["J"] / 7.0)
    assert abs(res["dkappa_A"] - res["J"] / 1.3) <= 1e-13 * abs(res["J"] / 1.3)


@pytest.mark.parametrize("drag,impact", [(0, 0), (1, 0), (0, 1), (2, 0)])
def test_gradient_matches_central_differences(drag, impact):
    c, g, lat, parts = _small(seed=11 + drag + 3 * impact, n=120)
    dt, nsteps = 2 * c.dt, 6
    p = oracle_params(c, U_c=2e3, drag_law=drag, impact_vel=impact)
    res = mean_charge_gradient(g, p, oracle_state(parts), lat, dt, nsteps)
    J0, imp0 = _J(g, p, parts, lat, dt, nsteps)
    assert imp0.sum() > 10

    def central(fp, fm, h):
        (jp, ip), (jm, im) = fp, fm
        assert np.array_equal(ip, imp0) and np.array_equal(im, imp0), "impact set changed under +-h"
        return (jp - jm) / (2 * h)

    h = 1e-4
    fd = central(_J(g, p.with_(U_c=p.U_c * (1 + h)), parts, lat, dt, nsteps),
                 _J(g, p.with_(U_c=p.U_c * (1 - h)), parts, lat, dt, nsteps), h * p.U_c)
    assert abs(fd - res["dU_c"]) <= 1e-6 * abs(res["dU_c"])
    fd = central(_J(g, p.with_(kappa_A=1 + h), parts, lat, dt, nsteps),
                 _J(g, p.with_(kappa_A=1 - h), parts, lat, dt, nsteps), h)
    assert abs(fd - res["dkappa_A"]) <= 1e-6 * abs(res["dkappa_A"])
    rng = np.random.default_rng(drag)
    dirn = rng.standard_normal(len(parts["d"])) * parts["d"]
    hd = 1e-6

    def shifted(sign):
        q = dict(parts)
        q["d"] = parts["d"] + sign * hd * dirn
        return _J(g, p, q, lat, dt, nsteps)

    fd = central(shifted(+1), shifted(-1), hd)
    ad = float(np.dot(res["dd"], dirn))
    assert abs(fd - ad) <= 1e-5 * np.abs(res["dd"] * dirn).sum()


def test_single_impact_closed_form():
    """Drag and field off: a particle flies into the bottom wall at constant
    velocity and hits it in the first step; J = q0 + dq.  The speed does not
    depend on d, so dJ/dd is the derivative of the condenser charge alone."""
    sp = pytest.importorskip("sympy")
    c, faces, lat, _ = problem(8, 6, 8, n=1, seed=1)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    d0, q0, U0, K0 = 1.1e-4, 3e-15, 40.0, 1.2
    vel = (0.3, -0.8, 0.2)
    parts = dict(x=np.array([0.01]), y=np.array([0.5 * d0 + 1e-5]), z=np.array([0.01]),
                 vx=np.array([vel[0]]), vy=np.array([vel[1]]), vz=np.array([vel[2]]),
                 d=np.array([d0]), q=np.array([q0]))
    p = oracle_params(c, U_c=U0, kappa_A=K0, drag_law=2, electrostatics=False)
    dt = 1e-4
    res = mean_charge_gradient(g, p, oracle_state(parts), lat, dt, 1)
    assert res["final"]["n_imp"][0] == 1
    d, U, K = sp.symbols("d U K", positive=True)
    s = math.sqrt(sum(v * v for v in vel))
    elastic = (1 - p.mu_p ** 2) / p.E_p + (1 - p.mu_w ** 2) / p.E_w
    alpha = (d / 2) * (sp.Rational(5, 8) * sp.pi * p.rho_p * (1 + p.k_e) * s ** 2 * elastic) ** sp.Rational(2, 5)
    area = K * sp.pi * (d / 2) * alpha
    cap = p.eps * area / p.h
    tw = p.eps_w * p.eps0 * p.phi_p
    dq = -cap * U * (1 - sp.exp(-2.94 * alpha / s / tw)) - area / (sp.pi * d ** 2) * q0
    subs = {d: d0, U: U0, K: K0}
    J = float((q0 + dq).subs(subs).evalf(30))
    assert abs(res["J"] - J) <= 1e-12 * abs(J)
    for sym, got in ((d, res["dd"][0]), (U, res["dU_c"]), (K, res["dkappa_A"])):
        ref = float(sp.diff(dq, sym).subs(subs).evalf(30))
        assert abs(got - ref) <= 1e-10 * abs(ref), (sym, got, ref)
