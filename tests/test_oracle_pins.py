"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks an oracle function against something other than itself: a
value printed in the paper, a closed-form solution, a textbook result solved
independently (e.g. by integrating an ODE), brute force on tiny inputs, or an
invariant.  None of these tests needs a GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.constants import (DRAG_OFF, DRAG_SCHILLER_NAUMANN, DRAG_STOKES,
                              IMPACT_NORMAL)
from oracle.particles import (condenser_wall, dplus, push, relaxation_time,
                              stokes_number, volume_fraction_ppm, wrap)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small_grid(nx=8, ny=6, nz=8, gamma=2.0):
    f = synth.y_faces(ny, 0.02, gamma)
    return oracle.Grid(nx, nz, 2 * math.pi * 0.02, math.pi * 0.02, f)


# ---------------------------------------------------------------- Table 2

def test_table2_units_and_constants():
    """Table 2: d+, St and omega follow from Table 1 and Sec. 3.1 formulas."""
    p = oracle.Params()
    rows = [l.split() for l in open(os.path.join(GOLD, "table2.txt")) if not l.startswith("#")]
    assert len(rows) == 15
    for kind, re, d_um, dp, uc, st, om in rows:
        d = float(d_um) * 1e-6
        # printed values carry two decimals (sometimes truncated): one unit
        assert abs(dplus(d, float(re), 0.02) - float(dp)) <= 0.0101
        assert abs(stokes_number(p, d, float(uc), 0.02) - float(st)) <= 0.0101
        assert abs(volume_fraction_ppm(1e8, d) - float(om)) <= 0.0101


# ---------------------------------------------------------------- grid

def test_locate_brute_force():
    g = small_grid(7, 9, 5)
    rng = np.random.default_rng(1)
    m = 12
    pick = lambda f: np.resize(f[:-1], m)       # points exactly on faces
    x = np.concatenate([rng.uniform(0, g.lx, 200), pick(g.xf)])
    y = np.concatenate([rng.uniform(0, g.ly, 200), pick(g.yf)])
    z = np.concatenate([rng.uniform(0, g.lz, 200), pick(g.zf)])
    i, j, k = oracle.locate(g, x, y, z)
    for n in range(x.shape[0]):
        ii = max(a for a in range(g.nx) if g.xf[a] <= x[n])
        jj = max(a for a in range(g.ny) if g.yf[a] <= y[n])
        kk = max(a for a in range(g.nz) if g.zf[a] <= z[n])
        assert (i[n], j[n], k[n]) == (ii, jj, kk)


def test_trilinear_reproduces_linear_fields():
    """Trilinear interpolation is exact for fields linear in x, y, z."""
    g = small_grid(10, 12, 9)
    xs = (np.arange(g.nx) + 0.5) * g.dx
    zs = (np.arange(g.nz) + 0.5) * g.dz
    Z, Y, X = np.meshgrid(zs, g.Y, xs, indexing="ij")
    coef = np.array([[1.5, -2.0, 0.7, 3.0], [0.2, 5.0, -1.0, -4.0]])
    lat = np.stack([c[0] + c[1] * X + c[2] * Y + c[3] * Z for c in coef], axis=-1)
    rng = np.random.default_rng(2)
    n = 500
    # stay inside the node hull in x and z (no periodic seam)
    x = rng.uniform(xs[0], xs[-1], n)
    z = rng.uniform(zs[0], zs[-1], n)
    y = np.concatenate([rng.uniform(0, g.ly, n - 4), [0.0, g.ly * (1 - 1e-16), g.yc[0], g.yc[-1]]])
    out = oracle.trilinear(g, lat, x, y, z)
    for c in range(2):
        ref = coef[c, 0] + coef[c, 1] * x + coef[c, 2] * y + coef[c, 3] * z
        assert np.allclose(out[:, c], ref, rtol=1e-13, atol=1e-13)


def test_deposit_conserves_charge():
    g = small_grid(6, 8, 4)
    rng = np.random.default_rng(3)
    n = 300
    x, y, z = rng.uniform(0, g.lx, n), rng.uniform(0, g.ly, n), rng.uniform(0, g.lz, n)
    q = rng.standard_normal(n) * 1e-14
    rho = oracle.deposit(g, q, *oracle.locate(g, x, y, z))
    total = np.sum(rho * g.vol_y[None, :, None])
    assert abs(total - q.sum()) <= 1e-12 * np.abs(q).sum()


# ---------------------------------------------------------------- Poisson

def test_poisson_matches_dense_direct_solve():
    """FFT(x,z) + Thomas(y) equals a dense LU solve of the same FV system."""
    g = small_grid(8, 6, 8)
    rng = np.random.default_rng(4)
    rho = rng.standard_normal((g.nz, g.ny, g.nx)) * 1e-6
    phi = oracle.poisson(g, rho, 8.854e-12)
    ref = oracle.dense_poisson(g, rho, 8.854e-12)
    assert np.max(np.abs(phi - ref)) <= 1e-11 * np.max(np.abs(ref))
    res = oracle.fv_apply(g, phi) + rho / 8.854e-12
    assert np.max(np.abs(res)) <= 1e-9 * np.max(np.abs(rho / 8.854e-12))


def test_poisson_manufactured_second_order():
    """phi = sin(2 pi x/Lx) cos(2 pi z/Lz) sin(pi y/Ly): error falls as h^2."""
    eps = 8.854e-12
    errs = []
    for n in (8, 16, 32):
        g = small_grid(n, n, n, gamma=1.5)
        xs = (np.arange(g.nx) + 0.5) * g.dx
        zs = (np.arange(g.nz) + 0.5) * g.dz
        Z, Y, X = np.meshgrid(zs, g.yc, xs, indexing="ij")
        kx, kz, ky = 2 * math.pi / g.lx, 2 * math.pi / g.lz, math.pi / g.ly
        exact = np.sin(kx * X) * np.cos(kz * Z) * np.sin(ky * Y)
        rho = eps * (kx * kx + ky * ky + kz * kz) * exact     # -eps lap(phi)
        phi = oracle.poisson(g, rho, eps)
        errs.append(np.max(np.abs(phi - exact)))
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3, errs


def _image_field(q, src, pts, lx, ly, lz, eps, nlat=(3, 6), nimg=300):
    """E of a point charge between grounded plates y=0, y=ly, periodic x, z.

    Direct Coulomb summation over the method of images (charges +q at
    y0 + 2 n ly, -q at -y0 + 2 n ly) and periodic copies in x and z.
    """
    E = np.zeros((pts.shape[0], 3))
    n = np.arange(-nimg, nimg + 1)
    ys = np.concatenate([src[1] + 2 * n * ly, -src[1] + 2 * n * ly])
    qs = np.concatenate([np.full(n.shape, q), np.full(n.shape, -q)])
    for a in range(-nlat[0], nlat[0] + 1):
        for b in range(-nlat[1], nlat[1] + 1):
            sx, sz = src[0] + a * lx, src[2] + b * lz
            dx = pts[:, 0:1] - sx
            dy = pts[:, 1:2] - ys[None, :]
            dz = pts[:, 2:3] - sz
            r3 = (dx * dx + dy * dy + dz * dz) ** 1.5
            f = qs[None, :] / (4 * math.pi * eps * r3)
            E[:, 0] += np.sum(f * dx, axis=1)
            E[:, 1] += np.sum(f * dy, axis=1)
            E[:, 2] += np.sum(f * dz, axis=1)
    return E


def test_mesh_field_matches_coulomb_image_sum():
    """Deposit -> FV Poisson -> E -> gather converges to the image-sum field."""
    eps = 8.854e-12
    q = 1e-12
    errs = []
    for n in (24, 48):
        f = synth.y_faces(n, 0.02, 1.0)
        g = oracle.Grid(n, n, 0.12, 0.08, f)
        i0, j0, k0 = n // 3, n // 2 - 1, n // 2
        src = np.array([(i0 + 0.5) * g.dx, g.yc[j0], (k0 + 0.5) * g.dz])
        rho = oracle.deposit(g, [q], [i0], [j0], [k0])
        E = oracle.efield(g, oracle.poisson(g, rho, eps))
        pts = np.array([[src[0] + 0.03, 0.012, src[2] + 0.02],
                        [src[0] - 0.025, 0.03, src[2] - 0.015],
                        [src[0] + 0.04, 0.02, src[2]],
                        [src[0], 0.006, src[2] + 0.03]])
        Em = oracle.trilinear(g, E, pts[:, 0] % g.lx, pts[:, 1], pts[:, 2] % g.lz)
        Ex = _image_field(q, src, pts, g.lx, g.ly, g.lz, eps)
        errs.append(np.max(np.linalg.norm(Em - Ex, axis=1) / np.linalg.norm(Ex, axis=1)))
    assert errs[0] < 0.05 and errs[1] < errs[0] / 3.0, errs


def test_efield_closed_forms():
    """Central difference of sin and Gauss-linear gradient of a linear phi."""
    g = small_grid(16, 10, 12)
    xs = (np.arange(g.nx) + 0.5) * g.dx
    th = 2 * math.pi / g.nx
    phi = np.broadcast_to(np.sin(2 * math.pi * xs / g.lx)[None, None, :], (g.nz, g.ny, g.nx)).copy()
    E = oracle.efield(g, phi)
    ref = -np.cos(2 * math.pi * xs / g.lx) * math.sin(th) / g.dx
    assert np.allclose(E[:, 1:-1, :, 0], ref[None, None, :], rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.all(E[:, 0, :, 0] == 0) and np.all(E[:, -1, :, 2] == 0)
    # phi = y - delta: interior faces interpolate exactly, walls are grounded
    phi = np.broadcast_to((g.yc - 0.02)[None, :, None], (g.nz, g.ny, g.nx)).copy()
    E = oracle.efield(g, phi)
    assert np.allclose(E[:, 2:-2, :, 1], -1.0, atol=1e-12)
    assert np.allclose(E[:, 1, :, 1], -(g.yf[1] - 0.02) / g.dy[0], rtol=1e-12)
    assert np.allclose(E[:, 0, :, 1], -(g.yc[0] - 0.02) / (g.dy[0] / 2), rtol=1e-12)
    assert np.allclose(E[:, -1, :, 1], (g.yc[-1] - 0.02) / (g.dy[-1] / 2), rtol=1e-12)


# ---------------------------------------------------------------- forces / integrator

def test_stokes_relaxation_closed_form():
    """Stokes drag F = 3 pi mu d (u - v): v(t) = u + (v0 - u) exp(-t/tau)."""
    p = oracle.Params(drag_law=DRAG_STOKES, rho_p=1200.0)
    d = np.array([50e-6, 111e-6])
    m = p.rho_p * math.pi * d ** 3 / 6
    tau = m / (3 * math.pi * p.rho * p.nu * d)
    u = np.array([[1.3, -0.2, 0.4]] * 2)
    v0 = np.array([[0.1, 0.5, -0.3], [2.0, 0.0, 0.0]])
    x0 = np.zeros((2, 3))
    x, v = x0.copy(), v0.copy()
    dt, nst = 3e-3, 25
    for _ in range(nst):
        x, v, _ = push(p, x, v, u, np.zeros((2, 3)), d, dt)
    t = dt * nst
    e = np.exp(-t / tau)[:, None]
    assert np.allclose(v, u + (v0 - u) * e, rtol=1e-12, atol=1e-14)
    xr = x0 + u * t + (v0 - u) * tau[:, None] * (1 - e)
    assert np.allclose(x, xr, rtol=1e-12, atol=1e-15)


def test_drag_plus_constant_force_terminal_velocity():
    p = oracle.Params(drag_law=DRAG_STOKES)
    d = np.array([80e-6])
    tau = p.rho_p * d ** 2 / (18 * p.rho * p.nu)
    a = np.array([[0.0, -9.81, 2.0]])
    u = np.array([[0.5, 0.0, 0.0]])
    v0 = np.zeros((1, 3))
    x, v = np.zeros((1, 3)), v0.copy()
    dt = 1e-4
    for _ in range(400):
        x, v, _ = push(p, x, v, u, a, d, dt)
    t = 400 * dt
    vt = u + a * tau[:, None]
    e = math.exp(-t / tau[0])
    assert np.allclose(v, vt + (v0 - vt) * e, rtol=1e-12, atol=1e-15)
    assert np.allclose(x, vt * t + (v0 - vt) * tau[0] * (1 - e), rtol=1e-11, atol=1e-16)


def test_ballistic_motion_in_uniform_field():
    """Drag off, f = qE/m with m = rho_p pi d^3 / 6: x = x0 + v0 t + a t^2 / 2."""
    p = oracle.Params(drag_law=DRAG_OFF, rho_p=1150.0)
    d = np.array([50e-6])
    q, E = 3e-13, np.array([100.0, -250.0, 40.0])
    a = (q / (p.rho_p * math.pi * d[0] ** 3 / 6)) * E
    assert np.allclose(a, q * E / oracle.particle_mass(p, d)[0], rtol=1e-15)
    x, v = np.array([[0.01, 0.02, 0.03]]), np.array([[1.0, -0.5, 0.25]])
    x0, v0 = x.copy(), v.copy()
    dt = 1e-5
    for _ in range(100):
        x, v, _ = push(p, x, v, np.zeros((1, 3)), a[None, :], d, dt)
    t = 100 * dt
    assert np.allclose(v, v0 + a * t, rtol=1e-13)
    assert np.allclose(x, x0 + v0 * t + 0.5 * a * t * t, rtol=1e-13)


def test_schiller_naumann_is_continuous_at_re_1000_and_stokes_at_low_re():
    """24/Re (1 + Re^(2/3)/6) at Re = 1000 equals the constant 0.424."""
    p = oracle.Params(drag_law=DRAG_SCHILLER_NAUMANN, rho_p=2400.0)
    d = 1e-3
    sp = np.array([1000.0 * (1 - 1e-9), 1000.0 * (1 + 1e-9)]) * p.nu / d
    t = relaxation_time(p, [d, d], sp)
    assert abs(t[0] / t[1] - 1) < 1e-3
    tau_p = p.rho_p * d ** 2 / (18 * p.rho * p.nu)
    t0 = relaxation_time(p, [d], [1e-12 * p.nu / d])
    assert abs(t0[0] / tau_p - 1) < 1e-6


def test_wrap_periodic():
    L = 0.1
    s = np.array([-1e-18, 0.0, 0.05, 0.1, 0.1 + 1e-3, -0.03])
    w = wrap(s, L)
    assert np.all((w >= 0) & (w < L))
    assert np.allclose(np.mod(w - s + L / 2, L) - L / 2, 0, atol=1e-15)


# ---------------------------------------------------------------- condenser charging

def _hertz_impact(m, R, Estar, v):
    """Integrate m d'' = -(4/3) E* sqrt(R) d^(3/2) from d=0, d'=v (RK4).

    Returns (max compression, contact duration).
    """
    k = 4.0 / 3.0 * Estar * math.sqrt(R)
    t_est = 3.0 * (15 * m * v * v / (16 * Estar * math.sqrt(R))) ** 0.4 / v
    h = t_est / 200000.0

    def f(s):
        d, w = s
        return np.array([w, -k * max(d, 0.0) ** 1.5 / m])

    s, t, dmax = np.array([0.0, v]), 0.0, 0.0
    while True:
        k1 = f(s); k2 = f(s + 0.5 * h * k1); k3 = f(s + 0.5 * h * k2); k4 = f(s + h * k3)
        sn = s + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        dmax = max(dmax, sn[0])
        if sn[0] < 0:
            t += h * s[0] / (s[0] - sn[0])
            return dmax, t
        s, t = sn, t + h


def test_hertz_contact_matches_impact_ode():
    """alpha_iw (k_e = 1) is the Hertz maximum compression, dt_w the contact
    time and A_iw = pi a^2 with the Hertz contact radius a = sqrt(R alpha)."""
    p = oracle.Params(k_e=1.0, rho_p=1150.0)
    d, v = 50e-6, 0.7
    R = d / 2
    m = p.rho_p * math.pi * d ** 3 / 6
    Estar = 1.0 / ((1 - p.mu_p ** 2) / p.E_p + (1 - p.mu_w ** 2) / p.E_w)
    dmax, tc = _hertz_impact(m, R, Estar, v)
    _, _, det = condenser_wall(p, [d], [v], [0.0])
    assert abs(det["alpha"][0] / dmax - 1) < 1e-6
    assert abs(det["dt_w"][0] / tc - 1) < 2e-3          # 2.94 vs 2.9432...
    assert abs(det["A"][0] / (math.pi * R * dmax) - 1) < 1e-6


def test_condenser_charge_is_rc_charging_of_contact_capacitor():
    """dq_c: charge of the parallel-plate capacitor eps A/h at U_c after
    charging through T_w for dt_w (dq/dt = -(q + C U_c)/T_w, q(0) = 0)."""
    p = oracle.Params(U_c=2.5, rho_p=1150.0)
    d, v = 90e-6, 0.3
    dq_c, dq_t, det = condenser_wall(p, [d], [v], [0.0])
    C = p.eps * det["A"][0] / p.h
    T = p.eps_w * p.eps0 * p.phi_p
    assert abs(T - 442.7) < 0.1                               # eps_w eps0 phi_p
    # integrate the RC ODE with RK4 over the contact time
    nst = 50
    h = det["dt_w"][0] / nst
    qv = 0.0
    fq = lambda s: -(s + C * p.U_c) / T
    for _ in range(nst):
        k1 = fq(qv); k2 = fq(qv + h / 2 * k1); k3 = fq(qv + h / 2 * k2); k4 = fq(qv + h * k3)
        qv += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert dq_c[0] < 0 and abs(dq_c[0] / qv - 1) < 1e-9
    assert dq_t[0] == 0.0


def test_condenser_parameter_elasticities():
    """d ln|dq_c| / d ln(parameter) takes the exponents the formulas fix."""
    base = oracle.Params(rho_p=1150.0, U_c=1.0)
    d0, v0 = 50e-6, 0.01

    def dq(p=base, d=d0, v=v0):
        return condenser_wall(p, [d], [v], [0.0])[0][0]

    ref = dq()
    f = 1.001
    lf = math.log(f)
    expect = dict(U_c=1.0, h=-1.0, eps_w=-1.0, phi_p=-1.0, rho_p=0.8,
                  kappa_A=1.0, eps=1.0, eps0=-1.0)
    for name, ex in expect.items():
        got = math.log(dq(p=base.with_(**{name: getattr(base, name) * f})) / ref) / lf
        assert abs(got - ex) < 1e-6, (name, got)
    assert abs(math.log(dq(d=d0 * f) / ref) / lf - 3.0) < 1e-6
    assert abs(math.log(dq(v=v0 * f) / ref) / lf - 0.6) < 1e-6
    # (1 + k_e)^(4/5)
    got = math.log(dq(p=base.with_(k_e=(1 + base.k_e) * f - 1)) / ref) / lf
    assert abs(got - 0.8) < 1e-6
    # a rigid wall leaves the particle's elastic term: E_p^(-4/5)
    rigid = base.with_(E_w=1e30)
    r0 = dq(p=rigid)
    got = math.log(dq(p=rigid.with_(E_p=base.E_p * f)) / r0) / lf
    assert abs(got + 0.8) < 1e-6


def test_precharge_transfer_is_contact_area_fraction():
    """dq_t = -(contact area / sphere area) q with the Hertz contact area."""
    p = oracle.Params(k_e=1.0)
    d, v, q = 60e-6, 0.4, 2e-14
    R = d / 2
    m = p.rho_p * math.pi * d ** 3 / 6
    Estar = 1.0 / ((1 - p.mu_p ** 2) / p.E_p + (1 - p.mu_w ** 2) / p.E_w)
    dmax, _ = _hertz_impact(m, R, Estar, v)
    frac = math.pi * R * dmax / (4 * math.pi * R * R)
    _, dq_t, _ = condenser_wall(p, [d], [v], [q])
    assert abs(dq_t[0] / (-frac * q) - 1) < 1e-6


# ---------------------------------------------------------------- the coupled step

def _uniform_lattice(g, u):
    lat = np.zeros((g.nz, g.ny + 2, g.nx, 3))
    lat[...] = u
    return lat


def test_specular_wall_reflection_and_bookkeeping():
    """Drag off, no field: y' = 2r - (y + vy dt); vx, vz, |v| kept; charge books."""
    g = small_grid(8, 16, 8)
    p = oracle.Params(drag_law=DRAG_OFF, electrostatics=False, U_c=3.0)
    d = np.array([100e-6, 100e-6, 80e-6])
    r = d / 2
    st = oracle.State.from_arrays(
        [0.01, 0.02, 0.03], [r[0] + 1e-6, g.ly - r[1] - 2e-6, 0.02], [0.01, 0.02, 0.03],
        [0.3, -0.1, 0.2], [-0.5, 0.8, 0.1], [0.05, 0.0, -0.2], [0.0, 1e-15, 0.0], d)
    dt = 1e-5
    lat = _uniform_lattice(g, 0.0)
    s1 = oracle.step(g, p, st, lat, dt)
    yfree = st.y + st.vy * dt
    assert abs(s1.y[0] - (2 * r[0] - yfree[0])) < 1e-18
    assert abs(s1.y[1] - (2 * (g.ly - r[1]) - yfree[1])) < 1e-18
    assert s1.y[2] == pytest.approx(yfree[2], abs=1e-18)
    assert np.array_equal(s1.n_imp, [1, 1, 0])
    assert np.allclose(s1.vy, [0.5, -0.8, 0.1]) and np.allclose(s1.vx, st.vx)
    assert np.allclose(s1.vz, st.vz)
    assert np.all(s1.q[:2] != st.q[:2]) and s1.q[2] == 0.0
    assert np.allclose(s1.q - st.q, s1.q_wall, rtol=0, atol=1e-30)
    # impact speed = |v'|; the normal-speed reading uses |v_y'|
    dq, dqt, _ = condenser_wall(p, d[:1], [math.sqrt(0.3 ** 2 + 0.5 ** 2 + 0.05 ** 2)], [0.0])
    assert s1.q[0] == pytest.approx(dq[0] + dqt[0], rel=1e-14)
    s2 = oracle.step(g, p.with_(impact_vel=IMPACT_NORMAL), st, lat, dt)
    dq, _, _ = condenser_wall(p, d[:1], [0.5], [0.0])
    assert s2.q[0] == pytest.approx(dq[0], rel=1e-14)


def _case_state(c, n, rng_seed=5, q_scale=0.0):
    f = synth.y_faces(c.ny, c.delta, c.gamma)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, f)
    P = synth.draw_particles(c, n)
    rng = np.random.default_rng(rng_seed)
    q = rng.standard_normal(n) * q_scale
    st = oracle.State.from_arrays(P.x, P.y, P.z, P.vx, P.vy + rng.standard_normal(n) * 0.3,
                                  P.vz, q, P.d)
    return g, f, st


def test_charge_bookkeeping_and_linearity_in_Uc():
    """Sum q(T) - Sum q(0) = recorded transfers; with no field and dq_t off,
    q(T) is proportional to U_c."""
    c = synth.case("re180_64").with_(nx=16, ny=24, nz=16)
    g, f, st = _case_state(c, 400)
    lat = synth.fluid_lattice(c, faces=f)
    p = oracle.Params(rho_p=c.rho_p, electrostatics=False, dq_t=False, U_c=1.0)
    s1 = oracle.run(g, p, st, lat, c.dt * 20, 15)
    assert s1.n_imp.sum() > 10
    assert np.allclose(s1.q - st.q, s1.q_wall, rtol=0, atol=1e-30)
    s2 = oracle.run(g, p.with_(U_c=7.0), st, lat, c.dt * 20, 15)
    assert np.array_equal(s1.n_imp, s2.n_imp)
    assert np.allclose(s2.q, 7.0 * s1.q, rtol=1e-12, atol=0)


def test_mirror_and_shift_symmetry():
    """Mirroring y (faces, field, particles) mirrors the trajectory; shifting
    by whole cells in x, z shifts it."""
    ny = 20
    half = synth.y_faces(ny, 0.02, 2.0)
    f = half.copy()
    f[ny // 2 + 1:] = 0.04 - half[: ny // 2][::-1]
    g = oracle.Grid(12, 10, 2 * math.pi * 0.02, math.pi * 0.02, f)
    c = synth.case("re180_64").with_(nx=12, ny=ny, nz=10)
    lat = synth.fluid_lattice(c, faces=f)
    _, _, st = _case_state(c, 300, q_scale=1e-13)
    p = oracle.Params(rho_p=c.rho_p, U_c=1e3)
    dt = c.dt * 10
    a = oracle.run(g, p, st, lat, dt, 4)
    mlat = lat[:, ::-1, :, :].copy()
    mlat[..., 1] *= -1
    ms = st.copy()
    ms.y = 0.04 - st.y
    ms.vy = -st.vy
    b = oracle.run(g, p, ms, mlat, dt, 4)
    assert np.allclose(b.y, 0.04 - a.y, rtol=0, atol=1e-15)
    assert np.allclose(b.vy, -a.vy, rtol=1e-9, atol=1e-14)
    assert np.allclose(b.x, a.x, rtol=0, atol=1e-15)
    assert np.allclose(b.q, a.q, rtol=1e-9, atol=1e-30)
    assert np.array_equal(b.n_imp, a.n_imp)
    # whole-cell shift in x and z
    sx, sz = 5, 3
    slat = np.roll(np.roll(lat, sx, axis=2), sz, axis=0)
    ss = st.copy()
    ss.x = wrap(st.x + sx * g.dx, g.lx)
    ss.z = wrap(st.z + sz * g.dz, g.lz)
    s = oracle.run(g, p, ss, slat, dt, 4)
    per = lambda u, v, L: np.abs(np.mod(u - v + L / 2, L) - L / 2)
    assert np.max(per(s.x, a.x + sx * g.dx, g.lx)) < 1e-15
    assert np.max(per(s.z, a.z + sz * g.dz, g.lz)) < 1e-15
    assert np.allclose(s.vx, a.vx, rtol=1e-9, atol=1e-14)
    assert np.allclose(s.q, a.q, rtol=1e-9, atol=1e-30)


# ---------------------------------------------------------------- C_rel statistics (Sec. 4.1)

def test_row_counts_by_brute_force():
    g = small_grid(ny=9)
    rng = np.random.default_rng(19)
    n = 500
    x, z = rng.uniform(0, g.lx, n), rng.uniform(0, g.lz, n)
    y = rng.uniform(g.yf[0], g.yf[-1], n)
    st = oracle.State.from_arrays(x, y, z, np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, 1e-5))
    counts = oracle.particles.ystats(g, st)
    brute = np.zeros(g.ny)
    for yy in y:                       # the row whose faces bracket y (a face belongs to the upper row)
        for j in range(g.ny):
            if g.yf[j] <= yy < g.yf[j + 1] or (j == g.ny - 1 and yy == g.yf[-1]):
                brute[j] += 1
                break
    assert np.array_equal(counts, brute) and counts.sum() == n


def test_relative_concentration_of_a_uniform_suspension_is_one():
    g = small_grid(ny=9)
    # counts in proportion to the rows' volumes: a uniform suspension
    counts = 1000.0 * g.vol_y * g.nx * g.nz / (g.lx * g.ly * g.lz)
    assert np.allclose(oracle.particles.c_rel(g, counts), 1.0, rtol=1e-13)
    # any counts: the volume-weighted mean of C_rel is one
    rng = np.random.default_rng(20)
    counts = rng.integers(0, 50, g.ny).astype(float)
    cr = oracle.particles.c_rel(g, counts)
    assert abs((cr * g.vol_y * g.nx * g.nz).sum() / (g.lx * g.ly * g.lz) - 1.0) < 1e-13
