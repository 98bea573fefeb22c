"""Momentum source of the particles on the gas (F_s of Eq. ns) on the GPU
against the oracle, through the C ABI (tribo_set_momentum_source).

Per cell, |F_s,gpu - F_s,oracle| <= tol * S_c + 4 u_R E_c (u_R the unit
roundoff of the particle precision):
  S_c = sum_p (m_p / (rho V_c dt)) ((|u| + |v|) phi1 + |a| tau phi2)
is the sum of the magnitudes of the cell's terms (the rounding bound of a sum
whose terms may cancel), and
  E_c = sum_p (m_p / (rho V_c dt)) G U_max phi1
bounds the error of the gathered u: U_max is the largest |u| among the
gather's eight nodes and G = 8 + x/dx + y/dY + z/dz, because the trilinear
weights are formed from absolute coordinates, so each carries an absolute
error of about u_R (x/dx) (and so on) that multiplies the node values, not
the possibly nearly cancelling interpolated u.  Both are averaged over the
steps.  FP64: ten steps (after a three-step call, so the source is
overwritten, not accumulated), tol 1e-12, with and without re-sorting.
Mixed: one step from the same rounded state (the cells are the same by
construction), tol 1e-5 (a few FP32 roundings per factor and float atomics,
about 10 u_32 = 6e-7 of S_c); over ten mixed steps near-face particles may
change cells, so there the sums of V_c F_s over all cells (the total
momentum) are compared, to 1e-4 S + 1e-5 E (ten FP32 steps move a particle
by up to about 1e-5 of the box from the oracle's path).
"""
import numpy as np
import pytest

import oracle
from _problems import TOL_FP64, compare_states, oracle_params, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2602_10761_gb300 as T  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10761_gb300 import build
    build.build()
    T.load()


def _case(real, seed=61, n=4000, shape=(32, 24, 16)):
    c, faces, lat, parts = problem(*shape, n=n, q_scale=2e-13, vy_scale=0.4, near_wall=0.2, seed=seed,
                                   dplus=(0.8, 2.5))
    pr = {k: (v if k == "q" else np.asarray(v).astype(real).astype(np.float64)) for k, v in parts.items()}
    return c, faces, lat.astype(real).astype(np.float64), pr


def _gather_scale(g, lat, st):
    """Per particle and component: U_max (largest |u| among the gather's
    nodes, from a 3x3x3 maximum taken around every node and interpolated)
    times G = 8 + x/dx + y/dY + z/dz."""
    from scipy.ndimage import maximum_filter
    m = np.empty_like(lat)
    for comp in range(3):
        a = np.abs(lat[..., comp])
        m[..., comp] = maximum_filter(a, size=3, mode=("wrap", "nearest", "wrap"))
    umax = oracle.trilinear(g, m, st.x, st.y, st.z)
    jn = np.clip(np.searchsorted(g.Y, st.y, side="right") - 1, 0, g.ny)
    G = 8.0 + st.x / g.dx + st.y / (g.Y[jn + 1] - g.Y[jn]) + st.z / g.dz
    return umax * G[:, None]


def _oracle(c, faces, lat, parts, nsteps, warm=0, **pkw):
    """Oracle state, mean F_s over nsteps (after warm steps) and its bounds (S_c, E_c)."""
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    p = oracle_params(c, U_c=2e3, **pkw)
    st = oracle.State.from_arrays(parts["x"], parts["y"], parts["z"], parts["vx"], parts["vy"], parts["vz"],
                                  parts["q"], parts["d"])
    st = oracle.run(g, p, st, lat, c.dt, warm)
    fs = np.zeros((3, g.nz, g.ny, g.nx))
    bound = np.zeros_like(fs)
    gbound = np.zeros_like(fs)
    for _ in range(nsteps):
        diag = {}
        V = np.stack([st.vx, st.vy, st.vz], axis=1)
        i, j, k = oracle.locate(g, st.x, st.y, st.z)
        key = g.cell_key(i, j, k)
        pre = st
        gs = _gather_scale(g, lat, st)
        st = oracle.step(g, p, st, lat, c.dt, diag=diag)
        fs += diag["F_s"] / nsteps
        s = c.dt / diag["tau"]
        phi1 = -np.expm1(-s)
        w = oracle.particle_mass(p, pre.d) / (p.rho * c.dt)
        for comp in range(3):
            t = w * ((np.abs(diag["uf"][:, comp]) + np.abs(V[:, comp])) * phi1 +
                     np.abs(diag["acc"][:, comp]) * diag["tau"] * (s - phi1))
            b = np.bincount(key, weights=t, minlength=g.ncells).reshape(g.nz, g.ny, g.nx)
            bound[comp] += b / (g.vol_y[None, :, None] * nsteps)
            b = np.bincount(key, weights=w * gs[:, comp] * phi1, minlength=g.ncells).reshape(g.nz, g.ny, g.nx)
            gbound[comp] += b / (g.vol_y[None, :, None] * nsteps)
    return g, st, fs, (bound, gbound)


def _gpu(c, faces, lat, parts, prec, nsteps, warm=0, **pkw):
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=2e3, **pkw)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params,
                   torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda(), max_particles=len(parts["x"]))
    F = ch.momentum_source()
    P = T.Particles.from_numpy(parts, prec, device="cuda")
    if warm:
        ch.step(P, c.dt, warm)
    ch.step(P, c.dt, nsteps)
    ch.sync()
    fs = F.cpu().numpy().astype(np.float64)
    out = P.to_numpy()
    ch.close()
    order = np.argsort(out["id"])
    return {k: np.asarray(v)[order].astype(np.float64) for k, v in out.items()}, fs


def _check(fs, ref, bounds, tol, unit, label):
    assert np.any(ref != 0)
    S, E = bounds
    lim = tol * S + 4.0 * unit * E
    err = np.abs(fs - ref)
    worst = (err / np.where(lim > 0, lim, 1.0)).max()
    assert np.all(err <= lim), f"{label}: worst error / bound {worst}"
    # in most cells the gather term is below the arithmetic one
    assert np.median((4.0 * unit * E / np.where(S > 0, tol * S, 1.0))[S > 0]) < 1.0
    return worst


@pytest.mark.parametrize("sort_every", [0, 3])
def test_momentum_source_fp64_matches_oracle(sort_every):
    c, faces, lat, parts = _case(np.float64)
    g, ref_st, ref, bound = _oracle(c, faces, lat, parts, 10, warm=3)
    got, fs = _gpu(c, faces, lat, parts, T.TRIBO_FP64, 10, warm=3, sort_every=sort_every)
    compare_states(g, got, ref_st, TOL_FP64, label="two-way fp64")
    _check(fs, ref, bound, 1e-12, 2.0 ** -53, f"fp64 sort={sort_every}")


@pytest.mark.parametrize("drag", [T.TRIBO_DRAG_STOKES, T.TRIBO_DRAG_SCHILLER_NAUMANN])
@pytest.mark.parametrize("sort_every", [0, 1])
def test_momentum_source_mixed_one_step(sort_every, drag):
    c, faces, lat, parts = _case(np.float32, seed=62)
    _, _, ref, bound = _oracle(c, faces, lat, parts, 1, drag_law=drag)
    _, fs = _gpu(c, faces, lat, parts, T.TRIBO_MIXED, 1, sort_every=sort_every, drag_law=drag)
    _check(fs, ref, bound, 1e-5, 2.0 ** -24, f"mixed drag={drag} sort={sort_every}")


def test_momentum_source_mixed_ten_steps_total():
    c, faces, lat, parts = _case(np.float32, seed=63)
    g, _, ref, bound = _oracle(c, faces, lat, parts, 10)
    _, fs = _gpu(c, faces, lat, parts, T.TRIBO_MIXED, 10, sort_every=4)
    vol = g.vol_y[None, None, :, None]
    tot, tot_ref = (fs * vol).sum(axis=(1, 2, 3)), (ref * vol).sum(axis=(1, 2, 3))
    # ten FP32 steps move the particles by up to about 1e-5 of the box from the
    # oracle's, which changes the gathered u by up to about 1e-5 G U_max
    tot_bound = (1e-4 * bound[0] * vol).sum(axis=(1, 2, 3)) + (1e-5 * bound[1] * vol).sum(axis=(1, 2, 3))
    assert np.all(np.abs(tot - tot_ref) <= tot_bound), (tot, tot_ref, tot_bound)


def test_momentum_source_is_overwritten_and_switched_off():
    c, faces, lat, parts = _case(np.float64, seed=64, n=500, shape=(16, 12, 8))
    params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(), max_particles=500)
    F = ch.momentum_source()
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    ch.step(P, c.dt, 2)
    ch.sync()
    assert torch.count_nonzero(F).item() > 0
    # drag off: no source; the previous call's values are gone
    ch.set_params(params.with_(drag_law=T.TRIBO_DRAG_OFF))
    ch.step(P, c.dt, 1)
    ch.sync()
    assert torch.count_nonzero(F).item() == 0
    # switched off: the buffer is left alone
    ch.set_params(params)
    F.fill_(7.0)
    ch.momentum_source(False)
    ch.step(P, c.dt, 1)
    ch.sync()
    assert bool((F == 7.0).all())
    # no particles: zero
    F2 = ch.momentum_source()
    F2.fill_(7.0)
    E = T.Particles.from_numpy({k: v[:0] for k, v in parts.items()}, T.TRIBO_FP64)
    ch.step(E, c.dt, 1)
    ch.sync()
    assert torch.count_nonzero(F2).item() == 0
    ch.close()


def test_momentum_source_rejects_misaligned_buffer():
    c, faces, lat, _ = _case(np.float64, seed=65, n=10, shape=(16, 12, 8))
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, T.Params(precision=T.TRIBO_FP64),
                   torch.from_numpy(lat).cuda(), max_particles=10)
    # FP64 planes must be 8-byte aligned: a float32 view one element in is not
    buf = torch.zeros(6 * c.nx * c.ny * c.nz + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(T.TriboError):
        T.tribo_set_momentum_source(ch.ctx, buf[1:])
    ch.close()


def test_momentum_source_of_a_host_pointer_call():
    """A host-pointer call (its last step in chunks, each sent back while the next
    runs) gives the momentum source of the same call on device arrays, up to the
    order of the float atomic sums."""
    c, faces, lat, parts = _case(np.float32, seed=66)
    out = []
    for host in (False, True):
        params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=2e3, sort_every=2)
        ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params,
                       torch.from_numpy(lat.astype(np.float32)).cuda(), max_particles=len(parts["x"]))
        F = ch.momentum_source()
        P = T.Particles.from_numpy(parts, T.TRIBO_MIXED, device=None if host else "cuda")
        ch.step(P, c.dt, 3)
        ch.sync()
        out.append(F.cpu().numpy().astype(np.float64))
        ch.close()
    a, b = out
    assert np.any(a != 0)
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
