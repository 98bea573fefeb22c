"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bar: FP64 mode agrees to 1e-12 relative per particle over 10 steps, mixed
mode to 1e-5; cell indices and impact counts are bit-exact (in mixed mode the
cell of every GPU position is bit-exact, and trajectory cells agree except
for particles within the position tolerance of a face).
"""
import math

import numpy as np
import pytest

import oracle
from _problems import (TOL_FP64, TOL_MIXED, compare_states, oracle_params, oracle_state, problem,
                       round_inputs)

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


def _real(prec):
    return np.float64 if prec == T.TRIBO_FP64 else np.float32


def run_gpu(c, faces, lat, parts, prec, nsteps, dt=None, host=False, **pkw):
    real = _real(prec)
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, **pkw)
    u = torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda()
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, u, max_particles=len(parts["x"]))
    P = T.Particles.from_numpy(parts, prec, device=None if host else "cuda", with_cell=True)
    ch.step(P, dt if dt is not None else c.dt, nsteps)
    ch.sync()
    out = P.to_numpy()
    st = ch.stats(P)
    ch.close()
    order = np.argsort(out["id"])
    got = {k: np.asarray(v)[order].astype(np.float64) if k not in ("n_imp", "id", "cell")
           else np.asarray(v)[order] for k, v in out.items()}
    return got, st


def run_oracle(c, faces, lat, parts, nsteps, dt=None, hist=None, **pkw):
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    st = oracle.run(g, oracle_params(c, **pkw), oracle_state(parts), lat, dt if dt is not None else c.dt,
                    nsteps, hist=hist)
    return g, st


def check_cells(g, got, ref, tol):
    i, j, k = oracle.locate(g, got["x"], got["y"], got["z"])
    own = g.cell_key(i, j, k)
    assert np.array_equal(got["cell"].astype(np.int64), own), "GPU cell != exact locate of GPU position"
    i2, j2, k2 = oracle.locate(g, ref.x, ref.y, ref.z)
    refkey = g.cell_key(i2, j2, k2)
    mism = own != refkey
    if tol <= TOL_FP64:
        assert not mism.any(), f"{mism.sum()} cell mismatches"
    else:
        # a mismatch is allowed only within the position tolerance of a face
        def near(s, faces, L):
            d = np.min(np.abs(s[:, None] - faces[None, :]), axis=1)
            return d <= 4 * tol * L
        nf = near(ref.x, g.xf, g.lx) | near(ref.y, g.yf, g.ly) | near(ref.z, g.zf, g.lz)
        assert not (mism & ~nf).any(), f"{(mism & ~nf).sum()} cell mismatches away from faces"


# ---------------------------------------------------------------- Poisson

@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
@pytest.mark.parametrize("shape", [
    (12, 10, 18), (48, 33, 36),                 # generic path (nz not a compiled length)
    (64, 64, 64), (6, 2, 4), (16, 8, 12), (96, 24, 48), (384, 20, 256), (128, 37, 96), (8, 5, 512),
    (16, 1024, 16), (8, 1023, 8),               # the tallest grids (y-solve shared memory, ragged chunk)
    (8, 3, 8), (16, 11, 8),                     # twisted y solve: one row per half, odd ny ((6, 2, 4): an empty half)
    (384, 64, 256),                             # fields beyond 64 MiB: the fused inverse pipeline
])
def test_poisson_matches_oracle(prec, shape):
    nx, ny, nz = shape
    c, faces, lat, _ = problem(nx, ny, nz, n=0)
    g = oracle.Grid(nx, nz, c.lx, c.lz, faces)
    rng = np.random.default_rng(11)
    rho = rng.standard_normal((nz, ny, nx)) * 1e-6 + 3e-7
    phi_ref = oracle.poisson(g, rho, 8.854e-12)
    E_ref = oracle.efield(g, phi_ref)
    params = T.Params(precision=prec)
    ch = T.Channel(nx, ny, nz, c.lx, c.lz, faces, params, None)
    phi, E = ch.poisson(torch.from_numpy(rho).cuda(), want_phi=True)
    ch.sync()
    phi = phi.cpu().numpy()
    E = E.cpu().numpy().astype(np.float64)
    ch.close()
    tol = 1e-12 if prec == T.TRIBO_FP64 else 2e-6
    assert np.abs(phi - phi_ref).max() <= tol * np.abs(phi_ref).max()
    assert E.shape == (3, nz, ny + 2, nx)
    for comp in range(3):
        ref = E_ref[..., comp]
        err = np.abs(E[comp] - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err <= tol, (comp, err)


# ---------------------------------------------------------------- coupled steps

@pytest.mark.parametrize("sort_every", [0, 4, 5])
@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_ten_steps_match_oracle(prec, sort_every):
    """Re_tau = 180, 64^3, 2,000 particles: charged, near-wall particles
    impacting, Stokes drag, mesh electrostatics every step; particles
    re-sorted by cell every 4 (three sorts) or 5 (two sorts) steps."""
    c, faces, lat, parts = problem(64, 64, 64, n=2000, q_scale=1e-12, vy_scale=0.3, near_wall=0.05)
    real = _real(prec)
    lat_r, parts_r = round_inputs(lat, parts, real)
    tol = TOL_FP64 if prec == T.TRIBO_FP64 else TOL_MIXED
    got, st = run_gpu(c, faces, lat_r, parts_r, prec, 10, U_c=1e3, sort_every=sort_every)
    hist = np.zeros(c.ny)
    g, ref = run_oracle(c, faces, lat_r, parts_r, 10, hist=hist, U_c=1e3)
    assert ref.n_imp.sum() >= 50
    errs = compare_states(g, got, ref, tol, label=f"prec={prec}")
    assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)
    check_cells(g, got, ref, tol)
    assert st["n_impacts"] == ref.n_imp.sum()
    assert np.array_equal(st["hist_y"], hist)
    assert st["n_samples"] == 10
    qs = max(np.abs(ref.q_wall).sum(), 1e-40)
    assert abs(st["sum_wall"] - ref.q_wall.sum()) <= tol * qs
    assert abs(st["sum_q"] - ref.q.sum()) <= tol * np.abs(ref.q).sum()
    print("max relative errors", errs)


@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_sort_into_unaligned_arrays_matches_oracle(prec):
    """The cell sort gathers four particles per thread with 16-byte stores when every
    destination array is 16-byte aligned, else one particle per thread.  Here the caller's x, q
    and n_imp start one element past an aligned address: of the two sorts in ten steps, the
    first writes the context's aligned set (four per thread), the second the caller's arrays
    (one per thread); 2,001 particles leave a ragged tail of one."""
    c, faces, lat, parts = problem(64, 64, 64, n=2001, q_scale=1e-12, vy_scale=0.3, near_wall=0.05)
    real = _real(prec)
    lat_r, parts_r = round_inputs(lat, parts, real)
    tol = TOL_FP64 if prec == T.TRIBO_FP64 else TOL_MIXED
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1e3, sort_every=4)
    u = torch.from_numpy(np.ascontiguousarray(lat_r.astype(real))).cuda()
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, u, max_particles=len(parts_r["x"]))
    P = T.Particles.from_numpy(parts_r, prec, with_cell=True)

    def shifted(t):
        buf = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)
        v = buf[1:]
        v.copy_(t)
        assert v.data_ptr() % 16 != 0
        return v

    P.x, P.q, P.n_imp = shifted(P.x), shifted(P.q), shifted(P.n_imp)
    ch.step(P, c.dt, 10)
    ch.sync()
    out = P.to_numpy()
    ch.close()
    order = np.argsort(out["id"])
    got = {k: np.asarray(v)[order].astype(np.float64) if k not in ("n_imp", "id", "cell")
           else np.asarray(v)[order] for k, v in out.items()}
    g, ref = run_oracle(c, faces, lat_r, parts_r, 10, U_c=1e3)
    assert ref.n_imp.sum() >= 50
    compare_states(g, got, ref, tol, label=f"prec={prec}")
    assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)
    assert np.array_equal(np.sort(got["id"]), np.arange(len(parts_r["x"])))
    check_cells(g, got, ref, tol)


@pytest.mark.parametrize("variant", [
    dict(drag_law=T.TRIBO_DRAG_SCHILLER_NAUMANN),
    dict(drag_law=T.TRIBO_DRAG_OFF),
    dict(impact_vel=T.TRIBO_IMPACT_NORMAL),
    dict(dq_t=0),
    dict(electrostatics=0),
])
def test_model_switches_fp64(variant):
    c, faces, lat, parts = problem(24, 30, 18, n=777, q_scale=2e-12, vy_scale=0.4, near_wall=0.1, seed=3,
                                   dplus=(0.5, 2.5))
    okw = dict(variant)
    okw["electrostatics"] = bool(okw.get("electrostatics", 1))
    if "dq_t" in okw:
        okw["dq_t"] = bool(okw["dq_t"])
    # particles heavy enough to reach Re_p > 1000 somewhere in the SN case
    got, _ = run_gpu(c, faces, lat, parts, T.TRIBO_FP64, 6, U_c=50.0, **variant)
    g, ref = run_oracle(c, faces, lat, parts, 6, U_c=50.0, **okw)
    compare_states(g, got, ref, TOL_FP64, label=str(variant))
    assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)
    check_cells(g, got, ref, TOL_FP64)


def test_schiller_naumann_high_reynolds_branch():
    """Large particles with a large slip exercise the C_D = 0.424 branch."""
    c, faces, lat, parts = problem(16, 20, 12, n=300, seed=5, dplus=(20.0, 40.0), density_ratio=2000.0)
    parts["vx"] = parts["vx"] + np.random.default_rng(5).uniform(0.0, 12.0, 300)
    p = oracle_params(c, drag_law=1)
    re = np.abs(parts["vx"]) * parts["d"] / p.nu
    assert (re > 1000).any() and (re < 1000).any()
    got, _ = run_gpu(c, faces, lat, parts, T.TRIBO_FP64, 3, drag_law=T.TRIBO_DRAG_SCHILLER_NAUMANN)
    g, ref = run_oracle(c, faces, lat, parts, 3, drag_law=1)
    compare_states(g, got, ref, TOL_FP64, label="SN high Re")


@pytest.mark.parametrize("prec", [T.TRIBO_MIXED, T.TRIBO_FP64])
def test_host_pointer_call_matches_device_call(prec):
    c, faces, lat, parts = problem(32, 24, 16, n=1500, q_scale=1e-12, vy_scale=0.3, near_wall=0.05, seed=9)
    lat_r, parts_r = round_inputs(lat, parts, _real(prec))
    a, sa = run_gpu(c, faces, lat_r, parts_r, prec, 5, U_c=1e3, sort_every=2)
    b, sb = run_gpu(c, faces, lat_r, parts_r, prec, 5, U_c=1e3, host=True, sort_every=2)
    rtol = 1e-6 if prec == T.TRIBO_MIXED else 1e-12
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.allclose(a[k], b[k], rtol=rtol, atol=rtol * np.abs(a[k]).max()), k
    assert np.array_equal(a["n_imp"], b["n_imp"])
    assert np.array_equal(a["cell"], b["cell"])
    assert sa["n_impacts"] == sb["n_impacts"]


@pytest.mark.parametrize("ssm", [False, True])
def test_host_pointer_single_steps_match_device_call(ssm):
    """Seven one-step host-pointer calls (the arrays the solve does not need
    copied beside it, the ids only in the calls that sort or when the SSM reads
    them) against one seven-step device call: the same FP64 oracle path, so
    the states agree to FP32 rounding (the call-start deposit sums in another
    order) and the impact counts and ids exactly."""
    c, faces, lat, parts = problem(32, 24, 16, n=2000, q_scale=1e-13, vy_scale=0.4, near_wall=0.2, seed=23)
    lat_r, parts_r = round_inputs(lat, parts, np.float32)
    params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1e3, sort_every=3)
    out = []
    for host in (False, True):
        ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat_r.astype(np.float32)).cuda(),
                       max_particles=2000)
        if ssm:
            ch.set_ssm(T.SSMParams(seed=3))
        P = T.Particles.from_numpy(parts_r, T.TRIBO_MIXED, device=None if host else "cuda")
        if host:
            for _ in range(7):
                ch.step(P, c.dt, 1)
        else:
            ch.step(P, c.dt, 7)
        ch.sync()
        o = P.to_numpy()
        ch.close()
        order = np.argsort(o["id"])
        out.append({k: np.asarray(v)[order] for k, v in o.items()})
    a, b = out
    assert np.array_equal(np.sort(b["id"]), np.arange(2000))
    for k in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall"):
        s = max(np.abs(a[k]).max(), 1e-30)
        assert np.abs(a[k].astype(np.float64) - b[k].astype(np.float64)).max() <= 1e-5 * s, k
    assert np.array_equal(a["n_imp"], b["n_imp"])
    assert a["n_imp"].sum() > 50


@pytest.mark.parametrize("n", [0, 1, 33, 257])
def test_small_and_ragged_ensembles(n):
    c, faces, lat, parts = problem(12, 8, 6, n=n, q_scale=1e-12, vy_scale=0.3, near_wall=0.3, seed=n + 1)
    got, st = run_gpu(c, faces, lat, parts, T.TRIBO_FP64, 4, U_c=10.0, sort_every=1)
    g, ref = run_oracle(c, faces, lat, parts, 4, U_c=10.0)
    if n:
        compare_states(g, got, ref, TOL_FP64, label=f"n={n}")
        assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)
    assert st["n_impacts"] == ref.n_imp.sum()


def test_device_error_word_reports_particles_outside():
    c, faces, lat, parts = problem(12, 8, 6, n=64, seed=2)
    parts["y"][5] = -1.0
    params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda())
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    ch.step(P, c.dt, 1)
    with pytest.raises(T.TriboError):
        ch.sync()
    assert ch.error_bits & T.TRIBO_DEV_OUTSIDE
    T.tribo_clear_error(ch.ctx)
    ch.sync()
    ch.close()
