"""In-cell Coulomb near field of the hybrid electrostatics (Sec. 2.2) on the
GPU against the oracle: clustered particles (about ten per cell), charged,
with mesh electrostatics, ten steps; FP64 to 1e-12 and mixed to 1e-5 per
particle, impact counts exact; with and without re-sorting."""
import numpy as np
import pytest

import oracle
from _problems import TOL_FP64, TOL_MIXED, compare_states, oracle_params, oracle_state, problem

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


def _case(n=2000, seed=31):
    return problem(8, 6, 4, n=n, q_scale=1.5e-12, vy_scale=0.2, near_wall=0.05, seed=seed, dplus=(0.8, 2.0))


def _gpu(c, faces, lat, parts, prec, nsteps, **pkw):
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, **pkw)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params,
                   torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda(), max_particles=len(parts["x"]))
    P = T.Particles.from_numpy(parts, prec, device="cuda")
    ch.step(P, c.dt, nsteps)
    ch.sync()
    out = P.to_numpy()
    ch.close()
    order = np.argsort(out["id"])
    return {k: np.asarray(v)[order].astype(np.float64) for k, v in out.items()}


@pytest.mark.parametrize("sort_every", [0, 3])
@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_near_field_matches_oracle(prec, sort_every):
    c, faces, lat, parts = _case()
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    pr = {k: (v if k == "q" else np.asarray(v).astype(real).astype(np.float64)) for k, v in parts.items()}
    lat_r = lat.astype(real).astype(np.float64)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    ref = oracle.run(g, oracle_params(c, U_c=100.0, coulomb=True), oracle_state(pr), lat_r, c.dt, 10)
    off = oracle.run(g, oracle_params(c, U_c=100.0), oracle_state(pr), lat_r, c.dt, 10)
    # the near field moves the particles well beyond the tolerance
    assert np.abs(ref.vx - off.vx).max() > 1e3 * TOL_MIXED * np.abs(ref.vx).max()
    got = _gpu(c, faces, lat_r, pr, prec, 10, U_c=100.0, coulomb=1, sort_every=sort_every)
    tol = TOL_FP64 if prec == T.TRIBO_FP64 else TOL_MIXED
    compare_states(g, got, ref, tol, label=f"near field prec={prec}")
    assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)


def test_near_field_rejections():
    c, faces, lat, parts = _case(n=50)
    params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p, coulomb=1)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(), max_particles=40)
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    with pytest.raises(T.TriboError):
        ch.step(P, c.dt, 1)                       # more particles than max_particles
    ch.close()
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(), max_particles=50)
    with pytest.raises(T.TriboError):
        T.tribo_adjoint(ch.ctx, P, c.dt, 2, 1)
    with pytest.raises(T.TriboError):
        T.Batch([ch])
    ch.close()
