"""4-way coupling on the GPU against the oracle: clustered large particles
(d+ 10-20, about fifteen per cell) collide with one another (about a hundred
pairs in ten steps) and exchange charge in each contact; FP64 to 1e-12 per
particle, impact counts exact, with and without re-sorting and together with
the Coulomb near field.

Mixed precision: the collision normal is the direction between two centres
about d_min = 1.1 mm apart, while FP32 positions in a channel of height
L_y = 40 mm carry a rounding of eps_32 L_y; each collision's velocity change
therefore carries a relative error up to eps_32 L_y / d_min = 2.2e-6, and a
particle colliding a few times in ten steps accumulates ~1e-5.  The bar for
this coupling in mixed precision is 5e-5 (the FP64 runs check the arithmetic
at 1e-12)."""
import numpy as np
import pytest

import oracle
from _problems import TOL_FP64, compare_states, oracle_params, oracle_state, problem

TOL_COLL_MIXED = 5e-5

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


def _case(n=3000, seed=41):
    return problem(8, 6, 4, n=n, q_scale=2e-14, vy_scale=0.3, near_wall=0.02, seed=seed, dplus=(10.0, 20.0))


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


@pytest.mark.parametrize("variant", [dict(sort_every=0), dict(sort_every=3), dict(sort_every=0, coulomb=1),
                                     dict(sort_every=3, coulomb=1)])
@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_collisions_match_oracle(prec, variant):
    c, faces, lat, parts = _case()
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    pr = {k: (v if k == "q" else np.asarray(v).astype(real).astype(np.float64)) for k, v in parts.items()}
    lat_r = lat.astype(real).astype(np.float64)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    okw = dict(U_c=100.0, collisions=True, coulomb=bool(variant.get("coulomb", 0)))
    p = oracle_params(c, **okw)
    st, npairs = oracle_state(pr), 0
    for _ in range(10):
        diag = {}
        st = oracle.step(g, p, st, lat_r, c.dt, diag=diag)
        npairs += len(diag.get("pairs", []))
    assert npairs > 50
    got = _gpu(c, faces, lat_r, pr, prec, 10, U_c=100.0, collisions=1, **variant)
    tol = TOL_FP64 if prec == T.TRIBO_FP64 else TOL_COLL_MIXED
    compare_states(g, got, st, tol, label=f"collisions prec={prec} {variant}")
    assert np.array_equal(got["n_imp"].astype(np.int64), st.n_imp)
    # particle-particle exchanges conserve the total charge up to the wall transfers
    assert abs(got["q"].sum() - pr["q"].sum() - got["q_wall"].sum()) <= 1e-12 * np.abs(pr["q"]).sum()


def test_collisions_rejected_where_not_available():
    c, faces, lat, parts = _case(n=50)
    params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p, collisions=1)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(), max_particles=50)
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    with pytest.raises(T.TriboError):
        T.tribo_adjoint(ch.ctx, P, c.dt, 2, 1)
    with pytest.raises(T.TriboError):
        T.Batch([ch])
    ch.close()
