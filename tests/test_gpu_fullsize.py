"""Full-size parity at Re_tau = 550: 384 x 256 x 256 cells, 8M particles,
mixed precision, particles re-sorted by cell every 20 steps (the benchmark's
launch configuration).  The oracle cannot run 8M particles, so it replays a
1-in-1000 subsample for one step from the GPU state 20 steps in, in the field
of all particles (deposit of the full ensemble, FP64 Poisson solve on the
full grid), and the full-grid field is compared as well.  Charges are
Gaussian (sigma = 0.01 q_sat) so that the field force is exercised, and half
of the subsample moves into a wall in the replayed step (synth.replay_state),
so that the impact charge is compared at full size too.  Tolerances follow
the per-particle reading of the parity bar (compare_states)."""
import numpy as np
import pytest

import oracle
import synth
from _problems import TOL_MIXED, compare_states, oracle_params

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


def _snapshot(P):
    out = P.to_numpy()
    order = np.argsort(out["id"])
    return {k: np.asarray(v)[order] for k, v in out.items()}


def test_full_size_sampled_one_step_replay():
    c = synth.case("re550_384")
    n = c.n_particles
    faces = synth.y_faces(c.ny, c.delta, c.gamma)
    lat32 = synth.fluid_lattice(c, faces=faces).astype(np.float32)
    P = synth.draw_particles(c)
    q0 = np.random.default_rng(550).standard_normal(n) * 0.01 * synth.Q_SAT
    parts = dict(x=P.x, y=P.y, z=P.z, vx=P.vx, vy=P.vy, vz=P.vz, d=P.d, q=q0)
    del P
    params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0, sort_every=20)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat32).cuda(),
                   max_particles=n)
    Pd = T.Particles.from_numpy(parts, T.TRIBO_MIXED, device="cuda", with_cell=True)
    del parts
    ch.step(Pd, c.dt, 20)                 # sorted at step 0
    s20 = _snapshot(Pd)
    del Pd
    # the state 20 steps in, with half of the 1-in-1000 subsample moving into a wall
    s0 = synth.replay_state(c, {k: s20[k] for k in ("x", "y", "z", "vx", "vy", "vz", "d")})
    del s20
    Pd = T.Particles.from_numpy(s0, T.TRIBO_MIXED, device="cuda", with_cell=True)
    ch.step(Pd, c.dt, 1)                  # sorted again before this step
    ch.sync()
    s1 = _snapshot(Pd)
    del Pd

    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    f64 = lambda a: np.asarray(a, np.float64)
    # field of the full ensemble at state n, FP64
    i, j, k = oracle.locate(g, f64(s0["x"]), f64(s0["y"]), f64(s0["z"]))
    rho = oracle.deposit(g, s0["q"], i, j, k)
    E_ref = oracle.efield(g, oracle.poisson(g, rho, params.eps))
    # the library's field from the same density
    _, E = ch.poisson(torch.from_numpy(rho).cuda())
    E = E.cpu().numpy()
    for comp in range(3):
        ref = E_ref[..., comp]
        err = np.abs(E[comp].astype(np.float64) - ref).max() / np.abs(ref).max()
        assert err <= 2e-6, (comp, err)
    del E, rho

    sel = np.arange(0, n, 1000)
    st = oracle.State.from_arrays(*(f64(s0[key][sel]) for key in ("x", "y", "z", "vx", "vy", "vz")),
                                  s0["q"][sel], f64(s0["d"][sel]))
    ref = oracle.step(g, oracle_params(c, U_c=1.0), st, lat32.astype(np.float64), c.dt, E_lat=E_ref)
    del E_ref
    # the near-wall half of the subsample impacts in this step, so the charge path is compared
    assert ref.n_imp.sum() >= 3000, ref.n_imp.sum()
    got = {key: f64(s1[key][sel]) for key in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall")}
    errs = compare_states(g, got, ref, TOL_MIXED, label="full size, one step")
    assert errs["q_wall"] > 0.0 or ref.n_imp.sum() == 0
    # impact counts bit-exact; the cell of every GPU position is exact
    assert np.array_equal(s1["n_imp"][sel].astype(np.int64), ref.n_imp)
    ii, jj, kk = oracle.locate(g, got["x"], got["y"], got["z"])
    assert np.array_equal(s1["cell"][sel].astype(np.int64), g.cell_key(ii, jj, kk))
    # ids survive the two sorts as a permutation
    assert np.array_equal(s1["id"], np.arange(n, dtype=np.uint32))
    ch.close()
