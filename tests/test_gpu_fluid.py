"""Synthetic time-varying gas field on the GPU (the input of the 128^3
time-varying workload): the mode-sum kernels against the host generator in
synth/ (an inverse 2-D DFT per lattice plane, FP64), and ten coupled steps in
the advected field against the oracle driven by the host generator."""
import math

import numpy as np
import pytest

import oracle
import synth
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


def _mode_inputs(c, faces):
    modes = synth.draw_modes(c)
    Y = synth.node_y(faces)
    return modes, synth.mean_velocity(Y, c), synth.damping(Y, c)


@pytest.mark.parametrize("shape", [(32, 24, 16), (48, 20, 36), (96, 40, 24)])
@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_mode_field_matches_host_generator(shape, prec):
    nx, ny, nz = shape
    c, faces, _, _ = problem(nx=nx, ny=ny, nz=nz, n=0, seed=11)
    modes, ubar, damp = _mode_inputs(c, faces)
    ch = T.Channel(nx, ny, nz, c.lx, c.lz, faces, T.Params(precision=prec))
    ch.set_modes(modes, ubar, damp, 0.0)
    tol = 1e-12 if prec == T.TRIBO_FP64 else 1e-6
    for t in (0.0, 250 * c.dt, 2000 * c.dt):
        ref = synth.fluid_lattice(c, modes, t, faces)              # (nz, ny+2, nx, 3)
        got = ch.eval_modes(t).cpu().numpy().astype(np.float64)    # (3, nz, ny+2, nx)
        got = np.moveaxis(got, 0, -1)
        scale = np.abs(ref).max()
        err = np.abs(got - ref).max() / scale
        assert err <= tol, f"t={t}: max error {err:.3e} of max |u|"
        # fluctuation part alone, against its own size
        fl = ref.copy()
        fl[..., 0] -= ubar[None, :, None]
        gf = got.copy()
        gf[..., 0] -= ubar[None, :, None]
        assert np.abs(gf - fl).max() <= 10 * tol * np.abs(fl).max()
    ch.close()


def test_mode_field_rejects_bad_input():
    c, faces, _, _ = problem(nx=32, ny=16, nz=16, n=0)
    modes, ubar, damp = _mode_inputs(c, faces)
    ch = T.Channel(32, 16, 16, c.lx, c.lz, faces, T.Params(precision=T.TRIBO_MIXED))
    with pytest.raises(T.TriboError):
        ch.eval_modes(0.0)                      # no modes set
    bad = synth.Modes(modes.nxi.copy(), modes.nzi.copy(), modes.kx, modes.ky, modes.kz, modes.amp, modes.phase)
    bad.nxi[0] = 16                             # |nxi| must be < nx/2
    with pytest.raises(T.TriboError):
        ch.set_modes(bad, ubar, damp)
    ch.close()


@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_ten_steps_in_advected_field(prec):
    nx, ny, nz, n = 48, 40, 32, 3000
    c, faces, _, parts = problem(nx=nx, ny=ny, nz=nz, n=n, q_scale=2e-15, vy_scale=0.3, near_wall=0.05,
                                 seed=21, dplus=(0.5, 2.0))
    modes, ubar, damp = _mode_inputs(c, faces)
    dt = 4 * c.dt                               # make the advection visible over ten steps
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    pr = {k: (v if k == "q" else np.asarray(v).astype(real).astype(np.float64)) for k, v in parts.items()}
    g = oracle.Grid(nx, nz, c.lx, c.lz, faces)
    ref = oracle.run(g, oracle_params(c, U_c=50.0), oracle_state(pr),
                     lambda t: synth.fluid_lattice(c, modes, t, faces), dt, 10)
    ch = T.Channel(nx, ny, nz, c.lx, c.lz, faces, T.Params(precision=prec, rho_p=c.rho_p, U_c=50.0),
                   max_particles=n)
    ch.set_modes(modes, ubar, damp, 0.0)
    P = T.Particles.from_numpy(pr, prec, device="cuda", with_cell=True)
    ch.step(P, dt, 10)
    ch.sync()
    out = P.to_numpy()
    ch.close()
    order = np.argsort(out["id"])
    got = {k: np.asarray(v)[order].astype(np.float64) for k, v in out.items()}
    compare_states(g, got, ref, TOL_FP64 if prec == T.TRIBO_FP64 else TOL_MIXED, label="advected field")
    assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)
    assert ref.n_imp.sum() > 0
