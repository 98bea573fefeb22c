"""Failure detection without a GPU fault: bad input injected from the host
sets the device error word, and a bounded wait of the pipelined inverse
transform that is made to run out (a producer task that never comes) ends with
TRIBO_DEV_TIMEOUT instead of a hang; in every case the context stays usable."""
import numpy as np
import pytest

import oracle
from _problems import problem

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


def _channel(c, faces, lat, prec, n):
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f)
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    return T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params,
                     torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda(), max_particles=n)


@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_nonfinite_state_is_reported(prec):
    c, faces, lat, parts = problem(12, 8, 6, n=64, seed=5)
    parts["vx"][7] = np.nan
    ch = _channel(c, faces, lat, prec, 64)
    P = T.Particles.from_numpy(parts, prec)
    ch.step(P, c.dt, 1)
    with pytest.raises(T.TriboError):
        ch.sync()
    assert ch.error_bits & T.TRIBO_DEV_NONFINITE
    T.tribo_clear_error(ch.ctx)
    ch.sync()
    ch.close()


def test_particle_still_outside_after_its_reflection_is_reported():
    c, faces, lat, parts = problem(12, 8, 6, n=64, seed=6)
    # three channel heights in one step: mirrored once about the upper contact plane it is still
    # far below the lower wall
    parts["vy"][3] = 3.0 * c.ly / c.dt
    ch = _channel(c, faces, lat, T.TRIBO_FP64, 64)
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    ch.step(P, c.dt, 1)
    with pytest.raises(T.TriboError):
        ch.sync()
    assert ch.error_bits & T.TRIBO_DEV_ESCAPED
    T.tribo_clear_error(ch.ctx)
    ch.sync()
    ch.close()


def test_pipeline_wait_runs_out_and_the_context_recovers():
    # a grid whose fields exceed 64 MiB runs the inverse transforms as the pipelined launch
    nx, ny, nz = 384, 64, 256
    c, faces, lat, _ = problem(nx, ny, nz, n=0)
    rng = np.random.default_rng(21)
    rho = rng.standard_normal((nz, ny, nx)) * 1e-6
    ch = T.Channel(nx, ny, nz, c.lx, c.lz, faces, T.Params(precision=T.TRIBO_MIXED), None)
    T.tribo_test_pipeline_wait(ch.ctx, 5)
    ch.poisson(torch.from_numpy(rho).cuda(), want_phi=True)
    with pytest.raises(T.TriboError):
        ch.sync()
    assert ch.error_bits & T.TRIBO_DEV_TIMEOUT
    T.tribo_clear_error(ch.ctx)
    T.tribo_test_pipeline_wait(ch.ctx, -1)
    phi, E = ch.poisson(torch.from_numpy(rho).cuda(), want_phi=True)
    ch.sync()
    assert ch.error_bits == 0
    g = oracle.Grid(nx, nz, c.lx, c.lz, faces)
    phi_ref = oracle.poisson(g, rho, 8.854e-12)
    E_ref = oracle.efield(g, phi_ref)
    E = E.cpu().numpy().astype(np.float64)
    for comp in range(3):
        ref = E_ref[..., comp]
        assert np.abs(E[comp] - ref).max() <= 2e-6 * np.abs(ref).max(), comp
    ch.close()
