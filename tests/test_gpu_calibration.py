"""Holding a simulation against the charging-rate correlation (Sec. 4): the
charge history sampled through tribo_stats against the oracle, and the Newton
calibration of U_c and kappa_A driven by the GPU adjoint, which must recover
the values that produced a target mean charge."""
import numpy as np
import pytest

import oracle
from _problems import oracle_params, oracle_state, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2602_10761_gb300 as T  # noqa: E402
from paper_2602_10761_gb300 import correlation as cor  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10761_gb300 import build
    build.build()
    T.load()


def _case(seed=81, q_scale=2e-14):
    return problem(16, 12, 8, n=200, q_scale=q_scale, vy_scale=0.4, near_wall=0.3, seed=seed, dplus=(0.8, 2.5))


def _channel(c, faces, lat, **kw):
    params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, **kw)
    return T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(), max_particles=200)


def test_charging_history_matches_oracle():
    c, faces, lat, parts = _case()
    ch = _channel(c, faces, lat, U_c=2e3)
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    tp, qrel = cor.charging_history(ch, P, c.dt, 9, 3, c.u_tau, c.nu)
    ch.close()
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    p = oracle_params(c, U_c=2e3)
    st = oracle_state(parts)
    ref = [st.q.mean() / cor.Q_SAT]
    for _ in range(3):
        st = oracle.run(g, p, st, lat, c.dt, 3)
        ref.append(st.q.mean() / cor.Q_SAT)
    assert np.allclose(tp, np.arange(4) * 3 * c.dt * c.u_tau ** 2 / c.nu, rtol=1e-14)
    scale = np.abs(ref).max()
    assert np.all(np.abs(qrel - np.array(ref)) <= 1e-12 * scale)
    assert st.n_imp.sum() > 10


@pytest.mark.parametrize("param,true,start", [("U_c", 2e3, 300.0), ("kappa_A", 1.7, 1.0)])
def test_adjoint_newton_calibration_recovers_the_parameter(param, true, start):
    # uncharged particles: the mean charge is what the impacts transfer
    c, faces, lat, parts = _case(seed=82, q_scale=0.0)
    dt, nsteps = 2 * c.dt, 7
    ch = _channel(c, faces, lat, U_c=2e3, kappa_A=1.0)
    ch.set_params(ch.params.with_(**{param: true}))
    J_true, _, _, _ = ch.adjoint(T.Particles.from_numpy(parts, T.TRIBO_FP64), dt, nsteps, 3, want_dd=False)
    ch.set_params(ch.params.with_(**{param: start}))
    theta, hist = cor.calibrate(ch, lambda: T.Particles.from_numpy(parts, T.TRIBO_FP64), dt, nsteps, J_true,
                                param=param, iters=8, rtol=1e-12, ckpt_every=3)
    ch.close()
    assert abs(theta / true - 1) < 1e-9, hist
    assert len(hist) <= 5, hist
