"""Long-run statistics against the oracle: the wall-normal concentration
profile (the per-row histogram of particle cells accumulated every step, the
C_rel(y) of Sec. 4.1) and the early-time charging rate (the slope of <q>_rel
over t+, Sec. 4) after 300 coupled steps on the Re_tau 180 64^3 grid, 4000
particles with random wall-normal velocities (so that several hundred impacts
charge them), condenser charging, mesh electrostatics every step.  Both must
agree within 1%: per bin for the profile (bins holding at least half the
mean count) and for the fitted slope.  The FP64 path is expected to agree far
closer (the same impacts, the same bins); the mixed path within the bound.
Inputs are FP32-rounded for both precisions, so one oracle run serves both."""
import numpy as np
import pytest

import oracle
from _problems import oracle_params, oracle_state, problem, round_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2602_10761_gb300 as T  # noqa: E402
from paper_2602_10761_gb300 import correlation as cor  # noqa: E402

STEPS, EVERY = 300, 20


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10761_gb300 import build
    build.build()
    T.load()


@pytest.fixture(scope="module")
def case():
    c, faces, lat, parts = problem(64, 64, 64, n=4000, q_scale=0.0, vy_scale=0.4, seed=41)
    lat, parts = round_inputs(lat, parts, np.float32)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    p = oracle_params(c, U_c=2e3)
    st = oracle_state(parts)
    hist = np.zeros(c.ny)
    q = [st.q.mean() / cor.Q_SAT]
    for _ in range(STEPS // EVERY):
        st = oracle.run(g, p, st, lat, c.dt, EVERY, hist=hist)
        q.append(st.q.mean() / cor.Q_SAT)
    tp = cor.t_plus(np.arange(len(q)) * EVERY * c.dt, c.u_tau, c.nu)
    return c, faces, lat, parts, dict(hist=hist, slope=cor.fit_rate(tp, q), impacts=int(st.n_imp.sum()))


@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_long_run_profile_and_charging_rate(case, prec):
    c, faces, lat, parts, ref = case
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=2e3, sort_every=20)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat.astype(real)).cuda(),
                   max_particles=len(parts["x"]))
    P = T.Particles.from_numpy(parts, prec)
    tp, qrel = cor.charging_history(ch, P, c.dt, STEPS, EVERY, c.u_tau, c.nu)
    st = ch.stats(P)
    ch.close()
    assert ref["impacts"] > 300 and ref["slope"] != 0        # (negative: the condenser charge at this U_c)
    assert abs(st["n_impacts"] - ref["impacts"]) <= 0.01 * ref["impacts"]
    slope = cor.fit_rate(tp, qrel)
    assert abs(slope - ref["slope"]) <= 0.01 * abs(ref["slope"]), (slope, ref["slope"])
    C, Cref = st["hist_y"] / st["hist_y"].sum(), ref["hist"] / ref["hist"].sum()
    full = Cref >= 0.5 / c.ny
    assert full.sum() >= c.ny // 2
    assert np.all(np.abs(C - Cref)[full] <= 0.01 * Cref[full])
    if prec == T.TRIBO_FP64:
        assert np.array_equal(st["hist_y"], ref["hist"])
        assert st["n_impacts"] == ref["impacts"]
        assert abs(slope - ref["slope"]) <= 1e-9 * abs(ref["slope"])
