"""Parity of tribo_adjoint (reverse mode on the GPU, through the C ABI) with
the oracle's gradient of the mean charge (autograd of the FP64 restatement
of the oracle step, pinned in test_oracle_adjoint.py).

FP64 mode: J to 1e-12, dJ/dU_c and dJ/dkappa_A to 1e-9, dJ/dd_p to 1e-9 of
the largest |dJ/dd_p|.  Mixed mode (FP32 particle state and adjoints, FP64
charge adjoints): 1e-4 for J, the parameter gradients and dJ/dd_p.
"""
import numpy as np
import pytest

import oracle
import synth
from _problems import oracle_params, oracle_state, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2602_10761_gb300 as T  # noqa: E402
from oracle.adjoint import mean_charge_gradient  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10761_gb300 import build
    build.build()
    T.load()


def _case(seed=4, n=150, shape=(16, 12, 8)):
    c, faces, lat, parts = problem(*shape, n=n, q_scale=2e-13, vy_scale=0.4, near_wall=0.3, seed=seed,
                                   dplus=(0.8, 2.5))
    return c, faces, lat, parts


def _round(parts, lat, prec):
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    pr = {k: (v if k == "q" else np.asarray(v).astype(real).astype(np.float64)) for k, v in parts.items()}
    return pr, lat.astype(real).astype(np.float64)


def gpu_adjoint(c, faces, lat, parts, prec, dt, nsteps, ckpt, modes=None, **pkw):
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, **pkw)
    u = torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda()
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, u, max_particles=len(parts["x"]))
    if modes is not None:
        m, ub, dm = modes
        ch.set_modes(m, ub, dm, 0.0)
    P = T.Particles.from_numpy(parts, prec, device="cuda")
    J, dU, dK, dd = ch.adjoint(P, dt, nsteps, ckpt)
    out = P.to_numpy()
    ch.close()
    return dict(J=J, dU_c=dU, dkappa_A=dK, dd=dd.cpu().numpy(), final=out)


def check(got, ref, tol, label):
    assert abs(got["J"] - ref["J"]) <= tol * max(abs(ref["J"]), 1e-40), (label, got["J"], ref["J"])
    for k in ("dU_c", "dkappa_A"):
        assert abs(got[k] - ref[k]) <= tol * abs(ref[k]), (label, k, got[k], ref[k])
    s = np.abs(ref["dd"]).max()
    err = np.abs(got["dd"] - ref["dd"]).max() / s
    assert err <= tol, (label, "dd", err)


VARIANTS = [
    dict(),
    dict(drag_law=T.TRIBO_DRAG_SCHILLER_NAUMANN),
    dict(drag_law=T.TRIBO_DRAG_OFF),
    dict(impact_vel=T.TRIBO_IMPACT_NORMAL),
    dict(dq_t=0),
    dict(electrostatics=0),
]


def _okw(v):
    o = dict(v)
    if "electrostatics" in o:
        o["electrostatics"] = bool(o["electrostatics"])
    if "dq_t" in o:
        o["dq_t"] = bool(o["dq_t"])
    return o


@pytest.mark.parametrize("variant", VARIANTS)
def test_adjoint_fp64_matches_oracle_gradient(variant):
    c, faces, lat, parts = _case(seed=5)
    dt, nsteps = 2 * c.dt, 7
    ref = mean_charge_gradient(oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces),
                               oracle_params(c, U_c=2e3, **_okw(variant)), oracle_state(parts), lat, dt, nsteps)
    assert ref["final"]["n_imp"].sum() > 10
    got = gpu_adjoint(c, faces, lat, parts, T.TRIBO_FP64, dt, nsteps, 3, U_c=2e3, **variant)
    assert np.array_equal(got["final"]["n_imp"].astype(np.int64), ref["final"]["n_imp"])
    check(got, ref, 1e-9, str(variant))


@pytest.mark.parametrize("ckpt", [1, 2, 7, 50])
def test_adjoint_independent_of_checkpoint_interval(ckpt):
    c, faces, lat, parts = _case(seed=6, shape=(24, 16, 12))
    dt, nsteps = 2 * c.dt, 7
    ref = mean_charge_gradient(oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces), oracle_params(c, U_c=2e3),
                               oracle_state(parts), lat, dt, nsteps)
    got = gpu_adjoint(c, faces, lat, parts, T.TRIBO_FP64, dt, nsteps, ckpt, U_c=2e3)
    check(got, ref, 1e-9, f"ckpt={ckpt}")


def test_adjoint_mixed_precision():
    c, faces, lat, parts = _case(seed=7, n=400, shape=(32, 24, 16))
    pr, lat_r = _round(parts, lat, T.TRIBO_MIXED)
    dt, nsteps = 2 * c.dt, 8
    ref = mean_charge_gradient(oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces), oracle_params(c, U_c=2e3),
                               oracle_state(pr), lat_r, dt, nsteps)
    got = gpu_adjoint(c, faces, lat_r, pr, T.TRIBO_MIXED, dt, nsteps, 3, U_c=2e3)
    assert np.array_equal(got["final"]["n_imp"].astype(np.int64), ref["final"]["n_imp"])
    check(got, ref, 1e-4, "mixed")


def test_adjoint_in_advected_field():
    c, faces, _, parts = _case(seed=8, shape=(24, 16, 12))
    modes = synth.draw_modes(c)
    Y = synth.node_y(faces)
    ub, dm = synth.mean_velocity(Y, c), synth.damping(Y, c)
    dt, nsteps = 4 * c.dt, 6
    lat_t = lambda t: synth.fluid_lattice(c, modes, t, faces)
    ref = mean_charge_gradient(oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces), oracle_params(c, U_c=2e3),
                               oracle_state(parts), lat_t, dt, nsteps)
    got = gpu_adjoint(c, faces, lat_t(0.0), parts, T.TRIBO_FP64, dt, nsteps, 4, modes=(modes, ub, dm), U_c=2e3)
    check(got, ref, 1e-9, "advected field")


def test_adjoint_forward_state_equals_step():
    c, faces, lat, parts = _case(seed=9, n=300, shape=(24, 16, 12))
    dt, nsteps = 2 * c.dt, 9
    got = gpu_adjoint(c, faces, lat, parts, T.TRIBO_FP64, dt, nsteps, 4, U_c=2e3)
    params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=2e3)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(), max_particles=300)
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    ch.step(P, dt, nsteps)
    ref = P.to_numpy()
    st = ch.stats(P)
    ch.close()
    for k in ("x", "y", "z", "vx", "vy", "vz", "q"):
        s = max(np.abs(ref[k]).max(), 1e-40)
        assert np.abs(got["final"][k] - ref[k]).max() <= 1e-13 * s, k
    assert np.array_equal(got["final"]["n_imp"], ref["n_imp"])
    assert abs(got["J"] - st["sum_q"] / 300) <= 1e-13 * np.abs(ref["q"]).max()


def test_adjoint_rejects_host_arrays():
    c, faces, lat, parts = _case(seed=2, n=10)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, T.Params(precision=T.TRIBO_FP64),
                   torch.from_numpy(lat).cuda(), max_particles=10)
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64, device=None)
    with pytest.raises(T.TriboError):
        T.tribo_adjoint(ch.ctx, P, c.dt, 2, 1)
    ch.close()


def test_autograd_function_matches_oracle_gradient():
    c, faces, lat, parts = _case(seed=12)
    dt, nsteps = 2 * c.dt, 6
    ref = mean_charge_gradient(oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces), oracle_params(c, U_c=2e3),
                               oracle_state(parts), lat, dt, nsteps)
    params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=2e3)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(),
                   max_particles=len(parts["x"]))
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    U = torch.tensor(2e3, dtype=torch.float64, requires_grad=True)
    K = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    d = torch.from_numpy(parts["d"].copy()).cuda().requires_grad_(True)
    J = T.mean_charge(ch, P, dt, nsteps, U, K, d, ckpt_every=4)
    (3.0 * J).backward()
    ch.close()
    got = dict(J=float(J), dU_c=float(U.grad) / 3, dkappa_A=float(K.grad) / 3, dd=d.grad.cpu().numpy() / 3)
    check(got, ref, 1e-9, "autograd")


def test_adjoint_with_and_without_the_kept_forward_fields():
    """The recomputed segments take the forward's fields when they are kept
    (default budget) or solve them again (budget 0): both match the oracle
    gradient and each other to rounding."""
    c, faces, lat, parts = _case(seed=13)
    dt, nsteps = 2 * c.dt, 7
    ref = mean_charge_gradient(oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces), oracle_params(c, U_c=2e3),
                               oracle_state(parts), lat, dt, nsteps)
    got = []
    for budget in (-1, 0):
        params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=2e3)
        ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(),
                       max_particles=len(parts["x"]))
        T.tribo_set_adjoint_memory(ch.ctx, budget)
        P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
        J, dU, dK, dd = ch.adjoint(P, dt, nsteps, 3)
        ch.close()
        g = dict(J=J, dU_c=dU, dkappa_A=dK, dd=dd.cpu().numpy())
        check(g, ref, 1e-9, f"budget {budget}")
        got.append(g)
    a, b = got
    assert abs(a["J"] - b["J"]) <= 1e-12 * abs(a["J"])
    assert np.abs(a["dd"] - b["dd"]).max() <= 1e-11 * np.abs(a["dd"]).max()


@pytest.fixture(scope="module")
def grid128_case():
    """The differentiation workload's grid (Re_tau 180, 128^3) with 1,000
    particles near the walls and the oracle gradient of 12 steps."""
    c, faces, lat, parts = problem(128, 128, 128, n=1000, q_scale=2e-13, vy_scale=0.4, near_wall=0.3, seed=14,
                                   dplus=(1.0, 1.0))
    dt, nsteps = 2 * c.dt, 12
    ref = mean_charge_gradient(oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces), oracle_params(c, U_c=2e3),
                               oracle_state(parts), lat, dt, nsteps)
    return c, faces, lat, parts, dt, nsteps, ref


@pytest.mark.parametrize("budget", [-1, 0])
def test_adjoint_on_the_differentiation_grid_matches_oracle_gradient(grid128_case, budget):
    """Twelve coupled steps on 128^3 with a state kept every 5, so that two of
    the three segments are recomputed, with the forward fields kept (budget
    -1) and solved again (budget 0); J, dJ/dU_c, dJ/dkappa_A and every dJ/dd_p
    against the oracle gradient (FP64 1e-9)."""
    c, faces, lat, parts, dt, nsteps, ref = grid128_case
    assert ref["final"]["n_imp"].sum() > 50
    params = T.Params(precision=T.TRIBO_FP64, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=2e3)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(),
                   max_particles=len(parts["x"]))
    T.tribo_set_adjoint_memory(ch.ctx, budget)
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64)
    J, dU, dK, dd = ch.adjoint(P, dt, nsteps, 5)
    fin = P.to_numpy()
    ch.close()
    assert np.array_equal(fin["n_imp"].astype(np.int64), ref["final"]["n_imp"])
    check(dict(J=J, dU_c=dU, dkappa_A=dK, dd=dd.cpu().numpy()), ref, 1e-9, f"128^3 budget {budget}")
