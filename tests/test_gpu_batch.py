"""Batched ensemble (tribo_batch_*): independent channels of different grids,
particle counts, diameters and Re_tau advanced together in one persistent
particle kernel per step, with graph-captured steps and per-channel Poisson
branches.  Each channel must match the same channel stepped alone with
tribo_step (FP64: 1e-13, mixed: 1e-6 relative; impact counts and statistics
exact) and, for FP64, the oracle at the 1e-12 bar."""
import math

import numpy as np
import pytest

import oracle
from _problems import TOL_FP64, compare_states, oracle_params, oracle_state, problem

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


SPECS = [  # (nx, ny, nz, n, re_tau, d+ range, seed)
    (16, 12, 8, 300, 180.0, (0.8, 2.0), 1),
    (24, 16, 12, 1000, 300.0, (1.0, 3.0), 2),
    (32, 20, 16, 0, 395.0, (0.5, 1.0), 3),       # an empty channel
    (12, 10, 6, 57, 550.0, (2.0, 2.0), 4),
    (32, 24, 32, 2500, 180.0, (0.5, 3.0), 5),
]


def _channels(prec, U_c=500.0, **pkw):
    out = []
    for nx, ny, nz, n, re, dp, seed in SPECS:
        c, faces, lat, parts = problem(nx, ny, nz, n=n, re_tau=re, dplus=dp, q_scale=1e-13, vy_scale=0.3,
                                       near_wall=0.1, seed=seed)
        out.append((c, faces, lat, parts))
    return out


def _make(c, faces, lat, parts, prec, sort_every, U_c, **pkw):
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=U_c, sort_every=sort_every, **pkw)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params,
                   torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda(),
                   max_particles=max(len(parts["x"]), 1))
    P = T.Particles.from_numpy(parts, prec, device="cuda")
    return ch, P


def _sorted(P):
    out = P.to_numpy()
    order = np.argsort(out["id"])
    return {k: np.asarray(v)[order] for k, v in out.items()}


@pytest.mark.parametrize("prec,sort_every,nsteps", [
    (T.TRIBO_FP64, 0, 21), (T.TRIBO_FP64, 3, 17), (T.TRIBO_MIXED, 4, 26), (T.TRIBO_MIXED, 0, 9)])
def test_batch_matches_single_channels(prec, sort_every, nsteps):
    data = _channels(prec)
    U_c = 500.0
    singles, batch_ch, batch_P, dts = [], [], [], []
    for c, faces, lat, parts in data:
        ch, P = _make(c, faces, lat, parts, prec, sort_every, U_c)
        ch.step(P, c.dt, nsteps)
        ch.sync()
        singles.append((_sorted(P), ch.stats(P)))
        ch.close()
        ch, P = _make(c, faces, lat, parts, prec, sort_every, U_c)
        batch_ch.append(ch)
        batch_P.append(P)
        dts.append(c.dt)
    B = T.Batch(batch_ch, sort_every=sort_every)
    choice = B.autotune(batch_P, dts)
    assert choice["threads"] in (128, 256, 512)
    # split the run so that both graph replays and direct launches occur
    B.step(batch_P, dts, nsteps - 5)
    B.step(batch_P, dts, 5)
    B.sync()
    assert B.launches > 0
    tol = 1e-13 if prec == T.TRIBO_FP64 else 1e-6
    for (c, faces, lat, parts), (ref, rst), ch, P in zip(data, singles, batch_ch, batch_P):
        got = _sorted(P)
        st = ch.stats(P)
        if len(parts["x"]) == 0:
            continue
        for k in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall"):
            s = max(np.abs(ref[k]).max(), 1e-40)
            assert np.abs(got[k].astype(np.float64) - ref[k].astype(np.float64)).max() <= tol * s, (c.name, k)
        assert np.array_equal(got["n_imp"], ref["n_imp"])
        assert st["n_impacts"] == rst["n_impacts"]
        assert np.array_equal(st["hist_y"], rst["hist_y"])
        assert st["n_samples"] == nsteps
    B.close()
    for ch in batch_ch:
        ch.close()


def test_batch_fp64_matches_oracle():
    data = _channels(T.TRIBO_FP64)
    chans, Ps, dts = [], [], []
    for c, faces, lat, parts in data:
        ch, P = _make(c, faces, lat, parts, T.TRIBO_FP64, 2, 500.0)
        chans.append(ch)
        Ps.append(P)
        dts.append(c.dt)
    B = T.Batch(chans, sort_every=2)
    B.step(Ps, dts, 10)
    B.sync()
    for (c, faces, lat, parts), P in zip(data, Ps):
        if len(parts["x"]) == 0:
            continue
        g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
        ref = oracle.run(g, oracle_params(c, U_c=500.0), oracle_state(parts), lat, c.dt, 10)
        got = {k: v.astype(np.float64) for k, v in _sorted(P).items()}
        compare_states(g, got, ref, TOL_FP64, label=c.name)
        assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)
    B.close()
    for ch in chans:
        ch.close()


def test_batch_rejects_mode_fields_and_oversize():
    c, faces, lat, parts = problem(16, 12, 8, n=50, seed=3)
    ch, P = _make(c, faces, lat, parts, T.TRIBO_MIXED, 0, 1.0)
    import synth
    ch.set_modes(synth.draw_modes(c), synth.mean_velocity(synth.node_y(faces), c),
                 synth.damping(synth.node_y(faces), c))
    with pytest.raises(T.TriboError):
        T.Batch([ch])
    ch.set_modes(None)
    B = T.Batch([ch])
    big = T.Particles.from_numpy({k: np.concatenate([v, v]) for k, v in parts.items()}, T.TRIBO_MIXED)
    with pytest.raises(T.TriboError):
        B.step([big], [c.dt], 1)
    B.close()
    ch.close()


GROUP_SPECS = [  # channels sharing a grid solve their Poisson passes as one launch each
    (32, 24, 32, 1500, 180.0, (0.5, 3.0), 11),
    (32, 24, 32, 0, 300.0, (1.0, 2.0), 12),        # an empty member: its field solves to zero
    (32, 24, 32, 800, 550.0, (0.8, 2.5), 13),
    (24, 16, 12, 600, 395.0, (1.0, 3.0), 14),
    (24, 16, 12, 900, 180.0, (0.5, 1.5), 15),
    (36, 12, 18, 300, 300.0, (1.0, 2.0), 16),      # no compiled transform length: solved alone
]


def _group_data():
    out = []
    for nx, ny, nz, n, re, dp, seed in GROUP_SPECS:
        out.append(problem(nx, ny, nz, n=n, re_tau=re, dplus=dp, q_scale=1e-13, vy_scale=0.3, near_wall=0.1,
                           seed=seed))
    return out


@pytest.mark.parametrize("sort_every,nsteps", [(0, 19), (3, 14)])
def test_batch_grouped_poisson_matches_single_channels(sort_every, nsteps):
    data = _group_data()
    U_c = 500.0
    singles, chans, Ps, dts = [], [], [], []
    for c, faces, lat, parts in data:
        ch, P = _make(c, faces, lat, parts, T.TRIBO_MIXED, sort_every, U_c)
        ch.step(P, c.dt, nsteps)
        ch.sync()
        singles.append((_sorted(P), ch.stats(P)))
        ch.close()
        ch, P = _make(c, faces, lat, parts, T.TRIBO_MIXED, sort_every, U_c)
        chans.append(ch)
        Ps.append(P)
        dts.append(c.dt)
    B = T.Batch(chans, sort_every=sort_every)
    B.step(Ps, dts, nsteps - 4)          # graph replays and direct launches
    B.step(Ps, dts, 4)
    B.sync()
    for (c, faces, lat, parts), (ref, rst), ch, P in zip(data, singles, chans, Ps):
        if len(parts["x"]) == 0:
            continue
        got = _sorted(P)
        st = ch.stats(P)
        for k in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall"):
            s = max(np.abs(ref[k]).max(), 1e-40)
            assert np.abs(got[k].astype(np.float64) - ref[k].astype(np.float64)).max() <= 1e-6 * s, (c.name, k)
        assert np.array_equal(got["n_imp"], ref["n_imp"])
        assert st["n_impacts"] == rst["n_impacts"]
        assert np.array_equal(st["hist_y"], rst["hist_y"])
    B.close()
    for ch in chans:
        ch.close()


def test_batch_group_launch_count_and_kernel_timing():
    # five channels in two groups, no sort: each step is the particle kernel plus five
    # passes per group, whether replayed from the graph or launched directly
    data = _group_data()[:5]
    chans, Ps, dts = [], [], []
    for c, faces, lat, parts in data:
        ch, P = _make(c, faces, lat, parts, T.TRIBO_MIXED, 0, 500.0)
        chans.append(ch)
        Ps.append(P)
        dts.append(c.dt)
    B = T.Batch(chans, sort_every=0)
    B.autotune(Ps, dts)
    l0 = B.launches
    B.step(Ps, dts, 9)                   # one 8-step graph and one direct step
    B.sync()
    deposits = sum(1 for _, _, _, parts in data if len(parts["x"]) > 0)
    assert B.launches - l0 == deposits + 9 * (1 + 2 * 5)
    B.timing(True)
    B.step(Ps, dts, 3)
    B.sync()
    ms, n = B.kernel_time()
    assert n == 3 and ms > 0.0
    assert B.kernel_time() == (0.0, 0)
    B.timing(False)
    B.close()
    for ch in chans:
        ch.close()
