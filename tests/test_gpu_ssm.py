"""Stochastic scaling model of wall impacts on the GPU against the oracle:
near-wall particles impacting over ten steps, each impact's charge drawn
from Philox4x32-10 with counter (particle id, impact count), so the result
must not depend on the particle order (re-sorting on and off); FP64 to 1e-12
and mixed to 1e-5 per particle, impact counts exact."""
import dataclasses

import numpy as np
import pytest

import oracle
from _problems import TOL_FP64, TOL_MIXED, compare_states, oracle_params, problem
from oracle.ssm import SSM

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


def _gpu(c, faces, lat, parts, prec, nsteps, ssm, **pkw):
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, **pkw)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params,
                   torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda(), max_particles=len(parts["x"]))
    ch.set_ssm(T.SSMParams(**dataclasses.asdict(ssm)))
    P = T.Particles.from_numpy(parts, prec, device="cuda")
    ch.step(P, c.dt, nsteps)
    ch.sync()
    out = P.to_numpy()
    ch.close()
    order = np.argsort(out["id"])
    return {k: np.asarray(v)[order].astype(np.float64) for k, v in out.items()}


@pytest.mark.parametrize("sort_every", [0, 3])
@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_ssm_matches_oracle(prec, sort_every):
    c, faces, lat, parts = problem(32, 24, 16, n=3000, q_scale=1e-14, vy_scale=0.4, near_wall=0.3, seed=51,
                                   dplus=(0.8, 2.5))
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    pr = {k: (v if k == "q" else np.asarray(v).astype(real).astype(np.float64)) for k, v in parts.items()}
    # earlier impacts: the counter's second word varies between particles
    pr["n_imp"] = np.random.default_rng(51).integers(0, 7, len(pr["x"]))
    lat_r = lat.astype(real).astype(np.float64)
    ssm = SSM(seed=0x1234567890ABCDEF)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    st0 = oracle.State.from_arrays(pr["x"], pr["y"], pr["z"], pr["vx"], pr["vy"], pr["vz"], pr["q"], pr["d"],
                                   n_imp=pr["n_imp"])
    ref = oracle.run(g, oracle_params(c, ssm=ssm), st0, lat_r, c.dt, 10)
    assert (ref.n_imp - st0.n_imp).sum() > 500
    got = _gpu(c, faces, lat_r, pr, prec, 10, ssm, sort_every=sort_every)
    tol = TOL_FP64 if prec == T.TRIBO_FP64 else TOL_MIXED
    compare_states(g, got, ref, tol, label=f"ssm prec={prec} sort={sort_every}")
    assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)
    # the stochastic charges are not all alike: both signs occur
    assert (ref.q_wall > 0).any() and (ref.q_wall < 0).any()


def test_ssm_needs_particle_ids():
    c, faces, lat, parts = problem(12, 8, 6, n=20, seed=2)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, T.Params(precision=T.TRIBO_FP64),
                   torch.from_numpy(lat).cuda(), max_particles=20)
    ch.set_ssm(T.SSMParams())
    P = T.Particles.from_numpy(parts, T.TRIBO_FP64, with_id=False)
    with pytest.raises(T.TriboError):
        ch.step(P, c.dt, 1)
    ch.set_ssm(None)
    ch.step(P, c.dt, 1)
    ch.sync()
    ch.close()


def _gpu_site(c, faces, lat, parts, prec, nsteps, ssm, host=False, calls=1, **pkw):
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, **pkw)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params,
                   torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda(), max_particles=len(parts["x"]))
    ch.set_ssm(T.SSMParams(**dataclasses.asdict(ssm)))
    P = T.Particles.from_numpy(parts, prec, device=None if host else "cuda", with_site=True)
    for _ in range(calls):
        ch.step(P, c.dt, nsteps // calls)
    ch.sync()
    out = P.to_numpy()
    ch.close()
    order = np.argsort(out["id"])
    return {k: np.asarray(v)[order].astype(np.float64) for k, v in out.items()}


@pytest.mark.parametrize("variant", ["device", "device_sorted", "host_one_step_calls"])
@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_ssm_site_history_matches_oracle(prec, variant):
    """The charging-site density c/c0 carried per particle: charged particles
    (towards saturation) impacting over ten steps, with initial densities in
    [0.2, 1] so that c/c0 changes the impact charge; c/c0 after each impact
    and the charges against the oracle, through sorts (the site array is
    permuted with the particles) and through one-step host-pointer calls
    (only the impacted particles' charges and densities come back)."""
    c, faces, lat, parts = problem(32, 24, 16, n=3000, vy_scale=0.4, near_wall=0.3, seed=53, dplus=(0.8, 2.5))
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    pr = {k: (v if k == "q" else np.asarray(v).astype(real).astype(np.float64)) for k, v in parts.items()}
    rng = np.random.default_rng(53)
    n = len(pr["x"])
    ssm = SSM(seed=0x0DDBA11)
    # charges between 0 and 0.9 of the saturation charge the wall drives them to (negative here)
    pr["q"] = -rng.uniform(0.0, 0.9, n) * ssm.c_sat * pr["d"] ** 2 / 4.0
    pr["site"] = rng.uniform(0.2, 1.0, n)
    pr["n_imp"] = rng.integers(0, 5, n)
    lat_r = lat.astype(real).astype(np.float64)
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    st0 = oracle.State.from_arrays(pr["x"], pr["y"], pr["z"], pr["vx"], pr["vy"], pr["vz"], pr["q"], pr["d"],
                                   n_imp=pr["n_imp"], site=pr["site"])
    ref = oracle.run(g, oracle_params(c, ssm=ssm), st0, lat_r, c.dt, 10)
    hit = ref.n_imp > st0.n_imp
    assert hit.sum() > 500
    assert np.abs(ref.site - st0.site)[hit].max() > 1e-6       # the history moved
    kw = dict(sort_every=3 if variant == "device_sorted" else 0)
    got = _gpu_site(c, faces, lat_r, pr, prec, 10, ssm, host=variant.startswith("host"),
                    calls=10 if variant.startswith("host") else 1, **kw)
    tol = TOL_FP64 if prec == T.TRIBO_FP64 else TOL_MIXED
    compare_states(g, got, ref, tol, label=f"ssm site prec={prec} {variant}")
    assert np.array_equal(got["n_imp"].astype(np.int64), ref.n_imp)
    err = np.abs(got["site"] - ref.site).max()
    assert err <= tol, err
    assert np.array_equal(got["site"][~hit], pr["site"][~hit])
