"""Host-pointer calls of tribo_step that do not re-sort send back positions and
velocities of all particles, and q, q_wall, n_imp only of the particles an
impact changed.  After such calls the caller's arrays must hold exactly what
the same calls leave in device arrays, whether the list of changed particles
fits the first copy (at most 4096), needs a second one, or is longer than the
list's capacity (max(1024, max_particles / 8)) and gives way to copying the
three arrays whole.  The byte counter reports what crossed the host link."""
import numpy as np
import pytest

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


def _run(c, faces, lat, parts, prec, host, nsteps=1, calls=2, sort_every=0, with_cell=False):
    real = np.float64 if prec == T.TRIBO_FP64 else np.float32
    params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1e3, sort_every=sort_every)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat.astype(real)).cuda(),
                   max_particles=len(parts["x"]))
    P = T.Particles.from_numpy(parts, prec, device=None if host else "cuda", with_cell=with_cell)
    n_imp = []
    for _ in range(calls):
        ch.step(P, c.dt, nsteps)
        ch.sync()
        n_imp.append(np.asarray(P.to_numpy()["n_imp"]).astype(np.int64))
    out = P.to_numpy()
    nb = T.tribo_transfer_bytes(ch.ctx)
    ch.close()
    order = np.argsort(out["id"])
    changed = [int((n_imp[0] > 0).sum())] + [int((b != a).sum()) for a, b in zip(n_imp, n_imp[1:])]
    return {k: np.asarray(v)[order] for k, v in out.items()}, nb, changed


@pytest.mark.parametrize("n,near,nsteps,lo,hi", [
    (3000, 0.05, 1, 1, 1024),          # the list fits the first copy (capacity 1024)
    (3000, 0.05, 3, 1, 1024),          # several steps in one call
    (60000, 0.09, 1, 4097, 7500),      # a second copy for the rest of the list
    (2000, 0.8, 1, 1025, 2000),        # longer than the list's capacity (1024): whole arrays
])
def test_host_calls_return_the_changed_charges(n, near, nsteps, lo, hi):
    c, faces, lat, parts = problem(16, 12, 8, n=n, q_scale=1e-13, vy_scale=0.2, near_wall=near, seed=31)
    a, _, changed = _run(c, faces, lat, parts, T.TRIBO_FP64, host=False, nsteps=nsteps)
    b, _, _ = _run(c, faces, lat, parts, T.TRIBO_FP64, host=True, nsteps=nsteps)
    assert lo <= changed[0] <= hi, changed        # the first call takes the intended path
    assert np.array_equal(a["n_imp"], b["n_imp"])
    for k in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall"):
        s = max(np.abs(a[k]).max(), 1e-300)
        assert np.abs(a[k].astype(np.float64) - b[k].astype(np.float64)).max() <= 1e-12 * s, k
    assert np.array_equal(np.sort(b["id"]), np.arange(n))


def test_mixed_host_calls_match_device_calls():
    c, faces, lat, parts = problem(16, 12, 8, n=4000, q_scale=1e-13, vy_scale=0.2, near_wall=0.1, seed=32)
    parts = {k: (v if k == "q" else np.asarray(v).astype(np.float32).astype(np.float64)) for k, v in parts.items()}
    lat = lat.astype(np.float32).astype(np.float64)
    a, _, changed = _run(c, faces, lat, parts, T.TRIBO_MIXED, host=False, calls=3, with_cell=True)
    b, _, _ = _run(c, faces, lat, parts, T.TRIBO_MIXED, host=True, calls=3, with_cell=True)
    assert changed[0] > 100
    assert np.array_equal(a["n_imp"], b["n_imp"])
    assert np.array_equal(a["cell"], b["cell"])
    for k in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall"):
        s = max(np.abs(a[k]).max(), 1e-300)
        assert np.abs(a[k].astype(np.float64) - b[k].astype(np.float64)).max() <= 1e-5 * s, k


def test_transfer_bytes_of_host_calls():
    n = 1000
    c, faces, lat, parts = problem(16, 12, 8, n=n, q_scale=1e-13, seed=33)
    # no re-sort and no SSM: the state arrays in except q_wall and n_imp (7 FP32 + q FP64 = 36 B:
    # the device collects the call's wall charge and impact count from zero and the host adds
    # them), positions and velocities out (24 B), and the list's count with its first entries
    # (capacity 1024 entries of 32 B: index, impact count, q, q_wall, site density)
    _, nb, _ = _run(c, faces, lat, parts, T.TRIBO_MIXED, host=True, calls=1)
    assert nb == (36 * n, 24 * n + 16 + 32 * 1024)
    # a call that sorts: the ids both ways, and every array back (44 B + 4 B of ids)
    _, nb, _ = _run(c, faces, lat, parts, T.TRIBO_MIXED, host=True, calls=1, sort_every=1)
    assert nb == (52 * n, 48 * n)
    # device arrays: nothing crosses
    _, nb, _ = _run(c, faces, lat, parts, T.TRIBO_MIXED, host=False, calls=1)
    assert nb == (0, 0)


def test_pinned_host_call_with_slow_copies_keeps_every_impact():
    """Pinned host arrays (the copies run asynchronously) and a tiny grid (the
    field solve ends long before the last range of the arrays has landed): the
    first ranges' chunks of the step run while later ranges are still being
    copied, and the impact counts they add must all come back."""
    n = 4_000_000
    c, faces, lat, parts = problem(16, 12, 8, n=n, q_scale=1e-13, vy_scale=0.2, near_wall=0.01, seed=34)
    a, _, changed = _run(c, faces, lat, parts, T.TRIBO_MIXED, host=False, calls=1)
    params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1e3, sort_every=0)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat.astype(np.float32)).cuda(),
                   max_particles=n)
    Pd = T.Particles.from_numpy(parts, T.TRIBO_MIXED, device="cuda")
    host = {}
    for k in ("x", "y", "z", "vx", "vy", "vz", "d", "q", "q_wall", "n_imp", "id"):
        v = getattr(Pd, k).cpu().pin_memory().numpy()
        host[k] = v.view(np.uint32) if k in ("n_imp", "id") else v
    del Pd
    Ph = T.Particles(**host)
    ch.step(Ph, c.dt, 1)
    ch.sync()
    ch.close()
    order = np.argsort(host["id"])
    b = {k: np.asarray(v)[order] for k, v in host.items()}
    assert changed[0] > 20000                     # impacts in every range, the first included
    first = np.arange(n) < n // 4
    assert (a["n_imp"][first] > 0).sum() > 1000
    assert np.array_equal(a["n_imp"], b["n_imp"])
    for k in ("q", "q_wall"):
        s = max(np.abs(a[k]).max(), 1e-300)
        assert np.abs(a[k] - b[k]).max() <= 1e-5 * s, k
