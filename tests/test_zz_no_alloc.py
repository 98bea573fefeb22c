"""The allocation-free Poisson entry point, called through the C ABI.

Callers that cannot allocate device memory while running (their allocator
already owns the device memory, or an allocation's latency or failure is not
acceptable mid-run) use tribo_poisson_noalloc, whose scratch is the library's
static 32 MiB device array.  Its result must equal the FP64 oracle's solve
and that of tribo_poisson on two calls in a row (the second call must not see
stale state from the first), on a generic-length grid, on a grid where the
context path runs its compiled-length kernels, and on a grid close to the
array's size; grids beyond the array must be rejected without touching the
GPU.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2602_10761_gb300 as T  # noqa: E402
from paper_2602_10761_gb300 import _abi  # noqa: E402
import synth  # noqa: E402

EPS = 8.854e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10761_gb300 import build
    build.build()
    T.load()


def _check(prec, shape, calls, stream=None):
    """Two (or more) calls in a row: each against the oracle and against the
    context solve of the same density; `calls` gives want_phi per call."""
    nx, ny, nz = shape
    lx, lz = 2 * math.pi * 0.02, math.pi * 0.02
    faces = synth.y_faces(ny, 0.02, 2.0)
    g = oracle.Grid(nx, nz, lx, lz, faces)
    rng = np.random.default_rng(21 + nx + ny)
    rdt = torch.float64 if prec == T.TRIBO_FP64 else torch.float32
    tol = 1e-12 if prec == T.TRIBO_FP64 else 2e-6
    ch = T.Channel(nx, ny, nz, lx, lz, faces, T.Params(precision=prec, eps=EPS), None)
    for call, want_phi in enumerate(calls):
        rho_h = rng.standard_normal((nz, ny, nx)) * 1e-6 + 1e-7 * (call + 1)
        phi_o = oracle.poisson(g, rho_h, EPS)
        E_o = oracle.efield(g, phi_o)
        rho = torch.from_numpy(rho_h).cuda()
        phi_ref, E_ref = ch.poisson(rho, want_phi=want_phi)
        E = torch.full((3, nz, ny + 2, nx), float("nan"), dtype=rdt, device="cuda")
        phi = torch.full((nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda") if want_phi else None
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())      # rho, phi and E are made on the default stream
        T.tribo_poisson_noalloc(nx, ny, nz, lx, lz, faces, EPS, prec, rho, phi, E, stream=stream)
        if stream is not None:
            stream.synchronize()
        torch.cuda.synchronize()
        En = E.double().cpu().numpy()
        Er = E_ref.double().cpu().numpy()
        for comp in range(3):
            ref = E_o[..., comp]
            scale = np.abs(ref).max()
            assert np.abs(En[comp] - ref).max() <= tol * scale, (call, comp, "vs oracle")
            assert np.abs(En[comp] - Er[comp]).max() <= tol * scale, (call, comp, "vs tribo_poisson")
        if want_phi:
            p = phi.cpu().numpy()
            assert np.abs(p - phi_o).max() <= tol * np.abs(phi_o).max(), (call, "phi vs oracle")
            pr = phi_ref.cpu().numpy()
            assert np.abs(p - pr).max() <= tol * np.abs(phi_o).max(), (call, "phi vs tribo_poisson")
    ch.close()


@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_noalloc_poisson_equals_oracle_and_context_poisson_twice(prec):
    _check(prec, (48, 40, 36), (True, False))


@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_noalloc_on_a_compiled_length_grid_and_a_side_stream(prec):
    # 64^3: the context solve runs its compiled-length kernels; phi absent first, then present
    _check(prec, (64, 64, 64), (False, True), stream=torch.cuda.Stream())


def test_noalloc_close_to_the_scratch_size():
    # 256 x 64 x 64 mixed: 28.6 MiB of the 32 MiB without phi
    _check(T.TRIBO_MIXED, (256, 64, 64), (False, False))


def _zeros(nx, ny, nz, prec, with_phi):
    rdt = torch.float64 if prec == T.TRIBO_FP64 else torch.float32
    rho = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
    phi = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda") if with_phi else None
    E = torch.zeros((3, nz, ny + 2, nx), dtype=rdt, device="cuda")
    return rho, phi, E


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    # 256 x 64 x 64 mixed with phi needs 32.8 MiB: rejected, while the same grid without phi runs
    nx, ny, nz = 256, 64, 64
    faces = synth.y_faces(ny, 0.02, 2.0)
    rho, phi, E = _zeros(nx, ny, nz, T.TRIBO_MIXED, True)
    with pytest.raises(T.TriboError) as ei:
        T.tribo_poisson_noalloc(nx, ny, nz, 0.1, 0.05, faces, EPS, T.TRIBO_MIXED, rho, phi, E)
    assert "limit" in str(ei.value) and ei.value.status == _abi.TRIBO_ERR_CAPACITY
    T.tribo_poisson_noalloc(nx, ny, nz, 0.1, 0.05, faces, EPS, T.TRIBO_MIXED, rho, None, E)
    torch.cuda.synchronize()
    assert torch.count_nonzero(E).item() == 0
    # more than 256 cells in a direction
    nx, ny, nz = 384, 64, 16
    faces = synth.y_faces(ny, 0.02, 2.0)
    rho, phi, E = _zeros(nx, ny, nz, T.TRIBO_MIXED, False)
    with pytest.raises(T.TriboError) as ei:
        T.tribo_poisson_noalloc(nx, ny, nz, 0.1, 0.05, faces, EPS, T.TRIBO_MIXED, rho, None, E)
    assert "limit" in str(ei.value) and ei.value.status == _abi.TRIBO_ERR_CAPACITY
