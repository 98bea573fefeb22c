"""The allocation-free Poisson entry point, called through the C ABI.

Callers that cannot allocate device memory while running (their allocator
already owns the device memory, or an allocation's latency or failure is not
acceptable mid-run) use tribo_poisson_noalloc, whose scratch is the library's
static device array.  Its result must equal that of tribo_poisson on two calls
in a row (the second call must not see stale state from the first), and grids
beyond the array's limit must be rejected without touching the GPU.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2602_10761_gb300 as T  # noqa: E402
import synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10761_gb300 import build
    build.build()
    T.load()


@pytest.mark.parametrize("prec", [T.TRIBO_FP64, T.TRIBO_MIXED])
def test_noalloc_poisson_equals_context_poisson_twice(prec):
    nx, ny, nz = 48, 40, 36
    lx, lz = 2 * math.pi * 0.02, math.pi * 0.02
    faces = synth.y_faces(ny, 0.02, 2.0)
    eps = 8.854e-12
    rng = np.random.default_rng(21)
    rdt = torch.float64 if prec == T.TRIBO_FP64 else torch.float32
    tol = 1e-12 if prec == T.TRIBO_FP64 else 2e-6
    ch = T.Channel(nx, ny, nz, lx, lz, faces, T.Params(precision=prec, eps=eps), None)
    for call, want_phi in ((0, True), (1, False)):
        rho = torch.from_numpy(rng.standard_normal((nz, ny, nx)) * 1e-6 + 1e-7 * call).cuda()
        phi_ref, E_ref = ch.poisson(rho, want_phi=want_phi)
        E = torch.full((3, nz, ny + 2, nx), float("nan"), dtype=rdt, device="cuda")
        phi = torch.full((nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda") if want_phi else None
        T.tribo_poisson_noalloc(nx, ny, nz, lx, lz, faces, eps, prec, rho, phi, E)
        torch.cuda.synchronize()
        Er = E_ref.double()
        err = (E.double() - Er).abs().max().item() / Er.abs().max().item()
        assert err <= tol, (call, err)
        if want_phi:
            perr = (phi - phi_ref).abs().max().item() / phi_ref.abs().max().item()
            assert perr <= tol, (call, perr)
    ch.close()


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    nx, ny, nz = 384, 256, 256
    faces = synth.y_faces(ny, 0.02, 2.0)
    with pytest.raises(T.TriboError) as ei:
        T.tribo_poisson_noalloc(nx, ny, nz, 0.1, 0.05, faces, 8.854e-12, T.TRIBO_MIXED,
                                torch.zeros(1, dtype=torch.float64, device="cuda"), None,
                                torch.zeros(1, device="cuda"))
    assert "limit" in str(ei.value)
