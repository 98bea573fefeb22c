"""Python binding of the C ABI (argument marshalling only).

Every function named tribo_* mirrors the C entry point of the same name in
include/tribo.h.  PyTorch is used for device memory and streams only; all
arithmetic of the hot path runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional

import numpy as np

from . import _abi
from ._abi import check, load


@dataclasses.dataclass
class Params:
    """Physical parameters (Table 1 of the paper) and switches.

    U_c, the particle-wall contact potential, is not given in the paper.
    """
    mu_p: float = 0.4          # Poisson's ratio, particle
    E_p: float = 1e8           # Young's modulus, particle [Pa]
    phi_p: float = 1e13        # resistivity, particle [Ohm m]
    k_e: float = 0.95          # restitution ratio
    mu_w: float = 0.28         # Poisson's ratio, wall
    E_w: float = 1e11          # Young's modulus, wall [Pa]
    eps_w: float = 5.0         # relative permittivity, wall
    h: float = 1e-9            # effective separation [m]
    eps: float = 8.854e-12     # gas permittivity [F/m]
    eps0: float = 8.854e-12    # vacuum permittivity [F/m]
    nu: float = 1.46e-5        # gas kinematic viscosity [m^2/s]
    rho: float = 1.2           # gas density [kg/m^3]
    rho_p: float = 1150.0      # particle density [kg/m^3]
    U_c: float = 1.0           # contact potential [V]
    kappa_A: float = 1.0       # contact-area factor
    drag_law: int = _abi.TRIBO_DRAG_STOKES
    impact_vel: int = _abi.TRIBO_IMPACT_SPEED
    dq_t: int = 1
    electrostatics: int = 1
    precision: int = _abi.TRIBO_MIXED
    sort_every: int = 0
    coulomb: int = 0          # in-cell Coulomb near field (hybrid electrostatics)
    collisions: int = 0       # 4-way coupling: particle-particle collisions with charge exchange

    def to_c(self) -> _abi.tribo_params:
        p = _abi.tribo_params()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p

    def with_(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)

    @property
    def real_dtype(self):
        return np.float64 if self.precision == _abi.TRIBO_FP64 else np.float32


def _ptr(a) -> Optional[int]:
    """Address of a contiguous torch tensor or numpy array (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _on_host(a) -> bool:
    return isinstance(a, np.ndarray) or (hasattr(a, "is_cuda") and not a.is_cuda)


class Particles:
    """Structure-of-arrays particle ensemble (torch CUDA tensors or numpy)."""
    REAL = ("x", "y", "z", "vx", "vy", "vz", "d")
    ALL = REAL + ("q", "q_wall", "n_imp", "id", "cell", "site")

    def __init__(self, **arrays):
        for name in self.ALL:
            setattr(self, name, arrays.get(name))
        self.n = int(self.x.shape[0])

    @classmethod
    def from_numpy(cls, src, precision: int, device: Optional[str] = "cuda", with_id: bool = True,
                   with_cell: bool = False, with_site: bool = False) -> "Particles":
        """src: object or dict with x, y, z, vx, vy, vz, d, q (and optionally
        q_wall, n_imp, site).  with_site: carry the SSM charging-site density
        c/c0 (src's site, else 1).  device=None keeps host (numpy) arrays."""
        get = (lambda k: src.get(k)) if isinstance(src, dict) else (lambda k: getattr(src, k, None))
        rdt = np.float64 if precision == _abi.TRIBO_FP64 else np.float32
        n = np.asarray(get("x")).shape[0]
        arr = {k: np.ascontiguousarray(np.asarray(get(k), dtype=rdt)) for k in cls.REAL}
        arr["q"] = np.ascontiguousarray(np.asarray(get("q"), dtype=np.float64))
        qw = get("q_wall")
        arr["q_wall"] = np.zeros(n) if qw is None else np.ascontiguousarray(np.asarray(qw, np.float64))
        ni = get("n_imp")
        arr["n_imp"] = np.zeros(n, np.uint32) if ni is None else np.ascontiguousarray(np.asarray(ni, np.uint32))
        if with_id:
            ids = get("id")
            arr["id"] = np.arange(n, dtype=np.uint32) if ids is None else np.asarray(ids, np.uint32)
        if with_cell:
            arr["cell"] = np.zeros(n, np.uint32)
        if with_site or get("site") is not None:
            si = get("site")
            arr["site"] = np.ones(n) if si is None else np.ascontiguousarray(np.asarray(si, np.float64))
        if device is None:
            return cls(**arr)
        import torch
        t = {}
        for k, v in arr.items():
            if v.dtype == np.uint32:
                t[k] = torch.from_numpy(v.view(np.int32)).to(device)
            else:
                t[k] = torch.from_numpy(v).to(device)
        return cls(**t)

    def to_numpy(self) -> dict:
        out = {}
        for k in self.ALL:
            v = getattr(self, k)
            if v is None:
                continue
            if not isinstance(v, np.ndarray):
                v = v.detach().cpu().numpy()
            if k in ("n_imp", "id", "cell"):
                v = v.view(np.uint32)
            out[k] = v
        return out

    @property
    def on_host(self) -> bool:
        return _on_host(self.x)

    def c_struct(self) -> _abi.tribo_particles:
        s = _abi.tribo_particles()
        s.n = self.n
        for k in self.ALL:
            setattr(s, k, _ptr(getattr(self, k)))
        s.on_host = 1 if self.on_host else 0
        return s


# ---------------------------------------------------------------- C-named calls

def tribo_init(nx: int, ny: int, nz: int, lx: float, lz: float, y_faces, params: Params,
               u_lattice=None, max_particles: int = 0, stream=None) -> int:
    lib = load()
    yf = np.ascontiguousarray(np.asarray(y_faces, dtype=np.float64))
    g = _abi.tribo_grid(nx, ny, nz, lx, lz, yf.ctypes.data_as(C.POINTER(C.c_double)))
    fl = None
    if u_lattice is not None:
        fl = _abi.tribo_fluid(_ptr(u_lattice), 1 if _on_host(u_lattice) else 0)
    ctx = C.c_void_p()
    sp = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    p = params.to_c()
    check(lib.tribo_init(C.byref(ctx), C.byref(g), C.byref(fl) if fl is not None else None, C.byref(p),
                         int(max_particles), sp), "tribo_init")
    return ctx.value


def tribo_set_fluid(ctx: int, u_lattice) -> None:
    fl = _abi.tribo_fluid(_ptr(u_lattice), 1 if _on_host(u_lattice) else 0)
    check(load().tribo_set_fluid(ctx, C.byref(fl)), "tribo_set_fluid")


def tribo_set_modes(ctx: int, modes, ubar, damp, t0: float = 0.0) -> None:
    """Time-varying synthetic gas field from Fourier modes (None: frozen lattice).

    modes: object with nxi, nzi (integer wavenumbers), ky, amp (n, 3), phase;
    ubar, damp: mean velocity and damping at the ny+2 lattice y nodes.
    """
    if modes is None:
        check(load().tribo_set_modes(ctx, None), "tribo_set_modes")
        return
    keep = dict(nxi=np.ascontiguousarray(modes.nxi, np.int32), nzi=np.ascontiguousarray(modes.nzi, np.int32),
                ky=np.ascontiguousarray(modes.ky, np.float64), amp=np.ascontiguousarray(modes.amp, np.float64),
                phase=np.ascontiguousarray(modes.phase, np.float64), ubar=np.ascontiguousarray(ubar, np.float64),
                damp=np.ascontiguousarray(damp, np.float64))
    m = _abi.tribo_modes(int(keep["nxi"].shape[0]), *(keep[k].ctypes.data for k in
                                                       ("nxi", "nzi", "ky", "amp", "phase", "ubar", "damp")),
                         float(t0))
    check(load().tribo_set_modes(ctx, C.byref(m)), "tribo_set_modes")


@dataclasses.dataclass
class SSMParams:
    """Stochastic scaling model of wall-impact charging (Sec. 2.3.2): the
    reference impact (radius r0, normal speed un0) with its charge statistics
    and C_sat, as given for the paper's particles in Sec. 3.1, and the seed of
    the Philox4x32-10 stream.  sigma0 = gamma0 = 0 makes the model
    deterministic."""
    r0: float = 2e-4          # reference particle radius [m]
    un0: float = 0.925        # reference normal impact speed [m/s]
    mu0: float = -4.12e-15    # mean charge of the reference impact [C]
    sigma0: float = 6.49e-15  # its standard deviation [C]
    gamma0: float = -0.191    # its skewness
    dq0_min: float = -2.19e-14   # minimum charge of the reference impact [C]
    c_sat: float = 500e-6     # saturation surface charge density C_sat [C/m^2]
    seed: int = 0


def tribo_set_ssm(ctx: int, ssm) -> None:
    """Stochastic scaling model of wall impacts (None: condenser model).  ssm:
    an SSMParams, or any object with its fields."""
    if ssm is None:
        check(load().tribo_set_ssm(ctx, None), "tribo_set_ssm")
        return
    s = _abi.tribo_ssm(*(float(getattr(ssm, k)) for k in ("r0", "un0", "mu0", "sigma0", "gamma0", "dq0_min",
                                                          "c_sat")), int(ssm.seed))
    check(load().tribo_set_ssm(ctx, C.byref(s)), "tribo_set_ssm")


def tribo_eval_modes(ctx: int, t: float, u_out=None) -> None:
    check(load().tribo_eval_modes(ctx, float(t), _ptr(u_out)), "tribo_eval_modes")


def tribo_set_momentum_source(ctx: int, F_s=None) -> None:
    """Momentum source of the particles on the gas (Eq. ns): device planes
    (3, Nz, Ny, Nx) of the real type, overwritten by every tribo_step with
    the mean over its steps; None switches it off."""
    check(load().tribo_set_momentum_source(ctx, _ptr(F_s)), "tribo_set_momentum_source")


def tribo_set_adjoint_memory(ctx: int, max_bytes: int = -1) -> None:
    """Budget of the adjoint's kept forward fields: < 0 half of the free device
    memory (default), 0 never keep them, > 0 at most that many bytes."""
    check(load().tribo_set_adjoint_memory(ctx, int(max_bytes)), "tribo_set_adjoint_memory")


def tribo_transfer_bytes(ctx: int) -> tuple:
    """(host to device, device to host) bytes the context's host-pointer calls
    have moved since tribo_init."""
    h2d, d2h = C.c_uint64(0), C.c_uint64(0)
    check(load().tribo_transfer_bytes(ctx, C.byref(h2d), C.byref(d2h)), "tribo_transfer_bytes")
    return int(h2d.value), int(d2h.value)


def tribo_set_params(ctx: int, params: Params) -> None:
    p = params.to_c()
    check(load().tribo_set_params(ctx, C.byref(p)), "tribo_set_params")


def tribo_step(ctx: int, particles: Particles, dt: float, nsteps: int = 1) -> None:
    s = particles.c_struct()
    check(load().tribo_step(ctx, C.byref(s), float(dt), int(nsteps)), "tribo_step")


def tribo_poisson(ctx: int, rho, phi, E) -> None:
    check(load().tribo_poisson(ctx, _ptr(rho), _ptr(phi), _ptr(E)), "tribo_poisson")


def tribo_adjoint(ctx: int, particles: Particles, dt: float, nsteps: int, ckpt_every: int, dJ_dd=None):
    """Advance the particles nsteps steps and return (J, dJ/dU_c, dJ/dkappa_A);
    dJ_dd (device, n doubles) receives dJ/dd_p if given."""
    s = particles.c_struct()
    J, dU, dK = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    check(load().tribo_adjoint(ctx, C.byref(s), float(dt), int(nsteps), int(ckpt_every), C.byref(J), C.byref(dU),
                               C.byref(dK), _ptr(dJ_dd)), "tribo_adjoint")
    return J.value, dU.value, dK.value


def _check_noalloc_args(nx, ny, nz, y_faces, precision, rho, phi, E):
    """Layout checks of tribo_poisson_noalloc's arrays, made before the C call
    (the C side sees raw pointers only): FP64 rho (nz, ny, nx), FP64 phi of
    the same shape or None, E (3, nz, ny+2, nx) of the precision's real type,
    all contiguous CUDA tensors on the current device; ny + 1 faces."""
    import torch
    yf = np.ascontiguousarray(np.asarray(y_faces, dtype=np.float64))
    if yf.ndim != 1 or yf.shape[0] != ny + 1:
        raise ValueError(f"y_faces must hold ny + 1 = {ny + 1} faces, got shape {yf.shape}")
    real = torch.float64 if precision == _abi.TRIBO_FP64 else torch.float32
    want = (("rho", rho, torch.float64, (nz, ny, nx)), ("phi", phi, torch.float64, (nz, ny, nx)),
            ("E", E, real, (3, nz, ny + 2, nx)))
    for name, t, dt, shape in want:
        if t is None and name == "phi":
            continue
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch CUDA tensor")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor (got a {t.device} tensor)")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on {t.device}, the current device is cuda:{torch.cuda.current_device()}")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    return yf


def tribo_poisson_noalloc(nx: int, ny: int, nz: int, lx: float, lz: float, y_faces, eps: float,
                          precision: int, rho, phi, E, stream=None) -> None:
    """Context-free Poisson solve that allocates no device memory (for callers
    that cannot allocate while running); scratch is the library's static
    32 MiB device array, shared by all calls.  rho, phi (or None) and E are
    torch CUDA tensors, checked for dtype, shape and device before the call."""
    yf = _check_noalloc_args(nx, ny, nz, y_faces, precision, rho, phi, E)
    g = _abi.tribo_grid(nx, ny, nz, lx, lz, yf.ctypes.data_as(C.POINTER(C.c_double)))
    sp = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    check(load().tribo_poisson_noalloc(C.byref(g), float(eps), int(precision), _ptr(rho), _ptr(phi), _ptr(E), sp),
          "tribo_poisson_noalloc")


def tribo_stats(ctx: int, particles: Optional[Particles], ny: int) -> dict:
    lib = load()
    sq = C.c_double(0.0)
    ni = C.c_uint64(0)
    sw = C.c_double(0.0)
    ns = C.c_int64(0)
    hist = np.zeros(ny)
    s = particles.c_struct() if particles is not None else None
    check(lib.tribo_stats(ctx, C.byref(s) if s is not None else None,
                          C.byref(sq) if s is not None else None, C.byref(ni), C.byref(sw),
                          hist.ctypes.data_as(C.POINTER(C.c_double)), C.byref(ns)), "tribo_stats")
    return dict(sum_q=sq.value if s is not None else None, n_impacts=ni.value, sum_wall=sw.value,
                hist_y=hist, n_samples=ns.value)


def tribo_reset_stats(ctx: int) -> None:
    check(load().tribo_reset_stats(ctx), "tribo_reset_stats")


def tribo_sync(ctx: int) -> None:
    check(load().tribo_sync(ctx), "tribo_sync")


def tribo_error_bits(ctx: int) -> int:
    return int(load().tribo_error_bits(ctx))


def tribo_clear_error(ctx: int) -> None:
    check(load().tribo_clear_error(ctx), "tribo_clear_error")


def tribo_test_pipeline_wait(ctx: int, plane: int) -> None:
    check(load().tribo_test_pipeline_wait(ctx, int(plane)), "tribo_test_pipeline_wait")


def tribo_launch_count(ctx: int) -> int:
    return int(load().tribo_launch_count(ctx))


def tribo_timing_enable(ctx: int, on: bool) -> None:
    check(load().tribo_timing_enable(ctx, 1 if on else 0), "tribo_timing_enable")


def tribo_timing_read(ctx: int) -> dict:
    """{kernel phase name: (total device ms, launches)} since the last enable."""
    lib = load()
    n = _abi.TRIBO_NPHASES
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    check(lib.tribo_timing_read(ctx, ms, cnt, n), "tribo_timing_read")
    return {lib.tribo_phase_name(i).decode(): (ms[i], cnt[i]) for i in range(n)}


def tribo_phase_name(phase: int):
    r = load().tribo_phase_name(phase)
    return None if r is None else r.decode()


def tribo_destroy(ctx: int) -> None:
    load().tribo_destroy(ctx)


# ---------------------------------------------------------------- batched ensemble

class Batch:
    """Independent channels advanced together (tribo_batch_*)."""

    def __init__(self, channels, sort_every: int = 0, stream=None):
        lib = load()
        self.channels = list(channels)
        arr = (C.c_void_p * len(self.channels))(*[ch.ctx for ch in self.channels])
        h = C.c_void_p()
        sp = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        check(lib.tribo_batch_create(C.byref(h), len(self.channels), arr, int(sort_every), sp), "tribo_batch_create")
        self.handle = h.value

    def _args(self, particles, dt):
        structs = [p.c_struct() for p in particles]
        ptrs = (C.POINTER(_abi.tribo_particles) * len(structs))(*[C.pointer(s) for s in structs])
        dts = (C.c_double * len(structs))(*[float(x) for x in dt])
        return structs, ptrs, dts

    def autotune(self, particles, dt):
        keep, ptrs, dts = self._args(particles, dt)
        choice = (C.c_int32 * 3)()
        check(load().tribo_batch_autotune(self.handle, ptrs, dts, choice), "tribo_batch_autotune")
        return dict(threads=choice[0], tile=choice[1], blocks_per_sm=choice[2])

    def step(self, particles, dt, nsteps: int) -> None:
        keep, ptrs, dts = self._args(particles, dt)
        check(load().tribo_batch_step(self.handle, ptrs, dts, int(nsteps)), "tribo_batch_step")

    def sync(self) -> None:
        check(load().tribo_batch_sync(self.handle), "tribo_batch_sync")

    @property
    def launches(self) -> int:
        return int(load().tribo_batch_launch_count(self.handle))

    def timing(self, enable: bool) -> None:
        """Start (True) or stop timing the particle kernel; while on, steps run as direct launches."""
        check(load().tribo_batch_timing(self.handle, 1 if enable else 0), "tribo_batch_timing")

    def kernel_time(self):
        """(total milliseconds, launches) of the timed particle-kernel launches; restarts the record."""
        ms = C.c_double()
        n = C.c_int64()
        check(load().tribo_batch_kernel_time(self.handle, C.byref(ms), C.byref(n)), "tribo_batch_kernel_time")
        return float(ms.value), int(n.value)

    def close(self) -> None:
        if self.handle:
            load().tribo_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- autograd

def _mean_charge_function():
    import torch

    class MeanCharge(torch.autograd.Function):
        """J = mean particle charge after nsteps steps, differentiable in U_c,
        kappa_A and the diameters.  The forward pass runs tribo_adjoint, which
        advances the particles and computes the gradients with the library's
        reverse-mode kernels; backward scales them by the upstream gradient."""

        @staticmethod
        def forward(ctx, U_c, kappa_A, d, channel, particles, dt, nsteps, ckpt_every):
            p = channel.params.with_(U_c=float(U_c), kappa_A=float(kappa_A))
            channel.set_params(p)
            particles.d.copy_(d.detach().to(particles.d.dtype))
            dd = torch.empty(particles.n, dtype=torch.float64, device=particles.d.device)
            J, dU, dK = tribo_adjoint(channel.ctx, particles, dt, nsteps, ckpt_every, dd)
            ctx.save_for_backward(dd)
            ctx.dU, ctx.dK = dU, dK
            ctx.d_dtype = d.dtype
            dev = lambda t: t.device if isinstance(t, torch.Tensor) else None
            ctx.devs = (dev(U_c), dev(kappa_A))
            return torch.tensor(J, dtype=torch.float64, device=d.device)

        @staticmethod
        def backward(ctx, gJ):
            (dd,) = ctx.saved_tensors
            gU = (gJ * ctx.dU).to(ctx.devs[0]) if ctx.needs_input_grad[0] else None
            gK = (gJ * ctx.dK).to(ctx.devs[1]) if ctx.needs_input_grad[1] else None
            gd = (gJ * dd).to(ctx.d_dtype) if ctx.needs_input_grad[2] else None
            return gU, gK, gd, None, None, None, None, None

    return MeanCharge


_MEAN_CHARGE = None


def mean_charge(channel: "Channel", particles: Particles, dt: float, nsteps: int, U_c, kappa_A, d,
                ckpt_every: int = 50):
    """Differentiable mean charge after nsteps steps (torch.autograd).

    U_c, kappa_A: 0-dim tensors; d: (n,) tensor of diameters on the device.
    The particles (device arrays) are advanced nsteps steps in place."""
    global _MEAN_CHARGE
    if _MEAN_CHARGE is None:
        _MEAN_CHARGE = _mean_charge_function()
    return _MEAN_CHARGE.apply(U_c, kappa_A, d, channel, particles, dt, nsteps, ckpt_every)


# ---------------------------------------------------------------- convenience

class Channel:
    """One channel context: grid, gas field, parameters and workspaces."""

    def __init__(self, nx, ny, nz, lx, lz, y_faces, params: Params, u_lattice=None,
                 max_particles: int = 0, stream=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.lx, self.lz = float(lx), float(lz)
        self.y_faces = np.asarray(y_faces, np.float64)
        self.params = params
        self.ctx = tribo_init(nx, ny, nz, lx, lz, self.y_faces, params, u_lattice, max_particles, stream)

    def step(self, particles: Particles, dt: float, nsteps: int = 1) -> None:
        tribo_step(self.ctx, particles, dt, nsteps)

    def set_fluid(self, u_lattice) -> None:
        tribo_set_fluid(self.ctx, u_lattice)

    def adjoint(self, particles: Particles, dt: float, nsteps: int, ckpt_every: int = 50, want_dd: bool = True):
        """(J, dJ/dU_c, dJ/dkappa_A, dJ/dd per particle or None); advances the particles."""
        import torch
        dd = torch.empty(particles.n, dtype=torch.float64, device="cuda") if want_dd else None
        J, dU, dK = tribo_adjoint(self.ctx, particles, dt, nsteps, ckpt_every, dd)
        return J, dU, dK, dd

    def set_modes(self, modes, ubar=None, damp=None, t0: float = 0.0) -> None:
        tribo_set_modes(self.ctx, modes, ubar, damp, t0)

    def eval_modes(self, t: float):
        """Mode field at time t as planes (3, Nz, Ny+2, Nx) on the device."""
        import torch
        rdt = torch.float64 if self.params.precision == _abi.TRIBO_FP64 else torch.float32
        u = torch.empty((3, self.nz, self.ny + 2, self.nx), dtype=rdt, device="cuda")
        tribo_eval_modes(self.ctx, t, u)
        return u

    def set_ssm(self, ssm) -> None:
        tribo_set_ssm(self.ctx, ssm)

    def momentum_source(self, on: bool = True):
        """Allocate (or drop, on=False) the planes F_s (3, Nz, Ny, Nx) of the
        particles' momentum source on the gas; every step() overwrites them
        with the mean over its steps.  Returns the tensor (or None)."""
        import torch
        if not on:
            tribo_set_momentum_source(self.ctx, None)
            self.F_s = None
            return None
        rdt = torch.float64 if self.params.precision == _abi.TRIBO_FP64 else torch.float32
        self.F_s = torch.zeros((3, self.nz, self.ny, self.nx), dtype=rdt, device="cuda")
        tribo_set_momentum_source(self.ctx, self.F_s)
        return self.F_s

    def set_params(self, params: Params) -> None:
        tribo_set_params(self.ctx, params)
        self.params = params

    def poisson(self, rho, want_phi: bool = False):
        import torch
        rdt = torch.float64 if self.params.precision == _abi.TRIBO_FP64 else torch.float32
        E = torch.empty((3, self.nz, self.ny + 2, self.nx), dtype=rdt, device=rho.device)
        phi = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float64, device=rho.device) if want_phi else None
        tribo_poisson(self.ctx, rho, phi, E)
        return phi, E

    def stats(self, particles: Optional[Particles] = None) -> dict:
        return tribo_stats(self.ctx, particles, self.ny)

    def reset_stats(self) -> None:
        tribo_reset_stats(self.ctx)

    def sync(self) -> None:
        tribo_sync(self.ctx)

    @property
    def error_bits(self) -> int:
        return tribo_error_bits(self.ctx)

    @property
    def launches(self) -> int:
        return tribo_launch_count(self.ctx)

    def close(self) -> None:
        if self.ctx:
            tribo_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
