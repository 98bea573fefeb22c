"""Gradient of the mean particle charge after N coupled steps (FP64, CPU).

Part of the FP64 CPU oracle: test infrastructure only.

J = (1/n) sum_p q_p(T) is the mean charge the charging-rate statistics of
Sec. 4.1 are built on.  Its derivatives with respect to the condenser model's
contact potential U_c and contact-area factor kappa_A (Sec. 2.3.1) and each
particle's diameter d_p are those of the step map of `oracle.particles.step`
with every discrete decision (cell index, interpolation stencil, wall
contact) held at its forward value: the map is piecewise smooth and this is
its derivative inside the piece.

The step is restated here with PyTorch CPU tensors in FP64, in the order and
notation of `oracle.particles.step`, `oracle.poisson` and `oracle.grid`, and
torch.autograd (a library primitive) differentiates it.  The restatement is
pinned to the numpy oracle's forward values and its gradient to central
differences of the numpy oracle, closed forms and linearity.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .constants import DRAG_OFF, DRAG_SCHILLER_NAUMANN, DRAG_STOKES, IMPACT_NORMAL, Params
from .grid import Grid, locate
from .poisson import modified_wavenumbers, y_coefficients

_F = torch.float64


def _t(a) -> torch.Tensor:
    return torch.as_tensor(np.asarray(a, np.float64), dtype=_F)


def _trilinear(g: Grid, lat: torch.Tensor, x, y, z) -> torch.Tensor:
    """Trilinear interpolation (oracle.grid.trilinear) with the stencil held fixed."""
    sx = x / g.dx - 0.5
    i0f = torch.floor(sx.detach())
    wx = sx - i0f
    i0 = i0f.long() % g.nx
    i1 = (i0 + 1) % g.nx
    sz = z / g.dz - 0.5
    k0f = torch.floor(sz.detach())
    wz = sz - k0f
    k0 = k0f.long() % g.nz
    k1 = (k0 + 1) % g.nz
    j0n = np.clip(np.searchsorted(g.Y, y.detach().numpy(), side="right") - 1, 0, g.ny)
    j0 = torch.as_tensor(j0n, dtype=torch.long)
    j1 = j0 + 1
    Y = _t(g.Y)
    wy = (y - Y[j0]) / (Y[j1] - Y[j0])
    out = torch.zeros((x.shape[0], lat.shape[-1]), dtype=_F)
    for kk, fz in ((k0, 1.0 - wz), (k1, wz)):
        for jj, fy in ((j0, 1.0 - wy), (j1, wy)):
            for ii, fx in ((i0, 1.0 - wx), (i1, wx)):
                out = out + (fz * fy * fx)[:, None] * lat[kk, jj, ii, :]
    return out


def _deposit(g: Grid, q: torch.Tensor, i, j, k) -> torch.Tensor:
    key = torch.as_tensor((np.asarray(k) * g.ny + np.asarray(j)) * g.nx + np.asarray(i), dtype=torch.long)
    Q = torch.zeros(g.ncells, dtype=_F).index_add(0, key, q)
    return Q.reshape(g.nz, g.ny, g.nx) / _t(g.vol_y)[None, :, None]


def _poisson(g: Grid, rho: torch.Tensor, eps: float) -> torch.Tensor:
    """oracle.poisson.poisson: DFT in x, z; Thomas sweep per pencil in y."""
    rhs = -rho / eps
    spec = torch.fft.fft(torch.fft.fft(rhs.to(torch.complex128), dim=2), dim=0)   # (mz, j, mx)
    lam = _t(modified_wavenumbers(g.nz, g.dz)[:, None] + modified_wavenumbers(g.nx, g.dx)[None, :])
    a, b, c = (_t(v) for v in y_coefficients(g))
    n = g.ny
    cp, dp = [], []
    den = b[0] - lam
    cp.append(c[0] / den)
    dp.append(spec[:, 0, :] / den)
    for j in range(1, n):
        den = b[j] - lam - a[j] * cp[j - 1]
        cp.append(c[j] / den)
        dp.append((spec[:, j, :] - a[j] * dp[j - 1]) / den)
    sol = [None] * n
    sol[n - 1] = dp[n - 1]
    for j in range(n - 2, -1, -1):
        sol[j] = dp[j] - cp[j] * sol[j + 1]
    s = torch.stack(sol, dim=1)
    return torch.fft.ifft(torch.fft.ifft(s, dim=0), dim=2).real


def _efield(g: Grid, phi: torch.Tensor) -> torch.Tensor:
    """oracle.poisson.efield: E = -grad(phi) on the wall-extended lattice."""
    nz, ny, nx = phi.shape
    zrow = torch.zeros((nz, 1, nx), dtype=_F)
    ex = -(torch.roll(phi, -1, dims=2) - torch.roll(phi, 1, dims=2)) / (2 * g.dx)
    ez = -(torch.roll(phi, -1, dims=0) - torch.roll(phi, 1, dims=0)) / (2 * g.dz)
    wgt = _t((g.yf[1:-1] - g.yc[:-1]) / (g.yc[1:] - g.yc[:-1]))
    inner = phi[:, :-1, :] + wgt[None, :, None] * (phi[:, 1:, :] - phi[:, :-1, :])
    phif = torch.cat([zrow, inner, zrow], dim=1)
    ey = -(phif[:, 1:, :] - phif[:, :-1, :]) / _t(g.dy)[None, :, None]
    ey0 = -(phi[:, :1, :] - 0.0) / (g.yc[0] - g.yf[0])
    eyn = -(0.0 - phi[:, -1:, :]) / (g.yf[-1] - g.yc[-1])
    Ex = torch.cat([zrow, ex, zrow], dim=1)
    Ey = torch.cat([ey0, ey, eyn], dim=1)
    Ez = torch.cat([zrow, ez, zrow], dim=1)
    return torch.stack([Ex, Ey, Ez], dim=-1)


def _phi12(s: torch.Tensor):
    phi1 = -torch.expm1(-s)
    small = s < 0.5
    ss = torch.where(small, s, torch.zeros_like(s))
    acc = torch.zeros_like(ss)
    pw = ss * ss
    for n in range(2, 23):
        acc = acc + pw * (((-1.0) ** n) / float(math.factorial(n)))
        pw = pw * ss
    return phi1, torch.where(small, acc, s - phi1)


def _relaxation_time(p: Params, d, rel):
    tau_p = p.rho_p * d ** 2 / (18.0 * p.rho * p.nu)
    if p.drag_law == DRAG_STOKES:
        return tau_p
    re_p = rel * d / p.nu
    pos = re_p > 0
    re_s = torch.where(pos, re_p, torch.ones_like(re_p))
    cd = torch.where(re_s <= 1000.0, 24.0 / re_s * (1.0 + re_s ** (2.0 / 3.0) / 6.0),
                     torch.full_like(re_s, 0.424))
    inv_tau = 0.75 * p.rho * p.nu * cd * re_s / (p.rho_p * d ** 2)
    return torch.where(pos, 1.0 / inv_tau, tau_p)


def _condenser(p: Params, U_c, kappa_A, d, speed, q, dq_t: bool):
    """oracle.particles.condenser_wall with U_c and kappa_A as tensors."""
    r = 0.5 * d
    elastic = (1.0 - p.mu_p ** 2) / p.E_p + (1.0 - p.mu_w ** 2) / p.E_w
    alpha = r * (0.625 * math.pi * p.rho_p * (1.0 + p.k_e) * speed ** 2 * elastic) ** 0.4
    A = kappa_A * math.pi * r * alpha
    C = p.eps * A / p.h
    dt_w = 2.94 * alpha / speed
    T_w = p.eps_w * p.eps0 * p.phi_p
    dq = -C * U_c * (-torch.expm1(-dt_w / T_w))
    if dq_t:
        dq = dq - (A / (math.pi * d ** 2)) * q
    return dq


def _step(g: Grid, p: Params, U_c, kappa_A, x, y, z, v, q, d, u_lat: torch.Tensor, dt: float):
    """One step of oracle.particles.step on tensors; returns the new state and hits."""
    n = x.shape[0]
    uf = _trilinear(g, u_lat, x, y, z)
    if p.electrostatics:
        i, j, k = locate(g, x.detach().numpy(), y.detach().numpy(), z.detach().numpy())
        rho = _deposit(g, q, i, j, k)
        E = _efield(g, _poisson(g, rho, p.eps))
        Ep = _trilinear(g, E, x, y, z)
        mass = math.pi * d ** 3 * p.rho_p / 6.0
        acc = (q / mass)[:, None] * Ep
    else:
        acc = torch.zeros((n, 3), dtype=_F)
    X = torch.stack([x, y, z], dim=1)
    if p.drag_law == DRAG_OFF:
        Xn = X + v * dt + 0.5 * acc * dt * dt
        Vn = v + acc * dt
    else:
        rel = torch.linalg.norm(v - uf, dim=1)
        tau = _relaxation_time(p, d, rel)
        s = dt / tau
        phi1, phi2 = _phi12(s)
        term = uf + acc * tau[:, None]
        Vn = v + (term - v) * phi1[:, None]
        Xn = X + tau[:, None] * (v * phi1[:, None] + term * phi2[:, None])

    def wrap(s_, L):
        w = s_ - L * torch.floor((s_ / L).detach())
        return torch.where(w.detach() >= L, w - L, w)

    xn = wrap(Xn[:, 0], g.lx)
    zn = wrap(Xn[:, 2], g.lz)
    r = 0.5 * d
    yv = Xn[:, 1]
    lo = (yv < r).detach()
    hi = (yv > g.ly - r).detach()
    yn = torch.where(lo, 2.0 * r - yv, torch.where(hi, 2.0 * (g.ly - r) - yv, yv))
    hit = lo | hi
    vy = torch.where(hit, -Vn[:, 1], Vn[:, 1])
    Vn = torch.stack([Vn[:, 0], vy, Vn[:, 2]], dim=1)
    if p.impact_vel == IMPACT_NORMAL:
        speed = torch.abs(Vn[:, 1])
    else:
        speed = torch.linalg.norm(Vn, dim=1)
    live = hit & (speed.detach() > 0)
    sp = torch.where(live, speed, torch.ones_like(speed))
    dq = _condenser(p, U_c, kappa_A, d, sp, q, bool(p.dq_t))
    qn = q + torch.where(live, dq, torch.zeros_like(dq))
    return xn, yn, zn, Vn, qn, hit


def mean_charge_gradient(g: Grid, p: Params, st, u_lat, dt: float, nsteps: int):
    """J = mean charge after nsteps and (dJ/dU_c, dJ/dkappa_A, dJ/dd_p).

    st: oracle State (the initial ensemble); u_lat: lattice (Nz, Ny+2, Nx, 3)
    or a callable t -> lattice (field at step n is u_lat(n dt)).
    Returns dict(J, dU_c, dkappa_A, dd, final) with `final` a dict of the
    forward end state (x, y, z, vx, vy, vz, q, n_imp) as numpy arrays.
    """
    U_c = torch.tensor(float(p.U_c), dtype=_F, requires_grad=True)
    kappa_A = torch.tensor(float(p.kappa_A), dtype=_F, requires_grad=True)
    d = _t(st.d).requires_grad_(True)
    x, y, z = _t(st.x), _t(st.y), _t(st.z)
    v = torch.stack([_t(st.vx), _t(st.vy), _t(st.vz)], dim=1)
    q = _t(st.q)
    n_imp = np.array(st.n_imp, np.int64)
    for s in range(nsteps):
        lat = u_lat(s * dt) if callable(u_lat) else u_lat
        x, y, z, v, q, hit = _step(g, p, U_c, kappa_A, x, y, z, v, q, d, _t(lat), dt)
        n_imp += hit.numpy().astype(np.int64)
    J = q.mean()
    gU, gK, gd = torch.autograd.grad(J, (U_c, kappa_A, d), allow_unused=True)
    zero = lambda t_, like: torch.zeros_like(like) if t_ is None else t_
    final = dict(x=x.detach().numpy(), y=y.detach().numpy(), z=z.detach().numpy(),
                 vx=v[:, 0].detach().numpy(), vy=v[:, 1].detach().numpy(), vz=v[:, 2].detach().numpy(),
                 q=q.detach().numpy(), n_imp=n_imp)
    return dict(J=float(J.detach()), dU_c=float(zero(gU, U_c)), dkappa_A=float(zero(gK, kappa_A)),
                dd=zero(gd, d).numpy().copy(), final=final)
