"""Benchmark: coupled particle steps of the Re_tau = 550 channel workload.

One step = deposit -> Poisson (FFT x,z + FP64 tridiagonal y) -> E -> gather
-> drag + q E / m integration -> wall impacts with condenser charging, for all
particles of one channel (384 x 256 x 256 grid, 8M particles, mixed precision).

Prints ONE JSON line.  --impl reference times the FP64 CPU oracle instead
(on the host cores, a bounded sample of the same workload).  Multi-GPU runs
(torchrun) advance one independent channel per rank (replicas; no collective
on the data path) and report the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "particle-steps/s"
WORKLOAD = "re550_384"
# algorithmic bytes of the particle kernel per launch (mixed precision):
PARTICLE_BYTES = 72      # per particle: state read (7 x f32 + q f64), state write (6 x f32), deposit
NODE_BYTES = 24          # per lattice node the gather touches: u (3 x f32) + E (3 x f32)
CELL_BYTES = 8           # per cell: the FP64 charge sum the deposit accumulates into
NOMINAL_HBM_GBS = 7900.0  # HBM3e nominal bandwidth of the GPU (context beside the measured copy peak)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device):
    """Largest value of x over all ranks of the process group (x on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, steps, seconds_max, world):
    """Whole-job throughput of replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank * steps / seconds_max


def shard(items, rank, world):
    """The share of independent work items (channels) that one rank takes."""
    return list(items)[rank::world]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_traffic(kernel, workload=WORKLOAD, alg_bytes=None):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, or None
    when the kernel's sources changed after the counters were taken.  A summary
    taken on a smaller case than the bench's records its algorithmic bytes; its
    traffic is then scaled to the bench's launch by the ratio of the
    algorithmic bytes (`alg_bytes`)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    m = re.search(r"<!-- traffic: (\{.*\}) -->", open(path).read())
    if not m:
        return None
    info = json.loads(m.group(1))
    h = hashlib.sha256()
    for f in info["files"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != info["source_hash"]:
        return None
    if info.get("alg_bytes_per_launch") and alg_bytes:
        return info["bytes_per_launch"] * alg_bytes / info["alg_bytes_per_launch"]
    return info["bytes_per_launch"]


def touched_nodes(c, faces, x, y, z):
    """Distinct lattice nodes the trilinear gather touches (host count)."""
    nx, ny, nz = c.nx, c.ny, c.nz
    Y = synth.node_y(faces)
    dx, dz = c.lx / nx, c.lz / nz
    i0 = np.floor(x / dx - 0.5).astype(np.int64) % nx
    k0 = np.floor(z / dz - 0.5).astype(np.int64) % nz
    j0 = np.clip(np.searchsorted(Y, y, side="right") - 1, 0, ny)
    mark = np.zeros(nz * (ny + 2) * nx, dtype=bool)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                mark[(((k0 + dk) % nz) * (ny + 2) + j0 + dj) * nx + (i0 + di) % nx] = True
    return int(mark.sum())


def make_inputs(c, n=None):
    faces = synth.y_faces(c.ny, c.delta, c.gamma)
    lat = synth.fluid_lattice(c, faces=faces).astype(np.float32)
    P = synth.draw_particles(c, n)
    return faces, lat, P


def oracle_step_time(c, faces, lat, P, n_sample):
    """Time one oracle step: the full-grid Poisson + a particle sample."""
    import oracle
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    p = oracle.Params(rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0)
    sel = slice(0, n_sample)
    st = oracle.State.from_arrays(P.x[sel], P.y[sel], P.z[sel], P.vx[sel], P.vy[sel], P.vz[sel],
                                  P.q[sel], P.d[sel])
    lat64 = lat.astype(np.float64)
    # the deposit of the full ensemble feeds the Poisson solve
    t0 = time.perf_counter()
    i, j, k = oracle.locate(g, P.x, P.y, P.z)
    rho = oracle.deposit(g, P.q, i, j, k)
    phi = oracle.poisson(g, rho, p.eps)
    oracle.efield(g, phi)
    t_field = time.perf_counter() - t0
    t1 = time.perf_counter()
    oracle.step(g, p.with_(electrostatics=False), st, lat64, c.dt)
    t_part = time.perf_counter() - t1
    # the per-particle gather of E (skipped in the electrostatics-off step) is one
    # more trilinear call; time it on the sample too
    t2 = time.perf_counter()
    oracle.trilinear(g, np.zeros((c.nz, c.ny + 2, c.nx, 3)), st.x, st.y, st.z)
    t_part += time.perf_counter() - t2
    return t_field, t_part


def adjoint_report(T, torch, steps=None, ckpt=50, h=1e-4):
    """Adjoint of the mean charge on the differentiation workload (Re_tau 180,
    128^3, 1M particles, 500 steps, a state kept every `ckpt` steps): forward
    and adjoint wall time, central differences with relative step h (and the
    fraction of particles whose impact count differs between +h and -h), and
    the mixed-precision gradients against the FP64 GPU path."""
    c = synth.case("re180_128_adj")
    nsteps = c.steps if steps is None else steps
    faces, lat, P = make_inputs(c)
    parts = dict(x=P.x, y=P.y, z=P.z, vx=P.vx, vy=P.vy, vz=P.vz, d=P.d, q=P.q)
    # the ensemble in cell order, as a simulation that sorts its particles holds it (neither the
    # forward call nor the adjoint re-sorts here)
    ix = np.floor(np.asarray(P.x) / (c.lx / c.nx)).astype(np.int64) % c.nx
    iz = np.floor(np.asarray(P.z) / (c.lz / c.nz)).astype(np.int64) % c.nz
    jy = np.clip(np.searchsorted(faces, np.asarray(P.y), side="right") - 1, 0, c.ny - 1)
    order = np.argsort((iz * c.ny + jy) * c.nx + ix, kind="stable")
    parts = {k: np.asarray(v)[order] for k, v in parts.items()}
    base = dict(rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0)

    def channel(prec):
        real = np.float32 if prec == T.TRIBO_MIXED else np.float64
        u = torch.from_numpy(np.ascontiguousarray(lat.astype(real))).cuda()
        return T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, T.Params(precision=prec, **base), u,
                         max_particles=c.n_particles)

    def fresh(prec, d_scale=1.0):
        q = dict(parts)
        q["d"] = parts["d"] * d_scale
        return T.Particles.from_numpy(q, prec, device="cuda")

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    mixed = channel(T.TRIBO_MIXED)
    mixed.step(fresh(T.TRIBO_MIXED), c.dt, 20)
    Pf = fresh(T.TRIBO_MIXED)
    _, fwd_ms = timed(lambda: mixed.step(Pf, c.dt, nsteps))
    mixed.adjoint(fresh(T.TRIBO_MIXED), c.dt, nsteps, ckpt)          # workspace allocation
    Pa = fresh(T.TRIBO_MIXED)
    (J, dU, dK, dd), adj_ms = timed(lambda: mixed.adjoint(Pa, c.dt, nsteps, ckpt))
    dd = dd.cpu().numpy()
    n_imp = int(Pa.to_numpy()["n_imp"].astype(np.int64).sum())

    def J_of(d_scale=1.0, **kw):
        mixed.set_params(T.Params(precision=T.TRIBO_MIXED, **{**base, **kw}))
        Pq = fresh(T.TRIBO_MIXED, d_scale)
        mixed.step(Pq, c.dt, nsteps)
        out = Pq.to_numpy()
        return out["q"].copy(), out["n_imp"].astype(np.int64)

    n = c.n_particles

    def central(plus, minus, step, per_particle=None):
        """Central difference of J; also restricted to the particles whose
        impact count is the same at +h and -h (a flip is a jump of J, not a
        derivative), against the adjoint's per-particle terms on that set."""
        (qp, ip), (qm, im) = plus, minus
        same = ip == im
        out = {"fd": float((qp.mean() - qm.mean()) / (2 * step)), "flip_frac": float(1.0 - same.mean())}
        if per_particle is not None:
            out["fd_same_impacts"] = float((qp[same] - qm[same]).sum() / n / (2 * step))
            out["adjoint_same_impacts"] = float(per_particle[same].sum())
        return out

    d32 = parts["d"].astype(np.float32).astype(np.float64)
    cU = central(J_of(U_c=1.0 + h), J_of(U_c=1.0 - h), h)
    cK = central(J_of(kappa_A=1.0 + h), J_of(kappa_A=1.0 - h), h)
    cD = central(J_of(d_scale=1.0 + h), J_of(d_scale=1.0 - h), h, per_particle=dd * d32)
    adjD = float(np.dot(dd, d32))
    mixed.close()

    fp64 = channel(T.TRIBO_FP64)
    fp64.adjoint(fresh(T.TRIBO_FP64), c.dt, nsteps, ckpt)
    P64 = fresh(T.TRIBO_FP64)
    (J64, dU64, dK64, dd64), adj64_ms = timed(lambda: fp64.adjoint(P64, c.dt, nsteps, ckpt))
    dd64 = dd64.cpu().numpy()
    fin32, fin64 = Pa.to_numpy(), P64.to_numpy()

    # Per-particle central differences in d on the FP64 path.  Changing every diameter at once
    # moves many particles across cell faces, and the NGP deposit jumps there: the difference
    # quotient of J then carries those jumps of the field, which the derivative with the cells
    # held (the adjoint) does not.  Changing only the diameters of the particles that hit a wall
    # (the only ones whose charge, and so whose term of dJ/dd, moves; 0.07% of the ensemble)
    # makes those jumps rare, and each such particle's own charge difference is its term of
    # dJ/dd (the others' charges move only through the field, second order).
    rel = lambda a, b: abs(a - b) / max(abs(b), 1e-300)
    d64 = np.asarray(parts["d"], np.float64)
    sel = np.nonzero(fin64["n_imp"] > 0)[0]

    def q64_of(sign, hh):
        q = dict(parts)
        dd_ = d64.copy()
        dd_[sel] *= 1.0 + sign * hh
        q["d"] = dd_
        Pq = T.Particles.from_numpy(q, T.TRIBO_FP64, device="cuda")
        fp64.step(Pq, c.dt, nsteps)
        out = Pq.to_numpy()
        return out["q"].copy(), out["n_imp"].astype(np.int64)

    adj64_p = (dd64 * d64)[sel]
    adj32_p = (dd * d32)[sel]

    def per_particle_fd(hh, fd_other=None):
        (qp, ip), (qm, im) = q64_of(+1, hh), q64_of(-1, hh)
        fd_p = (qp[sel] - qm[sel]) / (2 * hh * n)
        keep = (ip[sel] == im[sel]) & (dd64[sel] != 0)
        smooth = None
        if fd_other is not None:
            # the map is smooth at a particle where the differences at two steps h agree
            # (a jump between -h and +h makes the difference quotient scale with 1/h)
            smooth = keep & (np.abs(fd_p - fd_other) <= 1e-3 * np.abs(fd_other))
        r64 = np.abs(fd_p - adj64_p)[keep] / np.abs(adj64_p)[keep]
        r32 = np.abs(fd_p - adj32_p)[keep] / np.abs(fd_p)[keep].clip(1e-300)
        q_ = lambda r, x: float(np.percentile(r, x)) if r.size else None
        return {"h_rel": hh, "particles": int(keep.sum()), "flips": int((ip[sel] != im[sel]).sum()),
                "fp64_adjoint_rel_err": {"median": q_(r64, 50), "p90": q_(r64, 90), "p99": q_(r64, 99),
                                         "max": q_(r64, 100),
                                         "frac_within_1e-6": float((r64 <= 1e-6).mean()) if r64.size else None,
                                         "frac_within_1e-3": float((r64 <= 1e-3).mean()) if r64.size else None},
                "mixed_adjoint_rel_err": {"median": q_(r32, 50), "p90": q_(r32, 90), "p99": q_(r32, 99),
                                          "frac_within_1e-3": float((r32 <= 1e-3).mean()) if r32.size else None},
                "sum_rel_err_fp64": rel(float(adj64_p[keep].sum()), float(fd_p[keep].sum())) if keep.any() else None,
                **({} if smooth is None else {
                    "smooth_particles": int(smooth.sum()),
                    "sum_rel_err_fp64_smooth": rel(float(adj64_p[smooth].sum()), float(fd_p[smooth].sum()))
                    if smooth.any() else None,
                    "sum_rel_err_mixed_smooth": rel(float(adj32_p[smooth].sum()), float(fd_p[smooth].sum()))
                    if smooth.any() else None}), "_fd": fd_p}

    fd_particles = {
        "note": ("FP64 GPU path, the diameters of the particles that hit a wall changed by +-h; each such "
                 "particle's charge difference against its adjoint term dJ/dd_p d_p (those with the same "
                 "impact count at +h and -h).  The few that differ by O(1) cross a cell face or change the "
                 "step of an impact between -h and +h (a jump of the map, not of its derivative); their "
                 "share falls with h"),
        "smooth": ("h_1e-6 also sums over the particles whose differences at h = 1e-4 and 1e-6 agree "
                   "to 1e-3 (no jump of the map between -h and +h at either step)")}
    fd_particles["h_1e-4"] = per_particle_fd(h)
    fd_particles["h_1e-6"] = per_particle_fd(1e-6, fd_other=fd_particles["h_1e-4"]["_fd"])
    for k_ in ("h_1e-4", "h_1e-6"):
        del fd_particles[k_]["_fd"]
    fp64.close()
    match = fin32["n_imp"] == fin64["n_imp"]
    return {
        "workload": workload_desc(c) + f", {nsteps} steps, state kept every {ckpt}",
        "fwd_ms": fwd_ms, "adjoint_ms": adj_ms, "adjoint_over_fwd": adj_ms / fwd_ms,
        "J": J, "dJ_dUc": dU, "dJ_dkappaA": dK, "sum_d_dJ_dd": adjD, "impacts": n_imp,
        "central_differences": {
            "h_rel": h,
            "dJ_dUc": cU["fd"], "rel_err_Uc": rel(dU, cU["fd"]), "flip_frac_Uc": cU["flip_frac"],
            "dJ_dkappaA": cK["fd"], "rel_err_kappaA": rel(dK, cK["fd"]), "flip_frac_kappaA": cK["flip_frac"],
            "dJ_dlogd": cD["fd"], "flip_frac_d": cD["flip_frac"],
            "dJ_dlogd_same_impacts": cD["fd_same_impacts"],
            "adjoint_dJ_dlogd_same_impacts": cD["adjoint_same_impacts"],
            "rel_err_d_same_impacts": rel(cD["adjoint_same_impacts"], cD["fd_same_impacts"]),
            "d_per_particle": fd_particles},
        "vs_fp64_gpu": {
            "adjoint_ms_fp64": adj64_ms,
            "impact_count_mismatch_frac": float(1.0 - match.mean()),
            "rel_err_J": rel(J, J64),
            "rel_err_J_matched": rel(fin32["q"][match].sum(), fin64["q"][match].sum()),
            "rel_err_Uc": rel(dU, dU64), "rel_err_kappaA": rel(dK, dK64),
            "rel_err_dd_matched_max": float(np.abs(dd - dd64)[match].max() / np.abs(dd64[match]).max())},
    }


def per_particle_errors(a, b, lx, ly, lz, sel=None):
    """Errors of state `a` against reference state `b` (dicts of arrays in
    the same particle order) under the per-particle reading of the parity
    bar: positions per coordinate against the box extent (x, z periodic),
    the velocity vector against the particle's speed, the charge q and the
    received wall charge q_wall against the particle's charge scale
    max(|q|, |q_wall|, |q - q_wall|) (final, received, initial charge).
    Largest value and 99th percentile of each."""
    if sel is None:
        sel = slice(None)
    f = lambda k, src: np.asarray(src[k], np.float64)[sel]
    out = {}

    def put(name, r):
        r = np.asarray(r, np.float64)
        out[name] = {"max": float(r.max()) if r.size else 0.0,
                     "p99": float(np.percentile(r, 99)) if r.size else 0.0}

    for k, L in (("x", lx), ("y", ly), ("z", lz)):
        d = f(k, a) - f(k, b)
        if k != "y":
            d = (d + 0.5 * L) % L - 0.5 * L
        put(k, np.abs(d) / L)
    dv = np.sqrt(sum((f(k, a) - f(k, b)) ** 2 for k in ("vx", "vy", "vz")))
    sp = np.sqrt(sum(f(k, b) ** 2 for k in ("vx", "vy", "vz")))
    put("v", dv / np.maximum(sp, 1e-300))
    qs = np.maximum(np.maximum(np.abs(f("q", b)), np.abs(f("q_wall", b))), np.abs(f("q", b) - f("q_wall", b)))
    for k in ("q", "q_wall"):
        dq = np.abs(f(k, a) - f(k, b))
        put(k, np.where(qs > 0, dq / np.where(qs > 0, qs, 1.0), np.where(dq > 0, np.inf, 0.0)))
    return out


def fp64_report(T, torch, c, faces, lat, P, steps=10, sort_every=20):
    """The mixed-precision path against the plain FP64 GPU path on the full
    workload: both start from the same state (the FP32-rounded inputs, which
    FP64 holds exactly) and take `steps` coupled steps.  Per output, the
    per-particle errors of the parity bar's reading (per_particle_errors,
    all particles matched by id), beside each velocity component's largest
    difference against its largest FP64 magnitude; the fractions of
    particles whose cell or impact count differ; the FP64 path's time per
    step."""
    parts = dict(x=P.x, y=P.y, z=P.z, vx=P.vx, vy=P.vy, vz=P.vz, d=P.d, q=P.q)
    out, ms = {}, {}
    for prec in (T.TRIBO_MIXED, T.TRIBO_FP64):
        real = np.float32 if prec == T.TRIBO_MIXED else np.float64
        params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0, sort_every=sort_every)
        ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat.astype(real)).cuda(),
                       max_particles=c.n_particles)
        src = {k: (v if k == "q" else np.asarray(v).astype(np.float32).astype(real)) for k, v in parts.items()}
        Pd = T.Particles.from_numpy(src, prec, device="cuda", with_cell=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ch.step(Pd, c.dt, steps)
        e1.record()
        ch.sync()
        torch.cuda.synchronize()
        ms[prec] = e0.elapsed_time(e1) / steps
        o = Pd.to_numpy()
        ch.close()
        del Pd
        order = np.argsort(o["id"])
        out[prec] = {k: np.asarray(v)[order] for k, v in o.items()}
    a, b = out[T.TRIBO_MIXED], out[T.TRIBO_FP64]
    same = a["n_imp"] == b["n_imp"]

    def comp_max(k, q=None):
        d = np.abs(a[k].astype(np.float64) - b[k])
        return float((d.max() if q is None else np.percentile(d, q)) / max(np.abs(b[k]).max(), 1e-300))

    return {"steps": steps, "particles": int(len(b["x"])), "fp64_ms_per_step": ms[T.TRIBO_FP64],
            "mixed_ms_per_step": ms[T.TRIBO_MIXED],
            "reading": ("per particle: positions per coordinate against the box extent, the velocity vector "
                        "against the particle's speed, q and q_wall against the particle's charge scale "
                        "max(|q|, |q_wall|, |q - q_wall|)"),
            "rel_err": per_particle_errors(a, b, c.lx, c.ly, c.lz, sel=same),
            "rel_err_component_max": {k: comp_max(k) for k in ("vx", "vy", "vz")},
            "rel_err_component_max_p99": {k: comp_max(k, 99) for k in ("vx", "vy", "vz")},
            "max_abs_fp64": {k: float(np.abs(b[k]).max()) for k in ("vx", "vy", "vz")},
            "note": ("rel_err_component_max divides each velocity component's largest difference by that "
                     "component's largest FP64 magnitude (not the declared reading): v_y and v_z start at 0 "
                     "and stay small against v_x over 10 steps, so there they show the FP32 position "
                     "resolution (2.3e-5 of a cell at x = L_x) rather than the step's arithmetic"),
            "impact_mismatch_frac": float(1.0 - same.mean()),
            "cell_mismatch_frac": float((a["cell"] != b["cell"]).mean()),
            "impacts_fp64": int(b["n_imp"].sum())}


def oracle_subsample_report(T, torch, c, faces, lat, state, every=1000):
    """The mixed GPU path against the FP64 oracle at full size on a 1-in-
    `every` subsample: from the benchmark's own state after its timed steps
    (synth.replay_state: Gaussian charges, half of the subsample moving into
    a wall), the GPU takes one coupled step with all particles; the oracle
    deposits all particles' charges (FP64), solves the full-grid Poisson
    problem, and steps the subsample in that field.  Per output the
    per-particle errors (max and p99), cell and impact-count mismatches, and
    the field of the library's solve of the oracle's density against the
    oracle's field."""
    import oracle
    t0 = time.perf_counter()
    rs = synth.replay_state(c, state, sample_every=every, wall_every=2 * every)
    n = rs["x"].shape[0]
    params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0, sort_every=20)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(), max_particles=n)
    Pd = T.Particles.from_numpy({k: rs[k] for k in ("x", "y", "z", "vx", "vy", "vz", "d", "q")},
                                T.TRIBO_MIXED, device="cuda", with_cell=True)
    ch.step(Pd, c.dt, 1)
    ch.sync()
    o = Pd.to_numpy()
    order = np.argsort(o["id"])
    s1 = {k: np.asarray(v)[order] for k, v in o.items()}
    del Pd
    g = oracle.Grid(c.nx, c.nz, c.lx, c.lz, faces)
    f64 = lambda v: np.asarray(v, np.float64)
    i, j, k = oracle.locate(g, f64(rs["x"]), f64(rs["y"]), f64(rs["z"]))
    rho = oracle.deposit(g, rs["q"], i, j, k)
    E_ref = oracle.efield(g, oracle.poisson(g, rho, params.eps))
    _, E = ch.poisson(torch.from_numpy(rho).cuda())
    E = E.cpu().numpy()
    ch.close()
    field = {}
    for comp, name in enumerate(("Ex", "Ey", "Ez")):
        ref = E_ref[..., comp]
        field[name] = float(np.abs(E[comp].astype(np.float64) - ref).max() / np.abs(ref).max())
    del E, rho
    sel = np.arange(0, n, every)
    st = oracle.State.from_arrays(*(f64(rs[key][sel]) for key in ("x", "y", "z", "vx", "vy", "vz")),
                                  rs["q"][sel], f64(rs["d"][sel]))
    ref = oracle.step(g, oracle.Params(rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0), st, lat.astype(np.float64),
                      c.dt, E_lat=E_ref)
    del E_ref
    got = {key: s1[key][sel] for key in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall")}
    refd = {key: getattr(ref, key) for key in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall")}
    ii, jj, kk = oracle.locate(g, f64(got["x"]), f64(got["y"]), f64(got["z"]))
    i2, j2, k2 = oracle.locate(g, ref.x, ref.y, ref.z)
    return {"sample": f"{len(sel)} of {n} particles (every {every}th id), {int((sel % (2 * every) == 0).sum())} "
                      f"of them moving into a wall; one step from the benchmark's state",
            "reading": "per particle (see vs_fp64_gpu.reading)",
            "rel_err": per_particle_errors(got, refd, c.lx, c.ly, c.lz),
            "impacts_oracle": int(ref.n_imp.sum()),
            "impact_mismatch": int((s1["n_imp"][sel].astype(np.int64) != ref.n_imp).sum()),
            "cell_mismatch_vs_oracle_trajectory": int((g.cell_key(ii, jj, kk) != g.cell_key(i2, j2, k2)).sum()),
            "cell_vs_exact_locate_mismatch": int((s1["cell"][sel].astype(np.int64) != g.cell_key(ii, jj, kk)).sum()),
            "field_rel_err_vs_max": field,
            "seconds": time.perf_counter() - t0}


def batch_report(T, torch, steps=500, seq_steps=40, sort_every=20, rank=0, world=1, channels=64, scale=1.0,
                 timed_steps=40):
    """Batched ensemble of 64 independent channels (Re_tau in {180, 300, 395,
    550}, grids 64^3 to 192x128x128, 50k-2M particles each, d+ in [0.5, 3]):
    aggregate particle-steps/s of the batch (graph-captured steps, persistent
    particle kernel over all channels, autotuned shape) against the same
    channels stepped one after another with tribo_step.  With several ranks the
    channels are sharded over the ranks (independent problems, no exchange).
    The roofline of the batch particle kernel: per launch, every channel's
    particles x PARTICLE_BYTES + its touched lattice nodes (of the drawn
    positions) x NODE_BYTES + its cells x CELL_BYTES, over the kernel's mean
    event-timed duration in `timed_steps` further steps."""
    all_cases = synth.ensemble_cases(channels, scale=scale)
    cases = shard(all_cases, rank, world)
    chans, Ps, dts = [], [], []
    alg_bytes = 0                      # the batch particle kernel's algorithmic bytes per launch
    for c in cases:
        faces = synth.y_faces(c.ny, c.delta, c.gamma)
        params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0,
                          sort_every=sort_every)
        ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, None, max_particles=c.n_particles)
        Y = synth.node_y(faces)
        ch.set_modes(synth.draw_modes(c), synth.mean_velocity(Y, c), synth.damping(Y, c))
        T.tribo_eval_modes(ch.ctx, 0.0, None)          # frozen lattice from the device mode sum
        ch.set_modes(None)
        P = synth.draw_particles(c)
        alg_bytes += (c.n_particles * PARTICLE_BYTES + touched_nodes(c, faces, P.x, P.y, P.z) * NODE_BYTES
                      + c.nx * c.ny * c.nz * CELL_BYTES)
        Ps.append(T.Particles.from_numpy(dict(x=P.x, y=P.y, z=P.z, vx=P.vx, vy=P.vy, vz=P.vz, d=P.d, q=P.q),
                                         T.TRIBO_MIXED, device="cuda"))
        chans.append(ch)
        dts.append(c.dt)
    ntot = sum(c.n_particles for c in cases)
    B = T.Batch(chans, sort_every=sort_every)
    t0 = time.perf_counter()
    shape = B.autotune(Ps, dts)
    tune_s = time.perf_counter() - t0
    B.step(Ps, dts, 2 * sort_every)                  # graph capture and first replay
    B.sync()
    torch.cuda.synchronize()
    l0 = B.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    B.step(Ps, dts, steps)
    e1.record()
    torch.cuda.synchronize()
    B.sync()
    batch_ms = max_over_ranks(e0.elapsed_time(e1), "cuda")
    launches = B.launches - l0
    # the particle kernel alone: events around its launches (direct launches while timed)
    B.timing(True)
    B.step(Ps, dts, timed_steps)
    kern_ms, kern_n = B.kernel_time()
    B.timing(False)
    B.sync()
    kern_ms = max_over_ranks(kern_ms / max(kern_n, 1), "cuda")
    hbm_peak, peak_kind = measured_peaks()
    ach = alg_bytes / (kern_ms * 1e-3) / 1e9
    B.close()
    # the same channels one after another (tribo_step per channel)
    seq_ms = 0.0
    for ch, P, dt in zip(chans, Ps, dts):
        torch.cuda.synchronize()
        e0.record()
        ch.step(P, dt, seq_steps)
        e1.record()
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1)
    for ch in chans:
        ch.close()
    seq_ms = max_over_ranks(seq_ms, "cuda")
    check = batch_vs_fp64(T, torch, sorted(cases, key=lambda c: c.n_particles)[:2]) if rank == 0 else None
    ntot = sum(c.n_particles for c in all_cases)
    batch_rate = ntot * steps / (batch_ms * 1e-3)
    seq_rate = ntot * seq_steps / (seq_ms * 1e-3)
    return {"workload": (f"{channels} channels (synth.ensemble_cases): Re_tau in {{180,300,395,550}}, grids 64^3 to "
                         f"192x128x128, {ntot} particles in total, d+ in [0.5,3], sort every {sort_every}"),
            "steps": steps, "ms_per_step": batch_ms / steps, "particle_steps_per_s": batch_rate,
            "sequential_particle_steps_per_s": seq_rate, "sequential_steps": seq_steps,
            "speedup_vs_sequential": batch_rate / seq_rate, "autotuned_shape": shape, "autotune_s": tune_s,
            "kernels_per_step": launches / steps, "vs_fp64_gpu": check,
            "roofline": {"bound": "hbm", "kernel": "k_step_batch", "achieved": ach, "peak": hbm_peak,
                         "unit": "GB/s", "frac": ach / hbm_peak, "peak_kind": peak_kind,
                         "alg_bytes": alg_bytes, "ms_per_launch": kern_ms, "timed_launches": kern_n,
                         "traffic": measured_traffic("k_step_batch", "ensemble", alg_bytes)}}


def batch_vs_fp64(T, torch, cases, steps=10, sort_every=5):
    """Channels stepped together as one mixed-precision batch against each
    stepped alone on the plain FP64 GPU path, from the same FP32-rounded state:
    the per-particle errors of the declared reading (positions against the box
    extent, the velocity vector against the particle's speed, charges against
    the particle's charge scale) over the particles whose impact count agrees,
    the largest position and velocity differences relative to each quantity's
    largest FP64 magnitude, and the fraction of particles whose impact count
    differs, over all the channels' particles."""
    res = {"channels": [c.name for c in cases], "steps": steps}
    err = {k: 0.0 for k in ("x", "y", "z", "vx", "vy", "vz")}
    mism = n = 0
    outs = {T.TRIBO_MIXED: [], T.TRIBO_FP64: []}
    for prec in (T.TRIBO_MIXED, T.TRIBO_FP64):
        real = np.float32 if prec == T.TRIBO_MIXED else np.float64
        chans, Ps = [], []
        for c in cases:
            faces = synth.y_faces(c.ny, c.delta, c.gamma)
            lat = synth.fluid_lattice(c, faces=faces).astype(np.float32).astype(real)
            params = T.Params(precision=prec, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0, sort_every=sort_every)
            chans.append(T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(),
                                   max_particles=c.n_particles))
            P = synth.draw_particles(c)
            src = dict(x=P.x, y=P.y, z=P.z, vx=P.vx, vy=P.vy, vz=P.vz, d=P.d, q=P.q)
            Ps.append(T.Particles.from_numpy({k: (v if k == "q" else np.asarray(v).astype(np.float32).astype(real))
                                              for k, v in src.items()}, prec, device="cuda"))
        if prec == T.TRIBO_MIXED:
            B = T.Batch(chans, sort_every=sort_every)
            B.step(Ps, [c.dt for c in cases], steps)
            B.sync()
            B.close()
        else:
            for ch, P, c in zip(chans, Ps, cases):
                ch.step(P, c.dt, steps)
                ch.sync()
        for ch, P in zip(chans, Ps):
            o = P.to_numpy()
            order = np.argsort(o["id"])
            outs[prec].append({k: np.asarray(v)[order] for k, v in o.items()})
            ch.close()
    pp = {}
    for c, a, b in zip(cases, outs[T.TRIBO_MIXED], outs[T.TRIBO_FP64]):
        for k in err:
            d = a[k].astype(np.float64) - b[k]
            if k in ("x", "z"):
                L = c.lx if k == "x" else c.lz
                d = (d + 0.5 * L) % L - 0.5 * L
            err[k] = max(err[k], float(np.abs(d).max() / max(np.abs(b[k]).max(), 1e-300)))
        same = a["n_imp"] == b["n_imp"]
        for k, v in per_particle_errors(a, b, c.lx, c.ly, c.lz, sel=same).items():
            o = pp.setdefault(k, {"max": 0.0, "p99": 0.0})
            o["max"] = max(o["max"], v["max"])
            o["p99"] = max(o["p99"], v["p99"])
        mism += int((~same).sum())
        n += len(b["x"])
    res.update(reading="per particle, as vs_fp64_gpu.reading (p99: the largest of the channels' p99)",
               rel_err=pp, rel_err_component_max=err, impact_mismatch_frac=mism / max(n, 1), particles=n)
    return res


def timevarying_report(T, torch, steps=200, sort_every=20):
    """The 128^3 time-varying workload (Re_tau 180, 1M particles, d+ log-uniform
    in [0.5, 2], Gaussian initial charges): the gas field is re-evaluated from
    its 256 advected modes on the device before every step.  Reports
    particle-steps/s of the whole step and the per-kernel split, with the field
    evaluation (input generation) separate."""
    c = synth.case("re180_128")
    faces = synth.y_faces(c.ny, c.delta, c.gamma)
    params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0,
                      sort_every=sort_every)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, None, max_particles=c.n_particles)
    Y = synth.node_y(faces)
    ch.set_modes(synth.draw_modes(c), synth.mean_velocity(Y, c), synth.damping(Y, c), 0.0)
    P = synth.draw_particles(c)
    Pd = T.Particles.from_numpy(dict(x=P.x, y=P.y, z=P.z, vx=P.vx, vy=P.vy, vz=P.vz, d=P.d, q=P.q),
                                T.TRIBO_MIXED, device="cuda")
    ch.step(Pd, c.dt, 5)
    torch.cuda.synchronize()
    T.tribo_timing_enable(ch.ctx, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ch.step(Pd, c.dt, steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ph = T.tribo_timing_read(ch.ctx)
    T.tribo_timing_enable(ch.ctx, False)
    ch.sync()
    ch.close()
    per = {k: v[0] / steps for k, v in ph.items() if v[1]}
    field = per.get("fluid_modes", 0.0)
    poisson = sum(v for k, v in per.items() if k.startswith("poisson"))
    return {"workload": workload_desc(c) + ", time-varying field (256 advected modes, evaluated every step)",
            "steps": steps, "ms_per_step": ms / steps, "particle_steps_per_s": c.n_particles * steps / (ms * 1e-3),
            "field_ms_per_step": field, "poisson_ms_per_step": poisson,
            "particle_step_ms": per.get("particle_step", 0.0),
            "particle_steps_per_s_without_field": c.n_particles * steps / ((ms - field * steps) * 1e-3),
            "poisson_solves_per_s": 1e3 / poisson if poisson > 0 else None}


def interactions_report(T, torch, steps=100, sort_every=20):
    """Cost of the particle-particle interactions (the in-cell Coulomb near
    field and the 4-way collisions), of the stochastic scaling model of wall
    charging and of the momentum source on the gas (2-way coupling) on the
    128^3 workload with 1M particles: ms per step with each switch against
    the plain coupled step."""
    c = synth.case("re180_128")
    faces, lat, P = make_inputs(c)
    parts = dict(x=P.x, y=P.y, z=P.z, vx=P.vx, vy=P.vy, vz=P.vz, d=P.d, q=P.q)
    u = torch.from_numpy(lat).cuda()
    out = {"workload": workload_desc(c) + ", frozen field"}
    for name, kw in (("plain", {}), ("coulomb", dict(coulomb=1)), ("collisions", dict(collisions=1)),
                     ("coulomb_and_collisions", dict(coulomb=1, collisions=1)), ("ssm", {}), ("two_way", {})):
        params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0,
                          sort_every=sort_every, **kw)
        ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, u, max_particles=c.n_particles)
        if name == "ssm":
            ch.set_ssm(T.SSMParams(seed=1))
        if name == "two_way":
            ch.momentum_source()
        Pd = T.Particles.from_numpy(parts, T.TRIBO_MIXED, device="cuda")
        ch.step(Pd, c.dt, 5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ch.step(Pd, c.dt, steps)
        e1.record()
        torch.cuda.synchronize()
        ch.sync()
        ch.close()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "particle_steps_per_s": c.n_particles / (ms * 1e-3)}
    return out


_WORKER = {}


def _oracle_init(shm_name, shape, faces, geo):
    """Start-up of an all-core oracle worker: import the oracle and attach the
    shared lattice once per process."""
    import oracle
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)      # the parent owns and unlinks it
    nx, nz, lx, lz, rho_p, nu, rho_f, dt = geo
    _WORKER.update(oracle=oracle, shm=shm, lat=np.ndarray(shape, dtype=np.float64, buffer=shm.buf),
                   g=oracle.Grid(nx, nz, lx, lz, faces), dt=dt,
                   p=oracle.Params(rho_p=rho_p, nu=nu, rho=rho_f, U_c=1.0, electrostatics=False))


def _oracle_particles(arrays):
    """Task of an all-core oracle worker: the oracle's particle update (and one
    more trilinear call for the E gather) on one chunk; None is a start-up
    probe.  Returns the seconds it took."""
    if arrays is None:
        time.sleep(0.5)
        return 0.0
    w = _WORKER
    st = w["oracle"].State.from_arrays(*arrays)
    t0 = time.perf_counter()
    w["oracle"].step(w["g"], w["p"], st, w["lat"], w["dt"])
    w["oracle"].trilinear(w["g"], w["lat"], st.x, st.y, st.z)
    return time.perf_counter() - t0


def oracle_particles_all_cores(c, faces, lat, P, n_sample, workers):
    """Wall time of the oracle's particle update of n_sample particles split
    over `workers` spawned processes, all started before the timing."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import shared_memory
    lat64 = np.ascontiguousarray(lat, dtype=np.float64)
    shm = shared_memory.SharedMemory(create=True, size=lat64.nbytes)
    try:
        np.ndarray(lat64.shape, dtype=np.float64, buffer=shm.buf)[...] = lat64
        geo = (c.nx, c.nz, c.lx, c.lz, c.rho_p, c.nu, c.rho_f, c.dt)
        bounds = np.linspace(0, n_sample, workers + 1).astype(np.int64)
        tasks = [tuple(np.asarray(getattr(P, k)[a:b]) for k in ("x", "y", "z", "vx", "vy", "vz", "q", "d"))
                 for a, b in zip(bounds[:-1], bounds[1:])]
        # a worker that dies raises here (BrokenProcessPool) instead of leaving the pool waiting
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                 initializer=_oracle_init, initargs=(shm.name, lat64.shape, faces, geo)) as pool:
            list(pool.map(_oracle_particles, [None] * workers))
            list(pool.map(_oracle_particles, [tuple(x[:64] for x in t) for t in tasks]))
            t0 = time.perf_counter()
            list(pool.map(_oracle_particles, tasks))
            return time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()


def cpu_baseline(c, faces, lat, P, n_sample, all_sample=1_600_000):
    t_field, t_part = oracle_step_time(c, faces, lat, P, n_sample)
    t_full = t_field + t_part * (c.n_particles / n_sample)
    workers = os.cpu_count() or 1
    all_cores = None
    if workers > 1:
        n_all = min(all_sample, c.n_particles)
        t_all = oracle_particles_all_cores(c, faces, lat, P, n_all, workers)
        v_all = c.n_particles / (t_field + t_all * (c.n_particles / n_all))
        all_cores = {"value": v_all, "unit": METRIC, "cores": workers,
                     "sample": (f"the particle update of {n_all} particles over {workers} spawned oracle "
                                f"processes ({t_all:.2f} s), scaled to all particles, plus the single-threaded "
                                f"deposit+Poisson+E ({t_field:.2f} s)")}
    return {"value": c.n_particles / t_full, "unit": METRIC, "cores": 1, "kind": "oracle",
            "poisson_solves_per_s": 1.0 / t_field, "all_cores": all_cores,
            "sample": (f"one FP64 oracle step on the host: full {c.nx}x{c.ny}x{c.nz} deposit+Poisson+E "
                       f"({t_field:.2f} s) plus the particle update of {n_sample} of the "
                       f"{c.n_particles} particles ({t_part:.2f} s), scaled to all particles; "
                       f"numpy single-threaded; host has {os.cpu_count()} cores")}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    c = synth.case(args.config)
    faces, lat, P = make_inputs(c)
    n_sample = args.ref_sample
    for _ in range(args.warmup):
        oracle_step_time(c, faces, lat, P, min(n_sample, 20000))
    times, fields = [], []
    for _ in range(args.steps):
        tf, tp = oracle_step_time(c, faces, lat, P, n_sample)
        times.append(tf + tp * (c.n_particles / n_sample))
        fields.append((tf, tp))
    t = sum(times) / len(times)
    v = c.n_particles / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(c, f"FP64 oracle (numpy, one host core), each step "
                                                 f"extrapolated from {n_sample} of the {c.n_particles} "
                                                 f"particles")},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle", "extrapolated": True,
                             "poisson_solves_per_s": len(times) / sum(tf for tf, _ in fields),
                             "sample": f"each step: full-grid deposit+Poisson+E plus the particle update of "
                                       f"{n_sample} particles, the particle part extrapolated to "
                                       f"{c.n_particles}"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


MIXED_ARITH = ("mixed precision: FP32 particle state, interpolation, force math and x/z FFTs; FP64 cell "
               "charge sums, per-particle charges, wall-impact charge and charge totals; y tridiagonal "
               "solve with FP64-computed factors and double-single (hi+lo FP32) sweeps")
FP64_ARITH = "FP64 throughout"


def workload_desc(c, arith=MIXED_ARITH):
    return (f"{c.name}: Re_tau={c.re_tau:g}, {c.nx}x{c.ny}x{c.nz} grid (Lx=2 pi h, Lz=pi h, tanh y "
            f"stretching {c.gamma:g}), {c.n_particles} particles, d+={c.dplus[0]:g}, "
            f"rho_p/rho={c.density_ratio:g}, dt+={c.dt_plus:g}, Stokes drag, mesh electrostatics "
            f"every step, condenser wall charging; {arith}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tribo", choices=["tribo", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=20, help="end-to-end calls timed (20: one sort among them)")
    ap.add_argument("--cpu-sample", type=int, default=200_000)
    ap.add_argument("--ref-sample", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the mixed vs FP64 GPU comparison")
    ap.add_argument("--no-oracle-subsample", action="store_true",
                    help="skip the one-step comparison with the FP64 oracle on a 1-in-1000 subsample")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-timevarying", action="store_true")
    ap.add_argument("--no-interactions", action="store_true")
    ap.add_argument("--adj-steps", type=int, default=500, help="adjoint section: steps (500 = the workload)")
    ap.add_argument("--adj-ckpt", type=int, default=50, help="adjoint section: steps between stored states")
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--batch-channels", type=int, default=64)
    ap.add_argument("--batch-scale", type=float, default=1.0, help="batched section: particle-count factor")
    ap.add_argument("--sort-every", type=int, default=20)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_2602_10761_gb300 as T
    from paper_2602_10761_gb300 import build as B

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    T.load()

    c = synth.case(args.config)
    faces, lat, P = make_inputs(c)
    stream = torch.cuda.current_stream()
    params = T.Params(precision=T.TRIBO_MIXED, rho_p=c.rho_p, nu=c.nu, rho=c.rho_f, U_c=1.0,
                      sort_every=args.sort_every)
    ch = T.Channel(c.nx, c.ny, c.nz, c.lx, c.lz, faces, params, torch.from_numpy(lat).cuda(),
                   max_particles=c.n_particles, stream=stream)
    parts = dict(x=P.x, y=P.y, z=P.z, vx=P.vx, vy=P.vy, vz=P.vz, d=P.d, q=P.q)
    Pd = T.Particles.from_numpy(parts, T.TRIBO_MIXED, device=f"cuda:{local}")
    nodes = touched_nodes(c, faces, P.x, P.y, P.z)

    ch.step(Pd, c.dt, args.warmup)
    ch.sync()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    launches0 = ch.launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    ch.step(Pd, c.dt, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = ch.launches - launches0
    # the same number of steps again with CUDA events around every kernel, on the launching
    # stream (the library's phase timers): the kernels' durations for the roofline.  The timed
    # region above runs without them: an event between two kernels costs the step 1-2 us and
    # stops the next kernel from being scheduled while the previous one drains
    T.tribo_timing_enable(ch.ctx, True)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    ch.step(Pd, c.dt, args.steps)
    ev3.record(stream)
    torch.cuda.synchronize()
    ms_instr = ev2.elapsed_time(ev3)
    phases = T.tribo_timing_read(ch.ctx)
    T.tribo_timing_enable(ch.ctx, False)
    ch.sync()
    ms = max_over_ranks(ms, "cuda")
    ms_per_step = ms / args.steps
    value = aggregate_rate(c.n_particles, args.steps, ms * 1e-3, world)

    # end to end through the public call with HOST buffers (pinned), copies inside: the same
    # simulation continued, its state (cell-ordered by the last sort) held on the host
    host = {}
    for k in ("x", "y", "z", "vx", "vy", "vz", "d", "q", "q_wall", "n_imp", "id"):
        v = getattr(Pd, k).cpu().pin_memory().numpy()
        host[k] = v.view(np.uint32) if k in ("n_imp", "id") else v
    Ph = T.Particles(**host)
    # the bytes moved are the library's own count of the copies it issued (tribo_transfer_bytes):
    # every state array in; positions and velocities out, with q, q_wall, n_imp only of the
    # particles an impact changed, except in the call that sorts (the ids move then, and every
    # array comes back); the average over the timed calls is reported
    ch.step(Ph, c.dt, 1)
    if world > 1:
        dist.barrier()
    b0 = T.tribo_transfer_bytes(ch.ctx)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ch.step(Ph, c.dt, 1)          # copies in, one step, copies out, synchronises
    e2e_s = time.perf_counter() - t0
    b1 = T.tribo_transfer_bytes(ch.ctx)
    h2d = (b1[0] - b0[0]) // max(args.e2e_steps, 1)
    d2h = (b1[1] - b0[1]) // max(args.e2e_steps, 1)
    e2e_s = max_over_ranks(e2e_s, "cuda")
    e2e_value = aggregate_rate(c.n_particles, args.e2e_steps, e2e_s, world)

    hbm_peak, peak_kind = measured_peaks()
    kern = {}
    poisson_ms = 0.0
    for name, (tms, cnt) in phases.items():
        if cnt:
            kern[name] = {"ms_per_launch": tms / cnt, "launches": cnt, "share": tms / max(ms_instr, 1e-9)}
            if name.startswith("poisson"):
                poisson_ms += tms
    n_solves = phases["poisson_fwd_x"][1]
    poisson_per_solve = poisson_ms / max(n_solves, 1)
    cells = c.nx * c.ny * c.nz
    nodes_all = c.nx * (c.ny + 2) * c.nz
    alg = {
        "particle_step": c.n_particles * PARTICLE_BYTES + nodes * NODE_BYTES + cells * CELL_BYTES,
        "poisson": cells * CELL_BYTES + nodes_all * 12,
    }
    dom = max(kern, key=lambda k: kern[k]["ms_per_launch"] * kern[k]["launches"])
    step_ms = phases["particle_step"][0] / max(phases["particle_step"][1], 1)
    ach_step = alg["particle_step"] / (step_ms * 1e-3) / 1e9
    ach_pois = alg["poisson"] / (poisson_per_solve * 1e-3) / 1e9
    if dom.startswith("poisson"):
        roof = {"bound": "hbm", "achieved": ach_pois, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach_pois / hbm_peak, "traffic": None, "kernel": "poisson (all passes)",
                "peak_kind": peak_kind}
    else:
        roof = {"bound": "hbm", "achieved": ach_step, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach_step / hbm_peak, "traffic": measured_traffic("k_step"), "kernel": "k_step",
                "alg_bytes": alg["particle_step"], "peak_kind": peak_kind,
                "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": ach_step / NOMINAL_HBM_GBS}
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload_desc(c), "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set > L2 (lattices 2 x 406 MB, particles 0.5 GB); no flush",
                   "sort_every": args.sort_every},
        "poisson_solves_per_s": 1e3 / poisson_per_solve if poisson_per_solve > 0 else None,
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": args.e2e_steps},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_all": {
            "particle_step": {"achieved": ach_step, "frac": ach_step / hbm_peak,
                              "alg_bytes": alg["particle_step"], "ms": step_ms},
            "poisson": {"achieved": ach_pois, "frac": ach_pois / hbm_peak, "alg_bytes": alg["poisson"],
                        "ms": poisson_per_solve}},
        "kernels": kern,
        "kernels_timing": (f"a second run of {args.steps} steps with CUDA events around every kernel on the "
                           f"launching stream: {ms_instr / args.steps:.4f} ms per step with the events"),
        "clocks": clocks,
    }
    ch.close()
    del Pd
    if rank == 0 and world == 1 and not args.no_oracle_subsample:
        order = np.argsort(host["id"])
        state = {k: np.asarray(host[k])[order] for k in ("x", "y", "z", "vx", "vy", "vz", "d")}
        line["vs_oracle_subsample"] = oracle_subsample_report(T, torch, c, faces, lat, state)
        del state
    if rank == 0 and world == 1 and not args.no_fp64:
        line["vs_fp64_gpu"] = fp64_report(T, torch, c, faces, lat, P, sort_every=args.sort_every)
    if rank == 0 and world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_report(T, torch, steps=args.adj_steps, ckpt=args.adj_ckpt)
    if rank == 0 and world == 1 and not args.no_interactions:
        line["interactions"] = interactions_report(T, torch)
    if rank == 0 and world == 1 and not args.no_timevarying:
        line["timevarying"] = timevarying_report(T, torch)
    if not args.no_batch:
        line["batched"] = batch_report(T, torch, steps=args.batch_steps, rank=rank, world=world,
                                       channels=args.batch_channels, scale=args.batch_scale)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(c, faces, lat, P, args.cpu_sample)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
