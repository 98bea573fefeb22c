"""Host helpers of bench.py that enter the reported numbers (CPU):
* touched_nodes, the lattice nodes the trilinear gather reads (the per-node
  term of the particle kernel's algorithmic bytes): one particle touches the
  8 corners of its stencil; a particle at every cell centre touches every node
  row but the bottom wall row (the centre of cell j is node j+1, whose stencil
  is nodes j+1 and j+2);
* measured_traffic, which reports a profile's DRAM bytes only while the
  sources it was taken from are unchanged;
* measured_peaks, which falls back when the peak file is absent;
* per_particle_errors, the per-particle reading of the parity bar behind the
  bench's error reports, checked against values worked out by hand."""
import hashlib
import json
import os

import numpy as np
import pytest

import bench
import synth


def _case(nx=8, ny=6, nz=4):
    c = synth.case("re180_64").with_(nx=nx, ny=ny, nz=nz)
    return c, synth.y_faces(ny, c.delta, c.gamma)


def test_one_particle_touches_eight_nodes():
    c, faces = _case()
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = rng.uniform(0, c.lx, 1)
        y = rng.uniform(faces[0], faces[-1], 1)
        z = rng.uniform(0, c.lz, 1)
        assert bench.touched_nodes(c, faces, x, y, z) == 8


def test_cell_centres_touch_every_row_but_the_bottom_wall():
    c, faces = _case()
    yc = 0.5 * (faces[1:] + faces[:-1])
    k, j, i = np.meshgrid(np.arange(c.nz), np.arange(c.ny), np.arange(c.nx), indexing="ij")
    x = (i.ravel() + 0.5) * c.lx / c.nx
    z = (k.ravel() + 0.5) * c.lz / c.nz
    y = yc[j.ravel()]
    assert bench.touched_nodes(c, faces, x, y, z) == c.nz * (c.ny + 1) * c.nx


def test_measured_traffic_follows_its_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    info = {"kernel": "k_fake", "bytes_per_launch": 123, "source_hash": h, "files": ["kernel.cu"]}
    (tmp_path / "profiles" / "k_fake_re550_384.md").write_text("# k\n<!-- traffic: " + json.dumps(info) + " -->\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k_fake") == 123
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.measured_traffic("k_fake") is None
    assert bench.measured_traffic("k_absent") is None


def test_measured_peaks_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6794.1}))
    assert bench.measured_peaks() == (6794.1, "measured")


def test_per_particle_errors_by_hand():
    """Two particles in a box 2 x 1 x 4.  Particle 0: x off by 0.02 across the periodic
    seam (1.99 against 0.01: a distance of 0.02, 1% of L_x), velocity (3, 4, 0) against
    (3, 4, 0.05) (0.05 of a speed of 5: 1%), q -2e-15 against -1e-15 with q_wall -1e-15
    (charge scale max(1e-15, 1e-15, 0) = 1e-15: q off by 100%, q_wall exact).  Particle 1:
    exact.  The largest errors are those; the 99th percentile of two values interpolates."""
    ref = dict(x=np.array([0.01, 1.0]), y=np.array([0.5, 0.5]), z=np.array([1.0, 2.0]),
               vx=np.array([3.0, 1.0]), vy=np.array([4.0, 0.0]), vz=np.array([0.05, 0.0]),
               q=np.array([-1e-15, 2e-15]), q_wall=np.array([-1e-15, 0.0]))
    got = {k: v.copy() for k, v in ref.items()}
    got["x"][0] = 1.99
    got["vz"][0] = 0.0
    got["q"][0] = -2e-15
    e = bench.per_particle_errors(got, ref, 2.0, 1.0, 4.0)
    speed0 = np.sqrt(3.0 ** 2 + 4.0 ** 2 + 0.05 ** 2)
    assert e["x"]["max"] == pytest.approx(0.01, rel=1e-9)
    assert e["y"]["max"] == 0.0 and e["z"]["max"] == 0.0
    assert e["v"]["max"] == pytest.approx(0.05 / speed0, rel=1e-12)
    assert e["q"]["max"] == pytest.approx(1.0, rel=1e-12)
    assert e["q_wall"]["max"] == 0.0
    assert e["x"]["p99"] == pytest.approx(0.01 * 0.99, rel=1e-9)
    # a selection keeps only the chosen particles
    e1 = bench.per_particle_errors(got, ref, 2.0, 1.0, 4.0, sel=np.array([False, True]))
    assert all(e1[k]["max"] == 0.0 for k in ("x", "y", "z", "v", "q", "q_wall"))
