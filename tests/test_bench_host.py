"""Host helpers of bench.py that enter the reported numbers (CPU):
* touched_nodes, the lattice nodes the trilinear gather reads (the per-node
  term of the particle kernel's algorithmic bytes): one particle touches the
  8 corners of its stencil; a particle at every cell centre touches every node
  row but the bottom wall row (the centre of cell j is node j+1, whose stencil
  is nodes j+1 and j+2);
* measured_traffic, which reports a profile's DRAM bytes only while the
  sources it was taken from are unchanged;
* measured_peaks, which falls back when the peak file is absent."""
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
