"""The seeded synthetic inputs against their recipe (CPU).  The generators
hold none of the method's arithmetic, but every parity case and benchmark
rests on them, so the recipe's fixed points are pinned:
* the tanh-stretched faces: the first-cell and centre-cell spacings in wall
  units at Re_tau 180 on 64 rows and Re_tau 550 on 256 rows (0.876 / 11.65
  and 0.639 / 8.91), symmetry about the centreline, the walls at 0 and 2 delta;
* Reichardt's law of the wall: slope 1 at the wall and the log-law offset
  7.8 + ln(0.41) / 0.41 far from it;
* the near-wall damping y+ / (y+ + 10);
* the Fourier modes: amplitude vectors perpendicular to their wavenumber
  (divergence-free), x and z wavenumbers on the periodic lattice, and a total
  fluctuation energy of 3 u_tau^2 (per-component rms u_tau before damping);
* the particles inside the channel with their centres at least a radius from
  either wall.
"""
import math

import numpy as np
import pytest

import synth


@pytest.mark.parametrize("name,wall,centre", [("re180_64", 0.876, 11.65), ("re550_384", 0.639, 8.91)])
def test_stretched_faces(name, wall, centre):
    c = synth.case(name)
    f = synth.y_faces(c.ny, c.delta, c.gamma)
    dy = np.diff(f) * c.u_tau / c.nu
    assert abs(dy[0] - wall) < 5e-4 and abs(dy[c.ny // 2] - centre) < 5e-3
    assert f[0] == 0.0 and abs(f[-1] - 2 * c.delta) < 1e-15
    assert np.allclose(f + f[::-1], 2 * c.delta, atol=1e-15)
    assert np.all(np.diff(dy[: c.ny // 2]) > 0)          # cells grow towards the centre


def test_reichardt_law_limits():
    yp = np.array([1e-6, 1e-4])
    assert np.allclose(synth.reichardt_uplus(yp) / yp, 1.0, rtol=1e-3)
    big = np.array([1e4, 1e6])
    off = synth.reichardt_uplus(big) - np.log(big) / 0.41
    assert np.allclose(off, 7.8 + math.log(0.41) / 0.41, atol=1e-3)


def test_near_wall_damping():
    c = synth.case("re180_64")
    y = np.array([0.0, 10.0, 1e9]) * c.nu / c.u_tau
    y[-1] = c.delta
    d = synth.damping(y, c)
    yp = c.delta * c.u_tau / c.nu
    assert d[0] == 0.0 and abs(d[1] - 0.5) < 1e-12 and abs(d[2] - yp / (yp + 10.0)) < 1e-12


@pytest.mark.parametrize("name", ["re180_64", "re550_384"])
def test_modes_divergence_free_on_the_lattice_with_the_recipe_energy(name):
    c = synth.case(name)
    m = synth.draw_modes(c)
    k = np.stack([m.kx, m.ky, m.kz], axis=1)
    dot = np.abs(np.sum(m.amp * k, axis=1))
    assert np.all(dot <= 1e-12 * np.linalg.norm(m.amp, axis=1) * np.linalg.norm(k, axis=1) + 1e-300)
    assert np.allclose(m.kx, 2 * math.pi * m.nxi / c.lx) and np.allclose(m.kz, 2 * math.pi * m.nzi / c.lz)
    assert np.all(np.abs(m.nxi) < c.nx // 2) and np.all(np.abs(m.nzi) < c.nz // 2)
    assert abs(0.5 * np.sum(m.amp ** 2) / (3 * c.u_tau ** 2) - 1.0) < 1e-12


def test_particles_inside_the_channel():
    c = synth.case("re180_64")
    P = synth.draw_particles(c)
    r = 0.5 * P.d
    assert np.all(P.y >= r) and np.all(P.y <= c.ly - r)
    assert np.all((P.x >= 0) & (P.x < c.lx)) and np.all((P.z >= 0) & (P.z < c.lz))
