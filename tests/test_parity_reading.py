"""The per-particle tolerance reading that every GPU parity test asserts
(`_problems.compare_states`), checked on the CPU: a state within the tolerance
passes, and an error just above it in any one output (a position across the
periodic seam, the velocity vector, the charge, the received wall charge) fails,
each against the scale the reading fixes (the box extent, the particle's speed,
the particle's charge scale max(|q|, |q_wall|, |q - q_wall|))."""
import numpy as np
import pytest

import oracle
from _problems import compare_states

TOL = 1e-5


def _grid():
    faces = np.linspace(0.0, 1.0, 9)                 # ly = 1
    return oracle.Grid(8, 4, 2.0, 4.0, faces)         # lx = 2, lz = 4


def _ref():
    return oracle.State.from_arrays(
        x=[0.0005, 1.0], y=[0.5, 0.25], z=[1.0, 3.9999], vx=[3.0, 0.0], vy=[4.0, 1e-3], vz=[0.0, 0.0],
        q=[-2e-15, 0.0], d=[1e-4, 1e-4], n_imp=[1, 0], q_wall=[-1e-15, 0.0])


def _got(ref):
    return {k: np.array(getattr(ref, k), dtype=np.float64) for k in ("x", "y", "z", "vx", "vy", "vz", "q", "q_wall")}


def test_exact_state_passes():
    g, ref = _grid(), _ref()
    out = compare_states(g, _got(ref), ref, TOL)
    assert all(out[k] == 0.0 for k in ("x", "y", "z", "v", "q", "q_wall"))


@pytest.mark.parametrize("factor, ok", [(0.5, True), (2.0, False)])
def test_each_output_against_its_scale(factor, ok):
    g, ref = _grid(), _ref()
    e = factor * TOL
    cases = []
    # x of particle 0 moved across the periodic seam by e of L_x (0.0005 -> 0.0005 - e L_x, wrapped)
    got = _got(ref)
    got["x"][0] = np.mod(0.0005 - e * 2.0, 2.0)
    cases.append(got)
    # y of particle 1 by e of L_y
    got = _got(ref)
    got["y"][1] += e * 1.0
    cases.append(got)
    # z of particle 1 across the seam at L_z (3.9999 + e L_z, wrapped)
    got = _got(ref)
    got["z"][1] = np.mod(3.9999 + e * 4.0, 4.0)
    cases.append(got)
    # the velocity of particle 0 (speed 5) by e of its speed, in a component it does not have
    got = _got(ref)
    got["vz"][0] = e * 5.0
    cases.append(got)
    # the slow particle 1 (speed 1e-3) by e of its own speed, not of the fast particle's
    got = _got(ref)
    got["vx"][1] = e * 1e-3
    cases.append(got)
    # q of particle 0 (charge scale max(2e-15, 1e-15, 1e-15) = 2e-15) by e of that scale
    got = _got(ref)
    got["q"][0] += e * 2e-15
    cases.append(got)
    # q_wall of particle 0, same scale
    got = _got(ref)
    got["q_wall"][0] -= e * 2e-15
    cases.append(got)
    for got in cases:
        if ok:
            compare_states(g, got, ref, TOL)
        else:
            with pytest.raises(AssertionError):
                compare_states(g, got, ref, TOL)


def test_zero_reference_charge_must_match_exactly():
    g, ref = _grid(), _ref()
    got = _got(ref)
    got["q"][1] = 1e-40                # particle 1 carries no charge in the reference
    with pytest.raises(AssertionError):
        compare_states(g, got, ref, TOL)
