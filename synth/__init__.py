"""Seeded synthetic inputs for the channel-flow charging hot path.

This package draws the inputs that both the FP64 CPU oracle and the CUDA path
consume: the wall-stretched grid faces, the synthetic gas-velocity lattice
(Reichardt mean profile plus random Fourier modes with near-wall damping) and
the particle ensembles of the five workload cases.  It holds none of the
method's arithmetic (no interpolation, drag, impact charging, deposition or
Poisson solve); it only decides *what* the inputs are.  All random numbers are
drawn here, on the host, from numpy's counter-based Philox generator.
"""
from .channel import (  # noqa: F401
    Case, CASES, case, y_faces, node_y, friction_velocity, reichardt_uplus,
    Modes, draw_modes, fluid_lattice, Particles, draw_particles, ensemble_cases,
    Q_SAT, mean_velocity, damping, replay_state,
)
