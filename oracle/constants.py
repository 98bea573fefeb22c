"""Material constants (Table 1) and model switches of the oracle.

Part of the FP64 CPU oracle: test infrastructure only.
"""
from __future__ import annotations

import dataclasses

# Table 1 (material properties; PMMA particles, air, wall)
TABLE1 = dict(
    mu_p=0.4,          # Poisson's ratio, particle
    E_p=1e8,           # Young's modulus, particle [Pa]
    phi_p=1e13,        # resistivity, particle [Ohm m]
    k_e=0.95,          # particle restitution ratio
    mu_w=0.28,         # Poisson's ratio, wall
    E_w=1e11,          # Young's modulus, wall [Pa]
    eps_w=5.0,         # relative permittivity, wall
    h=1e-9,            # effective separation [m]
    eps=8.854e-12,     # air permittivity [F/m]
    nu=1.46e-5,        # air kinematic viscosity [m^2/s]
    rho=1.2,           # air density [kg/m^3]
    rho_p=1150.0,      # particle density [kg/m^3]
)

DRAG_STOKES = 0
DRAG_SCHILLER_NAUMANN = 1
DRAG_OFF = 2

IMPACT_SPEED = 0     # |u_i| = full particle speed at impact (literal reading)
IMPACT_NORMAL = 1    # |u_i| = wall-normal speed at impact


@dataclasses.dataclass
class Params:
    """Physical parameters and switches of one run.

    eps is the permittivity of the gas used in Poisson's equation and in the
    capacitor C = eps A / h (Sec. 2.2 and Eq. capacity-capacitor); eps0 is the
    vacuum permittivity in T_w = eps_w eps0 phi_p (Sec. 2.3.1).  The paper
    takes the gas permittivity equal to the vacuum one.
    U_c (contact potential) is not given in the paper (reading: a free
    parameter, default 1 V).  kappa_A scales the Hertz contact area (1 in the
    paper).  coulomb adds the near field of the hybrid electrostatics
    (Sec. 2.2): Coulomb's law between particles that share a cell.
    collisions adds 4-way coupling: hard-sphere particle-particle collisions
    (Sec. 2.2) with the condenser-model charge exchange (Sec. 2.3.1).
    ssm (an oracle.ssm.SSM) replaces the condenser model of wall impacts by
    the stochastic scaling model (Sec. 2.3.2).
    """
    mu_p: float = TABLE1["mu_p"]
    E_p: float = TABLE1["E_p"]
    phi_p: float = TABLE1["phi_p"]
    k_e: float = TABLE1["k_e"]
    mu_w: float = TABLE1["mu_w"]
    E_w: float = TABLE1["E_w"]
    eps_w: float = TABLE1["eps_w"]
    h: float = TABLE1["h"]
    eps: float = TABLE1["eps"]
    eps0: float = TABLE1["eps"]
    nu: float = TABLE1["nu"]
    rho: float = TABLE1["rho"]
    rho_p: float = TABLE1["rho_p"]
    U_c: float = 1.0
    kappa_A: float = 1.0
    drag_law: int = DRAG_STOKES
    impact_vel: int = IMPACT_SPEED
    dq_t: bool = True
    electrostatics: bool = True
    coulomb: bool = False
    collisions: bool = False
    ssm: object = None          # oracle.ssm.SSM: wall impacts charge by the SSM instead

    def with_(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)
