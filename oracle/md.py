"""Plain CPU oracle of velocity-Verlet NVE on the minimal Tersoff forces.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path. Independent of the
CUDA path. The integrator is not part of the paper's method (its MD runs, Sec. IV, use an external
MD code); it is the textbook velocity-Verlet scheme written out step by step, with forces from the
oracle's FP64 evaluation (Eq. 1-14):

    v(t + dt/2) = v(t) + F(t) dt / (2 m)
    x(t + dt)   = x(t) + v(t + dt/2) dt
    v(t + dt)   = v(t + dt/2) + F(t + dt) dt / (2 m)

Units: eV, A, amu (unified atomic mass unit), fs. Conversion factors follow from the CODATA 2018
exact elementary charge and the unified atomic mass unit.
"""
from __future__ import annotations

import numpy as np

from . import tersoff

E_CHARGE = 1.602176634e-19          # C (exact): 1 eV = E_CHARGE J
AMU = 1.66053906660e-27             # kg
ACCEL = E_CHARGE / (1e-10 * AMU) * 1e10 * 1e-30     # 1 eV/(A amu) in A/fs^2
KINETIC = AMU * 1e-20 / 1e-30 / E_CHARGE            # 1 amu A^2/fs^2 in eV
KB = 8.617333262e-5                 # Boltzmann constant, eV/K


def kinetic_energy(vel, mass) -> float:
    """sum_i m_i |v_i|^2 / 2 in eV."""
    vel = np.asarray(vel, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    return float(0.5 * KINETIC * np.sum(mass[:, None] * vel * vel))


def velocity_verlet(pos, vel, mass, box, params, dt: float, nsteps: int, R1=tersoff.R1_DEFAULT,
                    R2=tersoff.R2_DEFAULT, force_fn=None):
    """nsteps velocity-Verlet steps. Returns final (pos, vel) and the per-step Epot, Ekin [nsteps + 1]
    (before the first step and after every step). force_fn(pos) -> (E, F) replaces the Tersoff forces
    (for pins against other potentials)."""
    x = np.array(pos, dtype=np.float64)
    v = np.array(vel, dtype=np.float64)
    m = np.asarray(mass, dtype=np.float64)

    def forces(xx):
        if force_fn is not None:
            return force_fn(xx)
        r = tersoff.evaluate(xx, box, params, R1=R1, R2=R2)
        return r["E"], r["F"]

    E, F = forces(x)
    Ep, Ek = [E], [kinetic_energy(v, m)]
    for _ in range(nsteps):
        v = v + F * (0.5 * dt * ACCEL / m)[:, None]
        x = x + v * dt
        E, F = forces(x)
        v = v + F * (0.5 * dt * ACCEL / m)[:, None]
        Ep.append(E)
        Ek.append(kinetic_energy(v, m))
    return x, v, np.array(Ep), np.array(Ek)
