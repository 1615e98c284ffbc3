"""Pins of the velocity-Verlet oracle (test infrastructure for the NVE integrator): CODATA unit
factors, second-order convergence to an accurate solution of the Morse dimer, time reversibility,
and energy conservation in a periodic diamond cell."""
import math

import numpy as np
from scipy.integrate import solve_ivp

import oracle
from oracle import md as omd
from paper_1909_11474_gb300 import inputs as I

P2 = I.TABLE2_PARAMS


def test_unit_factors():
    # 1 eV/(A amu) = 9.6485332e-3 A/fs^2 and 1 amu A^2/fs^2 = 103.6427 eV (textbook values)
    assert abs(omd.ACCEL - 9.6485332e-3) < 1e-10
    assert abs(omd.KINETIC - 103.6427) < 1e-4
    assert abs(omd.ACCEL * omd.KINETIC - 1.0) < 1e-14


def _dimer_exact(r0, t_end, D0, al, re, mu):
    """Relative coordinate of the Morse pair U = D0 (x^2 - 2x), x = exp(-al (r - re)), solved by an
    8th-order Runge-Kutta at tolerance 1e-13."""
    def rhs(_, y):
        r, v = y
        x = math.exp(-al * (r - re))
        dU = -2.0 * al * D0 * (x * x - x)
        return [v, -dU / mu * omd.ACCEL]
    sol = solve_ivp(rhs, (0.0, t_end), [r0, 0.0], method="DOP853", rtol=1e-13, atol=1e-13)
    return sol.y[0, -1]


def test_verlet_converges_at_second_order_on_the_morse_dimer():
    """Two Si atoms at 2.30 A (inside R1, so f_C = 1 and, with zeta = 0, b = 1: the Morse pair)."""
    D0, al, re = P2[0], P2[1], P2[2]
    L = 40.0
    pos = np.array([[L / 2, L / 2, L / 2], [L / 2 + 2.30, L / 2, L / 2]])
    box = np.eye(3) * L
    m = np.full(2, I.SI_MASS)
    t_end = 60.0
    exact = _dimer_exact(2.30, t_end, D0, al, re, I.SI_MASS / 2)
    errs = []
    for dt in (1.0, 0.5):
        x, v, Ep, Ek = omd.velocity_verlet(pos, np.zeros((2, 3)), m, box, P2, dt, int(round(t_end / dt)))
        errs.append(abs((x[1, 0] - x[0, 0]) - exact))
        assert np.abs(x[:, 1:] - pos[:, 1:]).max() < 1e-12          # motion stays on the axis
    assert errs[0] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0                          # O(dt^2)


def _thermal_cell(T=300.0, seed=3):
    pos, box = I.diamond_supercell((1, 1, 1))
    rng = np.random.default_rng(seed)
    m = np.full(len(pos), I.SI_MASS)
    return pos, box, m, I.thermal_velocities(rng, m, T)


def test_verlet_is_time_reversible():
    pos, box, m, v = _thermal_cell()
    x1, v1, _, _ = omd.velocity_verlet(pos, v, m, box, P2, 1.0, 40)
    x2, v2, _, _ = omd.velocity_verlet(x1, -v1, m, box, P2, 1.0, 40)
    assert np.abs(x2 - pos).max() < 1e-9
    assert np.abs(v2 + v).max() < 1e-11


def test_verlet_conserves_energy_in_a_periodic_cell():
    """300 K in the 8-atom cell over 100 fs: the total energy stays within 1.5e-4 eV/atom at
    dt = 1 fs, and its excursion shrinks about fourfold at dt = 0.5 fs (second order)."""
    pos, box, m, v = _thermal_cell()
    dev = []
    for dt in (1.0, 0.5):
        _, _, Ep, Ek = omd.velocity_verlet(pos, v, m, box, P2, dt, int(round(100 / dt)))
        Et = Ep + Ek
        dev.append(np.abs(Et - Et[0]).max() / 8)
        assert np.abs(Ek - Ek[0]).max() > 1e-3                      # energy did move between the two
    assert dev[0] < 1.5e-4
    assert 3.0 < dev[0] / dev[1] < 5.5


def test_thermal_velocities_have_zero_momentum_and_the_drawn_temperature():
    """The seeded Maxwell-Boltzmann input draw: no centre-of-mass motion, and for 60,000 atoms the
    kinetic temperature 2 E_k / (3 N kB) within 2 % of T (statistical spread ~0.3 %)."""
    rng = np.random.default_rng(4)
    m = np.full(60000, I.SI_MASS)
    v = I.thermal_velocities(rng, m, 300.0)
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-9
    T = 2 * omd.kinetic_energy(v, m) / (3 * len(m) * omd.KB)
    assert abs(T / 300.0 - 1) < 0.02
