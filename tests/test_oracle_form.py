"""Pins of the oracle's Tersoff form (nine parameters: D0, alpha, r0, S, n, h, gamma, c, d; the
original angular function of Eq. 8 and a free S in Eq. 11-14) against closed forms and the
minimal-Tersoff limit of Sec. II.B."""
import math

import numpy as np
import pytest

import oracle
from paper_1909_11474_gb300 import inputs as I

P2 = I.TABLE2_PARAMS
# a Tersoff-form parameter set of the magnitudes Sec. II.B describes (c^2/d^2 >> 1, d^2 >> 1,
# gamma << 1), with S away from 2
XT = np.array([3.0, 1.5, 2.30, 1.8, 0.75, -0.55, 2.0e-5, 60.0, 12.0])


def _cluster(points, L=40.0):
    pos = np.asarray(points, dtype=np.float64) + L / 2
    return pos, np.eye(3) * L


def _pair(x, r):
    """f_R and f_A of Eq. 4-5 with Eq. 11-14 (free S), written out for one distance."""
    D0, al, r0, S = x[0], x[1], x[2], x[3]
    fR = D0 / (S - 1) * math.exp(-al * math.sqrt(2 * S) * (r - r0))
    fA = D0 * S / (S - 1) * math.exp(-al * math.sqrt(2 / S) * (r - r0))
    return fR, fA


@pytest.mark.parametrize("S", [1.5, 1.8, 2.0, 2.6])
def test_dimer_well_has_depth_D0_at_r0_for_any_S(S):
    """Two atoms: zeta = 0, b = 1, U = f_R - f_A, whose minimum is -D0 at r0 (Sec. II.B)."""
    x = XT.copy()
    x[3] = S
    for r in (x[2], x[2] + 0.2, x[2] - 0.15):
        out = oracle.evaluate(*_cluster([[0, 0, 0], [r, 0, 0]]), x)
        fR, fA = _pair(x, r)
        assert out["E"] == pytest.approx(fR - fA, rel=1e-13)
    out = oracle.evaluate(*_cluster([[0, 0, 0], [x[2], 0, 0]]), x)
    assert out["E"] == pytest.approx(-x[0], rel=1e-13)
    assert np.abs(out["F"]).max() < 1e-12


@pytest.mark.parametrize("theta_deg", [95.0, 109.47, 120.0, 150.0])
def test_trimer_bond_order_with_the_original_angular_function(theta_deg):
    """Atom 0 bonded to 1 and 2 (r = 2.3 A < R1, angle theta; 1-2 beyond R2): bonds 0-1 and 0-2 see
    zeta = g^T(theta) (Eq. 7-8), bonds 1-0 and 2-0 see zeta = 0, so
    U = (f_R - b f_A) + (f_R - f_A), b = (1 + g^n)^(-1/(2n))."""
    r, th = 2.3, math.radians(theta_deg)
    pts = [[0, 0, 0], [r, 0, 0], [r * math.cos(th), r * math.sin(th), 0]]
    assert 2 * r * math.sin(th / 2) > 3.2
    x = XT
    D0, al, r0, S, n, h, gam, c, d = x
    g = gam * (1 + c * c / (d * d) - c * c / (d * d + (math.cos(th) - h) ** 2))
    b = (1 + g ** n) ** (-1 / (2 * n))
    fR, fA = _pair(x, r)
    out = oracle.evaluate(*_cluster(pts), x)
    assert out["E"] == pytest.approx((fR - b * fA) + (fR - fA), rel=1e-13)


def test_tersoff_form_tends_to_the_minimal_potential():
    """Sec. II.B: with c^2 = kappa d^4 and gamma = beta / kappa, g^T = beta (cos - h)^2 + beta/kappa
    + O(beta u^4 / d^2); at S = 2 the Tersoff form then tends to the minimal one as kappa grows,
    with the error falling in proportion to 1/kappa."""
    rng = np.random.default_rng(0)
    pos, box = I.diamond_supercell((2, 2, 2))
    pos = pos + rng.normal(0, 0.08, pos.shape)
    ref = oracle.evaluate(pos, box, P2)
    D0, al, r0, be, n, h = P2
    errs = []
    for kappa in (1e3, 1e4):
        d = 300.0
        x = np.array([D0, al, r0, 2.0, n, h, be / kappa, math.sqrt(kappa) * d * d, d])
        out = oracle.evaluate(pos, box, x)
        errs.append((abs(out["E"] - ref["E"]) / abs(ref["E"]), np.abs(out["F"] - ref["F"]).max()))
    assert errs[0][0] < 5e-3 and errs[1][0] < 5e-4
    assert 5 < errs[0][0] / errs[1][0] < 20
    assert 5 < errs[0][1] / errs[1][1] < 20


def test_tersoff_form_forces_are_the_energy_gradient():
    """Central differences of E against F for the Tersoff form in a distorted periodic cell."""
    rng = np.random.default_rng(1)
    pos, box = I.diamond_supercell((1, 1, 1))
    pos = pos + rng.normal(0, 0.1, pos.shape)
    out = oracle.evaluate(pos, box, XT)
    h = 1e-5
    for i, k in ((0, 0), (3, 1), (6, 2)):
        p, m = pos.copy(), pos.copy()
        p[i, k] += h
        m[i, k] -= h
        fd = -(oracle.evaluate(p, box, XT)["E"] - oracle.evaluate(m, box, XT)["E"]) / (2 * h)
        assert out["F"][i, k] == pytest.approx(fd, rel=1e-6, abs=1e-8)
