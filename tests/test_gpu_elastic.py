"""Elastic constants through the device path (Table 3): the lattice constant, C11, C12 and the
internally relaxed C44 from the batched FP64 kernels, against Table 3 and against the same
stress-strain procedure run on the oracle."""
import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar

import oracle
from paper_1909_11474_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EV_A3_GPA = 160.21766208
P2 = I.TABLE2_PARAMS


def _oracle_cell(a, eps, u=np.zeros(3)):
    pos, box = I.diamond_supercell((1, 1, 1), a)
    pos = pos.copy()
    pos[4:] += u
    return I.apply_strain(pos, box, eps)


def _oracle_constants(e=1e-4):
    a0 = minimize_scalar(lambda a: oracle.evaluate(*I.diamond_supercell((1, 1, 1), a), P2)["E"] / 8.0,
                         bracket=(5.40, 5.43, 5.46), tol=1e-12).x
    V = a0 ** 3

    def W(eps, relax=False):
        u = np.zeros(3)
        if relax:
            def fg(uu):
                r = oracle.evaluate(*_oracle_cell(a0, eps, uu), P2)
                return r["E"], -r["F"][4:].sum(axis=0)
            u = minimize(fg, np.zeros(3), jac=True, method="BFGS", options={"gtol": 1e-11}).x
        return oracle.evaluate(*_oracle_cell(a0, eps, u), P2)["W"]

    ex = np.zeros((3, 3)); ex[0, 0] = e
    sh = np.zeros((3, 3)); sh[1, 2] = sh[2, 1] = e / 2
    Wp, Wm = W(ex), W(-ex)
    out = {"a0": a0, "C11": -(Wp[0] - Wm[0]) / (2 * e) / V * EV_A3_GPA, "C12": -(Wp[1] - Wm[1]) / (2 * e) / V * EV_A3_GPA}
    out["C44"] = -(W(sh, True)[4] - W(-sh, True)[4]) / (2 * e) / V * EV_A3_GPA
    return out


@pytest.fixture(scope="module")
def device_constants():
    from paper_1909_11474_gb300.elastic import elastic_constants
    return elastic_constants(P2)


def test_elastic_constants_match_table3(device_constants, golden):
    c = device_constants
    assert abs(c["a0"] - golden["lattice_constant"]) <= 1e-3
    for k in ("C11", "C12", "C44"):
        assert abs(c[k] - golden[k]) < 1.0, (k, c[k])
    # the internal relaxation lowers C44 (the unrelaxed shear is stiffer)
    assert c["C44_unrelaxed"] > c["C44"] + 10.0
    # by symmetry the relaxed shift under a yz shear lies along x
    u = np.asarray(c["shift_at_plus_shear"])
    assert abs(u[0]) > 1e-6 and np.abs(u[1:]).max() < 1e-3 * abs(u[0])


def test_elastic_constants_match_the_oracle(device_constants):
    ref = _oracle_constants()
    c = device_constants
    assert abs(c["a0"] - ref["a0"]) < 1e-7
    for k in ("C11", "C12", "C44"):
        assert abs(c[k] - ref[k]) < 1e-3, (k, c[k], ref[k])
