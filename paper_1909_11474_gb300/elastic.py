"""Zero-temperature elastic constants of diamond Si by stress-strain (arXiv:1909.11474, Table 3),
computed through the library's batched FP64 evaluation.

The stress of a strained conventional cell (8 atoms) is -W/V, with W the virial of the kernels.
* C11 and C12 are central differences of the xx and yy stress under a uniaxial strain +-e_xx.
* C44 is the central difference of the yz stress under an engineering shear +-gamma_yz. The second
  fcc sublattice is shifted rigidly to the position that minimises the energy of the sheared cell
  (internal relaxation), with forces from the same kernels.
* The lattice constant is the minimum of the energy per atom over the cubic lattice constant.

The minimisers (Brent over a, BFGS over the 3-vector shift) are host logic over a handful of
variables; every energy, force and virial comes from the device kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding
from . import inputs as I

EV_A3_GPA = 160.21766208  # 1 eV/A^3 in GPa


class _CellEval:
    """Batches of conventional diamond cells evaluated in FP64 on one context."""

    def __init__(self, params, ctx: binding.Context | None = None, R1: float = 2.8, R2: float = 3.2):
        self.ctx = ctx if ctx is not None else binding.Context(0)
        self.p = torch.as_tensor(np.asarray(params, dtype=np.float64).reshape(1, 6), device="cuda")
        self.R1, self.R2 = float(R1), float(R2)
        self.calls = 0

    def __call__(self, cells):
        """cells: list of (pos [8][3], box [3][3]). Returns E [C] (eV), F [C][8][3], W [C][6] (eV)."""
        pos = np.concatenate([c[0] for c in cells]).astype(np.float64)
        box = np.stack([c[1] for c in cells]).astype(np.float64)
        off = np.arange(len(cells) + 1, dtype=np.int32) * 8
        self.ctx.build_neighbors(off, torch.tensor(pos, device="cuda"), torch.tensor(box, device="cuda"),
                                 self.R1, self.R2, 16)
        E, F, W = self.ctx.eval(self.p, precision=64)
        st = self.ctx.get_status()
        if st != 0:
            raise RuntimeError(f"device status {st:#x} in the elastic-constant evaluation")
        self.calls += 1
        return (E[0].cpu().numpy(), F[0].cpu().numpy().reshape(len(cells), 8, 3), W[0].cpu().numpy())


def _cell(a: float, eps=None, u=None):
    pos, box = I.diamond_supercell((1, 1, 1), a)
    pos = pos.copy()
    if u is not None:
        pos[4:] += np.asarray(u, dtype=np.float64)   # rigid shift of the second fcc sublattice
    if eps is None:
        return pos, box
    return I.apply_strain(pos, box, np.asarray(eps, dtype=np.float64))


def lattice_constant(params, ctx: binding.Context | None = None, bracket=(5.40, 5.43, 5.46), tol=1e-12,
                     ev: _CellEval | None = None):
    """Cubic lattice constant (A) minimising the energy per atom, and that energy (eV/atom)."""
    from scipy.optimize import minimize_scalar
    ev = ev or _CellEval(params, ctx)
    res = minimize_scalar(lambda a: float(ev([_cell(a)])[0][0]) / 8.0, bracket=bracket, tol=tol)
    return float(res.x), float(res.fun)


def elastic_constants(params, ctx: binding.Context | None = None, e: float = 1e-4, a0: float | None = None,
                      R1: float = 2.8, R2: float = 3.2) -> dict:
    """C11, C12, C44 (GPa) at zero temperature, plus the unrelaxed C44 and the relaxed shift."""
    from scipy.optimize import minimize
    ev = _CellEval(params, ctx, R1, R2)
    if a0 is None:
        a0, _ = lattice_constant(params, ev=ev)
    V = a0 ** 3
    ex = np.zeros((3, 3))
    ex[0, 0] = e
    sh = np.zeros((3, 3))
    sh[1, 2] = sh[2, 1] = e / 2                      # engineering shear gamma_yz = e
    _, _, W = ev([_cell(a0, ex), _cell(a0, -ex), _cell(a0, sh), _cell(a0, -sh)])
    C11 = -(W[0, 0] - W[1, 0]) / (2 * e) / V * EV_A3_GPA
    C12 = -(W[0, 1] - W[1, 1]) / (2 * e) / V * EV_A3_GPA
    C44_0 = -(W[2, 4] - W[3, 4]) / (2 * e) / V * EV_A3_GPA

    def relaxed_W(eps):
        def fg(u):
            E, F, _ = ev([_cell(a0, eps, u)])
            return float(E[0]), -F[0, 4:].sum(axis=0)
        u = minimize(fg, np.zeros(3), jac=True, method="BFGS", options={"gtol": 1e-11}).x
        return ev([_cell(a0, eps, u)])[2][0], u

    Wp, up = relaxed_W(sh)
    Wm, _ = relaxed_W(-sh)
    C44 = -(Wp[4] - Wm[4]) / (2 * e) / V * EV_A3_GPA
    return {"a0": a0, "C11": float(C11), "C12": float(C12), "C44": float(C44), "C44_unrelaxed": float(C44_0),
            "shift_at_plus_shear": up.tolist(), "device_calls": ev.calls}
