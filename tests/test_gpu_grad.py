"""Parity of the adjoint kernel (loss gradient over the six parameters) with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_11474_gb300 import inputs as I

from ._util import targets_to_device, to_device

pytestmark = pytest.mark.gpu


def _setup(P, C, masks, seed_scale=None):
    from paper_1909_11474_gb300 import binding
    w = I.workload_adjoint(P=P, C=C)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0], mask=np.asarray(masks, np.uint8))
    ctx = binding.Context(0)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    params = w["params"]
    if seed_scale is not None:   # parameter sets near the hidden one (the polish regime)
        params = w["hidden"][None, :] * (1 + seed_scale * np.random.default_rng(7).normal(size=(P, 6)))
    return ctx, cs, t, params


@pytest.mark.parametrize("loss", [0, 1])
@pytest.mark.parametrize("regime", ["population", "near_optimum"])
def test_param_grad_matches_oracle(loss, regime):
    wts = (1.0, 0.7, 0.3)
    ctx, cs, t, params = _setup(P=9, C=3, masks=[7, 3, 5], seed_scale=None if regime == "population" else 0.02)
    L, dL = ctx.param_grad(torch.tensor(params, device="cuda"), targets_to_device(t), w=wts, loss=loss)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    L, dL = L.cpu().numpy(), dL.cpu().numpy()
    for p in range(len(params)):
        Lr, gr = oracle.loss_and_grad(cs, params[p], t, w=wts, loss="sq" if loss == 0 else "z")
        print(p, Lr, L[p], gr, dL[p])
        assert abs(L[p] - Lr) <= 1e-5 * abs(Lr)
        err = np.abs(dL[p] - gr)
        assert (err <= 1e-3 * np.abs(gr).max()).all(), (err, gr)
