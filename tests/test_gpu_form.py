"""The Tersoff form (nine parameters: Eq. 8 angular function, free S in Eq. 11-14) through the batched
kernels: E/F/W and fitness parity with the oracle, in FP32 and FP64, over cells that exercise the
small, large and cluster launch buckets; switching forms; the calls that take the minimal form only."""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_11474_gb300 import inputs as I

from ._util import (TOL32, TOL64, energy_rel_err, fitness_bounds, force_err, targets_to_device, to_device,
                    virial_rel_err)

pytestmark = pytest.mark.gpu

# g^T of magnitude like beta (cos - h)^2 near Table 2 (gamma c^2 / d^4 ~ 0.3), S away from 2
XG = np.array([3.2, 1.45, 2.25, 1.9, 0.65, -0.6, 0.06, 20.0, 3.0])


@pytest.fixture()
def ctx():
    from paper_1909_11474_gb300 import binding
    c = binding.Context(0)
    c.set_form(binding.FORM_TERSOFF)
    return c


def _params(P, seed):
    rng = np.random.default_rng(seed)
    x = XG[None, :] * rng.uniform(0.95, 1.05, size=(P, 9))
    x[0, 3] = 2.0                                     # one set at S = 2
    return x


def _mixed(seed, C):
    rng = np.random.default_rng(seed)
    sizes = [(1, 1, 1), (2, 2, 2), (1, 2, 3), (3, 2, 2), (2, 1, 1)]
    return I.make_cells(rng, C, lambda: sizes[rng.integers(0, len(sizes))],
                        lambda: I.random_strain(rng, 0.03), lambda: float(rng.uniform(0.05, 0.2)),
                        lambda: int(rng.integers(0, 3)))


def _compare(ctx, cs, params, precision):
    tol = TOL32 if precision == 32 else TOL64
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    E, F, W = ctx.eval(torch.tensor(params, device="cuda"), precision=precision)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    Er, Wr, Fr, ES, WS, FS = oracle.evaluate_batch(cs, params, scales=True, force_scales=True)
    E, F, W = E.cpu().numpy(), F.cpu().double().numpy(), W.cpu().numpy()
    assert energy_rel_err(E, Er, ES).max() < tol["E"]
    assert virial_rel_err(W, Wr, WS).max() < tol["W"]
    assert force_err(F, Fr, FS) < tol["F"]


@pytest.mark.parametrize("precision", [32, 64])
def test_tersoff_form_eval_matches_oracle_on_mixed_cells(ctx, precision):
    _compare(ctx, _mixed(5, 10), _params(5, 1), precision)


@pytest.mark.parametrize("precision", [32, 64])
def test_tersoff_form_eval_matches_oracle_on_large_cells(ctx, precision):
    """Cells of up to 512 atoms (several CTAs of a cluster per configuration)."""
    cs = I.workload_uneven(P=1, C=6)["configs"]
    assert cs.natoms.max() >= 128
    _compare(ctx, cs, _params(3, 2), precision)


def test_tersoff_form_fitness_matches_oracle(ctx):
    w = I.workload_ga_batch(P=4, C=5)
    cs = w["configs"]
    x = _params(9, 3)
    Eh, Wh, Fh = oracle.evaluate_batch(cs, XG[None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0],
                       mask=np.array([7, 3, 5, 6, 1], np.uint8))
    wts = (1.0, 0.7, 0.3)
    E, W, F, ES, WS, FS = oracle.evaluate_batch(cs, x, scales=True, force_scales=True)
    ref = oracle.fitness_from_predictions(cs, t, E, W, F, w=wts)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    Z, Zq, S = ctx.fitness(torch.tensor(x, device="cuda"), targets_to_device(t), w=wts, precision=32)
    Z, Zq, S = Z.cpu().numpy(), Zq.cpu().numpy(), S.cpu().numpy()
    B = fitness_bounds(cs, t, E, W, F, ES, WS, TOL32, FS=FS)
    D = ref["D"]
    assert (np.abs(np.sqrt(S) - np.sqrt(ref["S"])) <= B).all()
    assert (np.abs(Z - ref["Z"]) <= (np.asarray(wts)[None, :] * B / np.sqrt(D)[None, :]).sum(-1)).all()


def test_switching_forms_and_minimal_only_calls(ctx):
    """The fitness of the minimal form is the same before and after a Tersoff-form call on the same
    context (graph replay keyed by the form); calls that take the minimal form only refuse."""
    from paper_1909_11474_gb300 import binding
    w = I.workload_ga_batch(P=8, C=6)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    tg = targets_to_device(I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0]))
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    p6 = torch.tensor(w["params"], device="cuda")
    p9 = torch.tensor(_params(8, 4), device="cuda")
    ctx.set_form(binding.FORM_MINIMAL)
    z0 = ctx.fitness(p6, tg)[0].cpu().numpy()
    ctx.set_form(binding.FORM_TERSOFF)
    z9 = ctx.fitness(p9, tg)[0].cpu().numpy()
    with pytest.raises(binding.TersoffError) as ei:
        ctx.autotune(p6, tg)
    assert ei.value.code == binding.E_UNSUPPORTED
    with pytest.raises(binding.TersoffError):
        ctx.set_form(7)
    ctx.set_form(binding.FORM_MINIMAL)
    z1 = ctx.fitness(p6, tg)[0].cpu().numpy()
    assert np.array_equal(z0, z1)
    assert np.isfinite(z9).all() and not np.allclose(z9[:len(z0)], z0)
    assert ctx.get_status() == 0
