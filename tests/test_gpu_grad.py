"""Parity of the adjoint kernel (loss gradient over the six parameters) with the FP64 oracle, with
central finite differences of the library's FP64 loss, and through the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_11474_gb300 import inputs as I

from ._util import fitness_bounds, targets_to_device, to_device

pytestmark = pytest.mark.gpu

WTS = (1.0, 0.7, 0.3)
# Gradient bar: FP32 pair arithmetic, FP64 accumulation; each component within 1e-4 of the largest
# component of the FP64 oracle's gradient for that parameter set.
GRAD_TOL = 1e-4


def _setup(P, C, masks, near=None):
    from paper_1909_11474_gb300 import binding
    w = I.workload_adjoint(P=P, C=C)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0], mask=np.asarray(masks, np.uint8))
    ctx = binding.Context(0)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    params = w["params"]
    if near is not None:     # parameter sets near the hidden one: the regime of the gradient polish
        params = w["hidden"][None, :] * (1 + near * np.random.default_rng(7).normal(size=(P, 6)))
    return ctx, cs, t, params


def _loss_bound(cs, t, params, loss):
    """|dL| implied by the per-quantity parity bars: |d sqrt(S_q)| <= B_q (triangle inequality)."""
    E, W, F, ES, WS, FS = oracle.evaluate_batch(cs, params, scales=True, force_scales=True)
    ref = oracle.fitness_from_predictions(cs, t, E, W, F, w=WTS)
    B = fitness_bounds(cs, t, E, W, F, ES, WS, FS=FS)
    D = ref["D"]
    rs = np.sqrt(ref["S"])
    w = np.asarray(WTS)[None, :]
    if loss == 0:
        return (w * B * (2 * rs + B) / D[None, :]).sum(-1)
    return (w * B / np.sqrt(D)[None, :]).sum(-1)


@pytest.mark.parametrize("loss", [0, 1])
@pytest.mark.parametrize("regime", ["population", "near_optimum"])
def test_param_grad_matches_oracle(loss, regime):
    ctx, cs, t, params = _setup(P=9, C=3, masks=[7, 3, 5], near=None if regime == "population" else 0.02)
    L, dL = ctx.param_grad(torch.tensor(params, device="cuda"), targets_to_device(t), w=WTS, loss=loss)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    L, dL = L.cpu().numpy(), dL.cpu().numpy()
    bound = _loss_bound(cs, t, params, loss)
    for p in range(len(params)):
        Lr, gr = oracle.loss_and_grad(cs, params[p], t, w=WTS, loss="sq" if loss == 0 else "z")
        assert abs(L[p] - Lr) <= bound[p]
        assert (np.abs(dL[p] - gr) <= GRAD_TOL * np.abs(gr).max()).all(), (dL[p], gr)


def test_param_grad_two_tiles_and_fd_of_fp64_loss():
    """P = 40 spans two 32-wide parameter tiles; every component against central differences
    (h = 1e-6 relative) of the library's FP64 loss, and the oracle on sampled sets."""
    ctx, cs, t, params = _setup(P=40, C=4, masks=[7, 7, 6, 5])
    tg = targets_to_device(t)
    pt = torch.tensor(params, device="cuda")
    L, dL = ctx.param_grad(pt, tg, w=WTS, loss=0)
    dL = dL.cpu().numpy()
    for p in (0, 31, 32, 39):
        _, gr = oracle.loss_and_grad(cs, params[p], t, w=WTS, loss="sq")
        assert (np.abs(dL[p] - gr) <= GRAD_TOL * np.abs(gr).max()).all()
    fd = np.zeros((len(params), 6))
    for k in range(6):
        h = 1e-6 * np.abs(params[:, k])
        Lp = []
        for sgn in (1, -1):
            q = params.copy()
            q[:, k] += sgn * h
            _, Zq, _ = ctx.fitness(torch.tensor(q, device="cuda"), tg, w=WTS, precision=64)
            Lp.append((np.asarray(WTS)[None, :] * Zq.cpu().numpy() ** 2).sum(-1))
        fd[:, k] = (Lp[0] - Lp[1]) / (2 * h)
    assert (np.abs(dL - fd) <= GRAD_TOL * np.abs(fd).max(axis=1, keepdims=True)).all()


def test_autograd_function_backward():
    from paper_1909_11474_gb300.autograd import TersoffLoss
    ctx, cs, t, params = _setup(P=5, C=2, masks=[7, 7])
    tg = targets_to_device(t)
    x = torch.tensor(params, device="cuda", requires_grad=True)
    L = TersoffLoss.apply(x, ctx, tg, WTS, 0)
    g = torch.arange(1, 6, dtype=torch.float64, device="cuda")
    (L * g).sum().backward()
    _, dL = ctx.param_grad(x.detach(), tg, w=WTS, loss=0)
    assert torch.allclose(x.grad, g[:, None] * dL, rtol=1e-12, atol=0)


def test_param_grad_in_the_tersoff_form_matches_oracle():
    """Nine parameters (Eq. 8 angular function, free S): the adjoint's loss and gradient against the
    oracle's reverse-mode gradient, for sets spread around a Tersoff-form parameter set."""
    from paper_1909_11474_gb300 import binding
    xg = np.array([3.2, 1.45, 2.25, 1.9, 0.65, -0.6, 0.06, 20.0, 3.0])
    w = I.workload_adjoint(P=4, C=3)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, xg[None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0], mask=np.array([7, 3, 5], np.uint8))
    params = xg[None, :] * (1 + 0.03 * np.random.default_rng(11).normal(size=(5, 9)))
    ctx = binding.Context(0)
    ctx.set_form(binding.FORM_TERSOFF)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    L, dL = ctx.param_grad(torch.tensor(params, device="cuda"), targets_to_device(t), w=WTS, loss=0)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    L, dL = L.cpu().numpy(), dL.cpu().numpy()
    assert dL.shape == (5, 9)
    for p in range(len(params)):
        Lr, gr = oracle.loss_and_grad(cs, params[p], t, w=WTS, loss="sq")
        assert abs(L[p] - Lr) <= 1e-4 * abs(Lr) + 1e-9, (L[p], Lr)
        assert (np.abs(dL[p] - gr) <= GRAD_TOL * np.abs(gr).max()).all(), (dL[p], gr)


def _uneven_largest():
    """The two largest cells of the uneven batch (512 and 511 atoms: clusters of CTAs in the batched
    schedule), a middle one and the smallest (7 atoms), with targets from the hidden parameters."""
    w = I.workload_uneven(P=4, C=500)
    cs_all = w["configs"]
    order = np.argsort(cs_all.natoms, kind="stable")[::-1]
    pick = [int(order[0]), int(order[1]), int(order[len(order) // 2]), int(order[-1])]
    cs = I.pack_configs(*zip(*[cs_all.config(k) for k in pick]))
    rng = np.random.default_rng(11)
    return cs, w["hidden"], rng


@pytest.mark.parametrize("loss", [0, 1])
def test_param_grad_on_the_largest_uneven_cells(loss):
    """Configurations spread over clusters of CTAs take the split gradient path (evaluation, weights,
    per-slice tangent passes): loss and gradient against the oracle on the largest uneven-batch cells,
    mixed with cells that take the single-CTA adjoint kernel."""
    from paper_1909_11474_gb300 import binding
    cs, hidden, rng = _uneven_largest()
    Eh, Wh, Fh = oracle.evaluate_batch(cs, hidden[None, :])
    wd = {"configs": cs, "noise": I.target_noise(rng, cs.C, cs.natoms)}
    t = I.with_targets(wd, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0],
                       mask=np.array([7, 7, 3, 5], np.uint8))
    params = hidden[None, :] * (1 + 0.02 * rng.normal(size=(3, 6)))
    ctx = binding.Context(0)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    assert max(b["cluster"] for b in ctx.schedule_info()) > 1
    L, dL = ctx.param_grad(torch.tensor(params, device="cuda"), targets_to_device(t), w=WTS, loss=loss)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    L, dL = L.cpu().numpy(), dL.cpu().numpy()
    bound = _loss_bound(cs, t, params, loss)
    for p in range(len(params)):
        Lr, gr = oracle.loss_and_grad(cs, params[p], t, w=WTS, loss="sq" if loss == 0 else "z")
        assert abs(L[p] - Lr) <= bound[p], (L[p], Lr, bound[p])
        assert (np.abs(dL[p] - gr) <= GRAD_TOL * np.abs(gr).max()).all(), (dL[p], gr)


def test_param_grad_split_path_in_the_tersoff_form():
    """Nine parameters on the largest uneven cells: the split path's dual passes in the Tersoff form."""
    from paper_1909_11474_gb300 import binding
    cs, _, rng = _uneven_largest()
    xg = np.array([3.2, 1.45, 2.25, 1.9, 0.65, -0.6, 0.06, 20.0, 3.0])
    Eh, Wh, Fh = oracle.evaluate_batch(cs, xg[None, :])
    wd = {"configs": cs, "noise": I.target_noise(rng, cs.C, cs.natoms)}
    t = I.with_targets(wd, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0],
                       mask=np.array([7, 3, 5, 7], np.uint8))
    params = xg[None, :] * (1 + 0.03 * rng.normal(size=(2, 9)))
    ctx = binding.Context(0)
    ctx.set_form(binding.FORM_TERSOFF)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    L, dL = ctx.param_grad(torch.tensor(params, device="cuda"), targets_to_device(t), w=WTS, loss=0)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    L, dL = L.cpu().numpy(), dL.cpu().numpy()
    for p in range(len(params)):
        Lr, gr = oracle.loss_and_grad(cs, params[p], t, w=WTS, loss="sq")
        assert abs(L[p] - Lr) <= 1e-4 * abs(Lr) + 1e-9, (L[p], Lr)
        assert (np.abs(dL[p] - gr) <= GRAD_TOL * np.abs(gr).max()).all(), (dL[p], gr)
