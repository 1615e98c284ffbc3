"""The device GA generation against the oracle (bit for bit: ranks, genes and parameters), and a short
end-to-end fit with the gradient polish on synthetic data of a hidden parameter set."""
import numpy as np
import pytest
import torch

from oracle import ga as oga
from paper_1909_11474_gb300 import inputs as I

from ._util import targets_to_device, to_device

pytestmark = pytest.mark.gpu


XG = np.array([3.2, 1.45, 2.25, 1.9, 0.65, -0.6, 0.06, 20.0, 3.0])   # a Tersoff-form parameter set


def _case(seed, P, n_par, bad=0, ties=0, G=6):
    rng = np.random.default_rng(seed)
    Z = rng.uniform(0.0, 2.0, P)
    for k in range(ties):
        Z[(7 * k + 1) % P] = Z[(3 * k) % P]
    for k in range(bad):
        Z[(5 * k + 2) % P] = [np.nan, np.inf, -np.inf][k % 3]
    genes = rng.uniform(0.0, 1.0, (P, G))
    u = rng.uniform(0.0, 1.0, oga.n_uniforms(P, n_par, G) + 5)
    x = I.TABLE2_PARAMS if G == 6 else XG
    lo = x - 0.3 * np.abs(x)
    hi = x + 0.3 * np.abs(x)
    return Z, genes, u, lo, hi


@pytest.mark.parametrize("P,n_par,rate,bad,ties,G", [(200, 100, 0.2, 0, 0, 6), (200, 100, 0.05, 4, 6, 6),
                                                      (7, 3, 0.5, 1, 2, 6), (33, 33, 0.3, 0, 3, 6),
                                                      (1, 1, 1.0, 0, 0, 6), (4096, 1000, 0.1, 9, 20, 6),
                                                      (200, 100, 0.2, 3, 5, 9), (37, 11, 0.4, 1, 2, 1)])
def test_ga_step_matches_the_oracle_bit_for_bit(P, n_par, rate, bad, ties, G):
    from paper_1909_11474_gb300 import binding
    Z, genes, u, lo, hi = _case(P + n_par, P, n_par, bad, ties, G)
    if G == 1:
        lo, hi = lo[:1], hi[:1]
    want, order = oga.ga_step(Z, genes, u, n_par, rate)
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    g_out = torch.empty((P, G), dtype=torch.float64, device="cuda")
    x_out = torch.empty((P, G), dtype=torch.float64, device="cuda")
    o_out = torch.empty(P, dtype=torch.int32, device="cuda")
    binding.ga_step(d(Z), d(genes), d(u), d(lo), d(hi), n_par, rate, g_out, x_out, o_out)
    assert np.array_equal(o_out.cpu().numpy(), order)
    assert np.array_equal(g_out.cpu().numpy(), want)
    assert np.array_equal(x_out.cpu().numpy(), oga.phenotype(want, lo, hi))


def test_ga_step_rejects_bad_arguments():
    from paper_1909_11474_gb300 import binding
    Z, genes, u, lo, hi = _case(1, 8, 4)
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    g = d(genes)
    out = torch.empty((8, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.TersoffError):
        binding.ga_step(d(Z), g, d(u), d(lo), d(hi), 9, 0.1, out, out.clone())   # n_par > P
    with pytest.raises(binding.TersoffError):
        binding.ga_step(d(Z), g, d(u), d(lo), d(hi), 4, 1.5, out, out.clone())   # rate > 1
    with pytest.raises(binding.TersoffError):
        binding.ga_step(d(Z), g, d(u), d(lo), d(hi), 4, 0.1, g, out)             # in place


def test_ga_fit_then_polish_on_a_hidden_parameter_set():
    """20 configurations, noise-free targets of the Table 2 parameters: the elite never worsens (up to
    FP32 rounding), the GA cuts the best fitness by an order of magnitude, and the gradient polish
    lowers the loss."""
    from paper_1909_11474_gb300 import binding
    from paper_1909_11474_gb300.ga import GeneticFit, polish
    w = I.workload_ga_batch(P=4, C=20)
    cs = w["configs"]
    ctx = binding.Context(0)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    E, F, W = ctx.eval(torch.tensor(w["hidden"][None, :], device="cuda"), precision=64)
    natoms = cs.natoms.astype(np.float64)
    t = {"E": (E[0].cpu().numpy() / natoms), "W": W[0].cpu().numpy() / natoms[:, None],
         "F": F[0].cpu().numpy(), "mask": np.full(cs.C, 7, np.uint8)}
    tg = targets_to_device(t)
    lo = I.TABLE2_PARAMS - 0.3 * np.abs(I.TABLE2_PARAMS)
    hi = I.TABLE2_PARAMS + 0.3 * np.abs(I.TABLE2_PARAMS)
    fit = GeneticFit(ctx, tg, lo, hi, n_pop=200, n_par=100, seed=7)
    first = float(fit.evaluate().min())
    res = fit.run(n_gen=300, history=True)
    h = res["history"]
    # the elite is kept unaltered; its fitness is recomputed in whatever row it lands, and rows in a
    # narrow last tile sum their atoms in another FP32 order: near the optimum the force residuals are
    # small differences of FP32 forces, so equal up to 1e-4 relative
    worst = float(np.max(h[1:] / h[:-1] - 1.0))
    assert worst <= 1e-4, worst
    assert res["Z"] < 0.1 * first
    x, L0, L1 = polish(ctx, res["params"], tg, lo, hi, steps=30)
    assert L1 < L0
    rel = np.abs(x - w["hidden"]) / np.abs(w["hidden"])
    print("polish: L", L0, "->", L1, "max relative parameter error", rel.max())
    assert rel.max() < 1e-3, rel
    assert ctx.get_status() == 0


def test_ga_checkpoint_resume_is_bit_exact(tmp_path):
    """20 generations straight equal 10 generations, a checkpoint written to disk, a new GeneticFit
    loaded from it and 10 more generations: same population bit for bit, same best fitness."""
    from paper_1909_11474_gb300 import binding
    from paper_1909_11474_gb300.ga import GeneticFit
    w = I.workload_ga_batch(P=4, C=6)
    cs = w["configs"]
    ctx = binding.Context(0)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    E, F, W = ctx.eval(torch.tensor(w["hidden"][None, :], device="cuda"), precision=64)
    natoms = cs.natoms.astype(np.float64)
    tg = targets_to_device({"E": E[0].cpu().numpy() / natoms, "W": W[0].cpu().numpy() / natoms[:, None],
                            "F": F[0].cpu().numpy(), "mask": np.full(cs.C, 7, np.uint8)})
    lo = I.TABLE2_PARAMS - 0.3 * np.abs(I.TABLE2_PARAMS)
    hi = I.TABLE2_PARAMS + 0.3 * np.abs(I.TABLE2_PARAMS)
    a = GeneticFit(ctx, tg, lo, hi, n_pop=64, n_par=32, seed=11)
    ra = a.run(n_gen=20)
    b = GeneticFit(ctx, tg, lo, hi, n_pop=64, n_par=32, seed=11)
    b.run(n_gen=20, until=10)
    assert b.k == 10
    b.save(tmp_path / "ga.pt")
    del b
    c = GeneticFit.load(ctx, tg, tmp_path / "ga.pt")
    assert c.k == 10
    rc = c.run(n_gen=20)
    assert c.k == 20 and rc["generations"] == 20
    assert torch.equal(a.genes[a.cur], c.genes[c.cur])
    assert torch.equal(a.params, c.params)
    assert rc["Z"] == ra["Z"]
    with pytest.raises(ValueError):
        GeneticFit(ctx, tg, lo, hi, n_pop=32, n_par=16).load_state_dict(torch.load(tmp_path / "ga.pt", weights_only=True))


def test_ga_fits_in_the_tersoff_form():
    """Nine genes on a context in the Tersoff form: 200 generations on noise-free targets of a
    Tersoff-form parameter set; the elite never worsens (up to FP32 rounding) and the best fitness
    falls at least threefold."""
    from paper_1909_11474_gb300 import binding
    from paper_1909_11474_gb300.ga import GeneticFit
    w = I.workload_ga_batch(P=4, C=10)
    cs = w["configs"]
    ctx = binding.Context(0)
    ctx.set_form(binding.FORM_TERSOFF)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    E, F, W = ctx.eval(torch.tensor(XG[None, :], device="cuda"), precision=64)
    natoms = cs.natoms.astype(np.float64)
    tg = targets_to_device({"E": E[0].cpu().numpy() / natoms, "W": W[0].cpu().numpy() / natoms[:, None],
                            "F": F[0].cpu().numpy(), "mask": np.full(cs.C, 7, np.uint8)})
    lo, hi = XG - 0.3 * np.abs(XG), XG + 0.3 * np.abs(XG)
    with pytest.raises(ValueError):
        GeneticFit(ctx, tg, lo[:6], hi[:6])                 # six limits for a nine-parameter context
    fit = GeneticFit(ctx, tg, lo, hi, n_pop=100, n_par=50, seed=3)
    first = float(fit.evaluate().min())
    res = fit.run(n_gen=200, history=True)
    h = res["history"]
    assert float(np.max(h[1:] / h[:-1] - 1.0)) <= 1e-4
    assert res["Z"] < first / 3
    assert res["params"].shape == (9,)
    # the polish of this form (damped Newton on the nine-parameter adjoint gradient, and the variant
    # on finite differences of the FP64 fitness) drives the loss of the exact data towards zero; g^T's
    # three parameters are only loosely fixed by near-tetrahedral angles, so the test bars the loss,
    # not the parameters
    from paper_1909_11474_gb300.ga import polish
    x, L0, L1 = polish(ctx, res["params"], tg, lo, hi, steps=60)
    print("Tersoff-form polish: L", L0, "->", L1, "rel. parameter error", np.abs(x - XG) / np.abs(XG))
    assert L1 < 1e-4 * L0 and L1 < 1e-7
    x2, L0b, L2 = polish(ctx, res["params"], tg, lo, hi, steps=60, method="fd-newton")
    print("Tersoff-form polish on finite differences: L", L0b, "->", L2)
    assert L2 < 1e-3 * L0b
    assert ctx.get_status() == 0
