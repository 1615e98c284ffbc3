"""The FLOP model of the roofline figures: the op-counted formula listing (oracle/flops.py) and the
constants the benchmark freezes from it.

The listing writes out the per-atom terms of Eq. 2-10 and the derivative of the site energy with
respect to its bond vectors; before its counts mean anything, its values must be those of the method:
E, F and W from the listing in floating point equal the oracle's (autograd of Eq. 1-14) on cells with
bonds inside R1, in the switching region (R1, R2) and with several neighbour counts.
"""
import numpy as np
import pytest

import oracle
from oracle import flops
from paper_1909_11474_gb300 import inputs as I


def _cell(reps, a, sigma, seed, vacancies=0):
    rng = np.random.default_rng(seed)
    pos, box = I.diamond_supercell(reps, a=a)
    if vacancies:
        pos = np.delete(pos, rng.choice(len(pos), vacancies, replace=False), axis=0)
    return pos + rng.normal(0.0, sigma, pos.shape), box


@pytest.mark.parametrize("case", ["table2", "switching", "vacancy"])
def test_listing_equals_the_oracle(case):
    if case == "table2":
        pos, box = _cell((1, 1, 1), 5.431, 0.1, 1)
        x = I.TABLE2_PARAMS
    elif case == "switching":   # nearest neighbours near 2.94 A: every bond in (R1, R2)
        pos, box = _cell((1, 1, 1), 6.79, 0.05, 2)
        x = I.TABLE2_PARAMS * np.array([1.1, 0.9, 1.05, 1.2, 0.8, 1.1])
    else:
        pos, box = _cell((1, 1, 2), 5.3, 0.15, 3, vacancies=2)
        x = I.TABLE2_PARAMS * np.array([0.9, 1.1, 0.97, 0.8, 1.2, 0.9])
    ref = oracle.evaluate(pos, box, x)
    Ft = np.random.default_rng(9).normal(0.0, 1.0, pos.shape)
    E, F, W, res = flops.evaluate_listing(pos, box, x, F_target=Ft)
    assert abs(E - ref["E"]) <= 1e-11 * max(1.0, abs(ref["E"]))
    assert np.abs(F - ref["F"]).max() <= 1e-10
    assert np.abs(W - ref["W"]).max() <= 1e-10 * max(1.0, np.abs(ref["W"]).max())
    assert abs(res - ((ref["F"] - Ft) ** 2).sum()) <= 1e-9 * max(1.0, res)


def test_counts_follow_the_fitted_form_and_are_frozen_in_the_benchmark():
    import bench
    got = flops.count_per_unit()
    assert got == {"per_bond": 50.0, "per_triplet": 37.0, "per_atom": 10.0, "per_config": -2, "xu_per_bond": 6,
                   "xu_per_atom": 0}
    assert (bench.FLOP_PER_BOND, bench.FLOP_PER_TRIPLET, bench.FLOP_PER_ATOM, bench.FLOP_PER_CONFIG,
            bench.XU_PER_BOND) == (got["per_bond"], got["per_triplet"], got["per_atom"], got["per_config"],
                                   got["xu_per_bond"])


def test_counted_operations_match_the_whole_cell_count():
    """The per-unit form reproduces the count of a whole configuration run through the listing."""
    pos, box = _cell((1, 1, 1), 5.431, 0.05, 4)
    cnt = flops.Counter()
    flops.evaluate_listing(pos, box, I.TABLE2_PARAMS, counter=cnt, F_target=np.zeros_like(pos))
    nl = oracle.neighbor_list(pos, box)
    m = np.diff(nl["off"])
    u = flops.count_per_unit()
    want = u["per_bond"] * m.sum() + u["per_triplet"] * (m * (m - 1)).sum() + u["per_atom"] * len(m) + u["per_config"]
    method = {k: v for k, v in cnt.flop.items() if not k.startswith("geometry")}   # the build's part aside
    assert sum(method.values()) == want
    assert sum(v for k, v in cnt.xu.items() if not k.startswith("geometry")) == u["xu_per_bond"] * m.sum()


def test_dual_listing_tangents_equal_central_differences():
    """The forward-mode (dual-number) run of the listing, whose operations the adjoint's roofline counts,
    gives dE/dx, dW/dx and the tangent of the force residual equal to central differences of the
    floating-point listing (h = 1e-6 relative)."""
    pos, box = _cell((1, 1, 1), 6.2, 0.08, 5)           # bonds around 2.7 A: some inside, some beyond R1
    x = I.TABLE2_PARAMS * np.array([1.05, 0.95, 1.02, 1.1, 0.9, 1.05])
    Ft = np.random.default_rng(11).normal(0.0, 1.0, pos.shape)
    E, F, W, res = flops.evaluate_listing(pos, box, x, F_target=Ft, tangents=True)
    for q in range(6):
        h = 1e-6 * abs(x[q])
        xp, xm = x.copy(), x.copy()
        xp[q] += h
        xm[q] -= h
        Ep, _, Wp, rp = flops.evaluate_listing(pos, box, xp, F_target=Ft)
        Em, _, Wm, rm = flops.evaluate_listing(pos, box, xm, F_target=Ft)
        assert abs(E[1][q] - (Ep - Em) / (2 * h)) <= 1e-6 * max(1.0, abs(E[1][q]))
        assert abs(res[1][q] - (rp - rm) / (2 * h)) <= 1e-6 * max(1.0, abs(res[1][q]))
        dW = np.array([w[1][q] for w in W])
        assert np.abs(dW - (Wp - Wm) / (2 * h)).max() <= 1e-6 * max(1.0, np.abs(dW).max())


def test_md_and_adjoint_counts_are_frozen_in_the_benchmark():
    import bench
    md = flops.count_per_unit(geometry=True, inner=True)
    assert (bench.MD_FLOP_PER_BOND, bench.MD_FLOP_PER_TRIPLET, bench.MD_FLOP_PER_ATOM, bench.MD_XU_PER_BOND) == \
        (md["per_bond"], md["per_triplet"], md["per_atom"], md["xu_per_bond"])
    adj = flops.count_per_unit(tangents=True)
    assert (bench.ADJ_FLOP_PER_BOND, bench.ADJ_FLOP_PER_TRIPLET, bench.ADJ_FLOP_PER_ATOM, bench.ADJ_FLOP_PER_CONFIG,
            bench.ADJ_XU_PER_BOND) == (adj["per_bond"], adj["per_triplet"], adj["per_atom"], adj["per_config"],
                                       adj["xu_per_bond"])
