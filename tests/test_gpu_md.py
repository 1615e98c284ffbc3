"""Parity of the MD-scale force call (cell-list rebuild + E/F/W of one large cell) with the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_11474_gb300 import inputs as I

from ._util import TOL32, TOL64, energy_rel_err, force_err, virial_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1909_11474_gb300 import binding
    return binding.Context(0)


def _cell(reps, sigma, strain, seed, shift_images=False):
    rng = np.random.default_rng(seed)
    pos, box = I.diamond_supercell(reps)
    pos, box = I.apply_strain(pos, box, I.random_strain(rng, strain))
    pos = pos + rng.normal(0, sigma, pos.shape)
    if shift_images:   # some atoms given as periodic images outside the box
        k = rng.integers(-1, 2, size=(len(pos), 3))
        pos = pos + k @ box
    return pos, box


def _md(ctx, pos, box, params, precision):
    p = torch.tensor(pos, device="cuda")
    E, F, W = ctx.md_force(p, box, params, precision=precision)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    return float(E[0]), F.cpu().double().numpy(), W.cpu().numpy()


@pytest.mark.parametrize("case", [((3, 3, 3), 0.08, 0.0, False), ((4, 3, 3), 0.2, 0.03, True)])
def test_md_neighbor_lists_bit_exact(ctx, case):
    reps, sigma, strain, shifted = case
    pos, box = _cell(reps, sigma, strain, 3, shifted)
    _md(ctx, pos, box, I.TABLE2_PARAMS, 32)
    cnt, nbr, shift = ctx.md_export_neighbors()
    nl = oracle.neighbor_list(pos, box, 3.2)
    for i in range(len(pos)):
        e = slice(nl["off"][i], nl["off"][i + 1])
        assert cnt[i] == nl["off"][i + 1] - nl["off"][i]
        assert np.array_equal(nbr[i, :cnt[i]], nl["j"][e])
        assert np.array_equal(shift[i, :cnt[i]], nl["n"][e])


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("case", [((3, 3, 3), 0.08, 0.0, False), ((4, 3, 3), 0.2, 0.03, True)])
def test_md_energy_forces_virial(ctx, precision, case):
    reps, sigma, strain, shifted = case
    pos, box = _cell(reps, sigma, strain, 5, shifted)
    params = I.TABLE2_PARAMS * np.array([1.0, 1.01, 0.99, 1.1, 0.95, 1.02])
    E, F, W = _md(ctx, pos, box, params, precision)
    r = oracle.evaluate(pos, box, params)
    tol = TOL32 if precision == 32 else TOL64
    assert energy_rel_err(np.array([E]), np.array([r["E"]]), np.array([r["E_scale"]])).max() < tol["E"]
    assert virial_rel_err(W[None], r["W"][None], np.array([r["W_scale"]])).max() < tol["W"]
    assert force_err(F, r["F"], r["F_scale"]) < tol["F"]


def _cutout_force(pos, box, i, R2=3.2, pad=0.3):
    """F_i of the periodic cell from a non-periodic cut-out: every atom image within 2*R2 of atom i
    (the force on i depends on nothing farther), placed in a large empty box."""
    inv = np.linalg.inv(box)
    ds = (pos - pos[i]) @ inv
    pts = []
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for c in (-1, 0, 1):
                d = (ds - np.rint(ds) + np.array([a, b, c])) @ box
                keep = np.sqrt((d * d).sum(1)) < 2 * R2 + pad
                pts.append(d[keep])
    pts = np.concatenate(pts)
    order = np.argsort((pts * pts).sum(1))             # atom i itself (d = 0) first
    pts = pts[order]
    assert np.allclose(pts[0], 0.0)
    L = 60.0
    out = oracle.evaluate(pts + L / 2, np.eye(3) * L, I.TABLE2_PARAMS)
    return out["F"][0]


def test_md_full_size_sampled(ctx):
    """The 512,000-atom workload (40^3 conventional cells, sigma = 0.08 A): sampled neighbour lists
    and forces against the oracle, zero net force, translation invariance."""
    w = I.workload_md()
    pos, box = w["configs"].config(0)
    assert len(pos) == 512000
    E, F, W = _md(ctx, pos, box, I.TABLE2_PARAMS, 32)
    cnt, nbr, shift = ctx.md_export_neighbors()
    atoms = [0, 1, 777, 123457, 300001, 511999]
    for i, (j, n) in zip(atoms, oracle.neighbor_list_subset(pos, box, 3.2, atoms)):
        assert cnt[i] == len(j)
        assert np.array_equal(nbr[i, :cnt[i]], j) and np.array_equal(shift[i, :cnt[i]], n)
    for i in atoms[:4]:
        assert np.abs(F[i] - _cutout_force(pos, box, i)).max() < TOL32["F"]
    assert np.abs(F.sum(axis=0)).max() < 1e-3 * np.sqrt(len(pos)) * 1e-2
    E2, F2, W2 = _md(ctx, pos + np.array([0.37, -1.1, 2.3]), box, I.TABLE2_PARAMS, 32)
    assert abs(E2 - E) / abs(E) < 1e-5
    assert np.abs(F2 - F).max() < 1e-4
    # displaced diamond lies above the perfect-crystal minimum -2 D0 b0^2 = -4.62963 eV/atom
    # (closed form of the oracle pins) and within the thermal range of sigma = 0.08 A
    assert -4.62963 < E / len(pos) < -4.62963 + 0.3


def test_md_rejects_small_box(ctx):
    from paper_1909_11474_gb300 import binding
    pos, box = I.diamond_supercell((1, 1, 1))     # plane spacing 5.43 A < 3 R2 = 9.6 A
    with pytest.raises(binding.TersoffError) as ei:
        ctx.md_force(torch.tensor(pos, device="cuda"), box, I.TABLE2_PARAMS)
    assert ei.value.code == binding.E_ARG


@pytest.mark.parametrize("R2,per_atom", [(4.2, 16), (5.0, 28)])
def test_md_neighbor_lists_wide_cutoffs(ctx, R2, per_atom):
    """Long lists in a 4x4x4 diamond cell. R2 = 4.2 A: 16 neighbours, the records of a brick of cells
    and its surroundings staged in shared memory. R2 = 5 A: 28 neighbours, and the cells are the
    conventional cells (8 atoms each), so the surroundings of a brick hold more atoms than the stage
    and the records are read from global memory. The force kernel flags more than 8 neighbours and
    nothing else."""
    from paper_1909_11474_gb300 import binding
    pos, box = _cell((4, 4, 4), 0.05, 0.0, 9)
    ctx.md_force(torch.tensor(pos, device="cuda"), box, I.TABLE2_PARAMS, R1=R2 - 0.4, R2=R2, max_nbr=32)
    assert ctx.get_status() == binding.STATUS_MANY_NBRS
    cnt, nbr, shift = ctx.md_export_neighbors()
    nl = oracle.neighbor_list(pos, box, R2)
    assert (np.diff(nl["off"]) == per_atom).all()
    for i in range(len(pos)):
        e = slice(nl["off"][i], nl["off"][i + 1])
        assert cnt[i] == nl["off"][i + 1] - nl["off"][i]
        assert np.array_equal(nbr[i, :cnt[i]], nl["j"][e])
        assert np.array_equal(shift[i, :cnt[i]], nl["n"][e])


def test_md_short_lists_flag_overflow_and_count_every_neighbour(ctx):
    """max_nbr = 2 with 4 neighbours per atom: the overflow bit is set, the true count is returned and
    the kept entries are true neighbours in ascending order (which of them are kept is unspecified)."""
    from paper_1909_11474_gb300 import binding
    pos, box = _cell((3, 3, 3), 0.08, 0.0, 3)
    ctx.md_force(torch.tensor(pos, device="cuda"), box, I.TABLE2_PARAMS, max_nbr=2)
    assert ctx.get_status() & binding.STATUS_NBR_OVERFLOW
    cnt, nbr, shift = ctx.md_export_neighbors()
    nl = oracle.neighbor_list(pos, box, 3.2)
    for i in range(len(pos)):
        e = slice(nl["off"][i], nl["off"][i + 1])
        assert cnt[i] == nl["off"][i + 1] - nl["off"][i]
        full = {(int(j), tuple(n)) for j, n in zip(nl["j"][e], nl["n"][e])}
        kept = [(int(j), tuple(n)) for j, n in zip(nbr[i], shift[i])]
        assert all(k in full for k in kept) and kept == sorted(kept)


def test_md_nonfinite_atom_is_flagged_and_left_out(ctx):
    """An atom with a non-finite position gets no cell: the call flags it, its list is empty, and the
    other atoms' lists are the oracle's lists of the cell without it."""
    from paper_1909_11474_gb300 import binding
    pos, box = _cell((3, 3, 3), 0.08, 0.0, 3)
    bad = 17
    pos_nan = pos.copy()
    pos_nan[bad, 2] = np.nan
    ctx.md_force(torch.tensor(pos_nan, device="cuda"), box, I.TABLE2_PARAMS)
    assert ctx.get_status() & binding.STATUS_NONFINITE
    cnt, nbr, shift = ctx.md_export_neighbors()
    assert cnt[bad] == 0
    idx = np.flatnonzero(np.arange(len(pos)) != bad)
    nl = oracle.neighbor_list(pos[idx], box, 3.2)
    for a, i in enumerate(idx):
        e = slice(nl["off"][a], nl["off"][a + 1])
        assert cnt[i] == nl["off"][a + 1] - nl["off"][a]
        assert np.array_equal(nbr[i, :cnt[i]], idx[nl["j"][e]])
        assert np.array_equal(shift[i, :cnt[i]], nl["n"][e])
    _md(ctx, pos, box, I.TABLE2_PARAMS, 32)      # the next call on finite positions is clean
