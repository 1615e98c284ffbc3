"""Parity of the CUDA batched path (neighbour build, E/F/W, fitness) with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_11474_gb300 import inputs as I

from ._util import (TOL32, TOL64, energy_rel_err, fitness_bounds, force_err, targets_to_device, to_device,
                    virial_rel_err)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1909_11474_gb300 import binding
    return binding.Context(0)


def _build(ctx, cs, R1=2.8, R2=3.2, M=16):
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, R1, R2, M)
    return pos, box


def _oracle_lists(cs, R2=3.2):
    out = []
    for c in range(cs.C):
        nl = oracle.neighbor_list(*cs.config(c), R2)
        a = int(cs.atom_off[c])
        for i in range(cs.natoms[c]):
            e = slice(nl["off"][i], nl["off"][i + 1])
            out.append((nl["j"][e] + a, nl["n"][e]))
    return out


def _mixed_set(seed=5, C=10):
    rng = np.random.default_rng(seed)
    sizes = [(1, 1, 1), (2, 2, 2), (1, 2, 3), (3, 2, 2), (2, 1, 1)]
    return I.make_cells(rng, C, lambda: sizes[rng.integers(0, len(sizes))],
                        lambda: I.random_strain(rng, 0.03), lambda: float(rng.uniform(0.05, 0.2)),
                        lambda: int(rng.integers(0, 3)))


def _special_set():
    """Edge cases: a lone atom (no neighbours), a dimer (zeta = 0), one atom whose only neighbours are
    its own images, a compressed 8-atom cell with several images of the same j."""
    pos_list, box_list = [], []
    pos_list.append(np.array([[1.0, 2.0, 3.0]])); box_list.append(np.eye(3) * 12.0)
    pos_list.append(np.array([[0.0, 0.0, 0.0], [2.3, 0.1, 0.0]])); box_list.append(np.eye(3) * 15.0)
    pos_list.append(np.array([[0.1, 0.2, 0.3]])); box_list.append(np.eye(3) * 2.5)
    p, b = I.diamond_supercell((1, 1, 1), a=4.6)
    pos_list.append(p + np.random.default_rng(3).normal(0, 0.05, p.shape)); box_list.append(b)
    return I.pack_configs(pos_list, box_list)


@pytest.mark.parametrize("which", ["single", "ga", "mixed", "special"])
def test_neighbor_lists_bit_exact(ctx, which):
    cs = {"single": lambda: I.workload_single_cell()["configs"],
          "ga": lambda: I.workload_ga_batch(P=2, C=20)["configs"],
          "mixed": _mixed_set, "special": _special_set}[which]()
    _build(ctx, cs)
    cnt, nbr, shift = ctx.export_neighbors()
    ref = _oracle_lists(cs)
    assert len(ref) == cs.Ntot
    for i, (j, n) in enumerate(ref):
        assert cnt[i] == len(j), i
        assert np.array_equal(nbr[i, :cnt[i]], j), i
        assert np.array_equal(shift[i, :cnt[i]], n), i
        assert (nbr[i, cnt[i]:] == -1).all()


def _compare_eval(ctx, cs, params, precision, tol):
    P = len(params)
    pt = torch.tensor(params, dtype=torch.float64, device="cuda")
    E, F, W = ctx.eval(pt, precision=precision)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    Er, Wr, Fr, ES, WS, FS = oracle.evaluate_batch(cs, params, scales=True, force_scales=True)
    E, F, W = E.cpu().numpy(), F.cpu().double().numpy(), W.cpu().numpy()
    eE = energy_rel_err(E, Er, ES).max()
    eW = virial_rel_err(W, Wr, WS).max()
    eF = force_err(F, Fr, FS)
    assert eE < tol["E"], eE
    assert eW < tol["W"], eW
    assert eF < tol["F"], eF
    return eE, eW, eF


@pytest.mark.parametrize("precision", [32, 64])
def test_single_cell_eval(ctx, precision):
    w = I.workload_single_cell()
    _build(ctx, w["configs"])
    _compare_eval(ctx, w["configs"], w["params"], precision, TOL32 if precision == 32 else TOL64)


def test_physical_forces_strict_absolute_bar(ctx):
    """Table 2 parameters on strained, displaced 64-atom cells: |dF| < 1e-4 eV/A with no scaling."""
    w = I.workload_ga_batch(P=2, C=8)
    _build(ctx, w["configs"])
    params = np.stack([w["hidden"], w["hidden"] * np.array([1.02, 0.99, 1.0, 1.05, 0.97, 1.03])])
    E, F, W = ctx.eval(torch.tensor(params, device="cuda"), precision=32)
    _, _, Fr = oracle.evaluate_batch(w["configs"], params)
    assert np.abs(F.cpu().double().numpy() - Fr).max() < 1e-4


@pytest.mark.parametrize("precision", [32, 64])
def test_ga_batch_eval_ragged_tiles(ctx, precision):
    """P = 37 spans three parameter tiles of 16 with a ragged tail; 64-atom strained cells."""
    w = I.workload_ga_batch(P=37, C=6)
    _build(ctx, w["configs"])
    _compare_eval(ctx, w["configs"], w["params"], precision, TOL32 if precision == 32 else TOL64)


@pytest.mark.parametrize("precision", [32, 64])
def test_mixed_sizes_eval(ctx, precision):
    """8..96-atom cells with vacancies, strain and pairs inside the switching region."""
    cs = _mixed_set()
    _build(ctx, cs)
    params = I.population(np.random.default_rng(8), 5)[0]
    _compare_eval(ctx, cs, params, precision, TOL32 if precision == 32 else TOL64)


@pytest.mark.parametrize("precision", [32, 64])
def test_special_cases_eval(ctx, precision):
    cs = _special_set()
    _build(ctx, cs)
    _compare_eval(ctx, cs, I.TABLE2_PARAMS[None, :], precision, TOL32 if precision == 32 else TOL64)


@pytest.mark.parametrize("precision", [32, 64])
def test_fitness_matches_oracle(ctx, precision):
    w = I.workload_ga_batch(P=21, C=5)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0],
                       mask=np.array([7, 3, 5, 6, 1], np.uint8))
    wts = (1.0, 0.7, 0.3)
    E, W, F, ES, WS, FS = oracle.evaluate_batch(cs, w["params"], scales=True, force_scales=True)
    ref = oracle.fitness_from_predictions(cs, t, E, W, F, w=wts)
    _build(ctx, cs)
    Z, Zq, S = ctx.fitness(torch.tensor(w["params"], device="cuda"), targets_to_device(t),
                           w=wts, precision=precision)
    Z, Zq, S = Z.cpu().numpy(), Zq.cpu().numpy(), S.cpu().numpy()
    B = fitness_bounds(cs, t, E, W, F, ES, WS, TOL32 if precision == 32 else TOL64, FS=FS)
    D = ref["D"]
    assert (np.abs(np.sqrt(S) - np.sqrt(ref["S"])) <= B).all()
    assert (np.abs(Zq - ref["Zq"]) <= B / np.sqrt(D)[None, :]).all()
    assert (np.abs(Z - ref["Z"]) <= (np.asarray(wts)[None, :] * B / np.sqrt(D)[None, :]).sum(-1)).all()


def test_fitness_nonfinite_parameters_rank_last(ctx):
    w = I.workload_ga_batch(P=3, C=2)
    cs = w["configs"]
    _build(ctx, cs)
    params = w["params"].copy()
    params[1, 0] = np.nan
    t = {"E": np.full(cs.C, -4.6), "W": np.zeros((cs.C, 6)), "F": np.zeros((cs.Ntot, 3)),
         "mask": np.full(cs.C, 7, np.uint8)}
    Z, _, _ = ctx.fitness(torch.tensor(params, device="cuda"), targets_to_device(t))
    Z = Z.cpu().numpy()
    assert np.isinf(Z[1]) and np.isfinite(Z[0]) and np.isfinite(Z[2])


@pytest.mark.parametrize("which", ["ga", "mixed", "special"])
def test_plain_fp64_path(ctx, which):
    """The plain one-launch-per-(p, c) FP64 path against the oracle and the batched FP64 path."""
    if which == "ga":
        w = I.workload_ga_batch(P=3, C=4)
        cs, params = w["configs"], w["params"]
    elif which == "mixed":
        cs, params = _mixed_set(C=6), I.population(np.random.default_rng(9), 2)[0]
    else:
        cs, params = _special_set(), I.TABLE2_PARAMS[None, :]
    _build(ctx, cs)
    pt = torch.tensor(params, device="cuda")
    E, F, W = ctx.eval_plain(pt)
    Eb, Fb, Wb = ctx.eval(pt, precision=64)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    Er, Wr, Fr, ES, WS, FS = oracle.evaluate_batch(cs, params, scales=True, force_scales=True)
    E, F, W = E.cpu().numpy(), F.cpu().numpy(), W.cpu().numpy()
    assert energy_rel_err(E, Er, ES).max() < TOL64["E"]
    assert virial_rel_err(W, Wr, WS).max() < TOL64["W"]
    assert force_err(F, Fr, FS) < TOL64["F"]
    assert np.allclose(E, Eb.cpu().numpy(), rtol=1e-12, atol=1e-12)
    assert np.allclose(F, Fb.cpu().numpy(), rtol=1e-10, atol=1e-11)


def test_kernel_timer_and_launch_count(ctx):
    """The measurement hooks: one timed batched-kernel sequence per fitness call while enabled, none
    after disabling, and a launch count that grows by the same amount for identical calls."""
    w = I.workload_ga_batch(P=40, C=6)
    cs = w["configs"]
    _build(ctx, cs)
    t = {"E": np.full(cs.C, -4.6), "W": np.zeros((cs.C, 6)), "F": np.zeros((cs.Ntot, 3)),
         "mask": np.full(cs.C, 7, np.uint8)}
    params, tg = torch.tensor(w["params"], device="cuda"), targets_to_device(t)
    ctx.profile(True)
    n0 = ctx.kernel_launches()
    ctx.fitness(params, tg)
    n1 = ctx.kernel_launches()
    ctx.fitness(params, tg)
    ctx.fitness(params, tg)
    n3 = ctx.kernel_launches()
    count, ms = ctx.profile_read()
    assert count == 3 and ms > 0.0
    assert n1 - n0 >= 3 and n3 - n1 == 2 * (n1 - n0)   # prep + batched kernel(s) + finalize per call
    ctx.profile(False)
    ctx.fitness(params, tg)
    assert ctx.profile_read() == (0, 0.0)
    assert ctx.get_status() == 0


def test_fitness_graph_replay_matches_direct_launches(ctx):
    """The fitness call replayed from its captured CUDA graph (with programmatic dependent launch)
    gives the results of plain direct launches, and a change of arguments (targets, weights, P) or of
    the neighbour build re-captures."""
    w = I.workload_ga_batch(P=45, C=7)
    cs = w["configs"]
    _build(ctx, cs)
    rng = np.random.default_rng(11)
    t1 = {"E": np.full(cs.C, -4.6), "W": rng.normal(0, 0.01, (cs.C, 6)), "F": rng.normal(0, 0.3, (cs.Ntot, 3)),
          "mask": np.array([7, 1, 2, 4, 7, 3, 6], np.uint8)}
    t2 = dict(t1, E=np.full(cs.C, -4.5))
    params = torch.tensor(w["params"], device="cuda")
    tg1, tg2 = targets_to_device(t1), targets_to_device(t2)

    def run(graphs, tg, wts, P=None):
        ctx.set_launch_mode(graphs=graphs, pdl=graphs)
        Z, Zq, S = ctx.fitness(params[:P], tg, w=wts)
        return torch.cat([Z[:, None], Zq, S], 1).cpu().numpy()

    for tg, wts in [(tg1, (1.0, 1.0, 1.0)), (tg2, (1.0, 1.0, 1.0)), (tg2, (0.5, 2.0, 1.0)), (tg1, (1.0, 1.0, 1.0))]:
        direct = run(False, tg, wts)
        first = run(True, tg, wts)       # captures
        again = run(True, tg, wts)       # replays
        assert np.array_equal(direct, first) and np.array_equal(direct, again)
    assert np.array_equal(run(False, tg1, (1, 1, 1), P=33), run(True, tg1, (1, 1, 1), P=33))
    # a new neighbour build of other configurations: the replay must not reuse the old schedule
    w2 = I.workload_ga_batch(P=45, C=4)
    cs2 = w2["configs"]
    _build(ctx, cs2)
    t3 = targets_to_device({"E": np.full(cs2.C, -4.6), "W": np.zeros((cs2.C, 6)),
                            "F": np.zeros((cs2.Ntot, 3)), "mask": np.full(cs2.C, 7, np.uint8)})
    assert np.array_equal(run(False, t3, (1, 1, 1)), run(True, t3, (1, 1, 1)))
    ctx.set_launch_mode()
    assert ctx.get_status() == 0


def test_build_errors_reported_by_next_call(ctx):
    """The neighbour build is queued and checked by the next call that uses it: a list overflow and
    non-finite positions come back from that call, and a valid rebuild afterwards works."""
    from paper_1909_11474_gb300 import binding
    cs = I.workload_single_cell()["configs"]
    params = torch.tensor(I.TABLE2_PARAMS[None, :], device="cuda")
    _build(ctx, cs, M=2)                      # diamond has 4 neighbours per atom
    with pytest.raises(binding.TersoffError) as ei:
        ctx.eval(params)
    assert ei.value.code == binding.E_NBR_OVERFLOW
    pos, box = to_device(cs)
    pos[5, 1] = float("nan")
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    with pytest.raises(binding.TersoffError) as ei:
        ctx.build_info()
    assert ei.value.code == binding.E_NONFINITE
    ctx.get_status()                           # clear the status bits of the failed builds
    _build(ctx, cs)
    E, F, W = ctx.eval(params, precision=64)
    r = oracle.evaluate(*cs.config(0), I.TABLE2_PARAMS)
    assert abs(float(E[0, 0]) - r["E"]) < 1e-9 * abs(r["E"])
    assert ctx.get_status() == 0


def test_autotune_keeps_results_within_the_bars(ctx):
    """The schedule autotuner times its candidates, keeps the fastest, and the tuned fitness still
    meets the oracle bounds (a partly filled last tile here: P = 45 = 32 + 13)."""
    w = I.workload_ga_batch(P=45, C=5)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0])
    E, W, F, ES, WS, FS = oracle.evaluate_batch(cs, w["params"], scales=True, force_scales=True)
    ref = oracle.fitness_from_predictions(cs, t, E, W, F)
    B = fitness_bounds(cs, t, E, W, F, ES, WS, TOL32, FS=FS)
    _build(ctx, cs)
    params, tg = torch.tensor(w["params"], device="cuda"), targets_to_device(t)
    ms, tried = ctx.autotune(params, tg, reps=2)
    assert ms > 0.0 and tried >= 4             # chunkings 1, 2 x narrow last tile on / off
    Z, Zq, S = ctx.fitness(params, tg)
    S = S.cpu().numpy()
    assert (np.abs(np.sqrt(S) - np.sqrt(ref["S"])) <= B).all()
    assert ctx.get_status() == 0


@pytest.mark.parametrize("P", [45, 40, 7])
@pytest.mark.parametrize("tile,warps,items,narrow", [(32, 8, 1, 1), (32, 8, 3, 0), (16, 8, 1, 1), (16, 8, 2, 0),
                                                     (16, 8, 5, 1), (32, 12, 1, 1), (32, 12, 2, 0)])
def test_every_schedule_meets_the_oracle_bars(ctx, P, tile, warps, items, narrow):
    """Each schedule the autotuner can choose (tile width, work items per configuration, narrow last
    tile) gives a fitness within the oracle bounds, for full, half and small last tiles."""
    w = I.workload_ga_batch(P=P, C=5)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0])
    E, W, F, ES, WS, FS = oracle.evaluate_batch(cs, w["params"], scales=True, force_scales=True)
    ref = oracle.fitness_from_predictions(cs, t, E, W, F)
    B = fitness_bounds(cs, t, E, W, F, ES, WS, TOL32, FS=FS)
    _build(ctx, cs)
    ctx.set_schedule(P, tile=tile, items_per_config=items, narrow=bool(narrow), warps=warps)
    Z, Zq, S = ctx.fitness(torch.tensor(w["params"], device="cuda"), targets_to_device(t))
    S = S.cpu().numpy()
    assert (np.abs(np.sqrt(S) - np.sqrt(ref["S"])) <= B).all()
    assert ctx.get_status() == 0


@pytest.mark.parametrize("change_counts", [False, True])
def test_fitness_queued_before_rebuild_check(ctx, change_counts):
    """A fitness call right after a rebuild of the same layout is queued before the host has checked
    the new neighbour counts. Whether the counts stayed or changed, its results equal those of a fresh
    context built once on the new positions."""
    from paper_1909_11474_gb300 import binding
    w = I.workload_ga_batch(P=37, C=6)
    cs = w["configs"]
    t = {"E": np.full(cs.C, -4.6), "W": np.zeros((cs.C, 6)), "F": np.zeros((cs.Ntot, 3)),
         "mask": np.full(cs.C, 7, np.uint8)}
    params, tg = torch.tensor(w["params"], device="cuda"), targets_to_device(t)
    ctx.set_launch_mode()
    _build(ctx, cs)
    ctx.fitness(params, tg)
    pos2 = cs.pos.copy() + np.random.default_rng(4).normal(0, 0.01, cs.pos.shape)
    box2 = cs.box.copy()
    if change_counts:   # move one atom of configuration 2 by 0.7 A along <110>: it gains second-shell bonds
        a0 = cs.atom_off[2]
        pos2[a0] += 0.7 * np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    p2, b2 = torch.tensor(pos2, device="cuda"), torch.tensor(box2, device="cuda")
    n_before = ctx.export_neighbors()[0].copy()
    ctx.build_neighbors(cs.atom_off, p2, b2, 2.8, 3.2, 16)
    Z, Zq, S = ctx.fitness(params, tg)
    got = torch.cat([Z[:, None], Zq, S], 1).cpu().numpy()
    assert ctx.get_status() == 0
    n_after = ctx.export_neighbors()[0]
    assert (not np.array_equal(n_before, n_after)) == change_counts
    fresh = binding.Context(0)
    fresh.build_neighbors(cs.atom_off, p2, b2, 2.8, 3.2, 16)
    Z2, Zq2, S2 = fresh.fitness(params, tg)
    ref = torch.cat([Z2[:, None], Zq2, S2], 1).cpu().numpy()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("precision", [32, 64])
def test_large_cells_in_clusters_eval(ctx, precision):
    """Cells of up to 512 atoms with up to 6 neighbours per atom (the uneven workload's largest): the
    schedule spreads each over a thread-block cluster of up to 16 CTAs; E/F/W against the oracle."""
    w = I.workload_uneven(P=2, C=24)
    cs = w["configs"]
    big = np.argsort(cs.natoms)[-6:]
    pos_list = [cs.config(int(c))[0] for c in big]
    box_list = [cs.config(int(c))[1] for c in big]
    sub = I.pack_configs(pos_list, box_list)
    assert sub.natoms.max() >= 380
    _build(ctx, sub)
    _compare_eval(ctx, sub, w["params"][:2], precision, TOL32 if precision == 32 else TOL64)
    clusters = sorted({b["cluster"] for b in ctx.schedule_info(precision)})
    print("cluster sizes", clusters)
    assert max(clusters) >= 8
