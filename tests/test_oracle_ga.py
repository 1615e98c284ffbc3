"""Pins of the genetic-algorithm oracle (Sec. III.B) against brute force, its invariants and a
problem with a known optimum."""
import numpy as np

from oracle import ga


def _inputs(seed, n_pop=20, n_par=8, bad=()):
    rng = np.random.default_rng(seed)
    Z = rng.uniform(0.0, 1.0, n_pop)
    Z[3] = Z[5]                      # a tie
    for i in bad:
        Z[i] = [np.nan, np.inf, -np.inf][i % 3]
    genes = rng.uniform(0.0, 1.0, (n_pop, 6))
    u = rng.uniform(0.0, 1.0, ga.n_uniforms(n_pop, n_par))
    return Z, genes, u


def test_rank_is_the_brute_force_sort():
    Z, _, _ = _inputs(1, bad=(2, 7, 11))
    want = sorted(range(len(Z)), key=lambda i: (0 if np.isfinite(Z[i]) else 1, Z[i] if np.isfinite(Z[i]) else 0, i))
    assert list(ga.rank(Z)) == want


def test_uniform_count_and_layout():
    assert ga.n_uniforms(200, 100) == 8 * 100 + 12 * 199
    assert ga.n_uniforms(5, 5) == 12 * 4
    assert ga.n_uniforms(200, 100, 9) == 11 * 100 + 18 * 199


def test_nine_genes_take_the_same_steps():
    """G = 9 (the Tersoff form): children take each gene from one of their two drawn parents, the
    mutation replaces exactly the drawn genes, the elite is kept."""
    rng = np.random.default_rng(8)
    n_pop, n_par, G, rate = 16, 6, 9, 0.25
    Z = rng.uniform(0.0, 1.0, n_pop)
    genes = rng.uniform(0.0, 1.0, (n_pop, G))
    u = rng.uniform(0.0, 1.0, ga.n_uniforms(n_pop, n_par, G))
    new, order = ga.ga_step(Z, genes, u, n_par, rate)
    ranked = genes[order]
    assert np.array_equal(new[0], ranked[0])
    base = (G + 2) * (n_pop - n_par)
    for i in range(n_pop):
        for g in range(G):
            if i >= 1 and u[base + 2 * G * (i - 1) + 2 * g] < rate:
                assert new[i, g] == u[base + 2 * G * (i - 1) + 2 * g + 1]
            elif i < n_par:
                assert new[i, g] == ranked[i, g]
            else:
                c = i - n_par
                a, b = int(u[(G + 2) * c] * n_par), int(u[(G + 2) * c + 1] * n_par)
                assert new[i, g] == (ranked[a, g] if u[(G + 2) * c + 2 + g] < 0.5 else ranked[b, g])


def test_parents_are_the_best_in_rank_order_and_the_elite_is_kept():
    Z, genes, u = _inputs(2, bad=(4,))
    new, order = ga.ga_step(Z, genes, u, n_par=8, rate=0.0)
    assert np.array_equal(new[:8], genes[order[:8]])
    new1, _ = ga.ga_step(Z, genes, u, n_par=8, rate=1.0)   # every other gene mutates, never the elite's
    assert np.array_equal(new1[0], genes[np.argmin(np.where(np.isfinite(Z), Z, np.inf))])


def test_children_take_each_gene_from_one_of_their_two_parents():
    Z, genes, u = _inputs(3)
    n_pop, n_par = len(Z), 8
    new, order = ga.ga_step(Z, genes, u, n_par=n_par, rate=0.0)
    ranked = genes[order]
    for c in range(n_pop - n_par):
        a, b = int(u[8 * c] * n_par), int(u[8 * c + 1] * n_par)
        for g in range(6):
            want = ranked[a, g] if u[8 * c + 2 + g] < 0.5 else ranked[b, g]
            assert new[n_par + c, g] == want


def test_mutation_replaces_exactly_the_drawn_genes():
    Z, genes, u = _inputs(4)
    n_pop, n_par, rate = len(Z), 8, 0.3
    base_new, _ = ga.ga_step(Z, genes, u, n_par=n_par, rate=0.0)
    new, _ = ga.ga_step(Z, genes, u, n_par=n_par, rate=rate)
    base = 8 * (n_pop - n_par)
    changed = 0
    for i in range(1, n_pop):
        for g in range(6):
            k = base + 12 * (i - 1) + 2 * g
            if u[k] < rate:
                assert new[i, g] == u[k + 1]
                changed += 1
            else:
                assert new[i, g] == base_new[i, g]
    assert 0 < changed < (n_pop - 1) * 6
    assert np.array_equal(new[0], base_new[0])
    assert ((new >= 0.0) & (new <= 1.0)).all()


def test_mutation_rate_decreases_linearly_to_zero():
    n = 11
    r = [ga.mutation_rate(k, n) for k in range(n)]
    assert r[0] == 0.2 and r[-1] == 0.0
    assert np.allclose(np.diff(r), -0.02)


def test_phenotype_maps_the_unit_interval_onto_the_limits():
    lo, hi = np.array([1.0, -2.0, 0, 0, 0, 0]), np.array([3.0, 2.0, 1, 1, 1, 1])
    x = ga.phenotype(np.array([[0.0, 1.0, 0.5, 0, 0, 0]]), lo, hi)
    assert np.allclose(x[0, :3], [1.0, 2.0, 0.5])


def test_ga_finds_the_optimum_of_a_quadratic_and_the_elite_never_worsens():
    """A problem with a known optimum: Z(x) = |gene - g*|^2 with g* inside the unit box."""
    rng = np.random.default_rng(5)
    target = np.array([0.2, 0.7, 0.45, 0.9, 0.1, 0.6])
    n_pop, n_par, n_gen = 60, 30, 300
    genes = rng.uniform(0.0, 1.0, (n_pop, 6))
    best = []
    for k in range(n_gen):
        Z = ((genes - target) ** 2).sum(1)
        best.append(Z.min())
        u = rng.uniform(0.0, 1.0, ga.n_uniforms(n_pop, n_par))
        genes, _ = ga.ga_step(Z, genes, u, n_par, ga.mutation_rate(k, n_gen))
    Z = ((genes - target) ** 2).sum(1)
    assert all(b1 <= b0 for b0, b1 in zip(best, best[1:]))
    assert Z.min() < 1e-3
    assert np.abs(genes[np.argmin(Z)] - target).max() < 0.03
