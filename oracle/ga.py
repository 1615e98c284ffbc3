"""Plain CPU oracle of one generation of the genetic algorithm of arXiv:1909.11474 (Sec. III.B).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path. Independent of the
CUDA path; both sides receive the same fitness values, genes and uniform random numbers.

One generation, in the order the paper lists its steps:

* rank the population by fitness Z, smallest first (Sec. III.B, step 2a);
* keep the best individual (the elite) unaltered (step 2b);
* keep the N_par best as parents and drop the others (step 2c);
* refill the population with N_pop - N_par children made by crossover of the parents (step 2d);
* mutate randomly chosen genes of randomly chosen chromosomes (step 2e).

Genes are real numbers in [0, 1]; parameter x_g = lo_g + gene_g (hi_g - lo_g) (step 1).

Readings where the paper is silent (also listed in the design notes):

* a non-finite fitness ranks after every finite one; equal fitness values keep index order;
* the new population is the N_par parents in rank order (the elite first) followed by the children;
* crossover is uniform: a child draws two parents uniformly from the N_par (with replacement) and
  takes each gene from the first or the second with probability 1/2;
* mutation visits every gene of every individual except the elite; with probability `rate` the gene
  is replaced by a fresh uniform value;
* the random numbers are passed in, laid out for G genes per individual (G = 6 for the minimal
  potential, 9 for the Tersoff form) as: for child c, u[(G+2)c], u[(G+2)c+1] pick the two parents
  (index floor(u * N_par)) and u[(G+2)c+2+g] < 1/2 picks parent one for gene g; then, from
  base = (G+2) (N_pop - N_par), individual i >= 1 uses u[base + 2G(i-1) + 2g] < rate to decide a
  mutation of gene g and u[base + 2G(i-1) + 2g + 1] as its new value.
"""
from __future__ import annotations

import numpy as np

N_GENES = 6


def n_uniforms(n_pop: int, n_par: int, n_genes: int = N_GENES) -> int:
    """Uniform random numbers one generation consumes."""
    return (n_genes + 2) * (n_pop - n_par) + 2 * n_genes * (n_pop - 1)


def rank(Z: np.ndarray) -> np.ndarray:
    """Population indices from best to worst: ascending Z, non-finite last, ties by index."""
    Z = np.asarray(Z, dtype=np.float64)
    key = np.where(np.isfinite(Z), Z, np.inf)
    return np.lexsort((np.arange(len(Z)), key))


def ga_step(Z, genes, uniforms, n_par: int, rate: float):
    """One generation (Sec. III.B, steps 2a-2e). Returns (new genes [N_pop][G], rank order)."""
    genes = np.asarray(genes, dtype=np.float64)
    u = np.asarray(uniforms, dtype=np.float64)
    n_pop, G = genes.shape
    assert 1 <= n_par <= n_pop and G >= 1
    assert len(u) >= n_uniforms(n_pop, n_par, G)
    order = rank(Z)
    ranked = genes[order]
    new = np.empty_like(genes)
    new[:n_par] = ranked[:n_par]                        # elite first, then the other parents
    for c in range(n_pop - n_par):                      # uniform crossover
        a = min(int(u[(G + 2) * c] * n_par), n_par - 1)
        b = min(int(u[(G + 2) * c + 1] * n_par), n_par - 1)
        for g in range(G):
            new[n_par + c, g] = ranked[a, g] if u[(G + 2) * c + 2 + g] < 0.5 else ranked[b, g]
    base = (G + 2) * (n_pop - n_par)
    for i in range(1, n_pop):                           # mutation, the elite excepted
        for g in range(G):
            k = base + 2 * G * (i - 1) + 2 * g
            if u[k] < rate:
                new[i, g] = u[k + 1]
    return new, order


def phenotype(genes, lo, hi):
    """Parameter vectors of the genes (Sec. III.B, step 1): x = lo + gene (hi - lo)."""
    genes = np.asarray(genes, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + genes * (hi - lo)


def mutation_rate(gen: int, n_gen: int, rate0: float = 0.2) -> float:
    """Mutation rate decreasing linearly from rate0 to zero over the generations (Sec. III.B)."""
    return rate0 * (1.0 - gen / max(1, n_gen - 1)) if n_gen > 1 else rate0
