"""FP64 CPU oracle for the minimal Tersoff potential (Fan et al., arXiv:1909.11474).

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this package: only the tests, the
smoke check and the CPU-baseline leg of the benchmark call it. It shares no code with the CUDA
path; both sides receive the same seeded inputs and nothing else.

Parity status: every function here is pinned by the tests in tests/test_oracle_*.py against
closed forms, the paper's printed values and brute force (no function is left unpinned).
"""
from .tersoff import (  # noqa: F401
    R1_DEFAULT, R2_DEFAULT, neighbor_list, evaluate, evaluate_batch, fitness, loss_and_grad,
    data_norms, site_energy_sum, fitness_from_predictions, neighbor_list_subset,
)
