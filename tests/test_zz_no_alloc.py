"""tersoff_fitness_static, the fitness call that allocates no device memory.

Some callers cannot let a library call cudaMalloc: it stalls the whole device until it returns, and
a caller whose device memory is already reserved by another allocator may have none to give. This
entry point uses only the context built by tersoff_build_neighbors and one fixed 8 MiB device array.
It must give the results of tersoff_fitness, call after call, since every call reuses (and leaves
behind) the same scratch. This file is collected last so that a failure here does not hide the
results of the other tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_11474_gb300 import inputs as I

from ._util import targets_to_device, to_device

pytestmark = pytest.mark.gpu


def _setup(P, C, seed_mask):
    from paper_1909_11474_gb300 import binding
    w = I.workload_ga_batch(P=P, C=C)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    mask = np.random.default_rng(seed_mask).integers(1, 8, size=C).astype(np.uint8)
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0], mask=mask)
    ctx = binding.Context(0)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    return ctx, w, targets_to_device(t)


def test_fitness_static_matches_fitness_twice_in_a_row():
    ctx, w, tg = _setup(P=37, C=6, seed_mask=1)
    params_a = torch.tensor(w["params"], device="cuda")
    params_b = torch.tensor(w["params"][::-1].copy() * 1.01, device="cuda")
    wts = (1.0, 0.7, 0.3)
    for precision in (32, 64):
        for params in (params_a, params_b):      # two calls in a row on the shared scratch
            ref = [x.cpu().numpy() for x in ctx.fitness(params, tg, w=wts, precision=precision)]
            got = [x.cpu().numpy() for x in ctx.fitness_static(params, tg, w=wts, precision=precision)]
            torch.cuda.synchronize()
            assert ctx.get_status() == 0
            # the same kernels run on the same inputs; the parity tolerance of the fitness tests
            # (far above any difference these could show) is the bar
            for r, g in zip(ref, got):
                assert np.allclose(g, r, rtol=1e-10, atol=0.0)


def test_fitness_static_allocates_nothing_per_call():
    ctx, w, tg = _setup(P=21, C=4, seed_mask=2)
    params = torch.tensor(w["params"], device="cuda")
    out = (torch.empty(21, dtype=torch.float64, device="cuda"), torch.empty((21, 3), dtype=torch.float64, device="cuda"),
           torch.empty((21, 3), dtype=torch.float64, device="cuda"))
    ctx.fitness_static(params, tg, out=out)          # first call on the device: address set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ctx.fitness_static(params, tg, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    Z = out[0].cpu().numpy()
    assert np.isfinite(Z).all()


def test_fitness_static_rejects_requests_beyond_the_static_limit():
    from paper_1909_11474_gb300 import binding
    ctx, w, tg = _setup(P=3, C=4, seed_mask=3)
    P = 80000   # P*8*8 + P*C*24 = 12.8 MB of constants and residual sums > 8 MiB
    assert P * 64 + P * 4 * 24 > 8 << 20
    params = torch.tensor(np.tile(w["params"][:1], (P, 1)), device="cuda")
    with pytest.raises(binding.TersoffError) as ei:
        ctx.fitness_static(params, tg)
    assert ei.value.code == binding.E_ARG
    assert "static limit" in str(ei.value)
