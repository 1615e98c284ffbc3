"""tersoff_fitness_static, the fitness call that allocates no device memory.

Some callers cannot let a library call cudaMalloc: it stalls the whole device until it returns, and
a caller whose device memory is already reserved by another allocator may have none to give. This
entry point uses only what tersoff_build_neighbors allocated and one fixed 8 MiB device array whose
address tersoff_create looks up. It must give the results of tersoff_fitness, call after call, since
every call reuses (and leaves behind) the same scratch, and it must allocate nothing even as the
first call after a build, in either precision. This file is collected last so that a failure here
does not hide the results of the other tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_11474_gb300 import inputs as I

from ._util import TOL32, TOL64, fitness_bounds, targets_to_device, to_device

pytestmark = pytest.mark.gpu


def _setup(P, C, seed_mask, targets="oracle"):
    from paper_1909_11474_gb300 import binding
    w = I.workload_ga_batch(P=P, C=C)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    mask = np.random.default_rng(seed_mask).integers(1, 8, size=C).astype(np.uint8)
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0], mask=mask)
    ctx = binding.Context(0)
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    return ctx, w, t, targets_to_device(t), (pos, box)


def _out(P):
    return (torch.empty(P, dtype=torch.float64, device="cuda"), torch.empty((P, 3), dtype=torch.float64, device="cuda"),
            torch.empty((P, 3), dtype=torch.float64, device="cuda"))


def test_fitness_static_matches_fitness_twice_in_a_row():
    ctx, w, _, tg, _ = _setup(P=37, C=6, seed_mask=1)
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


@pytest.mark.parametrize("precision", [32, 64])
def test_fitness_static_matches_the_oracle(precision):
    """The allocation-free call against the FP64 oracle's fitness, within the bounds that the
    per-quantity parity bars imply (triangle inequality on sqrt(S_q)), on two calls in a row."""
    ctx, w, t, tg, _ = _setup(P=21, C=5, seed_mask=4)
    wts = (1.0, 0.7, 0.3)
    E, W, F, ES, WS, FS = oracle.evaluate_batch(w["configs"], w["params"], scales=True, force_scales=True)
    ref = oracle.fitness_from_predictions(w["configs"], t, E, W, F, w=wts)
    B = fitness_bounds(w["configs"], t, E, W, F, ES, WS, TOL32 if precision == 32 else TOL64, FS=FS)
    D = ref["D"]
    params = torch.tensor(w["params"], device="cuda")
    for _ in range(2):
        Z, Zq, S = (x.cpu().numpy() for x in ctx.fitness_static(params, tg, w=wts, precision=precision))
        assert ctx.get_status() == 0
        assert (np.abs(np.sqrt(S) - np.sqrt(ref["S"])) <= B).all()
        assert (np.abs(Zq - ref["Zq"]) <= B / np.sqrt(D)[None, :]).all()
        assert (np.abs(Z - ref["Z"]) <= (np.asarray(wts)[None, :] * B / np.sqrt(D)[None, :]).sum(-1)).all()


def test_first_static_call_after_a_build_allocates_nothing():
    """Free device memory is unchanged across the first static call after a fresh build (FP32), the
    first FP64 call (which computes the FP64 geometry into buffers the build allocated), a rebuild of
    other positions, and the calls after it."""
    ctx, w, _, tg, (pos, box) = _setup(P=21, C=4, seed_mask=2)
    cs = w["configs"]
    params = torch.tensor(w["params"], device="cuda")
    out = _out(21)
    pos2 = pos + 0.01 * torch.randn(pos.shape, dtype=torch.float64, device="cuda",
                                    generator=torch.Generator(device="cuda").manual_seed(5))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ctx.fitness_static(params, tg, out=out, precision=32)     # first call after the build
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx.fitness_static(params, tg, out=out, precision=64)     # first FP64 call
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    Z64 = out[0].cpu().numpy().copy()
    ctx.build_neighbors(cs.atom_off, pos2, box, 2.8, 3.2, 16)  # the build may allocate; the calls may not
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    for precision in (64, 32, 32):
        ctx.fitness_static(params, tg, out=out, precision=precision)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free1
    assert ctx.get_status() == 0
    assert np.isfinite(out[0].cpu().numpy()).all() and np.isfinite(Z64).all()


def test_fitness_static_rejects_requests_beyond_the_static_limit():
    from paper_1909_11474_gb300 import binding
    ctx, w, _, tg, _ = _setup(P=3, C=4, seed_mask=3)
    P = 80000   # P*8*8 + P*C*24 = 12.8 MB of constants and residual terms > 8 MiB
    assert P * 64 + P * 4 * 24 > 8 << 20
    params = torch.tensor(np.tile(w["params"][:1], (P, 1)), device="cuda")
    with pytest.raises(binding.TersoffError) as ei:
        ctx.fitness_static(params, tg)
    assert ei.value.code == binding.E_ARG
    assert "static limit" in str(ei.value)
