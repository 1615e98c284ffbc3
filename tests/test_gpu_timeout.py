"""The bounded device-side wait gives up, reports a timeout and leaves the context usable.

The batched kernel waits for the bulk copies that stage a configuration's geometry (an mbarrier);
it is the library's only wait on other work (the neighbour build has no cross-CTA wait).
tersoff_set_wait_limit bounds it in polls; with a bound of 0 the wait gives up at its first check.
Nothing faults or hangs: the wait returns, the CTA waits (with the built-in bound) for its copies in
flight and stops, the status word carries TERSOFF_STATUS_TIMEOUT, and the next call with the default
bound gives the results of a call that never timed out.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1909_11474_gb300 import inputs as I

from ._util import targets_to_device, to_device

pytestmark = pytest.mark.gpu


def _fitness_setup(ctx):
    w = I.workload_ga_batch(P=21, C=5)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0])
    pos, box = to_device(cs)
    ctx.build_neighbors(cs.atom_off, pos, box, 2.8, 3.2, 16)
    return torch.tensor(w["params"], device="cuda"), targets_to_device(t)


@pytest.mark.parametrize("graphs", [True, False])
def test_staging_wait_that_gives_up_reports_a_timeout(graphs):
    from paper_1909_11474_gb300 import binding
    ctx = binding.Context(0)
    ctx.set_launch_mode(graphs=graphs, pdl=True)
    params, tg = _fitness_setup(ctx)
    Z0 = ctx.fitness(params, tg)[0].cpu().numpy()
    E0, F0, W0 = (x.cpu().numpy() for x in ctx.eval(params))
    assert ctx.get_status() == 0

    ctx.set_wait_limit(0)                                  # every staging wait gives up at once
    ctx.fitness(params, tg)
    assert ctx.get_status() & binding.STATUS_TIMEOUT
    ctx.eval(params)
    assert ctx.get_status() & binding.STATUS_TIMEOUT

    ctx.set_wait_limit(-1)                                 # the built-in bound again
    Z1 = ctx.fitness(params, tg)[0].cpu().numpy()
    E1, F1, W1 = (x.cpu().numpy() for x in ctx.eval(params))
    assert ctx.get_status() == 0
    assert np.array_equal(Z1, Z0) and np.array_equal(E1, E0) and np.array_equal(F1, F0) and np.array_equal(W1, W0)
