"""Velocity-Verlet NVE on the device (tersoff_md_nve): parity with the oracle's integrator, energy
conservation, time reversibility, argument checks."""
import numpy as np
import pytest
import torch

from oracle import md as omd
from paper_1909_11474_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P2 = I.TABLE2_PARAMS


@pytest.fixture(scope="module")
def ctx():
    from paper_1909_11474_gb300 import binding
    return binding.Context(0)


def _system(reps, T, seed, sigma=0.05):
    rng = np.random.default_rng(seed)
    pos, box = I.diamond_supercell(reps)
    pos = pos + rng.normal(0.0, sigma, pos.shape)
    m = np.full(len(pos), I.SI_MASS)
    return pos, box, m, I.thermal_velocities(rng, m, T)


def _run(ctx, pos, box, m, v, dt, n, precision=64):
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    p, vv, mm = d(pos), d(v), d(m)
    Ep, Ek, F, W = ctx.md_nve(p, vv, mm, box, P2, dt, n, precision=precision)
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    return p.cpu().numpy(), vv.cpu().numpy(), Ep.cpu().numpy(), Ek.cpu().numpy(), F.cpu().double().numpy()


def test_nve_matches_the_oracle_integrator(ctx):
    """216 atoms at 600 K, 6 steps of 1 fs in FP64: positions, velocities and both energies of every
    step against the oracle's velocity-Verlet on its own forces."""
    pos, box, m, v = _system((3, 3, 3), 600.0, 1)
    x, vv, Ep, Ek, F = _run(ctx, pos, box, m, v, 1.0, 6)
    xo, vo, Epo, Eko = omd.velocity_verlet(pos, v, m, box, P2, 1.0, 6)
    assert np.abs(x - xo).max() < 1e-10
    assert np.abs(vv - vo).max() < 1e-11
    np.testing.assert_allclose(Ep, Epo, rtol=1e-11, atol=0)
    np.testing.assert_allclose(Ek, Eko, rtol=1e-11, atol=0)


@pytest.mark.parametrize("precision,bound", [(64, 1.5e-4), (32, 3e-4)])
def test_nve_conserves_energy(ctx, precision, bound):
    """512 atoms started on the perfect lattice at 300 K, 1000 steps of 1 fs: the total energy stays within `bound` eV/atom of its
    start (the velocity-Verlet excursion at this step; FP32 force rounding adds to it) while kinetic
    and potential energy exchange far more. In FP64, halving the step over the same time cuts the
    excursion about fourfold (second order), so it is the integrator's, not a force error."""
    pos, box, m, v = _system((4, 4, 4), 300.0, 2, sigma=0.0)     # perfect lattice at 300 K
    N = len(pos)
    _, _, Ep, Ek, _ = _run(ctx, pos, box, m, v, 1.0, 1000, precision)
    Et = Ep + Ek
    dev1 = np.abs(Et - Et[0]).max() / N
    assert dev1 < bound
    assert np.abs(Ek - Ek[0]).max() / N > 10 * bound
    # equipartition from the perfect lattice: about half the kinetic energy moves into the
    # potential, so the temperature settles near T0 / 2
    T_end = Ek[-500:].mean() / (1.5 * omd.KB * N)
    assert 120.0 < T_end < 180.0, T_end
    if precision == 64:
        _, _, Ep2, Ek2, _ = _run(ctx, pos, box, m, v, 0.5, 2000, precision)
        Et2 = Ep2 + Ek2
        dev2 = np.abs(Et2 - Et2[0]).max() / N
        assert 3.0 < dev1 / dev2 < 5.5, (dev1, dev2)


def test_nve_is_time_reversible(ctx):
    pos, box, m, v = _system((3, 3, 3), 300.0, 3)
    x1, v1, _, _, _ = _run(ctx, pos, box, m, v, 1.0, 200)
    x2, v2, _, _, _ = _run(ctx, x1, box, m, -v1, 1.0, 200)
    assert np.abs(x2 - pos).max() < 1e-8
    assert np.abs(v2 + v).max() < 1e-9


def test_nve_zero_steps_and_bad_arguments(ctx):
    from paper_1909_11474_gb300 import binding
    pos, box, m, v = _system((3, 3, 3), 300.0, 4)
    x, vv, Ep, Ek, F = _run(ctx, pos, box, m, v, 1.0, 0)
    assert np.array_equal(x, pos) and np.array_equal(vv, v) and len(Ep) == 1
    assert Ek[0] == pytest.approx(omd.kinetic_energy(v, m), rel=1e-13)
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    p = d(pos)
    with pytest.raises(binding.TersoffError):
        ctx.md_nve(p, d(v), d(m), box, P2, 0.0, 5)
    with pytest.raises(binding.TersoffError):
        ctx.md_nve(p, p, d(m), box, P2, 1.0, 5)
