"""Host logic of the damped Newton polish (CPU, no kernels): a stand-in context whose `param_grad`
returns a badly scaled least-squares loss with a known minimum, like the beta-n valley of the fit."""
import numpy as np
import torch

from paper_1909_11474_gb300.ga import _newton_polish


class _ValleyLoss:
    """L(x) = sum_k r_k(x)^2 with r = A (x - x*) + c (x - x*)_3 (x - x*)_4 e_0: a quadratic with
    condition number ~1e8 plus a mild nonlinearity; dL/dx exact."""

    def __init__(self):
        rng = np.random.default_rng(0)
        Q, _ = np.linalg.qr(rng.normal(size=(6, 6)))
        self.A = torch.tensor(Q @ np.diag([1.0, 0.3, 0.1, 1e-2, 1e-3, 1e-4]) @ Q.T)
        self.xs = torch.tensor([3.2, 1.43, 2.24, 0.28, 0.60, -0.64], dtype=torch.float64)
        self.calls = 0

    def param_grad(self, x, targets, w=None, loss=None):
        self.calls += 1
        d = x - self.xs
        r = d @ self.A.T
        r[:, 0] = r[:, 0] + 0.5 * d[:, 3] * d[:, 4]
        L = (r * r).sum(1)
        J = self.A.expand(x.shape[0], 6, 6).clone()
        J[:, 0, 3] += 0.5 * d[:, 4]
        J[:, 0, 4] += 0.5 * d[:, 3]
        dL = 2.0 * torch.einsum("pk,pkj->pj", r, J)
        return L, dL


def test_newton_polish_reaches_the_minimum_of_an_ill_conditioned_valley():
    f = _ValleyLoss()
    lo = f.xs - 0.3 * f.xs.abs()
    hi = f.xs + 0.3 * f.xs.abs()
    x0 = f.xs * torch.tensor([1.05, 0.97, 1.02, 1.2, 0.85, 1.1], dtype=torch.float64)
    g0 = (x0 - lo) / (hi - lo)
    L0 = float(f.param_grad(x0[None, :], None)[0][0])
    g = _newton_polish(f, g0, lo, hi, None, None, None, iters=40)
    x = lo + g * (hi - lo)
    L1 = float(f.param_grad(x[None, :], None)[0][0])
    assert L1 < 1e-20 * max(L0, 1.0) or L1 < 1e-24
    assert torch.allclose(x, f.xs, rtol=1e-8, atol=1e-10)


def test_newton_polish_never_raises_the_loss():
    f = _ValleyLoss()
    lo = f.xs - 0.3 * f.xs.abs()
    hi = f.xs + 0.3 * f.xs.abs()
    g0 = torch.full((6,), 0.9, dtype=torch.float64)
    L0 = float(f.param_grad((lo + g0 * (hi - lo))[None, :], None)[0][0])
    for iters in (0, 1, 3):
        g = _newton_polish(f, g0, lo, hi, None, None, None, iters=iters)
        L1 = float(f.param_grad((lo + g * (hi - lo))[None, :], None)[0][0])
        assert L1 <= L0


class _ValleyFitness(_ValleyLoss):
    """The same loss seen through a fitness call: S = (L, 0, 0) and Zq = (sqrt(L), 0, 0), so D = 1."""

    def fitness(self, x, targets, w=None, precision=64):
        L, _ = self.param_grad(x, targets)
        S = torch.stack([L, torch.zeros_like(L), torch.zeros_like(L)], 1)
        Zq = torch.sqrt(S)
        return Zq.sum(1), Zq, S


def test_finite_difference_newton_polish_reaches_the_minimum():
    """The polish of the Tersoff form (gradient and Hessian from loss values in one batch) on the
    same ill-conditioned valley: it reaches the minimum to finite-difference accuracy."""
    from paper_1909_11474_gb300.ga import _fd_newton_polish
    f = _ValleyFitness()
    lo = f.xs - 0.3 * f.xs.abs()
    hi = f.xs + 0.3 * f.xs.abs()
    x0 = f.xs * torch.tensor([1.05, 0.97, 1.02, 1.2, 0.85, 1.1], dtype=torch.float64)
    g0 = (x0 - lo) / (hi - lo)
    g = _fd_newton_polish(f, g0, lo, hi, None, (1.0, 1.0, 1.0), iters=40)
    x = lo + g * (hi - lo)
    assert torch.allclose(x, f.xs, rtol=1e-5, atol=1e-6)
    L1 = float(f.param_grad(x[None, :], None)[0][0])
    L0 = float(f.param_grad(x0[None, :], None)[0][0])
    assert L1 < 1e-10 * L0
