"""Genetic-algorithm fit of the minimal Tersoff parameters (arXiv:1909.11474, Sec. III.B) on the
device, and a gradient polish of the best individual.

Each generation evaluates the fitness Z of the whole population with `Context.fitness` and forms the
next population with one `tersoff_ga_step` kernel (rank, elite, parents, uniform crossover,
mutation); the uniform random numbers come from a seeded torch generator on the device. Nothing is
copied to the host inside the loop. `polish` then refines the best parameter set with the adjoint
gradient of the smooth loss (`TersoffLoss`), the use the gradient kernel serves beside the GA.
"""
from __future__ import annotations

import torch

from . import binding
from .autograd import TersoffLoss

N_GENES = 6


class GeneticFit:
    """GA over the context's configurations and targets (Sec. III.B): n_pop individuals, n_par
    parents, genes in [0, 1] mapped to [lo, hi] per parameter, mutation rate decreasing linearly from
    rate0 to zero over the generations."""

    def __init__(self, ctx: binding.Context, targets: dict, lo, hi, n_pop: int = 200, n_par: int = 100,
                 w=(1.0, 1.0, 1.0), seed: int = 0, device=None):
        device = torch.device(device or "cuda")
        self.ctx, self.targets, self.w = ctx, targets, tuple(float(x) for x in w)
        self.n_pop, self.n_par = int(n_pop), int(n_par)
        if not 1 <= self.n_par <= self.n_pop:
            raise ValueError("need 1 <= n_par <= n_pop")
        self.lo = torch.as_tensor(lo, dtype=torch.float64, device=device).contiguous()
        self.hi = torch.as_tensor(hi, dtype=torch.float64, device=device).contiguous()
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(int(seed))
        self.genes = [torch.rand((self.n_pop, N_GENES), generator=self.gen, dtype=torch.float64, device=device),
                      torch.empty((self.n_pop, N_GENES), dtype=torch.float64, device=device)]
        self.params = (self.lo + self.genes[0] * (self.hi - self.lo)).contiguous()
        self.Z = torch.empty(self.n_pop, dtype=torch.float64, device=device)
        self.order = torch.empty(self.n_pop, dtype=torch.int32, device=device)
        self.n_u = 8 * (self.n_pop - self.n_par) + 2 * N_GENES * (self.n_pop - 1)
        self.u = torch.empty(self.n_u, dtype=torch.float64, device=device)
        self.cur = 0

    def evaluate(self):
        self.ctx.fitness(self.params, self.targets, w=self.w, out=(self.Z, None, None))
        return self.Z

    def run(self, n_gen: int = 1000, rate0: float = 0.2, history: bool = False):
        """n_gen generations; returns the best parameter set, its fitness and (optionally) the best
        fitness of every generation (all device tensors until the end)."""
        best = []
        for k in range(n_gen):
            self.evaluate()
            if history:
                best.append(self.Z.min())
            rate = rate0 * (1.0 - k / (n_gen - 1)) if n_gen > 1 else rate0
            torch.rand(self.n_u, generator=self.gen, dtype=torch.float64, device=self.u.device, out=self.u)
            nxt = 1 - self.cur
            binding.ga_step(self.Z, self.genes[self.cur], self.u, self.lo, self.hi, self.n_par, rate,
                            self.genes[nxt], self.params, self.order)
            self.cur = nxt
        Z = self.evaluate()
        i = int(torch.argmin(Z))
        out = {"params": self.params[i].detach().cpu().numpy(), "Z": float(Z[i]), "genes": self.genes[self.cur][i].cpu().numpy()}
        if history:
            out["history"] = torch.stack(best).cpu().numpy()
        return out


def polish(ctx: binding.Context, params, targets: dict, lo, hi, steps: int = 200, lr: float = 2e-3,
           w=(1.0, 1.0, 1.0), loss: int = binding.LOSS_SQ):
    """Refine one parameter set by Adam in gene space on the smooth loss L = sum_q w_q S_q / D_q,
    with gradients from the adjoint kernel. Returns (params, loss before, loss after)."""
    dev = torch.device("cuda")
    lo = torch.as_tensor(lo, dtype=torch.float64, device=dev)
    hi = torch.as_tensor(hi, dtype=torch.float64, device=dev)
    x0 = torch.as_tensor(params, dtype=torch.float64, device=dev).reshape(1, N_GENES)
    g = ((x0 - lo) / (hi - lo)).clone().requires_grad_(True)
    opt = torch.optim.Adam([g], lr=lr)
    first = None
    for _ in range(steps):
        opt.zero_grad()
        x = (lo + g * (hi - lo)).contiguous()
        L = TersoffLoss.apply(x, ctx, targets, w, loss).sum()
        if first is None:
            first = float(L)
        L.backward()
        opt.step()
    x = (lo + g.detach() * (hi - lo)).contiguous()
    L, _ = ctx.param_grad(x, targets, w=w, loss=loss)
    return x[0].cpu().numpy(), first, float(L[0])
