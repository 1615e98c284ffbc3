"""Genetic-algorithm fit of the minimal Tersoff parameters (arXiv:1909.11474, Sec. III.B) on the
device, and a gradient polish of the best individual.

Each generation evaluates the fitness Z of the whole population with `Context.fitness` and forms the
next population with one `tersoff_ga_step` kernel (rank, elite, parents, uniform crossover,
mutation); the uniform random numbers come from a seeded torch generator on the device. Nothing is
copied to the host inside the loop. A run can be saved and resumed bit for bit (`save`, `load`).
`polish` then refines the best parameter set with the adjoint gradient of the smooth loss
(`TersoffLoss`), the use the gradient kernel serves beside the GA.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding
from .autograd import TersoffLoss

N_GENES = 6


class GeneticFit:
    """GA over the context's configurations and targets (Sec. III.B): n_pop individuals, n_par
    parents, genes in [0, 1] mapped to [lo, hi] per parameter (6 limits for the minimal potential, 9
    for a context in the Tersoff form), mutation rate decreasing linearly from rate0 to zero over the
    generations."""

    def __init__(self, ctx: binding.Context, targets: dict, lo, hi, n_pop: int = 200, n_par: int = 100,
                 w=(1.0, 1.0, 1.0), seed: int = 0, device=None):
        device = torch.device(device or "cuda")
        self.ctx, self.targets, self.w = ctx, targets, tuple(float(x) for x in w)
        self.n_pop, self.n_par = int(n_pop), int(n_par)
        if not 1 <= self.n_par <= self.n_pop:
            raise ValueError("need 1 <= n_par <= n_pop")
        self.lo = torch.as_tensor(lo, dtype=torch.float64, device=device).contiguous()
        self.hi = torch.as_tensor(hi, dtype=torch.float64, device=device).contiguous()
        self.n_genes = G = int(self.lo.numel())       # 6 (minimal potential) or 9 (Tersoff form)
        if G != getattr(ctx, "n_params", N_GENES):
            raise ValueError(f"{G} parameter limits for a context that takes {ctx.n_params} parameters")
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(int(seed))
        self.genes = [torch.rand((self.n_pop, G), generator=self.gen, dtype=torch.float64, device=device),
                      torch.empty((self.n_pop, G), dtype=torch.float64, device=device)]
        self.params = (self.lo + self.genes[0] * (self.hi - self.lo)).contiguous()
        self.Z = torch.empty(self.n_pop, dtype=torch.float64, device=device)
        self.order = torch.empty(self.n_pop, dtype=torch.int32, device=device)
        self.n_u = (G + 2) * (self.n_pop - self.n_par) + 2 * G * (self.n_pop - 1)
        self.u = torch.empty(self.n_u, dtype=torch.float64, device=device)
        self.cur = 0
        self.k = 0                      # generations done

    def evaluate(self):
        self.ctx.fitness(self.params, self.targets, w=self.w, out=(self.Z, None, None))
        return self.Z

    def run(self, n_gen: int = 1000, rate0: float = 0.2, history: bool = False, until: int | None = None):
        """Generations self.k .. min(until, n_gen) - 1 of an n_gen-generation schedule (mutation rate
        rate0 (1 - k / (n_gen - 1))); returns the best parameter set of the current population, its
        fitness and (optionally) the best fitness of every generation run. A run stopped by `until`
        continues, bit for bit, from where it stopped (also after `save` and `load`)."""
        best = []
        stop = n_gen if until is None else min(int(until), n_gen)
        for k in range(self.k, stop):
            self.evaluate()
            if history:
                best.append(self.Z.min())
            rate = rate0 * (1.0 - k / (n_gen - 1)) if n_gen > 1 else rate0
            torch.rand(self.n_u, generator=self.gen, dtype=torch.float64, device=self.u.device, out=self.u)
            nxt = 1 - self.cur
            binding.ga_step(self.Z, self.genes[self.cur], self.u, self.lo, self.hi, self.n_par, rate,
                            self.genes[nxt], self.params, self.order)
            self.cur = nxt
            self.k = k + 1
        Z = self.evaluate()
        i = int(torch.argmin(Z))
        out = {"params": self.params[i].detach().cpu().numpy(), "Z": float(Z[i]), "genes": self.genes[self.cur][i].cpu().numpy(),
               "generations": self.k}
        if history:
            out["history"] = torch.stack(best).cpu().numpy() if best else torch.zeros(0).numpy()
        return out

    # -- checkpoint / resume ------------------------------------------------------------------------
    def state_dict(self) -> dict:
        """Everything the next generations depend on: population (genes and parameters), generation
        count, random-number generator state, and the settings it was made with."""
        return {"genes": self.genes[self.cur].detach().cpu().clone(), "params": self.params.detach().cpu().clone(),
                "k": self.k, "rng": self.gen.get_state().cpu().clone(), "n_pop": self.n_pop, "n_par": self.n_par,
                "lo": self.lo.cpu().clone(), "hi": self.hi.cpu().clone(), "w": self.w}

    def load_state_dict(self, st: dict):
        if (int(st["n_pop"]), int(st["n_par"])) != (self.n_pop, self.n_par):
            raise ValueError("checkpoint of another population size")
        if not (torch.equal(st["lo"], self.lo.cpu()) and torch.equal(st["hi"], self.hi.cpu())):
            raise ValueError("checkpoint of other parameter limits")
        self.cur = 0
        self.genes[0].copy_(st["genes"])
        self.params.copy_(st["params"])
        self.k = int(st["k"])
        self.gen.set_state(st["rng"])
        self.w = tuple(float(x) for x in st["w"])

    def save(self, path):
        torch.save(self.state_dict(), path)

    @classmethod
    def load(cls, ctx: binding.Context, targets: dict, path, device=None) -> "GeneticFit":
        st = torch.load(path, weights_only=True)
        fit = cls(ctx, targets, st["lo"].numpy(), st["hi"].numpy(), n_pop=int(st["n_pop"]), n_par=int(st["n_par"]),
                  w=st["w"], device=device)
        fit.load_state_dict(st)
        return fit


def _newton_polish(ctx, g0, lo, hi, targets, w, loss, iters: int, h: float = 1e-4):
    """Damped Newton (Levenberg-Marquardt damping) in gene space. Each iteration evaluates the loss
    and its adjoint gradient at the point and at +-h along every gene in one batched call (13
    parameter sets), takes the Hessian by central differences of the gradients, and solves the 6x6
    system (H + lam diag(H)) d = -grad on the host; a step that lowers the loss is taken and lam
    shrinks, else lam grows. Stops when two accepted steps in a row gain less than 1e-10 relative."""
    span = hi - lo
    G = g0.numel()
    eye = torch.eye(G, dtype=torch.float64, device=g0.device)

    def batch(gg):
        pts = torch.cat([gg[None, :], gg[None, :] + h * eye, gg[None, :] - h * eye], 0)
        L, dL = ctx.param_grad((lo + pts * span).contiguous(), targets, w=w, loss=loss)
        grad = (dL * span).cpu().numpy()                  # d/dgene
        H = (grad[1:1 + G] - grad[1 + G:]) / (2 * h)
        return float(L[0]), grad[0], 0.5 * (H + H.T)

    def loss_at(gg):
        return float(ctx.param_grad((lo + gg * span)[None, :].contiguous(), targets, w=w, loss=loss)[0][0])

    g = g0.clone()
    L, grad, H = batch(g)
    lam = 1e-3
    stalled = 0
    for _ in range(iters):
        step = None
        for _ in range(12):
            A = H + lam * np.diag(np.maximum(np.diag(H), 1e-12))
            try:
                d = np.linalg.solve(A, -grad)
            except np.linalg.LinAlgError:
                d = None
            if d is not None and np.all(np.isfinite(d)):
                dt = torch.as_tensor(d, dtype=torch.float64, device=g.device)
                Ln = loss_at(g + dt)
                if Ln < L:
                    step = dt
                    break
            lam *= 10.0
        if step is None:
            break
        g = g + step
        lam = max(lam / 10.0, 1e-12)
        stalled = stalled + 1 if L - Ln <= 1e-10 * L else 0
        if stalled == 2:                               # at the rounding floor of the loss
            break
        L, grad, H = batch(g)
    return g


def _fd_newton_polish(ctx, g0, lo, hi, targets, w, iters: int, h: float = 1e-4):
    """Damped Newton in gene space on L = sum_q w_q S_q / D_q from FP64 fitness values alone (no
    gradient kernel): each iteration evaluates, in one batched call, the point, +-h along every gene
    and +-h along every pair of genes (1 + 2G + 2G(G-1) parameter sets), and takes the gradient and
    Hessian by central differences; steps as in `_newton_polish`."""
    G = g0.numel()
    span = hi - lo
    dev = g0.device
    offs = [np.zeros(G)]
    for i in range(G):
        for s in (1.0, -1.0):
            e = np.zeros(G)
            e[i] = s * h
            offs.append(e)
    pairs = [(i, j) for i in range(G) for j in range(i + 1, G)]
    for i, j in pairs:
        for si, sj in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
            e = np.zeros(G)
            e[i], e[j] = si * h, sj * h
            offs.append(e)
    offs = torch.as_tensor(np.stack(offs), dtype=torch.float64, device=dev)
    D = None

    def losses(pts):
        nonlocal D
        Z, Zq, S = ctx.fitness((lo + pts * span).contiguous(), targets, w=(1.0, 1.0, 1.0), precision=64)
        S, Zq = S.cpu().numpy(), Zq.cpu().numpy()
        if D is None:                                  # D_q = S_q / Zq_q^2 (Eq. 17-19), from the first point
            D = np.where(Zq[0] > 0, S[0] / np.maximum(Zq[0] ** 2, 1e-300), np.inf)
        return (np.asarray(w)[None, :] * S / D[None, :]).sum(-1)

    def batch(gg):
        L = losses(gg[None, :] + offs)
        L0, Lp, Lm = L[0], L[1:1 + 2 * G:2], L[2:2 + 2 * G:2]
        grad = (Lp - Lm) / (2 * h)
        H = np.diag((Lp - 2 * L0 + Lm) / (h * h))
        base = 1 + 2 * G
        for k, (i, j) in enumerate(pairs):
            a, b, c, d = L[base + 4 * k: base + 4 * k + 4]
            H[i, j] = H[j, i] = (a - b - c + d) / (4 * h * h)
        return float(L0), grad, H

    g = g0.clone()
    L, grad, H = batch(g)
    lam = 1e-3
    stalled = 0
    for _ in range(iters):
        step = None
        for _ in range(12):
            A = H + lam * np.diag(np.maximum(np.abs(np.diag(H)), 1e-12))
            try:
                d = np.linalg.solve(A, -grad)
            except np.linalg.LinAlgError:
                d = None
            if d is not None and np.all(np.isfinite(d)):
                dt = torch.as_tensor(d, dtype=torch.float64, device=dev)
                Ln = float(losses((g + dt)[None, :])[0])
                if Ln < L:
                    step = dt
                    break
            lam *= 10.0
        if step is None:
            break
        g = g + step
        lam = max(lam / 10.0, 1e-12)
        stalled = stalled + 1 if L - Ln <= 1e-12 * L else 0
        if stalled == 2:
            break
        L, grad, H = batch(g)
    return g


def polish(ctx: binding.Context, params, targets: dict, lo, hi, steps: int = 30, lr: float = 2e-3,
           w=(1.0, 1.0, 1.0), loss: int = binding.LOSS_SQ, method: str = "auto"):
    """Refine one parameter set on the smooth loss L = sum_q w_q S_q / D_q in gene space, with
    gradients from the adjoint kernel. The loss is a least-squares sum whose six directions are
    badly scaled (beta and n trade off along a long valley), so the default is a damped Newton method
    on a finite-difference Hessian of the adjoint gradient (`steps` iterations, one batched call of
    13 parameter sets each); `method="lbfgs"` (strong-Wolfe line search) and `method="adam"` (rate
    `lr`) are first-order alternatives. With `method="fd-newton"` the damped Newton step takes its
    gradient and Hessian by central differences of the FP64 fitness instead (no gradient kernel).
    "auto" is "newton", for either form. Returns (params, loss before, loss after)."""
    dev = torch.device("cuda")
    lo = torch.as_tensor(lo, dtype=torch.float64, device=dev)
    hi = torch.as_tensor(hi, dtype=torch.float64, device=dev)
    G = int(lo.numel())
    x0 = torch.as_tensor(params, dtype=torch.float64, device=dev).reshape(1, G)
    g0 = ((x0 - lo) / (hi - lo))
    if method == "auto":
        method = "newton"
    if method == "fd-newton":
        if loss != binding.LOSS_SQ:
            raise ValueError("the finite-difference polish minimises L_sq")

        def L_of(x):
            Z, Zq, S = ctx.fitness(x.contiguous(), targets, w=(1.0, 1.0, 1.0), precision=64)
            D = (S / torch.clamp(Zq * Zq, min=1e-300)).cpu().numpy()[0]
            return float((np.asarray(w) * S.cpu().numpy()[0] / D).sum())

        first = L_of(x0)
        g = _fd_newton_polish(ctx, g0[0], lo, hi, targets, w, int(steps)).reshape(1, G)
        x = (lo + g * (hi - lo)).contiguous()
        return x[0].cpu().numpy(), first, L_of(x)
    first = float(ctx.param_grad(x0.contiguous(), targets, w=w, loss=loss)[0][0])
    if method == "newton":
        g = _newton_polish(ctx, g0[0], lo, hi, targets, w, loss, int(steps)).reshape(1, G)
    elif method in ("lbfgs", "adam"):
        g = g0.clone().requires_grad_(True)

        def value(gg):
            return TersoffLoss.apply((lo + gg * (hi - lo)).contiguous(), ctx, targets, w, loss).sum()

        if method == "lbfgs":
            opt = torch.optim.LBFGS([g], lr=1.0, max_iter=int(steps), history_size=20, tolerance_grad=1e-14,
                                    tolerance_change=1e-16, line_search_fn="strong_wolfe")

            def closure():
                opt.zero_grad()
                L = value(g)
                L.backward()
                return L

            opt.step(closure)
        else:
            opt = torch.optim.Adam([g], lr=lr)
            for _ in range(steps):
                opt.zero_grad()
                value(g).backward()
                opt.step()
        g = g.detach()
    else:
        raise ValueError("method is 'auto', 'newton', 'fd-newton', 'lbfgs' or 'adam'")
    x = (lo + g * (hi - lo)).contiguous()
    L, _ = ctx.param_grad(x, targets, w=w, loss=loss)
    return x[0].cpu().numpy(), first, float(L[0])
