"""Plain FP64 CPU oracle of the minimal Tersoff potential, arXiv:1909.11474.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's CPU-baseline
leg, never by the product path. Independent of the CUDA path (no shared code, tables or helpers).

What it computes, in the paper's notation (all FP64, torch CPU tensors, autograd as a library step):

* neighbours: every periodic image (j, n) of every atom with |x_j - x_i + n.H| < R2, (j, n) != (i, 0)
  -- the index set of the sums over j (Eq. 2) and k (Eq. 7); a distinct periodic image counts as a
  distinct neighbour;
* U = sum_i U_i, U_i = 1/2 sum_j U_ij                                          (Eq. 1, 2)
* U_ij = f_C(r_ij) [f_R(r_ij) - b_ij f_A(r_ij)]                                 (Eq. 3)
* f_R = A exp(-lambda r), f_A = B exp(-mu r)                                   (Eq. 4, 5)
* A, B, lambda, mu from (D0, alpha, r0, S) with S fixed to 2                   (Eq. 11-14, Sec. II.B)
* b_ij = (1 + zeta_ij^n)^(-1/(2n)), zeta_ij = sum_k f_C(r_ik) g(theta_ijk)     (Eq. 6, 7)
* g = beta (cos theta_ijk - h)^2                                               (Eq. 10)
* f_C: 1 below R1, 1/2[1 + cos(pi (r - R1)/(R2 - R1))] between, 0 above R2     (Eq. 9)
* forces F_i = -dU/dx_i and virial W_mu,nu = -dU/d eps_mu,nu (homogeneous strain x -> (I+eps)x),
  both by reverse-mode autograd of U -- the plain definitions; the paper defers its force and
  virial formulas to another reference (Sec. III.C);
* fitness Z = w_e Z_e + w_v Z_v + w_f Z_f, each a relative RMS error          (Eq. 15, 17-19)
  over the parameter vector x = [D0, alpha, r0, beta, n, h]                    (Eq. 16)
* the Tersoff form: a parameter vector of nine, x = [D0, alpha, r0, S, n, h, gamma, c, d], takes
  the original angular function g^T = gamma (1 + c^2/d^2 - c^2/(d^2 + (cos - h)^2)) (Eq. 8) and a
  free S in Eq. 11-14; everything else as above

Readings where the paper is silent (also listed in the design notes):
* zeta_ij == 0 gives b_ij = 1, the value Eq. 6 takes in that limit; the branch is taken without
  evaluating 0^n, so derivatives stay finite for n < 1;
* energies and virials enter the fitness per atom (E_c / N_c, W_c / N_c); forces per atom as is;
* the virial components are ordered xx, yy, zz, xy, yz, zx (the six non-equivalent ones, Eq. 18);
* a quantity with no target anywhere (D_q = 0) drops out of Z;
* L_sq = sum_q w_q S_q / D_q is the smooth loss used for gradients; Z itself is also offered.
"""
from __future__ import annotations

import math

import numpy as np
import torch

R1_DEFAULT = 2.8   # Sec. II.B, Table 2
R2_DEFAULT = 3.2
S_FIXED = 2.0      # Sec. II.B: the Pauling-plot slope S is fixed to 2

_F64 = torch.float64


# ------------------------------------------------------------------------------------------------
# Neighbours (index set of the sums in Eq. 2 and Eq. 7)
# ------------------------------------------------------------------------------------------------

def _image_range(pos: np.ndarray, H: np.ndarray, R2: float):
    """Integer image ranges wide enough to contain every (j, n) with |x_j - x_i + n.H| < R2."""
    vol = abs(float(np.linalg.det(H)))
    s = pos @ np.linalg.inv(H)
    span = s.max(axis=0) - s.min(axis=0) if len(pos) else np.zeros(3)
    nmax = []
    for k in range(3):
        area = np.linalg.norm(np.cross(H[(k + 1) % 3], H[(k + 2) % 3]))
        plane_gap = vol / area
        nmax.append(int(math.ceil(R2 / plane_gap + span[k])) + 1)
    return nmax


def neighbor_list(pos, box, R2: float = R2_DEFAULT):
    """All neighbour entries (j, n0, n1, n2) of every atom i, in ascending (j, n0, n1, n2) order.

    The membership test is exact FP64 with a fixed evaluation order and no fused multiply-add:
        t   = (n0*a + n1*b) + n2*c            (a, b, c = rows of the box)
        d   = (x_j - x_i) + t                 (per component)
        r^2 = (d_x*d_x + d_y*d_y) + d_z*d_z,  kept when r^2 < R2*R2.
    Returns {"off": [N+1] int64, "j": [B] int64, "n": [B][3] int64}.
    """
    pos = np.asarray(pos, dtype=np.float64)
    H = np.asarray(box, dtype=np.float64)
    N = len(pos)
    nmax = _image_range(pos, H, R2)
    grid = np.array([(a, b, c)
                     for a in range(-nmax[0], nmax[0] + 1)
                     for b in range(-nmax[1], nmax[1] + 1)
                     for c in range(-nmax[2], nmax[2] + 1)], dtype=np.int64)
    g = grid.astype(np.float64)
    T = (g[:, 0:1] * H[0][None, :] + g[:, 1:2] * H[1][None, :]) + g[:, 2:3] * H[2][None, :]
    R2sq = R2 * R2
    offs = [0]
    js, ns = [], []
    zero_img = np.flatnonzero((grid == 0).all(axis=1))[0]
    for i in range(N):
        dx = (pos[:, 0] - pos[i, 0])[:, None] + T[None, :, 0]
        dy = (pos[:, 1] - pos[i, 1])[:, None] + T[None, :, 1]
        dz = (pos[:, 2] - pos[i, 2])[:, None] + T[None, :, 2]
        r2 = (dx * dx + dy * dy) + dz * dz
        keep = r2 < R2sq
        keep[i, zero_img] = False
        jj, kk = np.nonzero(keep)          # C order: j ascending, then image index ascending
        js.append(jj)
        ns.append(grid[kk])
        offs.append(offs[-1] + len(jj))
    return {"off": np.array(offs, dtype=np.int64),
            "j": np.concatenate(js).astype(np.int64) if js else np.zeros(0, np.int64),
            "n": np.concatenate(ns).astype(np.int64) if ns else np.zeros((0, 3), np.int64)}


def neighbor_list_subset(pos, box, R2: float, atoms):
    """Neighbour entries of the atoms listed in `atoms` only, for cells whose lattice-plane spacings
    all exceed 2*R2 (so every (j, n) with |d| < R2 has |s_j - s_i + n_k| < 1/2 on each axis and lies
    among the candidates n = -round(s_j - s_i) + {-1, 0, 1}^3). Same exact FP64 test and order as
    neighbor_list. Returns a list of (j [k], n [k][3]) per requested atom."""
    pos = np.asarray(pos, dtype=np.float64)
    H = np.asarray(box, dtype=np.float64)
    s = pos @ np.linalg.inv(H)
    off = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=np.int64)
    R2sq = R2 * R2
    out = []
    for i in atoms:
        base = -np.rint(s - s[i]).astype(np.int64)                 # [N][3]
        cand = base[:, None, :] + off[None, :, :]                   # [N][27][3]
        g = cand.astype(np.float64)
        T = (g[..., 0:1] * H[0] + g[..., 1:2] * H[1]) + g[..., 2:3] * H[2]
        dx = (pos[:, 0] - pos[i, 0])[:, None] + T[..., 0]
        dy = (pos[:, 1] - pos[i, 1])[:, None] + T[..., 1]
        dz = (pos[:, 2] - pos[i, 2])[:, None] + T[..., 2]
        r2 = (dx * dx + dy * dy) + dz * dz
        keep = r2 < R2sq
        keep[i] &= ~(cand[i] == 0).all(axis=1)
        jj, kk = np.nonzero(keep)
        n = cand[jj, kk]
        order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], jj))
        out.append((jj[order], n[order]))
    return out


def _triplets(off: np.ndarray):
    """Ordered pairs (a, b), a != b, of neighbour entries of the same atom: the (ij, ik) terms of Eq. 7."""
    ta, tb = [], []
    for i in range(len(off) - 1):
        e = np.arange(off[i], off[i + 1])
        if len(e) < 2:
            continue
        a, b = np.meshgrid(e, e, indexing="ij")
        sel = a != b
        ta.append(a[sel])
        tb.append(b[sel])
    if not ta:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(ta), np.concatenate(tb)


# ------------------------------------------------------------------------------------------------
# Energy (Eq. 1-14)
# ------------------------------------------------------------------------------------------------

def cutoff(r: torch.Tensor, R1: float, R2: float) -> torch.Tensor:
    """f_C of Eq. 9."""
    inner = 0.5 * (1.0 + torch.cos(math.pi * (r - R1) / (R2 - R1)))
    return torch.where(r <= R1, torch.ones_like(r), torch.where(r >= R2, torch.zeros_like(r), inner))


def site_energy_sum(d: torch.Tensor, owner: torch.Tensor, ta: torch.Tensor, tb: torch.Tensor,
                    natoms: int, params: torch.Tensor, R1: float, R2: float):
    """U and the site energies U_i from the neighbour vectors d (one row per entry (i; j, n)).

    owner[e] = i of entry e; (ta, tb) = ordered entry pairs of the same atom (Eq. 7's k != j).
    """
    tersoff_form = params.numel() == 9
    if tersoff_form:   # x = [D0, alpha, r0, S, n, h, gamma, c, d]: Eq. 8 angular function, free S
        D0, alpha, r0, S, n, h, gamma, c, dd = params.unbind()
        # Eq. 11-14
        A = D0 / (S - 1.0) * torch.exp(alpha * r0 * torch.sqrt(2.0 * S))
        B = D0 * S / (S - 1.0) * torch.exp(alpha * r0 * torch.sqrt(2.0 / S))
        lam = alpha * torch.sqrt(2.0 * S)
        mu = alpha * torch.sqrt(2.0 / S)
    else:
        D0, alpha, r0, beta, n, h = params.unbind()
        S = S_FIXED
        # Eq. 11-14
        A = D0 / (S - 1.0) * torch.exp(alpha * r0 * math.sqrt(2.0 * S))
        B = D0 * S / (S - 1.0) * torch.exp(alpha * r0 * math.sqrt(2.0 / S))
        lam = alpha * math.sqrt(2.0 * S)
        mu = alpha * math.sqrt(2.0 / S)

    r = torch.sqrt((d * d).sum(dim=1))
    fC = cutoff(r, R1, R2)
    fR = A * torch.exp(-lam * r)          # Eq. 4
    fA = B * torch.exp(-mu * r)           # Eq. 5

    # Eq. 7 with Eq. 10: zeta_ij = sum_{k != j} f_C(r_ik) beta (cos theta_ijk - h)^2, or with Eq. 8:
    # g = gamma (1 + c^2/d^2 - c^2 / (d^2 + (cos theta_ijk - h)^2))
    cos_t = (d[ta] * d[tb]).sum(dim=1) / (r[ta] * r[tb])
    if tersoff_form:
        g = gamma * (1.0 + c ** 2 / dd ** 2 - c ** 2 / (dd ** 2 + (cos_t - h) ** 2))
    else:
        g = beta * (cos_t - h) ** 2
    zeta = torch.zeros(len(r), dtype=_F64).index_add(0, ta, fC[tb] * g)

    # Eq. 6, with b = 1 taken directly when zeta = 0
    pos = zeta > 0
    zs = torch.where(pos, zeta, torch.ones_like(zeta))
    b = torch.where(pos, (1.0 + zs ** n) ** (-1.0 / (2.0 * n)), torch.ones_like(zeta))

    Uij = fC * (fR - b * fA)              # Eq. 3
    Ui = 0.5 * torch.zeros(natoms, dtype=_F64).index_add(0, owner, Uij)   # Eq. 2
    # magnitude of the summands of U (a conditioning scale for error bars, not part of U)
    scale = 0.5 * (fC * (fR.abs() + (b * fA).abs())).sum()
    return Ui.sum(), Ui, scale            # Eq. 1


class _Prepared:
    """Parameter-independent index data of one configuration."""

    def __init__(self, pos, box, R2):
        self.pos = np.asarray(pos, dtype=np.float64)
        self.box = np.asarray(box, dtype=np.float64)
        self.N = len(self.pos)
        self.nl = neighbor_list(self.pos, self.box, R2)
        off = self.nl["off"]
        self.owner = torch.from_numpy(np.repeat(np.arange(self.N), np.diff(off)))
        self.j = torch.from_numpy(self.nl["j"])
        ng = self.nl["n"].astype(np.float64)
        H = self.box
        T = (ng[:, 0:1] * H[0][None, :] + ng[:, 1:2] * H[1][None, :]) + ng[:, 2:3] * H[2][None, :]
        self.T = torch.from_numpy(T)
        ta, tb = _triplets(off)
        self.ta = torch.from_numpy(ta)
        self.tb = torch.from_numpy(tb)


def _energy_graph(prep: _Prepared, params: torch.Tensor, R1, R2, create_graph=False):
    x = torch.tensor(prep.pos, dtype=_F64, requires_grad=True)
    eps = torch.zeros((3, 3), dtype=_F64, requires_grad=True)
    d0 = (x[prep.j] - x[prep.owner]) + prep.T
    d = d0 + d0 @ eps.T                    # (I + eps) d, homogeneous strain
    U, Ui, scale = site_energy_sum(d, prep.owner, prep.ta, prep.tb, prep.N, params, R1, R2)
    gx, ge, gd = torch.autograd.grad(U, (x, eps, d), create_graph=create_graph)
    F = -gx
    Wm = -ge                               # W_mu,nu = -dU/d eps_mu,nu
    W6 = torch.stack([Wm[0, 0], Wm[1, 1], Wm[2, 2], Wm[0, 1], Wm[1, 2], Wm[2, 0]])
    # magnitude of the summands of W = -sum_bonds dU/dd (x) d (conditioning scale, diagnostics only)
    wscale = (gd.detach().norm(dim=1) * d.detach().norm(dim=1)).sum()
    # per atom: summed magnitudes of the bond terms of its force, F_i = sum_{e from i} g_e - sum_{e to i} g_e
    # (g_e = dU/dd_e), the conditioning scale of that sum (diagnostics only)
    gn = gd.detach().norm(dim=1)
    fscale = torch.zeros(prep.N, dtype=_F64).index_add(0, prep.owner, gn).index_add(0, prep.j, gn)
    return U, Ui, F, W6, Wm, scale.detach(), wscale, fscale


def evaluate(pos, box, params, R1: float = R1_DEFAULT, R2: float = R2_DEFAULT, prep=None):
    """E (eV, total), F [N][3] (eV/A), W [6] (eV, total; xx, yy, zz, xy, yz, zx), W3 [3][3], U_i [N]."""
    prep = prep or _Prepared(pos, box, R2)
    p = torch.as_tensor(np.asarray(params, dtype=np.float64))
    U, Ui, F, W6, Wm, es, ws, fs = _energy_graph(prep, p, R1, R2)
    return {"E": float(U.detach()), "F": F.detach().numpy(), "W": W6.detach().numpy(),
            "W3": Wm.detach().numpy(), "Ui": Ui.detach().numpy(),
            "E_scale": float(es), "W_scale": float(ws), "F_scale": fs.numpy()}


def evaluate_batch(configs, params, R1: float = R1_DEFAULT, R2: float = R2_DEFAULT, pairs=None,
                   scales: bool = False, force_scales: bool = False):
    """E [P][C], W [P][C][6], F [P][Ntot][3] for every (parameter set p, configuration c).

    `pairs` optionally restricts the work to a list of (p, c); other entries are left NaN.
    With scales=True also returns ES [P][C], WS [P][C]: the summed magnitudes of the summands of E
    and of W, the conditioning scales of the two sums; with force_scales=True also FS [P][Ntot], the
    summed magnitudes of the bond terms of each atom's force.
    """
    params = np.atleast_2d(np.asarray(params, dtype=np.float64))
    P, C = len(params), configs.C
    E = np.full((P, C), np.nan)
    W = np.full((P, C, 6), np.nan)
    F = np.full((P, configs.Ntot, 3), np.nan)
    ES = np.full((P, C), np.nan)
    WS = np.full((P, C), np.nan)
    FS = np.full((P, configs.Ntot), np.nan)
    todo = {}
    for p, c in (pairs if pairs is not None else [(p, c) for c in range(C) for p in range(P)]):
        todo.setdefault(c, []).append(p)
    for c, plist in todo.items():
        pos, box = configs.config(c)
        prep = _Prepared(pos, box, R2)
        a = int(configs.atom_off[c])
        for p in plist:
            r = evaluate(pos, box, params[p], R1, R2, prep=prep)
            E[p, c] = r["E"]
            W[p, c] = r["W"]
            F[p, a:a + len(pos)] = r["F"]
            ES[p, c] = r["E_scale"]
            WS[p, c] = r["W_scale"]
            FS[p, a:a + len(pos)] = r["F_scale"]
    if scales and force_scales:
        return E, W, F, ES, WS, FS
    if scales:
        return E, W, F, ES, WS
    return E, W, F


# ------------------------------------------------------------------------------------------------
# Fitness (Eq. 15-19)
# ------------------------------------------------------------------------------------------------

def data_norms(configs, targets):
    """D_e, D_v, D_f: the denominators of Eq. 17-19 (sums of squared targets over masked configs)."""
    mask = np.asarray(targets["mask"])
    De = Dv = Df = 0.0
    for c in range(configs.C):
        a, b = int(configs.atom_off[c]), int(configs.atom_off[c + 1])
        if mask[c] & 1:
            De += float(targets["E"][c]) ** 2
        if mask[c] & 2:
            Dv += float(np.sum(np.asarray(targets["W"][c]) ** 2))
        if mask[c] & 4:
            Df += float(np.sum(np.asarray(targets["F"][a:b]) ** 2))
    return De, Dv, Df


def _residual_sums(configs, targets, E, W, F):
    """S_e, S_v, S_f of one parameter set: E [C] total, W [C][6] total, F [Ntot][3]."""
    mask = np.asarray(targets["mask"])
    Se = Sv = Sf = 0.0
    for c in range(configs.C):
        a, b = int(configs.atom_off[c]), int(configs.atom_off[c + 1])
        N = b - a
        if mask[c] & 1:
            Se += (E[c] / N - targets["E"][c]) ** 2
        if mask[c] & 2:
            Sv += float(np.sum((np.asarray(W[c]) / N - targets["W"][c]) ** 2))
        if mask[c] & 4:
            Sf += float(np.sum((np.asarray(F[a:b]) - targets["F"][a:b]) ** 2))
    return Se, Sv, Sf


def fitness_from_predictions(configs, targets, E, W, F, w=(1.0, 1.0, 1.0)):
    """Z [P], Zq [P][3], L_sq [P] and S [P][3] from predictions E [P][C], W [P][C][6], F [P][Ntot][3]."""
    D = data_norms(configs, targets)
    P = E.shape[0]
    Z = np.zeros(P)
    Zq = np.zeros((P, 3))
    L = np.zeros(P)
    S = np.zeros((P, 3))
    for p in range(P):
        S[p] = _residual_sums(configs, targets, E[p], W[p], F[p])
        for q in range(3):
            if D[q] > 0:
                Zq[p, q] = math.sqrt(S[p, q] / D[q])
                L[p] += w[q] * S[p, q] / D[q]
        Z[p] = float(np.dot(w, Zq[p]))
        if not (np.isfinite(E[p]).all() and np.isfinite(W[p]).all() and np.isfinite(F[p]).all()):
            Z[p] = math.inf
            L[p] = math.inf
    return {"Z": Z, "Zq": Zq, "L": L, "S": S, "D": np.array(D)}


def fitness(configs, params, targets, w=(1.0, 1.0, 1.0), R1=R1_DEFAULT, R2=R2_DEFAULT):
    E, W, F = evaluate_batch(configs, params, R1, R2)
    return fitness_from_predictions(configs, targets, E, W, F, w)


def loss_and_grad(configs, params_row, targets, w=(1.0, 1.0, 1.0), loss: str = "sq",
                  R1=R1_DEFAULT, R2=R2_DEFAULT):
    """Loss of one parameter set and its gradient over x = [D0, alpha, r0, beta, n, h], or over the
    nine parameters of the Tersoff form (x = [D0, alpha, r0, S, n, h, gamma, c, d]).

    loss = "sq": L = sum_q w_q S_q / D_q; loss = "z": Z of Eq. 15.  Forces enter through
    F = -dU/dx built with create_graph, so the gradient is exact reverse-over-reverse autograd.
    """
    D = data_norms(configs, targets)
    p = torch.tensor(np.asarray(params_row, dtype=np.float64), requires_grad=True)
    mask = np.asarray(targets["mask"])
    S = [torch.zeros((), dtype=_F64) for _ in range(3)]
    for c in range(configs.C):
        pos, box = configs.config(c)
        a = int(configs.atom_off[c])
        N = len(pos)
        prep = _Prepared(pos, box, R2)
        need_graph = bool(mask[c] & 6)
        U, _, F, W6, _, _, _, _ = _energy_graph(prep, p, R1, R2, create_graph=need_graph)
        if mask[c] & 1:
            S[0] = S[0] + (U / N - float(targets["E"][c])) ** 2
        if mask[c] & 2:
            S[1] = S[1] + ((W6 / N - torch.as_tensor(targets["W"][c])) ** 2).sum()
        if mask[c] & 4:
            S[2] = S[2] + ((F - torch.as_tensor(targets["F"][a:a + N])) ** 2).sum()
    L = torch.zeros((), dtype=_F64)
    for q in range(3):
        if D[q] > 0:
            L = L + (w[q] * S[q] / D[q] if loss == "sq" else w[q] * torch.sqrt(S[q] / D[q]))
    (g,) = torch.autograd.grad(L, p)
    return float(L.detach()), g.numpy()
