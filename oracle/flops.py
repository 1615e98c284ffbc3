"""Operation count of the minimal-Tersoff E/F/W evaluation and its fitness residuals, by running the
formulas through a scalar type that counts what it computes.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the counts it yields are frozen as constants in
the benchmark, and tests/test_flop_model.py checks that the constants equal what this module counts.

The formula listing `site_terms` writes out, for one atom i with its bonds j (cached,
parameter-independent geometry: r_ij, the unit vector u_ij, f_C(r_ij), f_C'(r_ij) of Eq. 9 and the
cosines of the bond pairs), the steps of the method in the paper's notation:

  f_R = A e^{-lambda r}, f_A = B e^{-mu r} (Eq. 4-5) and their r-derivatives;
  g = beta (cos - h)^2 (Eq. 10) and g' = 2 beta (cos - h), per pair of bonds;
  zeta_ij = sum_{k != j} f_C(r_ik) g(theta_ijk) (Eq. 7);
  b_ij = (1 + zeta^n)^{-1/(2n)} (Eq. 6) and b'_ij = db/dzeta;
  U_i = 1/2 sum_j f_C (f_R - b f_A) (Eq. 2-3); c_ij = dU_i/dzeta_ij = -1/2 f_C f_A b';
  dU_i/dd_ij = 1/2 [f_C'(f_R - b f_A) + f_C (f_R' - b f_A')] u_ij
               + c_ij sum_{k != j} f_C(r_ik) g'(cos_ijk) (u_ik - cos_ijk u_ij) / r_ij
               + sum_{k != j} c_ik [f_C'(r_ij) g(cos_ijk) u_ij + f_C(r_ij) g'(cos_ijk) (u_ik - cos_ijk u_ij) / r_ij],
  the derivative of Eq. 2 with respect to the bond vector d_ij (F_i = -dU/dx_i gathers it:
  F_i = sum_j (dU_i/dd_ij - dU_j/dd_ji)), and the virial W = -sum_ij d_ij (x) dU_i/dd_ij;

and `residual_terms` the per-atom force residual of Eq. 19. Each quantity is computed once where the
formula names it (f_R, f_A, 1/r per bond; g, g' per pair of bonds; the vector (u_ik - cos u_ij)/r_ij
once per ordered pair), and nothing else is rearranged.

Counting conventions (the figures of the roofline): +, -, * and / of two operands are 1 FLOP each (a
fused multiply-add therefore counts 2); a sign change is free; exp and log are 1 transcendental (XU)
op each, and x**y = exp(y log x) is 2 XU ops and 1 FLOP. Work on per-parameter-set constants (A, B,
lambda, mu from Eq. 11-14, 2 beta, -1/(2n)) happens once per parameter set and is not per-atom work;
work on the geometry happens once per neighbour build. Both are left out, as the evaluation of a
parameter set over a cached geometry does not repeat them.

The listing is pinned, independently of the counts, by evaluating it in floating point: its E, F and W
equal the oracle's (autograd of Eq. 1-14) on cells with bonds in the switching region of f_C.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .tersoff import R1_DEFAULT, R2_DEFAULT, S_FIXED, cutoff, neighbor_list


class Counter:
    """Tallies of FLOP and XU ops, split by the loop they occur in."""

    def __init__(self):
        self.flop = {}
        self.xu = {}
        self.where = "none"

    def add(self, kind, n=1):
        d = self.flop if kind == "flop" else self.xu
        d[self.where] = d.get(self.where, 0) + n


class Num:
    """A float that reports each arithmetic operation to a Counter."""

    __slots__ = ("v", "c")

    def __init__(self, v, c):
        self.v = float(v)
        self.c = c

    def _o(self, x):
        return x.v if isinstance(x, Num) else float(x)

    def _r(self, v):
        self.c.add("flop")
        return Num(v, self.c)

    def __add__(self, x): return self._r(self.v + self._o(x))
    def __radd__(self, x): return self._r(self._o(x) + self.v)
    def __sub__(self, x): return self._r(self.v - self._o(x))
    def __rsub__(self, x): return self._r(self._o(x) - self.v)
    def __mul__(self, x): return self._r(self.v * self._o(x))
    def __rmul__(self, x): return self._r(self._o(x) * self.v)
    def __truediv__(self, x): return self._r(self.v / self._o(x))
    def __rtruediv__(self, x): return self._r(self._o(x) / self.v)
    def __neg__(self): return Num(-self.v, self.c)
    def __gt__(self, x): return self.v > self._o(x)
    def __le__(self, x): return self.v <= self._o(x)

    def sqrt(self):
        self.c.add("xu")
        return Num(math.sqrt(self.v), self.c)

    def __pow__(self, y):
        self.c.add("xu", 2)
        self.c.add("flop")
        return Num(self.v ** self._o(y), self.c)


def _exp(x):
    if isinstance(x, DNum):
        return x.exp()
    if isinstance(x, Num):
        x.c.add("xu")
        return Num(math.exp(x.v), x.c)
    return math.exp(x)


def _sqrt(x):
    if isinstance(x, (Num, DNum)):
        return x.sqrt()
    return math.sqrt(x)


def _cospi(x):
    if isinstance(x, DNum):
        x.c.add("xu")
        x.c.add("flop", 1 + x._k())
        sv = -math.pi * math.sin(math.pi * x.v)
        return DNum(math.cos(math.pi * x.v), [sv * a for a in x.d], x.c)
    if isinstance(x, Num):
        x.c.add("xu")
        return Num(math.cos(math.pi * x.v), x.c)
    return math.cos(math.pi * x)


def _sinpi(x):
    if isinstance(x, DNum):
        x.c.add("xu")
        x.c.add("flop", 1 + x._k())
        cv = math.pi * math.cos(math.pi * x.v)
        return DNum(math.sin(math.pi * x.v), [cv * a for a in x.d], x.c)
    if isinstance(x, Num):
        x.c.add("xu")
        return Num(math.sin(math.pi * x.v), x.c)
    return math.sin(math.pi * x)


class DNum:
    """A value with K tangents (forward-mode dual number) that reports its arithmetic to a Counter:
    the counted work of forward-mode differentiation of the listing with respect to the parameters.
    Per operation (value, then each tangent): a +- b: 1 + K; a * b: 1 + 3K (1 + K with a constant
    factor); a / b: 1 + 3K (1 + K with a constant denominator); exp: 1 XU + K; sqrt: 1 XU + 1 + K;
    x**y = exp(y log x): 2 XU + 1, plus 1 for y / x and 4 per tangent."""

    __slots__ = ("v", "d", "c")

    def __init__(self, v, d, c):
        self.v = float(v)
        self.d = list(d)
        self.c = c

    @staticmethod
    def const(v, K, c):
        return DNum(v, [0.0] * K, c)

    def _k(self):
        return len(self.d)

    def _lift(self, x):
        return x if isinstance(x, DNum) else None

    def __add__(self, x):
        y = self._lift(x)
        if y is None:
            self.c.add("flop")
            return DNum(self.v + float(x), self.d, self.c)
        self.c.add("flop", 1 + self._k())
        return DNum(self.v + y.v, [a + b for a, b in zip(self.d, y.d)], self.c)

    __radd__ = __add__

    def __sub__(self, x):
        y = self._lift(x)
        if y is None:
            self.c.add("flop")
            return DNum(self.v - float(x), self.d, self.c)
        self.c.add("flop", 1 + self._k())
        return DNum(self.v - y.v, [a - b for a, b in zip(self.d, y.d)], self.c)

    def __rsub__(self, x):
        self.c.add("flop")
        return DNum(float(x) - self.v, [-a for a in self.d], self.c)

    def __mul__(self, x):
        y = self._lift(x)
        if y is None:
            self.c.add("flop", 1 + self._k())
            return DNum(self.v * float(x), [a * float(x) for a in self.d], self.c)
        self.c.add("flop", 1 + 3 * self._k())
        return DNum(self.v * y.v, [a * y.v + self.v * b for a, b in zip(self.d, y.d)], self.c)

    __rmul__ = __mul__

    def __truediv__(self, x):
        y = self._lift(x)
        if y is None:
            self.c.add("flop", 1 + self._k())
            return DNum(self.v / float(x), [a / float(x) for a in self.d], self.c)
        q = self.v / y.v
        self.c.add("flop", 1 + 3 * self._k())
        return DNum(q, [(a - q * b) / y.v for a, b in zip(self.d, y.d)], self.c)

    def __rtruediv__(self, x):
        q = float(x) / self.v
        self.c.add("flop", 1 + 2 * self._k())
        return DNum(q, [-q * b / self.v for b in self.d], self.c)

    def __neg__(self):
        return DNum(-self.v, [-a for a in self.d], self.c)

    def __gt__(self, x):
        return self.v > (x.v if isinstance(x, DNum) else float(x))

    def __le__(self, x):
        return self.v <= (x.v if isinstance(x, DNum) else float(x))

    def exp(self):
        e = math.exp(self.v)
        self.c.add("xu")
        self.c.add("flop", self._k())
        return DNum(e, [e * a for a in self.d], self.c)

    def sqrt(self):
        q = math.sqrt(self.v)
        self.c.add("xu")
        self.c.add("flop", 1 + self._k())
        return DNum(q, [a * (0.5 / q) for a in self.d], self.c)

    def __pow__(self, y):
        yv = y.v if isinstance(y, DNum) else float(y)
        yd = y.d if isinstance(y, DNum) else [0.0] * self._k()
        v = self.v ** yv
        L = math.log(self.v)
        self.c.add("xu", 2)
        self.c.add("flop", 2 + 4 * self._k())
        return DNum(v, [v * (b * L + yv * a / self.v) for a, b in zip(self.d, yd)], self.c)


def _acc(s, x):
    """Running sum that starts at its first term (a sum of n terms takes n - 1 additions)."""
    return x if s is None else s + x


class _Stage:
    """Sets the loop label of the counter (no effect on plain floats)."""

    def __init__(self, c):
        self.c = c

    def __call__(self, where):
        if self.c is not None:
            self.c.where = where


def geometry_terms(dvec, R1, R2, stage):
    """Bond geometry from the bond vectors d_ij (lists of three scalars): r, u = d / r, f_C and f_C'
    (Eq. 9), and the cosines of the bond pairs. The batched evaluation caches these per neighbour build
    (they do not depend on the parameters); the MD-scale call computes them every step."""
    stage("geometry_bond")
    m = len(dvec)
    r, u, fc, fcp = [], [], [], []
    for d in dvec:
        r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
        rj = _sqrt(r2)
        inv = 1.0 / rj
        r.append(rj)
        u.append([d[a] * inv for a in range(3)])
        x = rj.v if isinstance(rj, (Num, DNum)) else rj
        if x <= R1:
            fc.append(1.0)
            fcp.append(0.0)
        elif x >= R2:
            fc.append(0.0)
            fcp.append(0.0)
        else:
            w = (rj - R1) * (1.0 / (R2 - R1))
            fc.append(0.5 * (1.0 + _cospi(w)))
            fcp.append((-0.5 * math.pi / (R2 - R1)) * _sinpi(w))
    stage("geometry_pair")
    cos = [[None] * m for _ in range(m)]
    for j in range(m):
        for k in range(j + 1, m):
            cos[j][k] = cos[k][j] = (u[j][0] * u[k][0] + u[j][1] * u[k][1]) + u[j][2] * u[k][2]
    return r, u, fc, fcp, cos


def site_terms(r, u, fc, fcp, cos, K, stage):
    """One atom: U_i, and P_j = dU_i/dd_ij for its m bonds (lists of three scalars).

    r, fc, fcp: [m] scalars; u: [m] lists of three scalars; cos[j][k]: cosine of bonds j, k (j != k).
    K: per-parameter-set constants A, B, lam, mu, beta, two_beta, h, n, m_inv2n (= -1/(2n)).
    """
    m = len(r)
    A, B, lam, mu = K["A"], K["B"], K["lam"], K["mu"]
    beta, two_beta, h, n, m_inv2n = K["beta"], K["two_beta"], K["h"], K["n"], K["m_inv2n"]
    # pair functions and their r-derivatives (Eq. 4-5), per bond
    stage("bond")
    fR, fA, dfR, dfA, inv_r = [], [], [], [], []
    for j in range(m):
        fR.append(A * _exp(-(lam * r[j])))
        fA.append(B * _exp(-(mu * r[j])))
        dfR.append(-(lam * fR[j]))
        dfA.append(-(mu * fA[j]))
        inv_r.append(1.0 / r[j])
    # angular function g and g' (Eq. 10), per pair of bonds (cos is symmetric in j, k)
    stage("pair")
    g = [[None] * m for _ in range(m)]
    gp = [[None] * m for _ in range(m)]
    for j in range(m):
        for k in range(j + 1, m):
            t = cos[j][k] - h
            g[j][k] = g[k][j] = beta * (t * t)
            gp[j][k] = gp[k][j] = two_beta * t
    # zeta_ij (Eq. 7), per ordered pair
    stage("triplet")
    zeta = [None] * m
    for j in range(m):
        for k in range(m):
            if k != j:
                zeta[j] = _acc(zeta[j], fc[k] * g[j][k])
        if zeta[j] is None:
            zeta[j] = 0.0
    # bond order (Eq. 6), bond energy (Eq. 3) and the coefficients of the derivative, per bond
    stage("bond")
    U = None
    c, rad = [], []
    for j in range(m):
        if zeta[j] > 0.0:
            zn = zeta[j] ** n
            opz = 1.0 + zn
            b = opz ** m_inv2n
            bp = -(0.5 * (b * (zn / (zeta[j] * opz))))
        else:                                   # zeta = 0: b = 1, b' = 0 (the limit of Eq. 6)
            b, bp = 1.0, 0.0
        e = fR[j] - b * fA[j]
        U = _acc(U, fc[j] * e)
        c.append(-(0.5 * (fc[j] * (fA[j] * bp))))
        rad.append(0.5 * (fcp[j] * e + fc[j] * (dfR[j] - b * dfA[j])))
    # angular part of dU_i/dd_ij: the two sums over k != j of the derivative, per ordered pair
    stage("triplet")
    Pang = [[None, None, None] for _ in range(m)]
    for j in range(m):
        for k in range(m):
            if k == j:
                continue
            v = [(u[k][a] - cos[j][k] * u[j][a]) * inv_r[j] for a in range(3)]
            s_a = c[j] * (fc[k] * gp[j][k])
            s_b1 = c[k] * (fcp[j] * g[j][k])
            s_b2 = c[k] * (fc[j] * gp[j][k])
            for a in range(3):
                Pang[j][a] = _acc(Pang[j][a], s_a * v[a])
                Pang[j][a] = _acc(Pang[j][a], s_b1 * u[j][a] + s_b2 * v[a])
    # radial part and the whole derivative, per bond
    stage("bond")
    P = [[rad[j] * u[j][a] + (Pang[j][a] if Pang[j][a] is not None else 0.0) for a in range(3)]
         for j in range(m)]
    stage("atom")
    return (0.5 * U if U is not None else 0.0), P


def virial_terms(r, u, P, W, stage):
    """W_{mu nu} -= d_mu P_nu for the atom's bonds, d = r u (components xx, yy, zz, xy, yz, zx)."""
    stage("bond")
    for j in range(len(r)):
        d = [r[j] * u[j][a] for a in range(3)]
        for q, (mu_, nu_) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0))):
            W[q] = W[q] - d[mu_] * P[j][nu_]
    stage("atom")


def residual_terms(F, Ft, stage):
    """|F_i - F*_i|^2 of one atom (Eq. 19)."""
    stage("atom")
    s = None
    for a in range(3):
        e = F[a] - Ft[a]
        s = _acc(s, e * e)
    return s


def constants(params):
    """Per-parameter-set constants of the listing from x = [D0, alpha, r0, beta, n, h] (Eq. 11-14, S = 2)."""
    D0, alpha, r0, beta, n, h = (float(v) for v in params)
    S = S_FIXED
    return {"A": D0 / (S - 1.0) * math.exp(alpha * r0 * math.sqrt(2.0 * S)),
            "B": D0 * S / (S - 1.0) * math.exp(alpha * r0 * math.sqrt(2.0 / S)),
            "lam": alpha * math.sqrt(2.0 * S), "mu": alpha * math.sqrt(2.0 / S),
            "beta": beta, "two_beta": 2.0 * beta, "h": h, "n": n, "m_inv2n": -1.0 / (2.0 * n)}


def constant_tangents(params):
    """d(constant)/dx for x = [D0, alpha, r0, beta, n, h], by the chain rule through Eq. 11-14."""
    D0, alpha, r0, beta, n, h = (float(v) for v in params)
    k = constants(params)
    s2, si = math.sqrt(2.0 * S_FIXED), math.sqrt(2.0 / S_FIXED)
    return {"A": [k["A"] / D0, k["A"] * r0 * s2, k["A"] * alpha * s2, 0, 0, 0],
            "B": [k["B"] / D0, k["B"] * r0 * si, k["B"] * alpha * si, 0, 0, 0],
            "lam": [0, s2, 0, 0, 0, 0], "mu": [0, si, 0, 0, 0, 0],
            "beta": [0, 0, 0, 1, 0, 0], "two_beta": [0, 0, 0, 2, 0, 0], "h": [0, 0, 0, 0, 0, 1],
            "n": [0, 0, 0, 0, 1, 0], "m_inv2n": [0, 0, 0, 0, 0.5 / (n * n), 0]}


def evaluate_listing(pos, box, params, R1=R1_DEFAULT, R2=R2_DEFAULT, counter=None, F_target=None,
                     tangents=False):
    """E, F [N][3], W [6] of one configuration from the listing (floats; counted with `counter`), and with
    F_target also the force residual sum of Eq. 19. tangents=True carries the derivatives with respect
    to x = [D0, alpha, r0, beta, n, h] (forward mode): each returned value is then (value, [6 tangents])."""
    pos = np.asarray(pos, dtype=np.float64)
    H = np.asarray(box, dtype=np.float64)
    N = len(pos)
    nl = neighbor_list(pos, H, R2)
    off, js, ns = nl["off"], nl["j"], nl["n"]
    c = counter if counter is not None else Counter()
    stage = _Stage(counter)
    if tangents:
        tk = constant_tangents(params)
        K = {k: DNum(v, tk[k], c) for k, v in constants(params).items()}
        wrap = lambda v: DNum.const(v, 6, c)
    elif counter is not None:
        K = {k: Num(v, counter) for k, v in constants(params).items()}
        wrap = lambda v: Num(v, counter)
    else:
        K = constants(params)
        wrap = lambda v: float(v)
    X = [[wrap(x) for x in row] for row in pos]
    E = None
    F = [[0.0, 0.0, 0.0] for _ in range(N)]
    W = [0.0] * 6
    for i in range(N):
        e0, e1 = int(off[i]), int(off[i + 1])
        m = e1 - e0
        T = ns[e0:e1].astype(np.float64) @ H                 # image shifts n.H of the bonds
        stage("geometry_bond")
        dvec = [[(X[int(js[e0 + e])][a] - X[i][a]) + float(T[e][a]) for a in range(3)] for e in range(m)]
        r, u, fc, fcp, cos = geometry_terms(dvec, R1, R2, stage)
        Ui, P = site_terms(r, u, fc, fcp, cos, K, stage)
        E = _acc(E, Ui)
        virial_terms(r, u, P, W, stage)
        # force gather F_i = sum_j (dU_i/dd_ij - dU_j/dd_ji): each bond's term added to i, taken from j
        stage("bond")
        for e in range(m):
            j = int(js[e0 + e])
            for a in range(3):
                F[i][a] = F[i][a] + P[e][a]
                F[j][a] = F[j][a] - P[e][a]
        stage("atom")
    res = None
    if F_target is not None:
        for i in range(N):
            res = _acc(res, residual_terms(F[i], [float(x) for x in F_target[i]], stage))

    def val(x):
        if isinstance(x, DNum):
            return (x.v, np.array(x.d))
        if isinstance(x, Num):
            return x.v
        return (float(x), np.zeros(6)) if tangents else float(x)
    return (val(E), [[val(x) for x in row] for row in F] if tangents else np.array([[val(x) for x in row] for row in F]),
            [val(x) for x in W] if tangents else np.array([val(x) for x in W]),
            None if res is None else val(res))


def count_atom(m, seed=0, tangents=False, geometry=False, inner=False):
    """FLOP and XU ops of one atom with m bonds: the listing's site terms, its virial terms, the force
    gather of its bonds (each bond's derivative added to the atom and taken from the neighbour) and its
    force residual; with geometry=True also its bond geometry from the bond vectors (as the MD-scale
    call does every step), and with tangents=True in forward-mode dual arithmetic carrying the six
    parameter tangents (the plain method of the parameter gradient). Synthetic geometry with every bond
    in the switching region (R1 < r < R2), so no f_C or f_C' term vanishes; inner=True puts every bond
    inside R1 instead (f_C = 1, f_C' = 0 need no evaluation: the case of the MD-scale cells)."""
    rng = np.random.default_rng(seed)
    cnt = Counter()
    stage = _Stage(cnt)
    x = [1.0, 1.5, 2.3, 0.1, 0.7, -0.3]
    if tangents:
        tk = constant_tangents(x)
        K = {k: DNum(v, tk[k], cnt) for k, v in constants(x).items()}
        wrap = lambda v: DNum.const(v, 6, cnt)
    else:
        K = {k: Num(v, cnt) for k, v in constants(x).items()}
        wrap = lambda v: Num(v, cnt)
    uu = rng.normal(size=(m, 3))
    uu /= np.linalg.norm(uu, axis=1, keepdims=True)
    rr = rng.uniform(2.2, 2.6, m) if inner else rng.uniform(R1_DEFAULT, R2_DEFAULT, m)
    if geometry:
        xi = [wrap(v) for v in rng.normal(size=3)]
        xj = [[wrap(v) for v in row] for row in rng.normal(size=(m, 3))]
        T = (np.array([[v.v for v in row] for row in xj]) - np.array([v.v for v in xi])) * -1.0 + uu * rr[:, None]
        stage("geometry_bond")
        dvec = [[(xj[e][a] - xi[a]) + float(T[e][a]) for a in range(3)] for e in range(m)]
        r, u, fc, fcp, cos = geometry_terms(dvec, R1_DEFAULT, R2_DEFAULT, stage)
    else:
        r = [wrap(v) for v in rr]
        u = [[wrap(v) for v in row] for row in uu]
        fc = [wrap(0.5) for _ in range(m)]
        fcp = [wrap(-1.0) for _ in range(m)]
        cos = [[wrap(float(uu[a] @ uu[b])) if a != b else None for b in range(m)] for a in range(m)]
    _, P = site_terms(r, u, fc, fcp, cos, K, stage)
    W = [0.0] * 6
    virial_terms(r, u, P, W, stage)
    stage("bond")
    Fi = [0.0, 0.0, 0.0]
    Fj = [[0.0, 0.0, 0.0] for _ in range(m)]
    for e in range(m):
        for a in range(3):
            Fi[a] = Fi[a] + P[e][a]
            Fj[e][a] = Fj[e][a] - P[e][a]
    residual_terms([Fi[a] for a in range(3)], [0.5, 0.5, 0.5], stage)
    return sum(cnt.flop.values()), sum(cnt.xu.values())


def count_per_unit(tangents=False, geometry=False, inner=False):
    """The counts as FLOP(atom with m bonds) = per_bond m + per_triplet m (m - 1) + per_atom and
    XU = xu_per_bond m, found exactly from the counts of atoms with m = 2 .. 6 bonds (every count is
    checked against the fitted form). The sums of the site energies and of the force residuals over a
    configuration's atoms add 2 FLOP per atom less 2 per configuration in plain arithmetic (each sum
    starts at its first term); they are included in per_atom and per_config (in dual arithmetic each of
    those additions also carries the six tangents)."""
    counts = {m: count_atom(m, tangents=tangents, geometry=geometry, inner=inner) for m in range(2, 7)}
    f2, f3, f4 = counts[2][0], counts[3][0], counts[4][0]
    c = ((f4 - f3) - (f3 - f2)) / 2.0          # second difference of a m + c m (m - 1) is 2 c
    a = (f3 - f2) - c * (3 * 2 - 2 * 1)
    d = f2 - a * 2 - c * 2
    x2, x3 = counts[2][1], counts[3][1]
    xu_b = x3 - x2
    for m, (f, x) in counts.items():
        if f != a * m + c * m * (m - 1) + d or x != xu_b * m + (x2 - 2 * xu_b):
            raise AssertionError(f"count of m = {m} ({f}, {x}) does not follow the fitted form")
    add = 1 + 6 if tangents else 1
    return {"per_bond": a, "per_triplet": c, "per_atom": d + 2 * add, "per_config": -2 * add,
            "xu_per_bond": xu_b, "xu_per_atom": x2 - 2 * xu_b}
