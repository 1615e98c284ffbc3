"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (no GPU).

Each test targets a plausible mistake: a dropped 1/2 in U_i (Eq. 2), a wrong exponent on the bond
order (Eq. 6), a sign of h (Eq. 10), a wrong A/B/lambda/mu conversion (Eq. 11-14), a wrong cutoff
(Eq. 9), a wrong virial sign or component order, a wrong neighbour/image set.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar

import oracle
from oracle import tersoff as T
from paper_1909_11474_gb300 import inputs as I

P2 = I.TABLE2_PARAMS
EV_A3_GPA = 160.21766208  # 1 eV/A^3 in GPa


def morse_parts(r, p=P2):
    """Closed form of Eq. 4-5 with Eq. 11-14 at S = 2: f_R = D0 x^2, f_A = 2 D0 x, x = e^{-alpha (r - r0)}."""
    D0, al, r0 = p[0], p[1], p[2]
    x = math.exp(-al * (r - r0))
    return D0 * x * x, 2.0 * D0 * x, x


def bond_order(zeta, p=P2):
    n = p[4]
    return 1.0 if zeta == 0 else (1.0 + zeta ** n) ** (-1.0 / (2.0 * n))


def diamond_closed_form(a, p=P2):
    """Perfect diamond: 4 neighbours at r = a sqrt(3)/4, all angles cos = -1/3."""
    D0, al, r0, be, n, h = p
    z0 = 3.0 * be * (-1.0 / 3.0 - h) ** 2
    b0 = bond_order(z0, p)
    r = a * math.sqrt(3.0) / 4.0
    fR, fA, x = morse_parts(r, p)
    E_atom = 2.0 * (fR - b0 * fA)                      # U_i = 1/2 * 4 * (f_R - b0 f_A)
    W_diag_atom = 4.0 / 3.0 * D0 * al * r * x * (x - b0)   # -(1/3) r dU_i/dr
    return E_atom, W_diag_atom, b0


# ------------------------------------------------------------------------------------------------
# Closed forms and the paper's printed values
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("reps", [(1, 1, 1), (2, 2, 2), (1, 2, 3)])
@pytest.mark.parametrize("a", [5.2, 5.431, 5.6])
def test_perfect_diamond_closed_form(reps, a):
    pos, box = I.diamond_supercell(reps, a)
    N = len(pos)
    r = oracle.evaluate(pos, box, P2)
    E_atom, W_atom, _ = diamond_closed_form(a)
    assert r["E"] / N == pytest.approx(E_atom, rel=1e-12, abs=1e-12)
    assert np.allclose(r["W"][:3] / N, W_atom, rtol=1e-10, atol=1e-12)
    assert np.allclose(r["W"][3:], 0.0, atol=1e-10)
    assert np.abs(r["F"]).max() < 1e-10
    # summand magnitude of Eq. 1-3: 4 bonds x 1/2 (f_R + b0 f_A) per atom
    _, _, b0 = diamond_closed_form(a)
    fR, fA, _ = morse_parts(a * math.sqrt(3.0) / 4.0)
    assert r["E_scale"] / N == pytest.approx(2.0 * (fR + b0 * fA), rel=1e-12)


def test_perfect_diamond_equilibrium_and_paper_values(golden):
    """Sec. III.C prints E_c = -4.63 eV/atom and a = 5.434 A for the Table 2 parameters."""
    D0, al, r0, be, n, h = P2
    _, _, b0 = diamond_closed_form(5.431)
    a_star = 4.0 * (r0 - math.log(b0) / al) / math.sqrt(3.0)   # x = b0 minimises 2D0(x^2 - 2 b0 x)
    E_star = -2.0 * D0 * b0 * b0
    res = minimize_scalar(lambda a: oracle.evaluate(*I.diamond_supercell((1, 1, 1), a), P2)["E"] / 8.0,
                          bracket=(5.40, 5.43, 5.46), tol=1e-12)
    assert res.x == pytest.approx(a_star, abs=2e-6)
    assert res.fun == pytest.approx(E_star, abs=1e-10)
    assert abs(res.x - golden["lattice_constant"]) <= 1e-3
    assert abs(res.fun - golden["cohesive_energy"]) <= 5e-3
    r = oracle.evaluate(*I.diamond_supercell((2, 2, 2), a_star), P2)
    assert np.abs(r["W"]).max() < 1e-9 and np.abs(r["F"]).max() < 1e-10


def _strained_cell(a, eps, u=np.zeros(3)):
    pos, box = I.diamond_supercell((1, 1, 1), a)
    pos = pos.copy()
    pos[4:] += u            # rigid shift of the second fcc sublattice (internal relaxation)
    return I.apply_strain(pos, box, eps)


def test_elastic_constants_table3(golden):
    """Table 3 (mini-Tersoff): C11 = 148, C12 = 65, C44 = 75 GPa from zero-temperature stress-strain.

    Stress is -W/V from the oracle's virial; C44 lets the internal sublattice coordinate relax.
    """
    a0 = minimize_scalar(lambda a: oracle.evaluate(*I.diamond_supercell((1, 1, 1), a), P2)["E"],
                         bracket=(5.40, 5.43, 5.46), tol=1e-12).x
    V = a0 ** 3
    e = 1e-4

    def W3(eps, relax=False):
        u = np.zeros(3)
        if relax:
            def fg(uu):
                r = oracle.evaluate(*_strained_cell(a0, eps, uu), P2)
                return r["E"], -r["F"][4:].sum(axis=0)
            u = minimize(fg, np.zeros(3), jac=True, method="BFGS", options={"gtol": 1e-12}).x
        return oracle.evaluate(*_strained_cell(a0, eps, u), P2)["W3"]

    ex = np.zeros((3, 3)); ex[0, 0] = e
    Wp, Wm = W3(ex), W3(-ex)
    C11 = -(Wp[0, 0] - Wm[0, 0]) / (2 * e) / V * EV_A3_GPA
    C12 = -(Wp[1, 1] - Wm[1, 1]) / (2 * e) / V * EV_A3_GPA
    sh = np.zeros((3, 3)); sh[1, 2] = sh[2, 1] = e / 2      # engineering shear gamma_yz = e
    Wp, Wm = W3(sh, relax=True), W3(-sh, relax=True)
    C44 = -(Wp[1, 2] - Wm[1, 2]) / (2 * e) / V * EV_A3_GPA
    assert abs(C11 - golden["C11"]) < 1.0
    assert abs(C12 - golden["C12"]) < 1.0
    assert abs(C44 - golden["C44"]) < 1.0


def _cluster(points, L=40.0):
    pos = np.asarray(points, dtype=np.float64) + L / 2
    return pos, np.eye(3) * L


@pytest.mark.parametrize("r", [2.0, 2.23801, 2.5, 2.8, 2.9, 3.0, 3.15, 3.2, 3.3])
def test_dimer_is_morse(r, golden):
    """Two atoms: zeta = 0 so b = 1 (Eq. 6), and U = f_C(r) D0 (x^2 - 2x): the Morse pair."""
    pos, box = _cluster([[0, 0, 0], [r, 0, 0]])
    out = oracle.evaluate(pos, box, P2)
    fR, fA, x = morse_parts(r)
    R1, R2 = golden["R1"], golden["R2"]
    if r <= R1:
        fc = 1.0
    elif r >= R2:
        fc = 0.0
    else:
        fc = 0.5 * (1 + math.cos(math.pi * (r - R1) / (R2 - R1)))
    assert out["E"] == pytest.approx(fc * (fR - golden["b_at_zeta0"] * fA), rel=1e-13, abs=1e-14)
    if abs(r - 3.0) < 1e-12:
        assert fc == pytest.approx(0.5)                     # midpoint of the switch
    if abs(r - P2[2]) < 1e-12:
        assert out["E"] == pytest.approx(-P2[0], rel=1e-14)  # Morse minimum -D0 at r0
        assert np.abs(out["F"]).max() < 1e-12


@pytest.mark.parametrize("theta_deg", [90.0, 100.0, 109.4712206, 120.0, 150.0, 180.0])
def test_single_triplet_angular_function(theta_deg):
    """Atom i with bonds to j and k (r = 2.3 A < R1, |jk| > R2): U = 2 f_R - (1 + b_ij(theta)) f_A,
    b_ij = (1 + (beta (cos theta - h)^2)^n)^(-1/2n) and b_ji = b_ki = 1."""
    th = math.radians(theta_deg)
    rr = 2.3
    pts = [[0, 0, 0], [rr, 0, 0], [rr * math.cos(th), rr * math.sin(th), 0]]
    pos, box = _cluster(pts)
    out = oracle.evaluate(pos, box, P2)
    D0, al, r0, be, n, h = P2
    g = be * (math.cos(th) - h) ** 2
    b = bond_order(g)
    fR, fA, _ = morse_parts(rr)
    assert out["E"] == pytest.approx(2 * fR - (1 + b) * fA, rel=1e-13)


# ------------------------------------------------------------------------------------------------
# Brute force on tiny cells (independent neighbour search, loops, Morse form of Eq. 11-14)
# ------------------------------------------------------------------------------------------------

def brute_force_energy(pos, box, p, R1=2.8, R2=3.2, nimg=3):
    D0, al, r0, be, n, h = p
    N = len(pos)

    def fc(r):
        if r <= R1:
            return 1.0
        if r >= R2:
            return 0.0
        return 0.5 * (1 + math.cos(math.pi * (r - R1) / (R2 - R1)))

    nb = []
    for i in range(N):
        lst = []
        for j in range(N):
            for a in range(-nimg, nimg + 1):
                for b in range(-nimg, nimg + 1):
                    for c in range(-nimg, nimg + 1):
                        if i == j and a == b == c == 0:
                            continue
                        d = pos[j] - pos[i] + a * box[0] + b * box[1] + c * box[2]
                        r = math.sqrt(float(d @ d))
                        if r < R2:
                            lst.append((d, r))
        nb.append(lst)
    U = 0.0
    for i in range(N):
        for jj, (dj, rj) in enumerate(nb[i]):
            zeta = 0.0
            for kk, (dk, rk) in enumerate(nb[i]):
                if kk == jj:
                    continue
                cos = float(dj @ dk) / (rj * rk)
                zeta += fc(rk) * be * (cos - h) ** 2
            bij = 1.0 if zeta == 0 else (1 + zeta ** n) ** (-1 / (2 * n))
            x = math.exp(-al * (rj - r0))
            U += 0.5 * fc(rj) * (D0 * x * x - bij * 2 * D0 * x)
    return U


@pytest.mark.parametrize("case", ["cell8", "cell16_strained", "small_box_images"])
def test_brute_force_triple_loop(case):
    rng = np.random.default_rng(7)
    if case == "cell8":
        pos, box = I.diamond_supercell((1, 1, 1))
        pos = pos + rng.normal(0, 0.12, pos.shape)
    elif case == "cell16_strained":
        pos, box = I.diamond_supercell((1, 1, 2))
        pos, box = I.apply_strain(pos, box, I.random_strain(rng, 0.04))
        pos = pos + rng.normal(0, 0.15, pos.shape)
    else:
        # 8-atom cell compressed so that R2 exceeds half the box: several images of one j
        pos, box = I.diamond_supercell((1, 1, 1), a=4.6)
        pos = pos + rng.normal(0, 0.05, pos.shape)
    ref = brute_force_energy(pos, box, P2)
    assert oracle.evaluate(pos, box, P2)["E"] == pytest.approx(ref, rel=1e-12)


# ------------------------------------------------------------------------------------------------
# Forces and virial against finite differences, invariances
# ------------------------------------------------------------------------------------------------

def _rand_cell(seed=3, reps=(1, 1, 1), sigma=0.15, strain=0.03, a=5.431):
    rng = np.random.default_rng(seed)
    pos, box = I.diamond_supercell(reps, a)
    pos, box = I.apply_strain(pos, box, I.random_strain(rng, strain))
    return pos + rng.normal(0, sigma, pos.shape), box


def test_forces_central_differences():
    pos, box = _rand_cell()
    out = oracle.evaluate(pos, box, P2)
    hstep = 1e-5
    for i in range(len(pos)):
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, c] += hstep
            pm[i, c] -= hstep
            fd = -(oracle.evaluate(pp, box, P2)["E"] - oracle.evaluate(pm, box, P2)["E"]) / (2 * hstep)
            assert out["F"][i, c] == pytest.approx(fd, abs=2e-7)
    assert np.abs(out["F"].sum(axis=0)).max() < 1e-12


def test_virial_finite_strain():
    pos, box = _rand_cell(seed=5)
    out = oracle.evaluate(pos, box, P2)
    hstep = 1e-6
    W = np.zeros((3, 3))
    for m in range(3):
        for v in range(3):
            e = np.zeros((3, 3)); e[m, v] = hstep
            Ep = oracle.evaluate(*I.apply_strain(pos, box, e), P2)["E"]
            Em = oracle.evaluate(*I.apply_strain(pos, box, -e), P2)["E"]
            W[m, v] = -(Ep - Em) / (2 * hstep)
    assert np.allclose(out["W3"], W, atol=2e-6)
    assert np.allclose(out["W3"], out["W3"].T, atol=1e-10)
    order = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0)]
    assert np.allclose(out["W"], [W[a, b] for a, b in order], atol=2e-6)


def test_cluster_virial_equals_sum_r_outer_f():
    """Non-periodic cluster: -dU/d eps_mu,nu = sum_i F_i,mu x_i,nu (position vs strain gradients)."""
    rng = np.random.default_rng(11)
    pos, _ = I.diamond_supercell((1, 1, 1))
    pos, box = _cluster(pos + rng.normal(0, 0.1, pos.shape) - 2.7)
    out = oracle.evaluate(pos, box, P2)
    W = np.einsum("im,in->mn", out["F"], pos)
    assert np.allclose(out["W3"], W, atol=1e-10)


def test_translation_rotation_permutation():
    pos, box = _rand_cell(seed=9, reps=(1, 1, 2))
    ref = oracle.evaluate(pos, box, P2)
    t = oracle.evaluate(pos + np.array([0.37, -1.2, 2.9]), box, P2)
    assert t["E"] == pytest.approx(ref["E"], rel=1e-12)
    assert np.allclose(t["F"], ref["F"], atol=1e-10)
    ang = 0.7
    Rz = np.array([[math.cos(ang), -math.sin(ang), 0], [math.sin(ang), math.cos(ang), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(0.3), -math.sin(0.3)], [0, math.sin(0.3), math.cos(0.3)]])
    R = Rz @ Rx
    rot = oracle.evaluate(pos @ R.T, box @ R.T, P2)
    assert rot["E"] == pytest.approx(ref["E"], rel=1e-12)
    assert np.allclose(rot["F"], ref["F"] @ R.T, atol=1e-10)
    assert np.allclose(rot["W3"], R @ ref["W3"] @ R.T, atol=1e-9)
    perm = np.random.default_rng(1).permutation(len(pos))
    pr = oracle.evaluate(pos[perm], box, P2)
    assert pr["E"] == pytest.approx(ref["E"], rel=1e-12)
    assert np.allclose(pr["F"], ref["F"][perm], atol=1e-10)


# ------------------------------------------------------------------------------------------------
# Neighbour list
# ------------------------------------------------------------------------------------------------

def _loop_neighbours(pos, box, R2, nimg=4):
    out = []
    for i in range(len(pos)):
        for j in range(len(pos)):
            for a in range(-nimg, nimg + 1):
                for b in range(-nimg, nimg + 1):
                    for c in range(-nimg, nimg + 1):
                        if i == j and a == b == c == 0:
                            continue
                        d = pos[j] - pos[i] + (a * box[0] + b * box[1] + c * box[2])
                        if float(d @ d) < R2 * R2:
                            out.append((i, j, a, b, c))
    return sorted(out)


@pytest.mark.parametrize("case", ["perfect8", "displaced16", "tiny_sc", "compressed8"])
def test_neighbor_list_exhaustive_and_symmetric(case):
    rng = np.random.default_rng(2)
    if case == "perfect8":
        pos, box = I.diamond_supercell((1, 1, 1))
    elif case == "displaced16":
        pos, box = _rand_cell(seed=4, reps=(2, 1, 1), sigma=0.2)
    elif case == "tiny_sc":
        pos, box = np.array([[0.1, 0.2, 0.3]]), np.eye(3) * 2.5   # only self-images are neighbours
    else:
        pos, box = I.diamond_supercell((1, 1, 1), a=4.6)
        pos = pos + rng.normal(0, 0.05, pos.shape)
    nl = oracle.neighbor_list(pos, box, 3.2)
    got = sorted((i, int(nl["j"][e]), *map(int, nl["n"][e]))
                 for i in range(len(pos)) for e in range(nl["off"][i], nl["off"][i + 1]))
    assert got == _loop_neighbours(pos, box, 3.2)
    S = set(got)
    for (i, j, a, b, c) in got:
        assert (j, i, -a, -b, -c) in S
    for i in range(len(pos)):   # canonical ascending order inside each atom's list
        e = range(nl["off"][i], nl["off"][i + 1])
        keys = [(int(nl["j"][k]), *map(int, nl["n"][k])) for k in e]
        assert keys == sorted(keys)
    if case == "perfect8":
        assert (np.diff(nl["off"]) == 4).all()
    if case == "tiny_sc":
        assert np.diff(nl["off"])[0] == 6 and set(nl["j"]) == {0}


def test_single_cell_workload_has_no_pair_in_switch_region():
    """Sec. II.B: the training structures put no pair between R1 and R2; the seeded 64-atom cell
    (sigma = 0.05 A) shares that property, so R1/R2 readings cannot change its results."""
    w = I.workload_single_cell()
    pos, box = w["configs"].config(0)
    nl = oracle.neighbor_list(pos, box, 3.3)
    d = (pos[nl["j"]] - pos[np.repeat(np.arange(len(pos)), np.diff(nl["off"]))]) + nl["n"] @ box
    r = np.sqrt((d * d).sum(axis=1))
    assert not ((r > 2.8) & (r < 3.2)).any()


# ------------------------------------------------------------------------------------------------
# Fitness (Eq. 15-19) and gradient
# ------------------------------------------------------------------------------------------------

def _small_set(C=3, seed=21):
    rng = np.random.default_rng(seed)
    return I.make_cells(rng, C, lambda: (1, 1, 1), lambda: I.random_strain(rng, 0.02),
                        lambda: 0.1, lambda: 0)


def test_fitness_zero_and_unit_cases():
    cs = _small_set()
    E, W, F = oracle.evaluate_batch(cs, P2[None, :])
    N = cs.natoms
    exact = {"E": E[0] / N, "W": W[0] / N[:, None], "F": F[0], "mask": np.full(cs.C, 7, np.uint8)}
    f0 = oracle.fitness(cs, P2[None, :], exact)
    assert f0["Z"][0] == pytest.approx(0.0, abs=1e-14)
    half = {"E": E[0] / N / 2, "W": W[0] / N[:, None] / 2, "F": F[0] / 2, "mask": exact["mask"]}
    f1 = oracle.fitness(cs, P2[None, :], half, w=(0.5, 0.25, 2.0))
    assert np.allclose(f1["Zq"][0], [1.0, 1.0, 1.0], rtol=1e-12)   # residual equals target
    assert f1["Z"][0] == pytest.approx(2.75, rel=1e-12)


def test_fitness_hand_computed_and_masks():
    cs = _small_set(C=2)
    E = np.array([[-36.0, -32.0]])
    W = np.array([[[1, 2, 3, 4, 5, 6], [0, 0, 0, 0, 0, 8.0]]])
    F = np.zeros((1, cs.Ntot, 3)); F[0, 0, 0] = 3.0
    tgt = {"E": np.array([-4.0, -4.5]), "W": np.zeros((2, 6)), "F": np.zeros((cs.Ntot, 3)),
           "mask": np.array([7, 1], np.uint8)}
    tgt["W"][0, 0] = 1.0
    tgt["F"][0, 0] = 1.0
    out = oracle.fitness_from_predictions(cs, tgt, E, W, F)
    # E per atom: -4.5, -4.0 -> residuals -0.5, 0.5; D_e = 16 + 20.25
    assert out["Zq"][0, 0] == pytest.approx(math.sqrt(0.5 / 36.25))
    # W only from config 0 (mask bit 2): residual W/8 - tgt
    rw = np.array([1, 2, 3, 4, 5, 6]) / 8.0 - np.array([1, 0, 0, 0, 0, 0])
    assert out["Zq"][0, 1] == pytest.approx(math.sqrt(float(rw @ rw) / 1.0))
    # F only config 0: residual (2, 0, 0) on atom 0; D_f = 1
    assert out["Zq"][0, 2] == pytest.approx(2.0)
    bad = oracle.fitness_from_predictions(cs, tgt, E * np.nan, W, F)
    assert math.isinf(bad["Z"][0])


@pytest.mark.parametrize("loss", ["sq", "z"])
def test_parameter_gradient_central_differences(loss):
    cs = _small_set(C=2, seed=33)
    E, W, F = oracle.evaluate_batch(cs, P2[None, :])
    N = cs.natoms
    rng = np.random.default_rng(4)
    tgt = {"E": E[0] / N + rng.normal(0, 0.01, cs.C), "W": W[0] / N[:, None] + rng.normal(0, 0.02, (cs.C, 6)),
           "F": F[0] + rng.normal(0, 0.05, F[0].shape), "mask": np.array([7, 5], np.uint8)}
    x = P2 * np.array([1.05, 0.97, 1.01, 1.1, 0.9, 1.05])
    L, g = oracle.loss_and_grad(cs, x, tgt, w=(1.0, 0.5, 2.0), loss=loss)
    for q in range(6):
        hq = 1e-6 * max(1.0, abs(x[q]))
        xp, xm = x.copy(), x.copy()
        xp[q] += hq
        xm[q] -= hq
        Lp, _ = oracle.loss_and_grad(cs, xp, tgt, w=(1.0, 0.5, 2.0), loss=loss)
        Lm, _ = oracle.loss_and_grad(cs, xm, tgt, w=(1.0, 0.5, 2.0), loss=loss)
        assert g[q] == pytest.approx((Lp - Lm) / (2 * hq), rel=2e-6, abs=1e-9)
    # the loss itself agrees with the fitness routine
    fz = oracle.fitness(cs, x[None, :], tgt, w=(1.0, 0.5, 2.0))
    assert L == pytest.approx(fz["L"][0] if loss == "sq" else fz["Z"][0], rel=1e-12)


def test_neighbor_subset_matches_full_list():
    """The large-cell neighbour helper equals the exhaustive list where its spacing condition holds."""
    pos, box = _rand_cell(seed=12, reps=(3, 3, 2), sigma=0.2, strain=0.03)
    full = oracle.neighbor_list(pos, box, 3.2)
    atoms = [0, 5, 17, 40, 71, len(pos) - 1]
    sub = oracle.neighbor_list_subset(pos, box, 3.2, atoms)
    for i, (j, n) in zip(atoms, sub):
        e = slice(full["off"][i], full["off"][i + 1])
        assert np.array_equal(j, full["j"][e]) and np.array_equal(n, full["n"][e])


def test_force_term_scale_dimer_and_triangle_inequality():
    """The per-atom conditioning scale of the force bar, S_F,i = sum of |dU/dd| over the bonds from and to
    atom i: for a dimer (zeta = 0, the two bond terms opposite and equal) it equals |F_i|; in any cell
    it bounds |F_i| from above (triangle inequality), with equality nowhere guaranteed."""
    x = I.TABLE2_PARAMS
    pos = np.array([[0.0, 0.0, 0.0], [2.45, 0.0, 0.0]])
    r = oracle.evaluate(pos, np.eye(3) * 20.0, x)
    assert np.allclose(r["F_scale"], np.linalg.norm(r["F"], axis=1), rtol=1e-13, atol=0.0)
    rng = np.random.default_rng(21)
    p, b = I.diamond_supercell((1, 1, 1))
    r = oracle.evaluate(p + rng.normal(0.0, 0.15, p.shape), b, x)
    assert (r["F_scale"] >= np.linalg.norm(r["F"], axis=1) - 1e-12).all()
    assert (r["F_scale"] > 1.5 * np.linalg.norm(r["F"], axis=1)).any()
