"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

None of these checks re-types the oracle's formulas: the optimum comes from
an independent KKT enumeration, the m = 1 case from a sort-based Euclidean
simplex projection, gaps from vertex enumeration with finite-difference
gradients, objective values from closed forms, step sizes from a grid search
of the objective, gradients from central finite differences.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2103_05857_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Independent references
# ----------------------------------------------------------------------------
def kkt_bruteforce(C, a, b, rho):
    """Optimal value and column sums of min <C,T> + rho/2 ||T^T 1 - b||^2 over
    {T >= 0, T 1 = a} by enumerating supports and solving the KKT system
    C_ij + rho (s_j - b_j) = mu_i on the support, row sums = a_i, then
    checking T >= 0 and dual feasibility off the support."""
    m, n = C.shape
    cells = [(i, j) for i in range(m) for j in range(n)]
    best = []
    row_sets = [list(s) for k in range(1, n + 1) for s in itertools.combinations(range(n), k)]
    for choice in itertools.product(row_sets, repeat=m):
        P = [(i, j) for i in range(m) for j in choice[i]]
        nv = len(P) + m
        A = np.zeros((nv, nv))
        rhs = np.zeros(nv)
        col = {c: k for k, c in enumerate(P)}
        for e, (i, j) in enumerate(P):
            # C_ij + rho * (sum_k T_kj - b_j) - mu_i = 0
            for (k2, j2), v in col.items():
                if j2 == j:
                    A[e, v] += rho
            A[e, len(P) + i] = -1.0
            rhs[e] = -C[i, j] + rho * b[j]
        for i in range(m):
            e = len(P) + i
            for j in choice[i]:
                A[e, col[(i, j)]] = 1.0
            rhs[e] = a[i]
        sol, *_ = np.linalg.lstsq(A, rhs, rcond=None)
        if np.max(np.abs(A @ sol - rhs)) > 1e-11:
            continue
        T = np.zeros((m, n))
        for (i, j), v in col.items():
            T[i, j] = sol[v]
        if T.min() < -1e-13:
            continue
        mu = sol[len(P):]
        s = T.sum(0)
        G = C + rho * (s - b)[None, :]
        if np.any(G < mu[:, None] - 1e-11):
            continue
        T = np.maximum(T, 0.0)
        f = float((C * T).sum() + 0.5 * rho * ((T.sum(0) - b) ** 2).sum())
        best.append((f, s, T))
    assert best, "no KKT point found"
    fs = np.array([x[0] for x in best])
    assert fs.max() - fs.min() <= 1e-12 * max(1.0, abs(fs.min())), "KKT values disagree"
    return best[0]


def project_simplex(v, z):
    """Euclidean projection of v onto {t >= 0, sum t = z} (sort-based; Held,
    Wolfe & Crowder 1974; Duchi et al. 2008)."""
    u = np.sort(v)[::-1]
    css = np.cumsum(u) - z
    k = np.arange(1, len(v) + 1)
    cond = u - css / k > 0
    r = k[cond][-1]
    theta = css[cond][-1] / r
    return np.maximum(v - theta, 0.0)


def random_problem(seed, m, n, rho):
    rng = np.random.default_rng(seed)
    X = rng.random((m, 3))
    Y = rng.random((n, 3))
    a = rng.random(m) + 0.2
    a /= a.sum()
    b = rng.random(n) + 0.2
    b /= b.sum()
    return X, Y, a, b, rho


def random_plan(rng, a, n, sparse=False):
    m = len(a)
    T = rng.random((m, n))
    if sparse:
        T *= rng.random((m, n)) < 0.5
        T[np.arange(m), rng.integers(0, n, m)] += 0.1
    return T / T.sum(1, keepdims=True) * a[:, None]


# ----------------------------------------------------------------------------
# Random numbers
# ----------------------------------------------------------------------------
def test_splitmix64_known_answers(oracle_mod):
    # First outputs of splitmix64 seeded with 0 (Steele, Lea & Flood 2014;
    # the reference generator's published test vector).
    assert oracle_mod.draw(0, 0, 0) == 0xE220A8397B1DCDAF
    assert oracle_mod.draw(0, 0, 1) == 0x6E789E6AA1B965F4
    assert oracle_mod.draw(0, 0, 2) == 0x06C45D188009454F
    # The input generator implements the same published generator.
    u = W._u64(0, 0, 3)
    assert [int(x) for x in u] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_permutation_is_uniform_permutation(oracle_mod):
    m = 37
    seen = set()
    for ep in range(50):
        p = oracle_mod.permutation(12345, ep, m)
        assert sorted(p.tolist()) == list(range(m))
        seen.add(tuple(p.tolist()))
    assert len(seen) == 50
    # position of element 0 should be roughly uniform over many epochs
    pos = np.array([int(np.where(oracle_mod.permutation(7, ep, 8) == 0)[0][0]) for ep in range(4000)])
    counts = np.bincount(pos, minlength=8)
    assert counts.min() > 400 and counts.max() < 600


# ----------------------------------------------------------------------------
# Cost and objective
# ----------------------------------------------------------------------------
def test_cost_closed_form(oracle_mod):
    X = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    Y = np.array([[1.0, 1.0, 1.0], [0.0, 0.0, 0.0], [0.5, 0.5, 0.0]])
    C = oracle_mod.cost(X, Y)
    np.testing.assert_array_equal(C, [[3.0, 0.0, 0.5], [2.25, 0.25, 0.25]])
    np.testing.assert_allclose(oracle_mod.cost(X, Y, squared=False), np.sqrt(C), rtol=0, atol=0)


def test_objective_closed_forms(oracle_mod):
    X, Y, a, b, rho = random_problem(3, 4, 5, 7.0)
    C = oracle_mod.cost(X, Y)
    # product plan a b^T has column sums b: the penalty vanishes, f = a^T C b
    cert = oracle_mod.certificate(C, a, b, rho, np.outer(a, b))
    assert abs(cert["f"] - a @ C @ b) <= 1e-15
    assert abs(cert["pen"]) <= 1e-30
    # zero cost, all mass on column 0: f = rho/2 ((1 - b_0)^2 + sum_{j>0} b_j^2)
    T0 = np.zeros((4, 5))
    T0[:, 0] = a
    cert = oracle_mod.certificate(np.zeros((4, 5)), a, b, rho, T0)
    ref = 0.5 * rho * ((1 - b[0]) ** 2 + (b[1:] ** 2).sum())
    assert abs(cert["f"] - ref) <= 1e-15
    # f is quadratic with curvature rho ||D^T 1||^2 along any direction D
    rng = np.random.default_rng(1)
    T = random_plan(rng, a, 5)
    D = rng.standard_normal((4, 5))
    h = 1e-3
    fp = oracle_mod.certificate(C, a, b, rho, T + h * D)["f"]
    f0 = oracle_mod.certificate(C, a, b, rho, T)["f"]
    fm = oracle_mod.certificate(C, a, b, rho, T - h * D)["f"]
    assert abs((fp - 2 * f0 + fm) / h**2 - rho * (D.sum(0) ** 2).sum()) < 1e-6


def fd_grad(oracle_mod, C, a, b, rho, T, h=1e-6):
    G = np.zeros_like(T)
    for idx in np.ndindex(*T.shape):
        E = np.zeros_like(T)
        E[idx] = h
        G[idx] = (oracle_mod.certificate(C, a, b, rho, T + E)["f"]
                  - oracle_mod.certificate(C, a, b, rho, T - E)["f"]) / (2 * h)
    return G


@pytest.mark.parametrize("seed,m,n", [(0, 2, 3), (1, 3, 3), (2, 3, 2), (3, 1, 4)])
def test_gap_is_max_over_vertices(oracle_mod, seed, m, n):
    """g(T) = max_{S in M} <T - S, grad f(T)> (Sec. 3.2, Thm 2): enumerate every
    vertex S of the product of simplices, with grad f by finite differences."""
    X, Y, a, b, rho = random_problem(seed, m, n, 5.0)
    C = oracle_mod.cost(X, Y)
    rng = np.random.default_rng(seed + 10)
    T = random_plan(rng, a, n)
    G = fd_grad(oracle_mod, C, a, b, rho, T)
    best = -np.inf
    for js in itertools.product(range(n), repeat=m):
        S = np.zeros((m, n))
        S[np.arange(m), js] = a
        best = max(best, float(((T - S) * G).sum()))
    cert = oracle_mod.certificate(C, a, b, rho, T)
    assert abs(cert["g"] - best) <= 1e-8
    assert cert["g"] >= 0
    # per-row gaps are the per-block maxima (eq. 11)
    for i in range(m):
        gi = max(float(((T[i] - a[i] * np.eye(n)[j]) * G[i]).sum()) for j in range(n))
        assert abs(cert["g_rows"][i] - gi) <= 1e-8


# ----------------------------------------------------------------------------
# Optimum: KKT brute force, closed forms
# ----------------------------------------------------------------------------
CASES = [(s, m, n, rho) for s, (m, n) in enumerate([(1, 2), (2, 2), (2, 3), (3, 2), (3, 3)])
         for rho in (0.7, 6.0, 40.0)]


@pytest.mark.parametrize("seed,m,n,rho", CASES)
def test_variants_reach_kkt_optimum(oracle_mod, seed, m, n, rho):
    X, Y, a, b, _ = random_problem(seed, m, n, rho)
    C = oracle_mod.cost(X, Y)
    fstar, sstar, Tstar = kkt_bruteforce(C, a, b, rho)
    o = oracle_mod
    for kw, tol_f, tol_s in [
        (dict(variant=o.BCPFW, step=o.ELS), 1e-12, 1e-8),
        (dict(variant=o.BCAFW, step=o.ELS), 1e-12, 1e-8),
        (dict(variant=o.BCPFW, step=o.ELS, order=o.UNIFORM, seed=5), 1e-12, 1e-8),
        (dict(variant=o.BCPFW, step=o.ELS, order=o.PERMUTE, seed=5), 1e-12, 1e-8),
        (dict(variant=o.BCPFW, step=o.ELS, order=o.GAP, seed=5), 1e-12, 1e-8),
        # plain FW directions are sublinear: bounded by 2m/(k+2m) (C_f + h_0)
        # of Thm 1 (the line search makes at least the decay rule's progress)
        (dict(variant=o.BCFW, step=o.ELS), 2 * m / (3000 * m + 2 * m) * (6 * rho + C.max()), 1.0),
        (dict(variant=o.BCFW, step=o.DEC, order=o.GAP, ga_global_only=1, seed=9),
         2 * m / (3000 * m + 2 * m) * (6 * rho + C.max()), 1.0),
        # full FW is sublinear: bound it by the deterministic rate 2 C_f/(k+2)
        (dict(variant=o.FW, step=o.ELS), 8 * rho / 3002, 1.0),
    ]:
        T, res, *_ = o.solve(C, a, b, rho=rho, max_epochs=3000, **kw)
        assert abs(res["f"] - fstar) <= tol_f * max(1.0, abs(fstar)), kw
        np.testing.assert_allclose(T.sum(0), sstar, atol=tol_s)
        np.testing.assert_allclose(T.sum(1), a, rtol=1e-12, atol=0)
        assert T.min() >= 0.0
        # weak duality: w(T) <= f* <= f(T), and f(T) - f* <= g(T)
        assert res["w"] <= fstar + 1e-12
        assert res["f"] - fstar <= res["g"] + 1e-12


@pytest.mark.parametrize("seed,n", [(0, 2), (1, 5), (2, 8)])
def test_single_row_is_simplex_projection(oracle_mod, seed, n):
    """m = 1: t* = Proj_{a_1 Delta_n}(b - c / rho) (completing the square)."""
    X, Y, a, b, rho = random_problem(seed, 1, n, 3.0)
    C = oracle_mod.cost(X, Y)
    tstar = project_simplex(b - C[0] / rho, a[0])
    T, res, *_ = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.BCPFW,
                                  step=oracle_mod.ELS, max_epochs=500)
    np.testing.assert_allclose(T[0], tstar, atol=1e-13)
    assert res["g"] <= 1e-15


def test_rho_zero_row_argmin(oracle_mod):
    """rho = 0: the problem separates into rows, T_ij = a_i [j = argmin_j C_ij];
    the line search reaches it in one epoch with zero gap."""
    inst = W.colour_instance(11, 40, 30, rho=0.0)
    C = oracle_mod.cost(inst.X, inst.Y)
    T, res, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=0.0, variant=oracle_mod.BCFW,
                                  step=oracle_mod.ELS, max_epochs=1)
    ref = np.zeros_like(C)
    ref[np.arange(40), C.argmin(1)] = inst.a
    np.testing.assert_array_equal(T, ref)
    assert res["g"] == 0.0
    assert abs(res["f"] - (inst.a * C.min(1)).sum()) <= 1e-15


def test_single_column(oracle_mod):
    """n = 1: the only feasible plan is T = a; gap zero."""
    X, Y, a, b, rho = random_problem(4, 5, 1, 2.0)
    C = oracle_mod.cost(X, Y)
    T, res, *_ = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.BCFW,
                                  step=oracle_mod.DEC, max_epochs=3)
    np.testing.assert_allclose(T[:, 0], a, rtol=4e-16, atol=0)
    assert abs(res["g"]) <= 1e-16
    assert abs(res["f"] - (C[:, 0] @ a + 0.5 * rho * (a.sum() - b[0]) ** 2)) <= 1e-15


# ----------------------------------------------------------------------------
# Steps
# ----------------------------------------------------------------------------
def _f_along(oracle_mod, C, a, b, rho, T, i, d, gam):
    T2 = T.copy()
    T2[i] = T[i] + gam * d
    return oracle_mod.certificate(C, a, b, rho, T2)["f"]


@pytest.mark.parametrize("variant", ["BCFW", "BCAFW", "BCPFW"])
def test_line_search_minimises_objective(oracle_mod, variant):
    """ELS (eq. 8, eq. 10) returns the minimiser of f along the chosen
    direction over [0, gamma_max]: compare with a grid of the objective."""
    o = oracle_mod
    X, Y, a, b, rho = random_problem(21, 4, 6, 9.0)
    C = o.cost(X, Y)
    rng = np.random.default_rng(5)
    checked = 0
    for trial in range(30):
        T = random_plan(rng, a, 6, sparse=True)
        r = T.sum(0) - b
        i = trial % 4
        T1, r1 = T.copy(), r.copy()
        js, v, dr, gam = o.block_step(C, a, T1, r1, i, 0, variant=getattr(o, variant),
                                      step=o.ELS, rho=rho)
        if gam == 0.0 and dr < 0:
            continue
        d = T1[i] - T[i]
        if np.abs(d).max() == 0:
            continue
        # direction of unit step length: recover from the reported gamma
        unit = d / gam
        if dr == 0:
            gmax = 1.0
            np.testing.assert_allclose(unit, a[i] * np.eye(6)[js] - T[i], atol=1e-12)
        elif dr == 1:
            alpha = T[i, v] / a[i]
            gmax = alpha / (1 - alpha)
            np.testing.assert_allclose(unit, T[i] - a[i] * np.eye(6)[v], atol=1e-9)
        else:
            gmax = T[i, v] / a[i]
            np.testing.assert_allclose(unit, a[i] * (np.eye(6)[js] - np.eye(6)[v]), atol=1e-9)
        grid = np.linspace(0, gmax, 2001)
        fs = [_f_along(o, C, a, b, rho, T, i, unit, g) for g in grid]
        fbest = min(fs)
        fgam = _f_along(o, C, a, b, rho, T, i, unit, gam)
        assert fgam <= fbest + 1e-15
        assert 0.0 <= gam <= gmax + 1e-15
        # the rank-1 update of the column sums matches the new plan
        np.testing.assert_allclose(r1, T1.sum(0) - b, atol=1e-15)
        checked += 1
    assert checked >= 10


def test_fw_direction_choice_and_drop_steps(oracle_mod):
    """BCAFW chooses the direction with the larger decrease rate (Alg. A.2) and
    a drop step zeroes the away atom exactly; BCPFW moves mass between two
    atoms only (Alg. A.3)."""
    o = oracle_mod
    X, Y, a, b, rho = random_problem(8, 3, 5, 50.0)
    C = o.cost(X, Y)
    rng = np.random.default_rng(3)
    saw_away = saw_drop = 0
    for trial in range(200):
        T = random_plan(rng, a, 5, sparse=True)
        r = T.sum(0) - b
        i = trial % 3
        G = C[i] + rho * r
        js = int(np.argmin(G))
        act = np.where(T[i] > 0)[0]
        v = int(act[np.argmax(G[act])])
        g_fw = T[i] @ G - a[i] * G[js]
        g_aw = a[i] * G[v] - T[i] @ G
        T1, r1 = T.copy(), r.copy()
        _, vv, dr, gam = o.block_step(C, a, T1, r1, i, 0, variant=o.BCAFW, step=o.ELS, rho=rho)
        assert vv == v
        expect_fw = len(act) == 1 or g_fw >= g_aw
        assert (dr == 0) == expect_fw
        if dr == 1:
            saw_away += 1
            alpha = T[i, v] / a[i]
            if gam >= alpha / (1 - alpha):
                saw_drop += 1
                assert T1[i, v] == 0.0
        T2, r2 = T.copy(), r.copy()
        _, _, dr2, gam2 = o.block_step(C, a, T2, r2, i, 0, variant=o.BCPFW, step=o.ELS, rho=rho)
        changed = np.where(T2[i] != T[i])[0]
        assert set(changed.tolist()) <= {js, v}
        np.testing.assert_allclose(T2[i].sum(), a[i], rtol=1e-15)
    assert saw_away > 5 and saw_drop > 0


def test_decay_rule_values(oracle_mod):
    """Decay rule 2m/(k+2m) for m blocks (Alg. 1): gamma_0 = 1, gamma_m = 2/3."""
    o = oracle_mod
    X, Y, a, b, rho = random_problem(2, 6, 4, 3.0)
    C = o.cost(X, Y)
    for k, ref in [(0, 1.0), (6, 2.0 / 3.0), (12, 0.5), (6 * 98, 0.02)]:
        T = np.outer(a, np.eye(4)[0])
        r = T.sum(0) - b
        _, _, _, gam = o.block_step(C, a, T, r, 1, k, variant=o.BCFW, step=o.DEC, rho=rho)
        assert abs(gam - ref) <= 1e-15
    with pytest.raises(ValueError):
        o.block_step(C, a, T, r, 1, 0, variant=o.BCPFW, step=o.DEC, rho=rho)


# ----------------------------------------------------------------------------
# Rates and duality
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed,m,n,rho", [(0, 2, 3, 5.0), (1, 3, 3, 20.0), (2, 3, 2, 1.0)])
def test_fw_decay_rate(oracle_mod, seed, m, n, rho):
    """FW with the 2/(k+2) rule: f(T_k) - f* <= 2 C_f / (k+2) with the
    curvature bound C_f <= 4/lambda = 4 rho (Thm 4 of App. B, restated)."""
    X, Y, a, b, _ = random_problem(seed, m, n, rho)
    C = oracle_mod.cost(X, Y)
    fstar = kkt_bruteforce(C, a, b, rho)[0]
    T, res, _, _, hist = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.FW,
                                          step=oracle_mod.DEC, max_epochs=300)
    for it, f, g in hist:
        if it >= 1:
            assert f - fstar <= 2 * 4 * rho / (it + 2) + 1e-12
        assert f - fstar <= g + 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bcfw_decay_rate_bound(oracle_mod, seed):
    """BCFW-U with the decay rule: f(T_k) - f* <= 2m/(k+2m) (C_f^x + h_0) with
    C_f^x <= 4 rho and h_0 = f(T_0) - f* (Thm 1); checked per run at epoch ends."""
    X, Y, a, b, rho = random_problem(seed + 40, 3, 3, 8.0)
    C = oracle_mod.cost(X, Y)
    fstar = kkt_bruteforce(C, a, b, rho)[0]
    T0 = np.zeros((3, 3))
    T0[:, 0] = a
    h0 = oracle_mod.certificate(C, a, b, rho, T0)["f"] - fstar
    # h_0 <= ||C||_inf + 2 rho (the h_0 bound of App. C, restated here)
    assert h0 <= C.max() + 2 * rho
    _, _, _, _, hist = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.BCFW,
                                        step=oracle_mod.DEC, order=oracle_mod.UNIFORM,
                                        seed=seed, max_epochs=400)
    m = 3
    for ep, f, g in hist:
        k = ep * m
        assert f - fstar <= 2 * m / (k + 2 * m) * (4 * rho + h0) + 1e-12


def test_weak_duality_along_trajectory(oracle_mod):
    """Weak duality (Thm 2, App. D): every dual value w(T_k) is below every
    primal value f(T_l), across iterates of different variants."""
    o = oracle_mod
    inst = W.colour_instance(5, 24, 20, rho=10.0)
    C = o.cost(inst.X, inst.Y)
    fs, ws = [], []
    for kw in [dict(variant=o.BCFW, step=o.DEC), dict(variant=o.BCPFW, step=o.ELS),
               dict(variant=o.BCAFW, step=o.ELS, order=o.UNIFORM, seed=2)]:
        T = None
        for ep in range(40):
            T, res, *_ = o.solve(C, inst.a, inst.b, T0=T, rho=10.0, max_epochs=1, **kw)
            fs.append(res["f"])
            ws.append(res["w"])
            assert res["g"] >= 0.0
            assert abs((res["f"] - res["w"]) - res["g"]) <= 1e-15
    assert max(ws) <= min(fs) + 1e-15
    # the bound is useful: after 40 epochs the best pair brackets f* within 2%
    assert min(fs) - max(ws) <= 2e-2 * min(fs)


# ----------------------------------------------------------------------------
# Gradients (envelope theorem)
# ----------------------------------------------------------------------------
def test_adjoint_matches_fd_at_fixed_plan(oracle_mod):
    """At a fixed plan, dX, dY, db are the exact gradients of
    <C(X, Y), T> + rho/2 ||T^T 1 - b||^2 (central differences of a quadratic)."""
    o = oracle_mod
    X, Y, a, b, rho = random_problem(6, 4, 5, 3.0)
    rng = np.random.default_rng(2)
    T = random_plan(rng, a, 5)
    dX, dY, db = o.adjoint(X, Y, b, rho, T)

    def phi(X_, Y_, b_):
        return o.certificate(o.cost(X_, Y_), a, b_, rho, T)["f"]

    h = 1e-5
    for (i, k) in [(0, 0), (1, 2), (3, 1)]:
        E = np.zeros_like(X)
        E[i, k] = h
        assert abs((phi(X + E, Y, b) - phi(X - E, Y, b)) / (2 * h) - dX[i, k]) < 1e-9
    for (j, k) in [(0, 1), (4, 2)]:
        E = np.zeros_like(Y)
        E[j, k] = h
        assert abs((phi(X, Y + E, b) - phi(X, Y - E, b)) / (2 * h) - dY[j, k]) < 1e-9
    for j in [0, 3]:
        E = np.zeros_like(b)
        E[j] = h
        assert abs((phi(X, Y, b + E) - phi(X, Y, b - E)) / (2 * h) - db[j]) < 1e-9


def test_envelope_gradient_of_optimal_value(oracle_mod):
    """d f*/dX (re-solving at X +- h) equals dX at the optimal plan."""
    o = oracle_mod
    X, Y, a, b, rho = random_problem(7, 5, 4, 6.0)

    def fstar(X_, Y_, b_):
        C = o.cost(X_, Y_)
        _, res, *_ = o.solve(C, a, b_, rho=rho, variant=o.BCPFW, step=o.ELS, max_epochs=4000)
        assert res["g"] <= 1e-13
        return res["f"]

    C = o.cost(X, Y)
    T, res, *_ = o.solve(C, a, b, rho=rho, variant=o.BCPFW, step=o.ELS, max_epochs=4000)
    dX, dY, db = o.adjoint(X, Y, b, rho, T)
    h = 1e-5
    for (i, k) in [(0, 0), (2, 1), (4, 2)]:
        E = np.zeros_like(X)
        E[i, k] = h
        fd = (fstar(X + E, Y, b) - fstar(X - E, Y, b)) / (2 * h)
        assert abs(fd - dX[i, k]) <= 1e-6 * max(1.0, abs(dX[i, k]))
    for j in [1, 3]:
        E = np.zeros_like(b)
        E[j] = h
        fd = (fstar(X, Y, b + E) - fstar(X, Y, b - E)) / (2 * h)
        assert abs(fd - db[j]) <= 1e-6


# ----------------------------------------------------------------------------
# Paper fixtures
# ----------------------------------------------------------------------------
def test_paper_printed_iterates_are_feasible():
    """The 3x3 plans printed in Figs. 5 and 6 (BCFW-P-DEC on the three-colour
    images) keep the exact marginal b_paper = (0.6, 0.3, 0.1) on their columns;
    in this library's orientation (rows are the blocks) their transposes have
    row sums close to (0.6, 0.3, 0.1). The printed values are rounded to three
    decimals and some column sums are off by up to 0.01, so the check is loose; one
    printed matrix is garbled and is listed separately in the fixture."""
    with open(os.path.join(GOLDEN, "paper_fig5_fig6_iterates.json")) as fh:
        fx = json.load(fh)
    target = np.array(fx["b_paper"])
    for it in fx["iterates"]:
        Tb = np.array(it["T_paper"]).T  # build orientation
        np.testing.assert_allclose(Tb.sum(1), target, atol=0.011, err_msg=it["where"])
        assert Tb.min() >= 0


def test_gap_adaptive_sampling_support(oracle_mod):
    """Alg. A.4 draws block i with probability proportional to max(g_i, 0):
    rows of zero weight (g_i = 0 at every feasible T) are never drawn, and
    every row with a positive gap is drawn within a few epochs."""
    X, Y, a, b, rho = random_problem(11, 12, 9, 5.0)
    a = a.copy()
    a[::3] = 0.0
    a /= a.sum()
    C = oracle_mod.cost(X, Y)
    _, _, ti, _, _ = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.BCFW, step=oracle_mod.ELS,
                                      order=oracle_mod.GAP, seed=3, max_epochs=6, trace=True)
    drawn = set(ti.tolist())
    assert not drawn & set(range(0, 12, 3))
    assert drawn == {i for i in range(12) if i % 3}


def _chi2_pvalue(counts, probs):
    from scipy.stats import chi2
    counts = np.asarray(counts, dtype=np.float64)
    exp = counts.sum() * np.asarray(probs, dtype=np.float64)
    keep = exp > 0
    stat = float((((counts - exp) ** 2)[keep] / exp[keep]).sum())
    return float(chi2.sf(stat, int(keep.sum()) - 1))


def test_gap_adaptive_sampling_frequencies(oracle_mod):
    """Alg. A.4 samples block i with probability g_i / sum_k g_k over the
    clamped gaps max(g_i, 0). 10^5 draws of the sampling step, fed with
    64-bit uniforms from numpy's own generator, match those probabilities by
    a chi-square test; entries with zero or negative gap are never drawn; and
    the same counts reject the plausible mistakes (weights g_i^2, or uniform
    over the rows with a positive gap)."""
    g = np.array([0.5, 0.0, -0.2, 1.0, 2.5, 0.0, 0.3, 1e-3, 0.7, -1e-9, 0.05])
    rng = np.random.default_rng(2024)
    draws = rng.integers(0, 2**64, size=100_000, dtype=np.uint64)
    counts = np.zeros(len(g), dtype=np.int64)
    for u in draws.tolist():
        counts[oracle_mod.sample_from(g, u)] += 1
    gp = np.maximum(g, 0.0)
    assert counts[gp == 0].sum() == 0
    assert _chi2_pvalue(counts, gp / gp.sum()) > 1e-4
    assert _chi2_pvalue(counts, gp ** 2 / (gp ** 2).sum()) < 1e-12
    pos = (gp > 0).astype(float)
    assert _chi2_pvalue(counts, pos / pos.sum()) < 1e-12


def test_gap_adaptive_sampling_interval_boundaries(oracle_mod):
    """Inverse-transform sampling gives block i the half-open interval
    [cum_{i-1}, cum_i) of u * total, so each block's probability is exactly
    its weight's share: a draw landing on cum_i belongs to the next block of
    positive weight, u = 0 to the first, the largest u to the last; with all
    gaps zero the draw falls back to a uniform index."""
    g = np.array([1.0, 1.0, 0.0, 2.0])  # total 4: cum = 1, 2, 2, 4
    u = lambda x: int(x * 2**64)  # x a multiple of 2^-53 is represented exactly
    assert oracle_mod.sample_from(g, 0) == 0
    assert oracle_mod.sample_from(g, u(0.25) - 2048) == 0   # u just below 1/4
    assert oracle_mod.sample_from(g, u(0.25)) == 1          # target 1.0 = cum_0
    assert oracle_mod.sample_from(g, u(0.5) - 2048) == 1
    assert oracle_mod.sample_from(g, u(0.5)) == 3           # target 2.0: block 2 has no weight
    assert oracle_mod.sample_from(g, 2**64 - 1) == 3
    assert oracle_mod.sample_from(np.array([0.0, 0.0, 3.0]), 0) == 2
    z = np.zeros(5)
    assert [oracle_mod.sample_from(z, -(-(k * 2**64) // 5)) for k in range(5)] == [0, 1, 2, 3, 4]


def test_uniform_order_draws(oracle_mod):
    """The uniform block order (Sec. 3.1) picks floor(u m): the index is the
    j with u in [j 2^64 / m, (j+1) 2^64 / m), checked at both ends of every
    interval for m = 10 and 7; the block frequencies of a uniform-order run
    (m = 7, 21,000 updates) pass a chi-square test against 1/m."""
    for m in (10, 7):
        for j in range(m):
            lo = -(-(j * 2**64) // m)          # smallest u with floor(u m / 2^64) = j
            hi = -(-((j + 1) * 2**64) // m) - 1
            assert oracle_mod.uniform_index(lo, m) == j
            assert oracle_mod.uniform_index(hi, m) == j
    X, Y, a, b, rho = random_problem(3, 7, 4, 2.0)
    C = oracle_mod.cost(X, Y)
    _, _, ti, _, _ = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.BCFW, step=oracle_mod.DEC,
                                      order=oracle_mod.UNIFORM, seed=77, max_epochs=3000, trace=True)
    counts = np.bincount(ti, minlength=7)
    assert _chi2_pvalue(counts, np.full(7, 1 / 7)) > 1e-4


def _gap_rows(oracle_mod, C, a, b, rho, T):
    return oracle_mod.certificate(C, a, b, rho, T)["g_rows"]


def test_gap_adaptive_global_update_cadence(oracle_mod):
    """Alg. A.4 with inner updates (GAD-M, M = 3): the sampling gaps are all
    recomputed after epochs 3 and 6 (and once at the start), and only then.
    At those epochs every stored g_i equals the gap of row i at the epoch's
    plan (the certificate, Thm 2); at the others, rows not drawn in the epoch
    keep their previous value bit for bit, and the row drawn last holds its
    gap after its own update (the post-update reading of the inner update).
    The first draw of every epoch is the sampling step applied to the gaps
    stored at the end of the epoch before."""
    X, Y, a, b, rho = random_problem(21, 16, 12, 4.0)
    C = oracle_mod.cost(X, Y)
    m, M, E, seed = 16, 3, 7, 5
    _, res, ti, _, _ = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.BCFW, step=oracle_mod.ELS,
                                        order=oracle_mod.GAP, ga_M=M, seed=seed, max_epochs=E, trace=True,
                                        epoch_state=True)
    gh, Th = res["ga_hist"], res["T_hist"]
    T0 = np.zeros((m, 12))
    T0[:, 0] = a
    prev = _gap_rows(oracle_mod, C, a, b, rho, T0)  # the exact update at k = 0
    for e in range(E):
        cert = _gap_rows(oracle_mod, C, a, b, rho, Th[e])
        drawn = ti[e * m:(e + 1) * m]
        assert drawn[0] == oracle_mod.sample_from(prev, oracle_mod.draw(seed, 3, e * m))
        if (e + 1) % M == 0:
            np.testing.assert_allclose(gh[e], cert, rtol=1e-10, atol=1e-15)
        else:
            rest = np.setdiff1d(np.arange(m), drawn)
            assert len(rest) > 0
            np.testing.assert_array_equal(gh[e][rest], prev[rest])
            last = drawn[-1]
            assert abs(gh[e][last] - cert[last]) <= 1e-10 * abs(cert[last]) + 1e-13 * np.abs(cert).max()
            assert np.abs(gh[e] - cert).max() > 1e-9 * np.abs(cert).max()  # not a global update
        prev = gh[e]


def test_gap_adaptive_global_only_cadence(oracle_mod):
    """BCFW-GAS (global updates only): the sampling gaps are recomputed after
    every epoch and frozen within it, so every draw of epoch e is the
    sampling step applied to the certificate's row gaps at the end of epoch
    e - 1 (at T0 for the first epoch)."""
    X, Y, a, b, rho = random_problem(22, 14, 10, 3.0)
    C = oracle_mod.cost(X, Y)
    m, E, seed = 14, 5, 9
    _, res, ti, _, _ = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.BCFW, step=oracle_mod.ELS,
                                        order=oracle_mod.GAP, ga_global_only=1, ga_M=4, seed=seed,
                                        max_epochs=E, trace=True, epoch_state=True)
    gh, Th = res["ga_hist"], res["T_hist"]
    T0 = np.zeros((m, 10))
    T0[:, 0] = a
    prev = _gap_rows(oracle_mod, C, a, b, rho, T0)
    for e in range(E):
        for k in range(e * m, (e + 1) * m):
            assert ti[k] == oracle_mod.sample_from(prev, oracle_mod.draw(seed, 3, k))
        np.testing.assert_allclose(gh[e], _gap_rows(oracle_mod, C, a, b, rho, Th[e]), rtol=1e-10, atol=1e-15)
        prev = gh[e]


def test_apply_step_reproduces_block_steps(oracle_mod):
    """Applying a block step's own decision to a copy of the state gives the
    state that the block step produced, bit for bit, for every direction
    (Frank-Wolfe, away with and without a drop, pairwise)."""
    X, Y, a, b, rho = random_problem(31, 9, 11, 6.0)
    C = oracle_mod.cost(X, Y)
    rng = np.random.default_rng(0)
    seen = set()
    for variant in (oracle_mod.BCFW, oracle_mod.BCAFW, oracle_mod.BCPFW):
        T = random_plan(rng, a, 11, sparse=True)
        r = T.sum(0) - b
        for k in range(60):
            i = k % 9
            T2, r2 = T.copy(), r.copy()
            js, v, dr, gam = oracle_mod.block_step(C, a, T, r, i, k, variant=variant,
                                                   step=oracle_mod.ELS, rho=rho)
            oracle_mod.apply_step(a, T2, r2, i, dr, js, v, gam)
            np.testing.assert_array_equal(T2, T)
            np.testing.assert_array_equal(r2, r)
            seen.add(dr)
    assert seen >= {0, 1, 2}


# ----------------------------------------------------------------------------
# Colour-transfer tail (Sec. 5.1 projection, Sec. 5 metrics iii and iv)
# ----------------------------------------------------------------------------
def test_barycentric_is_the_weighted_least_squares_point(oracle_mod):
    """The projection minimises sum_j T_ij ||x - y_j||^2: its gradient vanishes
    there and every perturbation raises the objective."""
    rng = np.random.default_rng(5)
    m, n, d = 6, 9, 3
    Y = rng.random((n, d))
    T = rng.random((m, n)) * (rng.random((m, n)) < 0.6)
    T[0] = 0.0  # a row with no mass
    T[1] = 0.0
    T[1, 4] = 0.37  # all its mass on one column
    Xh = oracle_mod.barycentric(Y, T)
    assert np.all(Xh[0] == 0.0)
    np.testing.assert_allclose(Xh[1], Y[4], rtol=0, atol=1e-15)

    def obj(i, x):
        return float(sum(T[i, j] * np.sum((x - Y[j]) ** 2) for j in range(n)))
    for i in range(2, m):
        grad = sum(2.0 * T[i, j] * (Xh[i] - Y[j]) for j in range(n))
        assert np.abs(grad).max() <= 1e-12
        for _ in range(20):
            dx = rng.normal(size=d) * 1e-3
            assert obj(i, Xh[i] + dx) > obj(i, Xh[i])


def test_transfer_stats_special_plans(oracle_mod):
    """e_c vanishes for a plan that meets both marginals (the product plan a
    b^T); for the initial plan of Thm 1 (all mass in column 0) only the column
    term remains and equals ||e_0 - b||; sparsity counts zero cells."""
    rng = np.random.default_rng(6)
    m, n = 7, 5
    a = rng.random(m); a /= a.sum()
    b = rng.random(n); b /= b.sum()
    s = oracle_mod.transfer_stats(a, b, np.outer(a, b))
    assert s["e_c"] <= 1e-15 and s["sparsity"] == 0.0
    T0 = np.zeros((m, n)); T0[:, 0] = a
    s0 = oracle_mod.transfer_stats(a, b, T0)
    e0 = np.zeros(n); e0[0] = 1.0
    assert s0["row_err"] <= 1e-15
    assert abs(s0["col_err"] - np.sqrt(((e0 - b) ** 2).sum())) <= 1e-15
    assert abs(s0["e_c"] - s0["col_err"]) <= 1e-15
    zeros = sum(1 for i in range(m) for j in range(n) if T0[i, j] == 0.0)
    assert s0["sparsity"] == zeros / (m * n) == (n - 1) / n


def test_euclidean_cost_pins(oracle_mod):
    """The paper's cost ||x_i - y_j||_2 (Sec. 5.1): equal to numpy's vector
    norm cell by cell, its square is the squared cost, it is a metric
    (symmetric, zero on the diagonal of a cloud with itself, triangle
    inequality through any third point), and a 3-4-5 pair gives 5."""
    rng = np.random.default_rng(12)
    X, Y, Z = rng.random((9, 4)), rng.random((7, 4)), rng.random((5, 4))
    E = oracle_mod.cost(X, Y, squared=False)
    for i in range(9):
        for j in range(7):
            assert abs(E[i, j] - np.linalg.norm(X[i] - Y[j])) <= 1e-15
    np.testing.assert_allclose(E ** 2, oracle_mod.cost(X, Y), rtol=1e-14, atol=0)
    XX = oracle_mod.cost(X, X, squared=False)
    assert np.all(np.diag(XX) == 0.0) and np.array_equal(XX, XX.T)
    XZ, ZY = oracle_mod.cost(X, Z, squared=False), oracle_mod.cost(Z, Y, squared=False)
    for k in range(5):
        assert np.all(E <= XZ[:, k:k + 1] + ZY[k:k + 1, :] + 1e-15)
    P = oracle_mod.cost(np.array([[0.0, 0.0, 0.0]]), np.array([[3.0, 4.0, 0.0]]), squared=False)
    assert P[0, 0] == 5.0


# ----------------------------------------------------------------------------
# Reference plan of the LP-based metrics (Sec. 5, metrics v and vi)
# ----------------------------------------------------------------------------
def _lp_vertices(C, a, b):
    """Brute force over the vertices of the transportation polytope: every
    set of m + n - 1 cells whose equality system (row sums a, column sums b)
    has a unique nonnegative solution is a basic feasible solution; return
    the cheapest one and its cost."""
    m, n = C.shape
    cells = [(i, j) for i in range(m) for j in range(n)]
    best, best_T = np.inf, None
    for basis in itertools.combinations(range(m * n), m + n - 1):
        A = np.zeros((m + n, m + n - 1))
        for k, cidx in enumerate(basis):
            i, j = cells[cidx]
            A[i, k] = 1.0
            A[m + j, k] = 1.0
        if np.linalg.matrix_rank(A) < m + n - 1:
            continue
        x, *_ = np.linalg.lstsq(A, np.concatenate([a, b]), rcond=None)
        if np.abs(A @ x - np.concatenate([a, b])).max() > 1e-12 or x.min() < -1e-13:
            continue
        T = np.zeros((m, n))
        for k, cidx in enumerate(basis):
            T[cells[cidx]] = x[k]
        v = float((T * C).sum())
        if v < best - 1e-14:
            best, best_T = v, T
    return best, best_T


@pytest.mark.parametrize("seed,m,n", [(1, 2, 3), (2, 3, 3), (3, 3, 2), (4, 1, 4)])
def test_transport_lp_is_the_cheapest_vertex(oracle_mod, seed, m, n):
    """T*_LP is the cheapest vertex of the transportation polytope
    (enumerated by brute force on tiny sizes) and is feasible."""
    rng = np.random.default_rng(seed)
    C = rng.random((m, n))
    a = rng.random(m) + 0.1
    a /= a.sum()
    b = rng.random(n) + 0.1
    b /= b.sum()
    L = oracle_mod.transport_lp(C, a, b)
    v, Tv = _lp_vertices(C, a, b)
    assert abs(float((L * C).sum()) - v) <= 1e-12
    np.testing.assert_allclose(L, Tv, atol=1e-12)
    np.testing.assert_allclose(L.sum(1), a, atol=1e-12)
    np.testing.assert_allclose(L.sum(0), b, atol=1e-12)
    assert L.min() >= 0.0


def test_transport_lp_dual_certificate(oracle_mod):
    """Optimality of T*_LP without the solver: potentials u, v solved from
    u_i + v_j = C_ij on its support (a spanning tree of cells for a
    non-degenerate problem) are dual feasible, u_i + v_j <= C_ij everywhere,
    and <a, u> + <b, v> = <C, T*_LP> (LP duality)."""
    rng = np.random.default_rng(9)
    m, n = 7, 9
    C = rng.random((m, n))
    a = rng.random(m) + 0.1
    a /= a.sum()
    b = rng.random(n) + 0.1
    b /= b.sum()
    L = oracle_mod.transport_lp(C, a, b)
    supp = np.argwhere(L > 1e-14)
    assert len(supp) == m + n - 1  # non-degenerate basis
    A = np.zeros((len(supp) + 1, m + n))
    rhs = np.zeros(len(supp) + 1)
    for k, (i, j) in enumerate(supp):
        A[k, i] = 1.0
        A[k, m + j] = 1.0
        rhs[k] = C[i, j]
    A[-1, 0] = 1.0  # fix the free constant: u_0 = 0
    uv = np.linalg.solve(A, rhs)
    u, v = uv[:m], uv[m:]
    assert (u[:, None] + v[None, :] - C).max() <= 1e-12
    assert abs(a @ u + b @ v - float((L * C).sum())) <= 1e-12


def test_semi_relaxed_value_tends_to_the_lp_value(oracle_mod):
    """The semi-relaxed problem penalises the column marginal with weight
    rho / 2 (Sec. 3, eq. 5 with rho = 1/lambda): its optimal value increases
    with rho and approaches the LP value from below as rho grows, at rate
    O(1/rho)."""
    X, Y, a, b, _ = random_problem(5, 4, 5, 1.0)
    C = oracle_mod.cost(X, Y)
    lp = float((oracle_mod.transport_lp(C, a, b) * C).sum())
    vals = []
    for rho in (1.0, 10.0, 100.0, 1000.0):
        _, r, *_ = oracle_mod.solve(C, a, b, rho=rho, variant=oracle_mod.BCPFW, step=oracle_mod.ELS,
                                    max_epochs=200000, tol_rel_gap=1e-13, gap_every=10)
        vals.append(r["f"])
    assert all(x < y for x, y in zip(vals, vals[1:]))
    assert vals[-1] <= lp + 1e-12
    gaps = [lp - v for v in vals]
    assert gaps[-1] <= 1.5 * gaps[-2] / 10.0 and gaps[-1] >= 0.0


def test_lp_metrics_closed_forms(oracle_mod):
    """e_m and e_v of Sec. 5 on plans with known answers: the product plan
    (all entries 1/9) against the diagonal plan (1/3 on the diagonal) has
    ||T - L|| = sqrt(18)/9 and ||L|| = sqrt(3)/3, so e_m = sqrt(6)/3; with
    C = [[1,2,3],[2,1,2],[3,2,1]] the values are <L, C> = 1 and
    <T, C> = 17/9, so e_v = 8/9; a plan against itself gives 0."""
    L = np.eye(3) / 3.0
    T = np.full((3, 3), 1.0 / 9.0)
    C = np.array([[1.0, 2, 3], [2, 1, 2], [3, 2, 1]])
    r = oracle_mod.lp_metrics(C, T, L)
    assert abs(r["e_m"] - np.sqrt(6.0) / 3.0) <= 1e-15
    assert abs(r["e_v"] - 8.0 / 9.0) <= 1e-15
    r0 = oracle_mod.lp_metrics(C, L, L)
    assert r0["e_m"] == 0.0 and r0["e_v"] == 0.0

