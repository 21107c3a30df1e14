"""Parity of the single-instance CUDA path with the FP64 oracle.

Every GPU call goes through the C ABI (libsr_ot.so via ctypes). Tolerances:
FP64 decay-rule trajectories are compared bit for bit (argmin sequence and
plan); everything else uses objective <= 1e-5 relative and
max |T - T_oracle| <= 1e-6 on the same trajectory, as stated for this
library's parity targets.
"""
import numpy as np
import pytest
import torch

from paper_2103_05857_gb300 import workloads as W

from .gpu_util import dev, f32, host, rel

pytestmark = pytest.mark.gpu

OBJ_RTOL = 1e-5
T_ATOL = 1e-6


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_05857_gb300 import sr_ot
    return sr_ot


@pytest.fixture(scope="module")
def h(S):
    hd = S.Handle(0)
    yield hd
    hd.close()


def random_plan(rng, a, n, density=0.3):
    m = len(a)
    T = rng.random((m, n)) * (rng.random((m, n)) < density)
    T[np.arange(m), rng.integers(0, n, m)] += 0.5
    return T / T.sum(1, keepdims=True) * a[:, None]


# ---------------------------------------------------------------------------
# Certificate (Thm 2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,mode", [(37, 53, "pts"), (300, 517, "pts"), (300, 517, "C"),
                                      (1024, 1000, "pts"), (4096, 4096, "pts")])
def test_certificate_fp64(S, h, oracle_mod, m, n, mode):
    inst = W.colour_instance(7 + m, m, n, rho=10.0, b_dirichlet=True)
    rng = np.random.default_rng(m + n)
    T = random_plan(rng, inst.a, n)
    C = oracle_mod.cost(inst.X, inst.Y)
    ref = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, T)
    g_rows = torch.empty(m, dtype=torch.float64, device="cuda")
    kw = dict(C=dev(C, torch.float64)) if mode == "C" else dict(X=dev(inst.X, torch.float64),
                                                                 Y=dev(inst.Y, torch.float64))
    res = h.gap(dev(inst.a, torch.float64), dev(inst.b, torch.float64), dev(T, torch.float64),
                g_rows=g_rows, precision=S.FP64, rho=inst.rho, **kw)
    assert rel(res["objective"], ref["f"]) <= 1e-13
    assert abs(res["gap"] - ref["g"]) <= 1e-12 * ref["f"]
    assert abs(res["dual"] - ref["w"]) <= 1e-12 * ref["f"]
    np.testing.assert_allclose(host(g_rows), ref["g_rows"], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("m,n,mode", [(37, 53, "pts"), (300, 517, "pts"), (300, 517, "C"),
                                      (4096, 4096, "pts"), (4096, 4096, "C")])
def test_certificate_fp32(S, h, oracle_mod, m, n, mode):
    """FP32 plan and cost, FP64 accumulation: the oracle sees the same FP32
    values (plan, points or cost) promoted to double."""
    inst = W.colour_instance(11 + m, m, n, rho=10.0, b_dirichlet=True).rounded()
    rng = np.random.default_rng(m * 3 + n)
    T = f32(random_plan(rng, inst.a, n))
    if mode == "C":
        C = f32(oracle_mod.cost(inst.X, inst.Y))
        kw = dict(C=dev(C, torch.float32))
    else:
        C = oracle_mod.cost(inst.X, inst.Y)
        kw = dict(X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32))
    ref = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, T)
    g_rows = torch.empty(m, dtype=torch.float64, device="cuda")
    res = h.gap(dev(inst.a, torch.float32), dev(inst.b, torch.float32), dev(T, torch.float32),
                g_rows=g_rows, precision=S.FP32, rho=inst.rho, **kw)
    # C mode: FP32 products summed with compensation, so about FP64 accuracy;
    # points mode: the cost itself is evaluated in FP32 (one rounding per entry)
    ftol = 1e-9 if mode == "C" else 2e-7
    assert rel(res["objective"], ref["f"]) <= ftol
    assert abs(res["gap"] - ref["g"]) <= 2e-7 * ref["f"] + 1e-9 * abs(ref["g"])
    assert abs(res["dual"] - ref["w"]) <= 2e-7 * ref["f"] + 1e-9 * abs(ref["g"])
    np.testing.assert_allclose(host(g_rows), ref["g_rows"], rtol=1e-4, atol=1e-6 * ref["f"] / m)


# ---------------------------------------------------------------------------
# FP64 decay-rule trajectories are bit-identical to the oracle's
# ---------------------------------------------------------------------------
def _trace_buf(cap):
    return torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")


@pytest.mark.parametrize("order,epochs", [("CYCLIC", 200), ("PERMUTE", 25), ("UNIFORM", 25)])
def test_fp64_dec_trajectory_bit_identical(S, h, oracle_mod, order, epochs):
    """colour256_fp64: m = n = 256, rho = 10, BCFW-DEC; the argmin sequence and
    the plan match the oracle bit for bit."""
    inst = W.workload("colour256_fp64")
    m, n = inst.m, inst.n
    C = oracle_mod.cost(inst.X, inst.Y)
    seed = 20250101
    To, ro, ti, tj, _ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                         step=oracle_mod.DEC, order=getattr(oracle_mod, order),
                                         seed=seed, max_epochs=epochs, trace=True)
    cap = epochs * m
    tr = _trace_buf(cap)
    T = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    res = h.solve(dev(inst.a, torch.float64), dev(inst.b, torch.float64), T,
                  X=dev(inst.X, torch.float64), Y=dev(inst.Y, torch.float64),
                  precision=S.FP64, variant=S.BCFW, step=S.DEC, order=getattr(S, order), seed=seed,
                  rho=inst.rho, max_epochs=epochs, trace=tr, trace_capacity=cap)
    trh = tr.cpu().numpy().reshape(-1, 4)
    np.testing.assert_array_equal(trh[:, 0], ti)
    np.testing.assert_array_equal(trh[:, 1], tj)
    np.testing.assert_array_equal(host(T), To)
    assert res["block_updates"] == ro["updates"]
    assert rel(res["objective"], ro["f"]) <= 1e-13
    assert abs(res["gap"] - ro["g"]) <= 1e-12 * ro["f"]


@pytest.mark.parametrize("m,n,order,mode", [(50, 97, "CYCLIC", "pts"), (64, 1, "CYCLIC", "pts"),
                                             (33, 512, "UNIFORM", "pts"), (300, 65, "PERMUTE", "C"),
                                             (7, 2, "UNIFORM", "C"), (120, 130, "CYCLIC", "C")])
def test_fp64_dec_single_warp_kernel_edges(S, h, oracle_mod, m, n, order, mode):
    """FP64 BCFW rows of width <= 512 run on the single-warp kernel: odd
    widths (8-byte copies and padded columns), one column, the widest rows it
    takes, repeated rows in uniform order, given or point costs. The argmin
    sequence and the plan equal the oracle's bit for bit."""
    inst = W.colour_instance(m * 7 + n, m, n, rho=10.0, b_dirichlet=True)
    C = oracle_mod.cost(inst.X, inst.Y)
    ep, seed = 12, 4
    To, ro, ti, tj, _ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                         step=oracle_mod.DEC, order=getattr(oracle_mod, order), seed=seed,
                                         max_epochs=ep, trace=True)
    cap = ep * m
    tr = _trace_buf(cap)
    T = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    kw = dict(C=dev(C, torch.float64)) if mode == "C" else dict(X=dev(inst.X, torch.float64),
                                                                 Y=dev(inst.Y, torch.float64))
    res = h.solve(dev(inst.a, torch.float64), dev(inst.b, torch.float64), T, precision=S.FP64, variant=S.BCFW,
                  step=S.DEC, order=getattr(S, order), seed=seed, rho=inst.rho, max_epochs=ep, trace=tr,
                  trace_capacity=cap, **kw)
    trh = tr.cpu().numpy().reshape(-1, 4)
    np.testing.assert_array_equal(trh[:, 0], ti)
    np.testing.assert_array_equal(trh[:, 1], tj)
    np.testing.assert_array_equal(host(T), To)
    assert rel(res["objective"], ro["f"]) <= 1e-13


@pytest.mark.parametrize("order", ["CYCLIC", "UNIFORM"])
def test_fp64_line_search_single_warp_kernel(S, h, oracle_mod, order):
    """FP64 BCFW with the exact line search (eq. 8) on the single-warp
    kernel: the same trajectory as the oracle up to the order of the two dot
    products."""
    inst = W.colour_instance(15, 180, 300, rho=10.0, b_dirichlet=True)
    C = oracle_mod.cost(inst.X, inst.Y)
    ep = 15
    To, ro, _, tj, _ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                        step=oracle_mod.ELS, order=getattr(oracle_mod, order), seed=2,
                                        max_epochs=ep, trace=True)
    cap = ep * 180
    tr = _trace_buf(cap)
    T = torch.zeros((180, 300), dtype=torch.float64, device="cuda")
    res = h.solve(dev(inst.a, torch.float64), dev(inst.b, torch.float64), T, X=dev(inst.X, torch.float64),
                  Y=dev(inst.Y, torch.float64), precision=S.FP64, variant=S.BCFW, step=S.ELS,
                  order=getattr(S, order), seed=2, rho=inst.rho, max_epochs=ep, trace=tr, trace_capacity=cap)
    js = tr.cpu().numpy().reshape(-1, 4)[:, 1]
    assert rel(res["objective"], ro["f"]) <= 1e-10
    assert np.abs(host(T) - To).max() <= 1e-10
    assert (js != tj).mean() <= 0.01


@pytest.mark.parametrize("d,order", [(3, "CYCLIC"), (5, "PERMUTE")])
def test_fp64_euclidean_cost_trajectory_bit_identical(S, h, oracle_mod, d, order):
    """The paper's cost ||x_i - y_j||_2 (Sec. 5.1) from points: the argmin
    sequence and the plan of BCFW-DEC match the oracle run on the oracle's
    Euclidean cost bit for bit (the cost is built with the oracle's summation
    order and a correctly rounded square root)."""
    m, n = 120, 250
    rng = np.random.default_rng(d)
    X, Y = rng.random((m, d)), rng.random((n, d))
    a = W.dirichlet_weights(d, m)
    b = W.dirichlet_weights(d + 1, n)
    C = oracle_mod.cost(X, Y, squared=False)
    seed, epochs = 8, 6
    To, ro, ti, tj, _ = oracle_mod.solve(C, a, b, rho=5.0, variant=oracle_mod.BCFW, step=oracle_mod.DEC,
                                         order=getattr(oracle_mod, order), seed=seed, max_epochs=epochs,
                                         trace=True)
    cap = epochs * m
    tr = _trace_buf(cap)
    T = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    res = h.solve(dev(a, torch.float64), dev(b, torch.float64), T, X=dev(X, torch.float64),
                  Y=dev(Y, torch.float64), precision=S.FP64, variant=S.BCFW, step=S.DEC,
                  order=getattr(S, order), seed=seed, rho=5.0, max_epochs=epochs, trace=tr,
                  trace_capacity=cap, cost_kind=S.COST_EUCLIDEAN)
    trh = tr.cpu().numpy().reshape(-1, 4)
    np.testing.assert_array_equal(trh[:, 0], ti)
    np.testing.assert_array_equal(trh[:, 1], tj)
    np.testing.assert_array_equal(host(T), To)
    assert rel(res["objective"], ro["f"]) <= 1e-13
    # the certificate of the same plan under the Euclidean cost
    g = h.gap(dev(a, torch.float64), dev(b, torch.float64), T, X=dev(X, torch.float64), Y=dev(Y, torch.float64),
              precision=S.FP64, rho=5.0, cost_kind=S.COST_EUCLIDEAN)
    cert = oracle_mod.certificate(C, a, b, 5.0, To)
    assert rel(g["objective"], cert["f"]) <= 1e-13 and abs(g["gap"] - cert["g"]) <= 1e-12 * cert["f"]


def test_fp32_euclidean_cost_converges_to_oracle_optimum(S, h, oracle_mod):
    inst = W.colour_instance(41, 300, 400, rho=10.0, b_dirichlet=True).rounded()
    C = oracle_mod.cost(inst.X, inst.Y, squared=False)
    _, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCPFW, step=oracle_mod.ELS,
                                 max_epochs=50000, tol_rel_gap=1e-10, gap_every=5)
    T = torch.zeros((inst.m, inst.n), dtype=torch.float32, device="cuda")
    res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
                  Y=dev(inst.Y, torch.float32), precision=S.FP32, variant=S.BCPFW, step=S.ELS, rho=inst.rho,
                  max_epochs=20000, tol_rel_gap=1e-6, cost_kind=S.COST_EUCLIDEAN)
    assert res["status"] == S.OK, res
    assert ro["f"] - 1e-9 <= res["objective"] <= ro["f"] * (1 + 1.2e-6)


def test_euclidean_cost_rejected_where_unsupported(S, h):
    m, n = 8, 12
    X = torch.rand((m, 3), device="cuda")
    Y = torch.rand((n, 3), device="cuda")
    a = torch.full((m,), 1.0 / m, device="cuda")
    b = torch.full((n,), 1.0 / n, device="cuda")
    T = torch.zeros((m, n), device="cuda")
    o = S.options(precision=S.FP32, cost_kind=S.COST_EUCLIDEAN)
    dX = torch.empty((m, 3), device="cuda")
    assert S.lib.sr_ot_grad(h._h, o, m, n, 3, S._ptr(X), S._ptr(Y), None, S._ptr(b), S._ptr(T), None,
                            S._ptr(dX), None, None) == S.EUNSUPPORTED
    o2 = S.options(precision=S.FP32_BF16COST, cost_kind=S.COST_EUCLIDEAN)
    X64 = torch.rand((m, 64), device="cuda")
    Y64 = torch.rand((n, 64), device="cuda")
    res = S.Result()
    assert S.lib.sr_ot_solve(h._h, o2, m, n, 64, None, S._ptr(X64), S._ptr(Y64), S._ptr(a), S._ptr(b),
                             S._ptr(T), 0, res) == S.EUNSUPPORTED
    o3 = S.options(precision=S.FP32, cost_kind=7)
    assert S.lib.sr_ot_solve(h._h, o3, m, n, 3, None, S._ptr(X), S._ptr(Y), S._ptr(a), S._ptr(b),
                             S._ptr(T), 0, res) == S.EINVAL


def test_fp64_given_cost_matches_point_cost(S, h, oracle_mod):
    inst = W.colour_instance(3, 150, 333, rho=25.0)
    C = oracle_mod.cost(inst.X, inst.Y)
    To, ro, _, tj, _ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                        step=oracle_mod.DEC, max_epochs=30, trace=True)
    cap = 30 * 150
    tr = _trace_buf(cap)
    T = torch.zeros((150, 333), dtype=torch.float64, device="cuda")
    h.solve(dev(inst.a, torch.float64), dev(inst.b, torch.float64), T, C=dev(C, torch.float64),
            precision=S.FP64, rho=inst.rho, max_epochs=30, trace=tr, trace_capacity=cap)
    np.testing.assert_array_equal(tr.cpu().numpy().reshape(-1, 4)[:, 1], tj)
    np.testing.assert_array_equal(host(T), To)


# ---------------------------------------------------------------------------
# FP64 line-search variants: same trajectory up to rounding
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("variant", ["BCFW", "BCAFW", "BCPFW"])
@pytest.mark.parametrize("order", ["CYCLIC", "UNIFORM"])
def test_fp64_line_search_variants(S, h, oracle_mod, variant, order):
    """FP64 line search: the only difference from the oracle is the order of
    the two dot products in eq. 8 / eq. 10, so the runs agree to rounding."""
    inst = W.colour_instance(5, 200, 600, rho=10.0, b_dirichlet=True)
    C = oracle_mod.cost(inst.X, inst.Y)
    ep = 12
    To, ro, _, tj, _ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho,
                                        variant=getattr(oracle_mod, variant), step=oracle_mod.ELS,
                                        order=getattr(oracle_mod, order), seed=9, max_epochs=ep,
                                        trace=True)
    cap = ep * 200
    tr = _trace_buf(cap)
    T = torch.zeros((200, 600), dtype=torch.float64, device="cuda")
    res = h.solve(dev(inst.a, torch.float64), dev(inst.b, torch.float64), T,
                  X=dev(inst.X, torch.float64), Y=dev(inst.Y, torch.float64), precision=S.FP64,
                  variant=getattr(S, variant), step=S.ELS, order=getattr(S, order), seed=9,
                  rho=inst.rho, max_epochs=ep, trace=tr, trace_capacity=cap)
    js = tr.cpu().numpy().reshape(-1, 4)[:, 1]
    # same trajectory to rounding: the plans agree; a recorded LMO vertex may
    # differ only where the row is converged (zero step), i.e. at exact ties
    assert rel(res["objective"], ro["f"]) <= 1e-10
    assert np.abs(host(T) - To).max() <= 1e-10
    assert (js != tj).mean() <= 0.01


# ---------------------------------------------------------------------------
# Epoch replay: from one state, one GPU epoch against one oracle epoch
# ---------------------------------------------------------------------------
def _trace_rows(tr):
    """Per update (i, j*, v, gamma) from a device trace buffer (word 2 holds
    v in bits 0..28, all ones for none, and the direction above)."""
    t = tr.cpu().numpy().reshape(-1, 4)
    v = t[:, 2] & 0x1FFFFFFF
    v = np.where(v == 0x1FFFFFFF, -1, v)
    return t[:, 0], t[:, 1], v, t[:, 3].copy().view(np.float32).astype(np.float64)


def _trace_dirs(tr):
    """Per update the direction the GPU stepped in: 0 toward j*, 1 away from
    v, 2 pairwise, -1 no step."""
    d = (tr.cpu().numpy().reshape(-1, 4)[:, 2] >> 29) & 3
    return np.where(d == 3, -1, d)


def near_tie(C, a, T, r, i, rho, variant, tol_rel=2e-6):
    """Whether some discrete decision of the block update of row i at state
    (T, r) is within FP32 rounding of flipping: the LMO argmin (eq. 7), the
    away vertex, the FW-or-away choice (Alg. A.2), a step at the boundary of
    [0, gamma_max] (drop step or clip), or a row whose step is ~zero."""
    g = C[i] + rho * r
    tol = tol_rel * max(1.0, np.abs(g).max())
    ai, t = a[i], T[i]
    gs = np.sort(g)
    if len(g) > 1 and gs[1] - gs[0] <= tol:
        return "argmin"
    js = int(np.argmin(g))
    act = np.where(t > 0)[0]
    if len(act) >= 2:
        ga = np.sort(g[act])[::-1]
        if ga[0] - ga[1] <= tol:
            return "away vertex"
    dot = t @ g
    g_fw = dot - ai * g[js]
    if abs(g_fw) <= 4 * ai * tol:
        return "zero step"
    if variant == "BCFW" or variant == "BCAFW":
        d = -t.copy()
        d[js] += ai
        dd = d @ d
        if rho * dd > 0 and abs(g_fw / (rho * dd) - 1.0) <= 1e-4:
            return "clip at 1"
    if len(act) == 0:
        return None
    v = int(act[np.argmax(g[act])])
    if variant == "BCAFW":
        g_aw = ai * g[v] - dot
        if abs(g_fw - g_aw) <= 4 * ai * tol:
            return "FW or away"
        alpha = t[v] / ai
        if alpha < 1:
            d = t.copy()
            d[v] -= ai
            dd = d @ d
            gmax = alpha / (1 - alpha)
            if rho * dd > 0 and abs(g_aw / (rho * dd) - gmax) <= 1e-4 * max(gmax, 1e-12):
                return "drop"
    if variant == "BCPFW" and v != js:
        gam = (g[v] - g[js]) / (2 * rho * ai) if rho > 0 else np.inf
        gmax = t[v] / ai
        if abs(gam - gmax) <= 1e-4 * max(gmax, 1e-12) + tol / (2 * rho * ai):
            return "drop"
    return None


def _fw_away_gammas(C, a, T, r, i, rho, j, v):
    """Exact line-search steps (eq. 8) of row i toward vertex j (FW) and away
    from atom v, at state (T, r); None where the direction does not exist."""
    g = C[i] + rho * r
    t = T[i]
    ai = a[i]
    s2 = float(t @ t)
    tg = float(t @ g)
    out = [None, None]
    dd = (s2 - t[j] * t[j]) + (ai - t[j]) ** 2
    if dd > 0:
        out[0] = min(max((tg - ai * g[j]) / (rho * dd), 0.0), 1.0)
    if 0 <= v < len(t) and 0 < t[v] < ai:
        dd = (s2 - t[v] * t[v]) + (ai - t[v]) ** 2
        alpha = t[v] / ai
        if dd > 0:
            out[1] = min(max((ai * g[v] - tg) / (rho * dd), 0.0), alpha / (1.0 - alpha))
    return out


def _followed_gamma(direction, row, ai, v, gam_g):
    """The step the oracle applies when the GPU's gamma matched its own: the
    GPU's. A GPU gamma within 1e-6 of gamma_max is the drop step it was in
    FP32 (atom v removed); below that the GPU kept atom v with the mass its
    gamma leaves, whatever the oracle's own step would have done (a drop the
    GPU did not take leaves an atom of up to 1e-7 of mass that later
    decisions see)."""
    if direction in (1, 2) and 0 <= v < len(row) and 0 < row[v] < ai:
        alpha = row[v] / ai
        gmax = alpha if direction == 2 else alpha / (1.0 - alpha)
        if gam_g >= gmax * (1.0 - 1e-6):
            return gmax
    return gam_g


EPS32 = 2.0 ** -24   # unit roundoff of binary32
NEGLIGIBLE = 1e-6    # an atom lighter than this fraction of a_i is below what an FP32 step resolves


def fp32_step_allowance(C, a, T, r, i, rho, direction, js, v, gam):
    """How far an FP32 step size gamma may lie from the FP64 one for the same
    decision. gamma = num / (rho dd) (eq. 8 / eq. 10). The numerator is a
    difference of sums of O(|supp| + 2) terms of size t_ij |grad_ij|, each
    carrying a few FP32 roundings (cost, residual, product, sum); the
    curvature dd is a difference and sum of squares of the row's entries (for
    away and FW steps it cancels when one atom holds almost all the row's
    mass), and the dense kernel takes a_i - t_v from the stored mass of the
    other atoms, which also carries the row's drift from a_i. Each error is
    bounded by ~8 (|supp| + 4) eps32 times the magnitudes of its terms; gamma
    inherits the numerator's error over the curvature plus the curvature's
    relative error."""
    g = C[i] + rho * r
    t = T[i]
    ai = a[i]
    supp = np.nonzero(t > 0)[0]
    k = 8.0 * (len(supp) + 4) * EPS32
    if direction == 2:  # pairwise: numerator a_i (g_v - g_js), curvature 2 a_i^2
        dd = 2.0 * ai * ai
        num_mag = ai * (abs(g[v]) + abs(g[js]))
        err_dd = k * dd
    else:  # FW (towards js) or away (from v)
        x = js if direction == 0 else v
        tx = float(t[x])
        s2 = float(t @ t)
        oth = ai - tx
        dd = (s2 - tx * tx) + oth * oth
        num_mag = float(t @ np.abs(g)) + ai * abs(g[x])
        err_dd = k * (s2 + tx * tx + (ai + tx) ** 2)
        if direction == 1:
            drift = abs(float(t.sum()) - ai)
            err_dd += 2.0 * abs(oth) * (drift + k * ai)
    den = rho * dd
    if not den > 0 or err_dd >= dd:
        return np.inf  # the curvature is below FP32 resolution: gamma is not determined
    return k * num_mag / den + (err_dd / dd + k) * abs(gam)


def replay_epochs(S, h, O, inst, C, kw, variant, step, order, epochs, prec=None, seed=3,
                  dense_only=0, T0=None, max_tie_frac=0.05):
    """Run `epochs` epochs one at a time; before each, the oracle starts from
    the GPU's current plan. Within an epoch every GPU decision (block i, LMO
    vertex j*, away vertex v, step gamma; from the device trace) is compared
    with the oracle's block step at the same state, update by update:
      - the same vertices and gamma within 1e-7 + 1e-5 gamma (in units of
        a_i): the oracle continues from the GPU's gamma (a drop stays a drop),
        so that every later update is judged from the GPU's own state;
      - the same vertices and gamma within what FP32 resolves for this step
        (fp32_step_allowance: the line-search numerator cancels when the row
        is nearly converged, the away curvature when alpha_v is near 1) -- an
        "ill-conditioned step" (not a different decision, and not counted as
        one);
      - other vertices: the decision must be a near tie at the oracle's state
        (one FP32 cannot order, see near_tie), or the vertex that differs is an
        atom lighter than 1e-6 a_i on one side (a mass below FP32 resolution
        that one run holds and the other rounded away).
    In the last two cases the oracle adopts the GPU's decision for that update
    (its own update arithmetic applied to the GPU's j*, v and gamma; a step
    within FP32 rounding of gamma_max is taken as the drop it was, and atoms
    below FP32 resolution in the row are cleared first), and the comparison
    goes on with the next update, so no update of the epoch goes unchecked.
    Every epoch must end with the oracle's plan within 1e-6 of the GPU's and
    its objective within 1e-5. Adopted different decisions may not exceed
    `max_tie_frac` of the updates (at least 2). Returns the per-epoch numbers
    of adopted different decisions."""
    prec = S.FP32 if prec is None else prec
    dt = torch.float32 if prec != S.FP64 else torch.float64
    m, n = inst.m, inst.n
    if T0 is None:
        T = torch.zeros((m, n), dtype=dt, device="cuda")
        start = np.zeros((m, n))
        start[:, 0] = inst.a
    else:
        T = dev(T0, dt)
        start = host(T)
    var_o, step_o, order_o = getattr(O, variant), getattr(O, step), getattr(O, order)
    ties = []
    kinds = {}
    events = []
    steps_ill = 0
    for ep in range(epochs):
        tr = torch.full((4 * m,), -1, dtype=torch.int32, device="cuda")
        res = h.solve(dev(inst.a, dt), dev(inst.b, dt), T, warm_start=ep > 0 or T0 is not None,
                      dense_only=dense_only, precision=prec,
                      variant=getattr(S, variant), step=getattr(S, step), order=getattr(S, order),
                      seed=seed + ep, rho=inst.rho, max_epochs=1, trace=tr, trace_capacity=m, **kw)
        Tg = host(T)
        gi, gj, gv, gg = _trace_rows(tr)
        gd = _trace_dirs(tr)
        _, ro, ti, _, _ = O.solve(C, inst.a, inst.b, T0=start, rho=inst.rho, variant=var_o,
                                  step=step_o, order=order_o, seed=seed + ep, max_epochs=1, trace=True)
        np.testing.assert_array_equal(gi, ti)  # same block order
        assert Tg.min() >= 0.0
        np.testing.assert_allclose(Tg.sum(1), inst.a, rtol=2e-5, atol=0)
        assert rel(res["objective"], ro["f"]) <= 1e-3  # free-running oracle epoch: gross check
        Tr = start.copy()
        rr = Tr.sum(0) - inst.b
        nt = 0
        for p in range(m):
            i = int(ti[p])
            ai = inst.a[i]
            row_before, r_before = Tr[i].copy(), rr.copy()
            js, v, dr, gam = O.block_step(C, inst.a, Tr, rr, i, p, variant=var_o, step=step_o,
                                          rho=inst.rho)
            if gam == 0.0 and gg[p] == 0.0:
                continue  # neither moved: the state is the same whatever vertex was named
            same_vertices = gj[p] == js and (variant == "BCFW" or gv[p] == v) and (gd[p] == dr or gam == 0.0)
            if same_vertices and abs(gg[p] - gam) * ai <= 1e-7 + 1e-5 * abs(gam) * ai:
                # the same decision: the oracle takes the GPU's gamma from here on, so
                # that the states both sides decide from do not drift apart by the
                # tolerance of this comparison over the epoch
                gam_f = _followed_gamma(dr, row_before, ai, v, float(gg[p]))
                if gam_f != gam:
                    Tr[i] = row_before
                    rr[:] = r_before
                    O.apply_step(inst.a, Tr, rr, i, dr, js, v, gam_f)
                continue
            Tpre = Tr.copy()
            Tpre[i] = row_before
            if same_vertices:
                tie = "ill-conditioned step" if abs(gg[p] - gam) <= fp32_step_allowance(
                    C, inst.a, Tpre, r_before, i, inst.rho, dr, js, v, gam) else None
                tie = near_tie(C, inst.a, Tpre, r_before, i, inst.rho, variant) if tie is None else tie
            else:
                tie = near_tie(C, inst.a, Tpre, r_before, i, inst.rho, variant)
                if tie is None and variant != "BCFW":
                    light = lambda c: 0 <= c < n and row_before[c] <= NEGLIGIBLE * ai
                    if light(int(gv[p])) or light(v):
                        tie = "negligible atom"
            if tie is None:  # report what the decision looked like at the oracle's state
                gr = C[i] + inst.rho * r_before
                tt = row_before
                info = dict(dir=dr, alpha_v=(tt[v] / ai if 0 <= v < n else None),
                            g_fw=float(tt @ gr - ai * gr[js]),
                            g_aw=(float(ai * gr[v] - tt @ gr) if 0 <= v < n else None),
                            allowance=fp32_step_allowance(C, inst.a, Tpre, r_before, i, inst.rho, dr, js, v, gam)
                            if same_vertices else None, nnz=int((tt > 0).sum()), row_drift=float(tt.sum() - ai),
                            gammas_fw_away=_fw_away_gammas(C, inst.a, Tpre, r_before, i, inst.rho, int(gj[p]),
                                                           int(gv[p])),
                            r_consistent=float(np.abs(r_before - (Tpre.sum(0) - inst.b)).max()),
                            kinds=dict(kinds), steps_ill=steps_ill,
                            events_here=[e for e in events if e[2] == i or e[5] in (js, v) or e[6] in (js, v)][-8:],
                            last_events=events[-5:])
            assert tie is not None, repr((ep, p, i, (gj[p], js), (gv[p], v), (gg[p], gam), info))
            kinds[tie] = kinds.get(tie, 0) + 1
            if tie == "ill-conditioned step":
                steps_ill += 1  # the same decision, a step FP32 resolves only this far
            else:
                nt += 1
            # follow the GPU's decision from here on
            Tr[i] = row_before
            rr[:] = r_before
            light = (Tr[i] > 0) & (Tr[i] <= NEGLIGIBLE * ai)
            rr[light] -= Tr[i][light]
            Tr[i][light] = 0.0
            gdir, gam_g = int(gd[p]), float(gg[p])  # the direction the GPU took (from its trace)
            events.append((ep, p, i, tie, gdir, int(gj[p]), int(gv[p]), gam_g))
            gvc = int(gv[p])
            if gdir in (1, 2) and 0 <= gvc < n and Tr[i, gvc] > 0:
                alpha = Tr[i, gvc] / ai
                gmax = alpha if gdir == 2 else alpha / (1.0 - alpha)
                if gam_g >= gmax * (1.0 - 1e-6):
                    gam_g = gmax  # the GPU dropped the atom
                elif tie == "drop" and gam >= gmax:
                    gam_g = min(gam_g, float(np.nextafter(gmax, 0.0)))  # the GPU kept it
            O.apply_step(inst.a, Tr, rr, i, gdir, int(gj[p]), gvc, gam_g)
        ties.append(nt)
        assert np.abs(Tg - Tr).max() <= T_ATOL, (ep, np.abs(Tg - Tr).max(), nt)
        fr = O.certificate(C, inst.a, inst.b, inst.rho, Tr)["f"]
        assert rel(res["objective"], fr) <= OBJ_RTOL, (ep, res["objective"], fr, nt)
        start = Tg
    assert sum(ties) <= max(2, max_tie_frac * m * epochs), (ties, kinds)
    return ties


@pytest.mark.parametrize("m,n,ep", [(700, 1100, 20), (64, 1, 5)])
def test_fp32_decay_trajectory(S, h, oracle_mod, m, n, ep):
    """Decay rule in FP32: whole trajectory against the oracle."""
    inst = W.colour_instance(m + 3 * n, m, n, rho=10.0, b_dirichlet=True).rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    To, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                  step=oracle_mod.DEC, max_epochs=ep)
    T = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T,
                  X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32), precision=S.FP32,
                  variant=S.BCFW, step=S.DEC, rho=inst.rho, max_epochs=ep)
    assert rel(res["objective"], ro["f"]) <= OBJ_RTOL
    Tg = host(T)
    assert np.abs(Tg - To).max() <= T_ATOL
    assert Tg.min() >= 0.0
    np.testing.assert_allclose(Tg.sum(1), inst.a, rtol=1e-5)


CASES32 = [
    ("BCFW", "ELS", "PERMUTE", 700, 1100, 12),
    ("BCAFW", "ELS", "UNIFORM", 700, 1100, 12),
    ("BCPFW", "ELS", "CYCLIC", 700, 1100, 12),
    ("BCPFW", "ELS", "PERMUTE", 257, 3000, 8),
    ("BCFW", "ELS", "CYCLIC", 1, 513, 10),
    ("BCPFW", "ELS", "UNIFORM", 300, 257, 10),
]


@pytest.mark.parametrize("dense_only", [0, 1])
@pytest.mark.parametrize("variant,step,order,m,n,ep", CASES32)
def test_fp32_line_search_replay(S, h, oracle_mod, variant, step, order, m, n, ep, dense_only):
    """Away and pairwise steps run on the active-set kernel by default and on
    the dense row kernel with dense_only; both replay the oracle."""
    if variant == "BCFW" and dense_only:
        pytest.skip("BCFW always uses the dense kernel")
    inst = W.colour_instance(m + 3 * n, m, n, rho=10.0, b_dirichlet=True).rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    replay_epochs(S, h, oracle_mod, inst, C,
                  dict(X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32)),
                  variant, step, order, ep, dense_only=dense_only)


@pytest.mark.parametrize("dense_only", [0, 1])
def test_fp32_given_cost(S, h, oracle_mod, dense_only):
    inst = W.colour_instance(99, 500, 2000, rho=100.0).rounded()
    C = f32(oracle_mod.cost(inst.X, inst.Y))
    replay_epochs(S, h, oracle_mod, inst, C, dict(C=dev(C, torch.float32)), "BCPFW", "ELS",
                  "CYCLIC", 8, dense_only=dense_only)


def test_active_set_overflow_falls_back_to_dense(S, h, oracle_mod):
    """A row whose active set would exceed the 31-atom record hands the epoch
    to the dense kernel at that update; the result still replays the oracle."""
    m, n = 40, 300
    inst = W.colour_instance(123, m, n, rho=10.0).rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    T0 = np.zeros((m, n))
    T0[:, 0] = inst.a
    # row 5: 31 atoms on its most expensive columns, so its FW step adds a 32nd
    cols = np.argsort(C[5])[-31:]
    T0[5] = 0.0
    T0[5, cols] = inst.a[5] / 31
    T0 = f32(T0)
    replay_epochs(S, h, oracle_mod, inst, C,
                  dict(X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32)),
                  "BCAFW", "ELS", "CYCLIC", 3, T0=T0)
    # a start with a row beyond the record size goes dense from the first update
    T1 = T0.copy()
    T1[7] = 0.0
    T1[7, :40] = inst.a[7] / 40
    replay_epochs(S, h, oracle_mod, inst, C,
                  dict(X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32)),
                  "BCPFW", "ELS", "CYCLIC", 2, T0=f32(T1))


@pytest.mark.parametrize("order", ["CYCLIC", "PERMUTE"])
def test_pairwise_overflow_mid_epoch_all_kernels(S, h, oracle_mod, order):
    """Row 5 starts with 63 atoms (the record's limit) on its most expensive
    columns, so its pairwise step must append a 64th: every active-set kernel
    stops at that update and the dense kernel finishes the epoch. The trace and
    the plan agree bit for bit across the three kernels, and the epochs replay
    the oracle."""
    m, n = 48, 300
    inst = W.colour_instance(321, m, n, rho=10.0).rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    T0 = np.zeros((m, n))
    T0[:, 0] = inst.a
    cols = np.argsort(C[5])[-63:]
    T0[5] = 0.0
    T0[5, cols] = inst.a[5] / 63
    T0 = f32(T0)
    ep = 3
    out = []
    for ek in (S.EPOCH_TWO_PHASE, S.EPOCH_PIPELINED, S.EPOCH_SPECULATIVE, S.EPOCH_SPECULATIVE_ONE_CHAIN,
               S.EPOCH_SPECULATIVE_SPLIT):
        cap = ep * m
        tr = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
        T = dev(T0, torch.float32).contiguous()
        res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
                      Y=dev(inst.Y, torch.float32), precision=S.FP32, variant=S.BCPFW, step=S.ELS,
                      order=getattr(S, order), seed=5, rho=inst.rho, max_epochs=ep, warm_start=True,
                      trace=tr, trace_capacity=cap, epoch_kernel=ek)
        assert res["status"] in (S.OK, S.NOT_CONVERGED), res
        out.append((tr.cpu().numpy(), T.cpu().numpy()))
    for k in (1, 2, 3, 4):
        np.testing.assert_array_equal(out[0][0], out[k][0])
        np.testing.assert_array_equal(out[0][1], out[k][1])
    tr0 = out[0][0].reshape(-1, 4)
    first5 = tr0[np.nonzero(tr0[:, 0] == 5)[0][0]]
    assert first5[1] not in set(cols.tolist())  # its LMO vertex is a 64th atom: the overflow happens
    if order == "CYCLIC":
        replay_epochs(S, h, oracle_mod, inst, C,
                      dict(X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32)),
                      "BCPFW", "ELS", "CYCLIC", 2, T0=T0)


@pytest.mark.parametrize("variant,step", [("BCFW", "DEC"), ("BCPFW", "ELS"), ("BCAFW", "ELS")])
def test_fp32_full_size_colour4096(S, h, oracle_mod, variant, step):
    """colour4096_fp32 (m = n = 4096, Dirichlet b) in the launch configuration
    the benchmark times: the decay rule over 3 epochs of trajectory, the line
    search variants by epoch replay."""
    inst = W.workload("colour4096_fp32").rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    kw = dict(X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32))
    if step == "DEC":
        To, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                      step=oracle_mod.DEC, max_epochs=3)
        T = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")
        res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, precision=S.FP32,
                      variant=S.BCFW, step=S.DEC, rho=inst.rho, max_epochs=3, **kw)
        assert rel(res["objective"], ro["f"]) <= OBJ_RTOL
        assert np.abs(host(T) - To).max() <= T_ATOL
    else:
        # from T0 the rows are far from converged: FP32 may flip at most 1% of
        # the decisions
        replay_epochs(S, h, oracle_mod, inst, C, kw, variant, step, "CYCLIC", 3, max_tie_frac=0.01)


def _optima():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "colour4096_fp32_optima.json")) as fh:
        return json.load(fh)["optima"]


@pytest.mark.parametrize("rho", [1.0, 10.0, 100.0])
def test_fp32_headline_converged_to_oracle_optimum(S, h, oracle_mod, rho):
    """colour4096_fp32 solved as the benchmark solves it (BCPFW-ELS, cyclic,
    FP32 with FP64 certificate, default kernel, rel. gap 1e-6), for rho = 1,
    10, 100. The returned plan is certified again by the oracle: its gap
    (Thm 2) is at most 1.2e-6 of its objective, and that objective is within
    1.2e-6 of the optimal value f* the oracle reached on the same inputs
    (stored by tests/golden/make_optima.py; f* is unique). The library's own
    objective agrees with the oracle's evaluation of its plan to the FP32
    rounding of the cost entries."""
    opt = _optima()[f"{rho:g}"]
    inst = W.workload("colour4096_fp32").rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    T = torch.zeros((inst.m, inst.n), dtype=torch.float32, device="cuda")
    res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
                  Y=dev(inst.Y, torch.float32), precision=S.FP32, variant=S.BCPFW, step=S.ELS, order=S.CYCLIC,
                  rho=rho, tol_rel_gap=1e-6, max_epochs=6000, gap_every=1, refresh_every=1)
    assert res["status"] == S.OK and res["rel_gap"] <= 1e-6, res
    cert = oracle_mod.certificate(C, inst.a, inst.b, rho, host(T))
    assert cert["g"] <= 1.2e-6 * cert["f"], (cert["g"] / cert["f"], res)
    # below f* only by what the FP32 row sums' rounding allows (the plan is
    # feasible to ~1e-7 of a_i)
    assert opt["f_lower"] * (1 - 2e-7) <= cert["f"] <= opt["f"] * (1 + 1.2e-6), (cert["f"], opt)
    assert rel(res["objective"], cert["f"]) <= 2e-7
    assert abs(res["gap"] - cert["g"]) <= 2e-7 * cert["f"]


def test_fp32_reaches_relative_gap(S, h, oracle_mod):
    """Pairwise steps in FP32 reach rel. gap 1e-6 and agree with the oracle's
    converged objective."""
    inst = W.colour_instance(77, 512, 512, rho=10.0, b_dirichlet=True).rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    _, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCPFW,
                                 step=oracle_mod.ELS, max_epochs=5000, tol_rel_gap=1e-7)
    T = torch.zeros((512, 512), dtype=torch.float32, device="cuda")
    res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T,
                  X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32), precision=S.FP32,
                  variant=S.BCPFW, step=S.ELS, rho=inst.rho, max_epochs=5000, tol_rel_gap=1e-6)
    assert res["status"] == S.OK
    assert res["rel_gap"] <= 1e-6
    assert rel(res["objective"], ro["f"]) <= 2e-6


# ---------------------------------------------------------------------------
# Edge cases and error handling
# ---------------------------------------------------------------------------
def test_zero_weight_rows_and_warm_start(S, h, oracle_mod):
    inst = W.colour_instance(8, 90, 140, rho=5.0)
    a = inst.a.copy()
    a[[3, 50, 89]] = 0.0
    a /= a.sum()
    C = oracle_mod.cost(inst.X, inst.Y)
    T1, _, *_ = oracle_mod.solve(C, a, inst.b, rho=5.0, variant=oracle_mod.BCFW, step=oracle_mod.DEC,
                                 max_epochs=7)
    To, ro, *_ = oracle_mod.solve(C, a, inst.b, T0=T1, rho=5.0, variant=oracle_mod.BCPFW,
                                  step=oracle_mod.ELS, max_epochs=9)
    T = dev(T1, torch.float64)
    res = h.solve(dev(a, torch.float64), dev(inst.b, torch.float64), T, C=dev(C, torch.float64),
                  warm_start=True, precision=S.FP64, variant=S.BCPFW, step=S.ELS, rho=5.0,
                  max_epochs=9)
    assert rel(res["objective"], ro["f"]) <= 1e-10
    assert np.abs(host(T) - To).max() <= 1e-9
    assert np.all(host(T)[[3, 50, 89]] == 0.0)


def test_zero_epochs_returns_initial_certificate(S, h, oracle_mod):
    inst = W.colour_instance(2, 33, 44, rho=3.0)
    C = oracle_mod.cost(inst.X, inst.Y)
    T0 = np.zeros((33, 44))
    T0[:, 0] = inst.a
    ref = oracle_mod.certificate(C, inst.a, inst.b, 3.0, T0)
    T = torch.full((33, 44), 7.0, dtype=torch.float64, device="cuda")
    res = h.solve(dev(inst.a, torch.float64), dev(inst.b, torch.float64), T,
                  X=dev(inst.X, torch.float64), Y=dev(inst.Y, torch.float64), precision=S.FP64,
                  rho=3.0, max_epochs=0)
    np.testing.assert_array_equal(host(T), T0)
    assert rel(res["objective"], ref["f"]) <= 1e-13
    assert res["epochs"] == 0


def test_general_dimension_points(S, h, oracle_mod):
    rng = np.random.default_rng(0)
    X, Y = rng.standard_normal((120, 7)), rng.standard_normal((90, 7))
    a, b = np.full(120, 1 / 120), np.full(90, 1 / 90)
    C = oracle_mod.cost(X, Y)
    To, ro, *_ = oracle_mod.solve(C, a, b, rho=50.0, variant=oracle_mod.BCFW, step=oracle_mod.DEC,
                                  max_epochs=10)
    T = torch.zeros((120, 90), dtype=torch.float64, device="cuda")
    res = h.solve(dev(a, torch.float64), dev(b, torch.float64), T, X=dev(X, torch.float64),
                  Y=dev(Y, torch.float64), precision=S.FP64, rho=50.0, max_epochs=10)
    assert rel(res["objective"], ro["f"]) <= 1e-12
    assert np.abs(host(T) - To).max() <= 1e-12


def test_errors(S, h):
    m, n = 16, 20
    a = torch.full((m,), 1 / m, dtype=torch.float32, device="cuda")
    b = torch.full((n,), 1 / n, dtype=torch.float32, device="cuda")
    X = torch.rand((m, 3), device="cuda")
    Y = torch.rand((n, 3), device="cuda")
    T = torch.zeros((m, n), device="cuda")
    st, _ = h.solve_raw(a, b, T, X=X, Y=Y, variant=S.BCPFW, step=S.DEC)
    assert st == S.EINVAL
    st, _ = h.solve_raw(a, b, T, X=X, Y=Y, rho=-1.0)
    assert st == S.EINVAL
    st, _ = h.solve_raw(a, b, T, X=X, Y=Y, C=torch.zeros((m, n), device="cuda"))
    assert st == S.EINVAL
    bad = a.clone()
    bad[3] = float("nan")
    st, _ = h.solve_raw(bad, b, T, X=X, Y=Y)
    assert st == S.EINVAL and "a has" in h.last_error()
    Xn = X.clone()
    Xn[0, 0] = float("inf")
    st, _ = h.solve_raw(a, b, T, X=Xn, Y=Y)
    assert st == S.ENUMERIC
    big = torch.zeros((2, 9000), device="cuda")
    st, _ = h.solve_raw(torch.full((2,), 0.5, device="cuda"), torch.full((9000,), 1 / 9000, device="cuda"),
                        big, C=torch.rand((2, 9000), device="cuda"))
    assert st == S.EUNSUPPORTED
    # the handle stays usable after errors
    res = h.solve(a, b, T, X=X, Y=Y, max_epochs=2)
    assert res["status"] == S.OK


def test_bounded_wait_times_out_and_handle_stays_usable(S, h):
    """The speculative epoch kernel's waits are bounded. With a start gate
    that nothing opens and a limit of 2000 probes, its first wait runs out:
    the kernel stops without making an update, the call returns
    SR_OT_ETIMEOUT, and the same handle and stream then solve normally -- the
    result equal, bit for bit, to a solve on a fresh handle and to a solve
    through an opened gate."""
    inst = W.colour_instance(61, 300, 500, rho=10.0, b_dirichlet=True).rounded()
    a, b = dev(inst.a, torch.float32), dev(inst.b, torch.float32)
    X, Y = dev(inst.X, torch.float32), dev(inst.Y, torch.float32)
    kw = dict(precision=S.FP32, variant=S.BCPFW, step=S.ELS, rho=10.0, max_epochs=4,
              epoch_kernel=S.EPOCH_SPECULATIVE)
    gate = torch.zeros(1, dtype=torch.int32, device="cuda")
    T = torch.zeros((inst.m, inst.n), dtype=torch.float32, device="cuda")
    st, _ = h.solve_raw(a, b, T, X=X, Y=Y, start_gate=gate, spin_limit=2000, **kw)
    assert st == S.ETIMEOUT and "bounded device wait" in h.last_error()
    Tz = host(T)
    assert np.all(Tz[:, 1:] == 0.0) and np.allclose(Tz[:, 0], inst.a)  # no update was made
    res = h.solve(a, b, T, X=X, Y=Y, **kw)
    h2 = S.Handle(0)
    T2 = torch.zeros_like(T)
    res2 = h2.solve(a, b, T2, X=X, Y=Y, **kw)
    h2.close()
    assert torch.equal(T, T2) and res["objective"] == res2["objective"]
    gate.fill_(1)
    T3 = torch.zeros_like(T)
    res3 = h.solve(a, b, T3, X=X, Y=Y, start_gate=gate, spin_limit=2000, **kw)
    assert torch.equal(T, T3) and res3["objective"] == res["objective"]
    st, _ = h.solve_raw(a, b, T3, X=X, Y=Y, spin_limit=-1, **kw)
    assert st == S.EINVAL


def test_reading_b_lambda_as_inverse_weight(S, h, oracle_mod):
    """The paper's weight is 1/(2 lambda) (Sec. 3, eq. 5): read literally, the
    workload's "lambda = 10" is rho = 1/10. colour256_fp64 at rho = 0.1,
    BCFW-DEC, 200 epochs: argmin sequence and plan bit-identical to the
    oracle, as for rho = 10."""
    inst = W.workload("colour256_fp64")
    m, n, rho = inst.m, inst.n, 0.1
    C = oracle_mod.cost(inst.X, inst.Y)
    To, ro, ti, tj, _ = oracle_mod.solve(C, inst.a, inst.b, rho=rho, variant=oracle_mod.BCFW,
                                         step=oracle_mod.DEC, max_epochs=200, trace=True)
    cap = 200 * m
    tr = _trace_buf(cap)
    T = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    res = h.solve(dev(inst.a, torch.float64), dev(inst.b, torch.float64), T, X=dev(inst.X, torch.float64),
                  Y=dev(inst.Y, torch.float64), precision=S.FP64, variant=S.BCFW, step=S.DEC, rho=rho,
                  max_epochs=200, trace=tr, trace_capacity=cap)
    trh = tr.cpu().numpy().reshape(-1, 4)
    np.testing.assert_array_equal(trh[:, 0], ti)
    np.testing.assert_array_equal(trh[:, 1], tj)
    np.testing.assert_array_equal(host(T), To)
    assert rel(res["objective"], ro["f"]) <= 1e-13


def test_not_converged_status(S, h):
    m, n = 64, 64
    inst = W.colour_instance(1, m, n)
    T = torch.zeros((m, n), device="cuda")
    st, res = h.solve_raw(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T,
                          X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32),
                          tol_rel_gap=1e-12, max_epochs=3)
    assert st == S.NOT_CONVERGED and res["status"] == S.NOT_CONVERGED and res["epochs"] == 3


@pytest.mark.parametrize("variant,order", [("BCPFW", "CYCLIC"), ("BCPFW", "GAP_ADAPTIVE"),
                                           ("BCAFW", "GAP_ADAPTIVE")])
def test_fp32_dense_steps_conserve_row_mass(S, h, oracle_mod, variant, order):
    """Thousands of FP32 away / pairwise steps on the dense row kernels keep
    every row sum at a_i (the stopping test requires it): pairwise moves are
    rounded so both entries change exactly, away steps take the other atoms'
    stored mass instead of a_i - t_v. (Cyclic dense BCAFW, whose FW and away
    steps rescale every entry in FP32, drifts by ~4e-5 over 8000 epochs; the
    default BCAFW path keeps double-float atoms and does not.)"""
    inst = W.colour_instance(79, 150, 210, rho=10.0, b_dirichlet=True).rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    _, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCPFW,
                                 step=oracle_mod.ELS, max_epochs=50000, tol_rel_gap=1e-10, gap_every=5)
    T = torch.zeros((inst.m, inst.n), dtype=torch.float32, device="cuda")
    res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
                  Y=dev(inst.Y, torch.float32), precision=S.FP32, variant=getattr(S, variant), step=S.ELS,
                  order=getattr(S, order), seed=3, rho=inst.rho, max_epochs=12000, tol_rel_gap=1e-6,
                  dense_only=1)
    assert res["status"] == S.OK and res["row_err"] <= 1e-5, res
    Tc = host(T)
    assert Tc.min() >= 0.0
    assert np.abs(Tc.sum(1) - inst.a).max() <= 1e-5 * inst.a.max()
    assert ro["f"] - 1e-9 <= res["objective"] <= ro["f"] * (1 + 1.2e-6)


@pytest.mark.parametrize("order,m,n,ep,mode", [("CYCLIC", 300, 700, 30, "pts"), ("UNIFORM", 257, 515, 20, "pts"),
                                               ("PERMUTE", 200, 1500, 15, "pts"), ("CYCLIC", 190, 600, 20, "cost"),
                                               ("CYCLIC", 1024, 4096, 3, "pts"), ("PERMUTE", 2048, 3000, 4, "pts"),
                                               ("CYCLIC", 3, 40, 200, "pts"), ("CYCLIC", 5000, 1025, 2, "pts"),
                                               ("UNIFORM", 6, 300, 60, "pts"), ("UNIFORM", 40, 2000, 12, "pts"),
                                               ("CYCLIC", 256, 8192, 3, "cost"), ("PERMUTE", 300, 2048, 6, "cost"),
                                               ("CYCLIC", 3, 4100, 40, "cost"), ("CYCLIC", 100, 1001, 10, "cost")])
def test_pairwise_kernels_match_two_phase(S, h, oracle_mod, order, m, n, ep, mode):
    """The pipelined BCPFW kernel takes the next row's LMO and away vertex over
    the columns the current update leaves unchanged and completes them at the
    two changed columns afterwards; the speculative kernel takes the LMOs of
    the next rows against an older residual and repairs them at every column
    changed since. Every decision (block, LMO vertex, away vertex, step) and
    the final plan equal the two-phase active-set kernel's bit for bit (where
    a kernel does not apply, the fallback runs and must match as well). In
    uniform order rows come back within a few updates (m = 6: every few
    updates), which the split chain handles by re-reading the record. With a
    given cost matrix the speculative kernel reads C (n a multiple of 4, up
    to 8192 = the widest rows, where the last column can be the away vertex;
    n = 1001 takes the fallback)."""
    inst = W.colour_instance(17 + m, m, n, rho=10.0, b_dirichlet=True).rounded()
    C = dev(oracle_mod.cost(inst.X, inst.Y), torch.float32) if mode == "cost" else None
    out = []
    for ek in (S.EPOCH_TWO_PHASE, S.EPOCH_PIPELINED, S.EPOCH_SPECULATIVE, S.EPOCH_SPECULATIVE_ONE_CHAIN,
               S.EPOCH_SPECULATIVE_SPLIT):
        cap = ep * m
        tr = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
        T = torch.zeros((m, n), dtype=torch.float32, device="cuda")
        kw = dict(C=C) if C is not None else dict(X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32))
        res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, precision=S.FP32,
                      variant=S.BCPFW, step=S.ELS, order=getattr(S, order), seed=11, rho=inst.rho,
                      max_epochs=ep, trace=tr, trace_capacity=cap, epoch_kernel=ek, **kw)
        assert res["status"] in (S.OK, S.NOT_CONVERGED), res
        out.append((tr.cpu().numpy(), T.cpu().numpy(), res))
    for k in (1, 2, 3, 4):
        np.testing.assert_array_equal(out[0][0], out[k][0])
        np.testing.assert_array_equal(out[0][1], out[k][1])
        assert out[0][2]["objective"] == out[k][2]["objective"]


def test_chain_floor_probe(S, h):
    """The chain-floor probe (observability) runs its dependent hand-overs
    to the end for one and three chain warps and reports a positive time per
    update below that of any real block update; bad arguments are refused."""
    for cw in (1, 3):
        ns = h.chain_floor(cw, 1 << 14)
        assert 1.0 < ns < 5000.0, (cw, ns)
    r = S.ct.c_double()
    assert S.lib.sr_ot_profile_chain_floor(h._h, 2, 100, S.ct.byref(r)) == S.EINVAL
    assert S.lib.sr_ot_profile_chain_floor(h._h, 3, 0, S.ct.byref(r)) == S.EINVAL


def test_predicted_certificate_schedule(S, h, oracle_mod):
    """cert_schedule = 1 takes the certificate only when the gap's decay
    predicts the tolerance: colour4096_fp32 (the benchmark's solve) reaches
    rel. gap 1e-6 with fewer certificates and within 8 epochs of the solve
    with a certificate every epoch, and the returned plan is certified by the
    oracle against the stored optimum."""
    inst = W.workload("colour4096_fp32").rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    opt = _optima()["10"]
    out = {}
    for sched in (0, 1):
        T = torch.zeros((inst.m, inst.n), dtype=torch.float32, device="cuda")
        l0 = h.launch_count()
        res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
                      Y=dev(inst.Y, torch.float32), precision=S.FP32, variant=S.BCPFW, step=S.ELS, rho=inst.rho,
                      tol_rel_gap=1e-6, max_epochs=6000, gap_every=1, cert_schedule=sched)
        assert res["status"] == S.OK and res["rel_gap"] <= 1e-6, res
        cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, host(T))
        assert cert["g"] <= 1.2e-6 * cert["f"]
        assert cert["f"] <= opt["f"] * (1 + 1.2e-6)
        out[sched] = (res["epochs"], h.launch_count() - l0)
    # each certificate also refreshes the residual from exact column sums, so
    # the two trajectories differ by rounding: epoch counts within 8
    (e0, l0), (e1, l1) = out[0], out[1]
    assert abs(e1 - e0) <= 8, out
    assert l1 < l0, out  # fewer certificate launches


@pytest.mark.parametrize("sched", [0, 1])
def test_record_overflow_with_either_certificate_schedule(S, h, oracle_mod, sched):
    """A row that must grow a 64th atom hands the solve to the dense kernel
    at that update; with certificates far apart the active-set kernels see
    the overflow themselves in the next epochs and leave them to the dense
    kernel. Either way the solve converges and the oracle certifies it."""
    m, n = 48, 300
    inst = W.colour_instance(321, m, n, rho=10.0).rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    T0 = np.zeros((m, n))
    T0[:, 0] = inst.a
    cols = np.argsort(C[5])[-63:]
    T0[5] = 0.0
    T0[5, cols] = inst.a[5] / 63
    T = dev(f32(T0), torch.float32).contiguous()
    res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
                  Y=dev(inst.Y, torch.float32), precision=S.FP32, variant=S.BCPFW, step=S.ELS, rho=inst.rho,
                  tol_rel_gap=1e-6, max_epochs=20000, warm_start=True, cert_schedule=sched)
    assert res["status"] == S.OK and res["rel_gap"] <= 1e-6, res
    Tg = host(T)
    cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, Tg)
    assert cert["g"] <= 1.2e-6 * cert["f"]
    assert Tg.min() >= 0.0
    np.testing.assert_allclose(Tg.sum(1), inst.a, rtol=2e-5)
