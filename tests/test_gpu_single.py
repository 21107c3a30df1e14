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
    """Per update (i, j*, v, gamma) from a device trace buffer."""
    t = tr.cpu().numpy().reshape(-1, 4)
    return t[:, 0], t[:, 1], t[:, 2], t[:, 3].copy().view(np.float32).astype(np.float64)


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


def replay_epochs(S, h, O, inst, C, kw, variant, step, order, epochs, prec=None, seed=3,
                  dense_only=0, T0=None):
    """Run `epochs` epochs one at a time; before each, the oracle starts from
    the GPU's current plan. Within an epoch the GPU's decisions (block i,
    LMO vertex j*, away vertex v, step gamma; from the device trace) are
    compared update by update with the oracle's block steps. They must agree
    until the first update where a discrete decision is a near tie at the
    oracle's state (which FP32 cannot order); the epoch is then accepted
    without further comparison. Epochs without a tie must reproduce the
    oracle's plan to 1e-6 and its objective to 1e-5. Returns the number of
    epochs that ended at a tie."""
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
    ties = 0
    for ep in range(epochs):
        tr = torch.full((4 * m,), -1, dtype=torch.int32, device="cuda")
        res = h.solve(dev(inst.a, dt), dev(inst.b, dt), T, warm_start=ep > 0 or T0 is not None,
                      dense_only=dense_only, precision=prec,
                      variant=getattr(S, variant), step=getattr(S, step), order=getattr(S, order),
                      seed=seed + ep, rho=inst.rho, max_epochs=1, trace=tr, trace_capacity=m, **kw)
        Tg = host(T)
        gi, gj, gv, gg = _trace_rows(tr)
        _, ro, ti, _, _ = O.solve(C, inst.a, inst.b, T0=start, rho=inst.rho, variant=var_o,
                                  step=step_o, order=order_o, seed=seed + ep, max_epochs=1, trace=True)
        np.testing.assert_array_equal(gi, ti)  # same block order
        assert Tg.min() >= 0.0
        np.testing.assert_allclose(Tg.sum(1), inst.a, rtol=2e-5, atol=0)
        assert rel(res["objective"], ro["f"]) <= 1e-3  # gross check, holds across ties
        Tr = start.copy()
        rr = Tr.sum(0) - inst.b
        tie = None
        for p in range(m):
            i = int(ti[p])
            row_before, r_before = Tr[i].copy(), rr.copy()
            js, v, _, gam = O.block_step(C, inst.a, Tr, rr, i, p, variant=var_o, step=step_o,
                                         rho=inst.rho)
            same = gj[p] == js and (variant == "BCFW" or gv[p] == v or abs(gam) + abs(gg[p]) == 0)
            same = same and abs(gg[p] - gam) * inst.a[i] <= 1e-7 + 1e-5 * abs(gam) * inst.a[i]
            if not same:
                Tpre = Tr.copy()
                Tpre[i] = row_before
                tie = near_tie(C, inst.a, Tpre, r_before, i, inst.rho, variant)
                assert tie is not None, (ep, p, i, (gj[p], js), (gv[p], v), (gg[p], gam))
                break
        if tie is None:
            assert np.abs(Tg - Tr).max() <= T_ATOL, ep
            assert rel(res["objective"], ro["f"]) <= OBJ_RTOL, ep
        else:
            ties += 1
        start = Tg
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
    for ek in (S.EPOCH_TWO_PHASE, S.EPOCH_PIPELINED, S.EPOCH_SPECULATIVE):
        cap = ep * m
        tr = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
        T = dev(T0, torch.float32).contiguous()
        res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
                      Y=dev(inst.Y, torch.float32), precision=S.FP32, variant=S.BCPFW, step=S.ELS,
                      order=getattr(S, order), seed=5, rho=inst.rho, max_epochs=ep, warm_start=True,
                      trace=tr, trace_capacity=cap, epoch_kernel=ek)
        assert res["status"] in (S.OK, S.NOT_CONVERGED), res
        out.append((tr.cpu().numpy(), T.cpu().numpy()))
    for k in (1, 2):
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
        replay_epochs(S, h, oracle_mod, inst, C, kw, variant, step, "CYCLIC", 3)


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
                                               ("CYCLIC", 3, 40, 200, "pts"), ("CYCLIC", 5000, 1025, 2, "pts")])
def test_pairwise_kernels_match_two_phase(S, h, oracle_mod, order, m, n, ep, mode):
    """The pipelined BCPFW kernel takes the next row's LMO and away vertex over
    the columns the current update leaves unchanged and completes them at the
    two changed columns afterwards; the speculative kernel takes the LMOs of
    the next rows against an older residual and repairs them at every column
    changed since. Every decision (block, LMO vertex, away vertex, step) and
    the final plan equal the two-phase active-set kernel's bit for bit (where
    a kernel does not apply, the fallback runs and must match as well)."""
    inst = W.colour_instance(17 + m, m, n, rho=10.0, b_dirichlet=True).rounded()
    C = dev(oracle_mod.cost(inst.X, inst.Y), torch.float32) if mode == "cost" else None
    out = []
    for ek in (S.EPOCH_TWO_PHASE, S.EPOCH_PIPELINED, S.EPOCH_SPECULATIVE):
        cap = ep * m
        tr = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
        T = torch.zeros((m, n), dtype=torch.float32, device="cuda")
        kw = dict(C=C) if C is not None else dict(X=dev(inst.X, torch.float32), Y=dev(inst.Y, torch.float32))
        res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, precision=S.FP32,
                      variant=S.BCPFW, step=S.ELS, order=getattr(S, order), seed=11, rho=inst.rho,
                      max_epochs=ep, trace=tr, trace_capacity=cap, epoch_kernel=ek, **kw)
        assert res["status"] in (S.OK, S.NOT_CONVERGED), res
        out.append((tr.cpu().numpy(), T.cpu().numpy(), res))
    for k in (1, 2):
        np.testing.assert_array_equal(out[0][0], out[k][0])
        np.testing.assert_array_equal(out[0][1], out[k][1])
        assert out[0][2]["objective"] == out[k][2]["objective"]
