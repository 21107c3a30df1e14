"""The evaluation metrics (v) and (vi) of Sec. 5 on the GPU (sr_ot_lp_metrics)
against the oracle.

e_m = ||T - T_lp|| / ||T_lp|| and e_v = |<T, C> - <T_lp, C>| / |<T_lp, C>| of
a plan T against the reference plan T_lp, which the paper takes as the
optimal plan of the unrelaxed transport problem (the oracle's transport_lp,
pinned on the CPU). The GPU pass is compared with the oracle's lp_metrics on
the same plans, element sums in FP64 for FP64 plans and compensated FP32 sums
for FP32 plans, at sizes that span several blocks with ragged rows, and at the
2048 x 2048 size of the differentiable workload.
"""
import numpy as np
import pytest
import torch

from paper_2103_05857_gb300 import workloads as W

from .gpu_util import dev, f32, host, rel

pytestmark = pytest.mark.gpu


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


def _check(g, o, fp64, scale_v):
    """GPU metrics g against the oracle's o. FP64: sums agree to rounding.
    FP32: each sum carries a few FP32 roundings per term, so the values
    agree to ~1e-6 and e_v (a difference of two values) to 1e-6 of their
    magnitudes over |<T_lp, C>|."""
    tol = 1e-12 if fp64 else 1e-6
    assert rel(g["diff_norm"], o["diff_norm"]) <= tol
    assert rel(g["lp_norm"], o["lp_norm"]) <= tol
    assert rel(g["value"], o["value"]) <= tol
    assert rel(g["lp_value"], o["lp_value"]) <= tol
    assert rel(g["e_m"], o["e_m"]) <= 2 * tol
    assert abs(g["e_v"] - o["e_v"]) <= 2 * tol * scale_v


@pytest.mark.parametrize("m,n,mode,prec,kind", [(37, 53, "pts", "FP64", "SQUARED"), (60, 45, "C", "FP64", "SQUARED"),
                                                (300, 517, "pts", "FP32", "SQUARED"),
                                                (257, 300, "C", "FP32", "SQUARED"),
                                                (90, 140, "pts", "FP32", "EUCLIDEAN"),
                                                (64, 1, "pts", "FP64", "EUCLIDEAN")])
def test_lp_metrics_match_oracle(S, h, oracle_mod, m, n, mode, prec, kind):
    """A converged semi-relaxed plan against the exact LP plan of the same
    instance (the paper's setting), every cost form the library takes."""
    fp64 = prec == "FP64"
    dt = torch.float64 if fp64 else torch.float32
    inst = W.colour_instance(m * 5 + n, m, n, rho=10.0, b_dirichlet=True)
    if not fp64:
        inst = inst.rounded()
    C = oracle_mod.cost(inst.X, inst.Y, squared=kind == "SQUARED")
    if not fp64 and (mode == "C" or kind == "EUCLIDEAN"):
        C = f32(C)  # the FP32 cost the GPU reads (C mode) or builds (Euclidean, one rounding)
    T, _, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCPFW, step=oracle_mod.ELS,
                                max_epochs=200)
    L = oracle_mod.transport_lp(C, inst.a, inst.b)
    if not fp64:
        T, L = f32(T), f32(L)
    o = oracle_mod.lp_metrics(C, T, L)
    kw = dict(C=dev(C, dt)) if mode == "C" else dict(X=dev(inst.X, dt), Y=dev(inst.Y, dt))
    g = h.lp_metrics(dev(T, dt), dev(L, dt), precision=getattr(S, prec), cost_kind=getattr(S, "COST_" + kind), **kw)
    _check(g, o, fp64 and kind == "SQUARED", (o["value"] + o["lp_value"]) / o["lp_value"])
    assert 0.0 <= g["e_v"] and (0.0 < g["e_m"] or n == 1)  # one column: every feasible plan is the LP plan


def test_lp_metrics_full_size(S, h, oracle_mod):
    """At 2048 x 2048 (the differentiable workload's instance size): a plan
    returned by the solver against a sparse feasible reference plan (any
    plan exercises the pass; the LP plan itself is not needed for parity)."""
    inst = W.workload("colour_batch64_2048")[0].rounded()
    m, n = inst.m, inst.n
    T = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    X, Y = dev(inst.X, torch.float32), dev(inst.Y, torch.float32)
    h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=X, Y=Y, precision=S.FP32,
            variant=S.BCPFW, step=S.ELS, rho=inst.rho, tol_rel_gap=1e-6, max_epochs=5000)
    r, c, v = W.feasible_plan(17, inst.a, n, support=6)
    L = np.zeros((m, n))
    L[r, c] = v
    L = f32(L)
    g = h.lp_metrics(T, dev(L, torch.float32), X=X, Y=Y, precision=S.FP32)
    o = oracle_mod.lp_metrics(oracle_mod.cost(inst.X, inst.Y), host(T), L)
    _check(g, o, False, (o["value"] + o["lp_value"]) / o["lp_value"])


def test_lp_metrics_argument_errors(S, h):
    m, n = 8, 12
    T = torch.zeros((m, n), device="cuda")
    X = torch.rand((m, 3), device="cuda")
    Y = torch.rand((n, 3), device="cuda")
    C = torch.rand((m, n), device="cuda")
    o = S.options(precision=S.FP32)
    r = S.LpMetrics()
    p = S._ptr
    assert S.lib.sr_ot_lp_metrics(h._h, o, m, n, 3, p(C), p(X), p(Y), p(T), p(T), r) == S.EINVAL
    assert S.lib.sr_ot_lp_metrics(h._h, o, m, n, 0, None, None, None, p(T), p(T), r) == S.EINVAL
    assert S.lib.sr_ot_lp_metrics(h._h, o, m, n, 3, None, p(X), p(Y), p(T), None, r) == S.EINVAL
    X5 = torch.rand((m, 5), device="cuda")
    Y5 = torch.rand((n, 5), device="cuda")
    assert S.lib.sr_ot_lp_metrics(h._h, o, m, n, 5, None, p(X5), p(Y5), p(T), p(T), r) == S.EUNSUPPORTED
    # the handle stays usable
    g = h.lp_metrics(T + 1.0 / (m * n), T + 1.0 / (m * n), C=C, precision=S.FP32)
    assert g["e_m"] == 0.0 and g["e_v"] == 0.0
