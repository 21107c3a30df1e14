"""Gap-adaptive block sampling (Alg. A.4) and full Frank-Wolfe (Alg. A.1) on
the GPU against the FP64 oracle.

GA: in FP64 with the decay rule the sampled blocks and LMO vertices follow
the oracle's sequence (the sampling decision is taken in FP64 on both sides;
the running gaps agree to rounding, so a different draw would need a target
within a few ulps of a cumulative-weight boundary). With the line search
and in FP32 the converged optimal value is compared (it is unique).
FW: the FP64 decay-rule iterates match the oracle's to rounding; the line
search and FP32 runs are compared on the objective after the same number of
iterations and at convergence.
"""
import numpy as np
import pytest
import torch

from paper_2103_05857_gb300 import workloads as W

from .gpu_util import dev, host, rel

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


def _solve64(S, h, inst, **kw):
    T = torch.zeros((inst.m, inst.n), dtype=torch.float64, device="cuda")
    res = h.solve(dev(inst.a, torch.float64), dev(inst.b, torch.float64), T,
                  X=dev(inst.X, torch.float64), Y=dev(inst.Y, torch.float64), precision=S.FP64,
                  rho=inst.rho, **kw)
    return T, res


@pytest.mark.parametrize("ga_M,glob", [(1, 0), (3, 0), (1, 1)])
def test_ga_fp64_decay_sequence(S, h, oracle_mod, ga_M, glob):
    inst = W.colour_instance(77, 96, 130, rho=10.0, b_dirichlet=True)
    C = oracle_mod.cost(inst.X, inst.Y)
    ep = 12
    To, ro, ti, tj, _ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                         step=oracle_mod.DEC, order=oracle_mod.GAP, seed=4,
                                         ga_M=ga_M, ga_global_only=glob, max_epochs=ep, trace=True)
    cap = ep * inst.m
    tr = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
    T, res = _solve64(S, h, inst, variant=S.BCFW, step=S.DEC, order=S.GAP_ADAPTIVE, seed=4,
                      ga_M=ga_M, ga_global_only=glob, max_epochs=ep, trace=tr, trace_capacity=cap)
    trh = tr.cpu().numpy().reshape(-1, 4)
    np.testing.assert_array_equal(trh[:, 0], ti)
    np.testing.assert_array_equal(trh[:, 1], tj)
    assert np.abs(host(T) - To).max() <= 1e-13
    assert rel(res["objective"], ro["f"]) <= 1e-12


@pytest.mark.parametrize("m", [8192, 8193, 12000])
def test_ga_fp64_decay_sequence_large_m(S, h, oracle_mod, m):
    """Past 8192 rows the draw goes through a third level of sums (super
    nodes of 32 chunks of 32 rows); 8192 is the largest two-level case."""
    inst = W.colour_instance(81, m, 24, rho=10.0, b_dirichlet=True)
    C = oracle_mod.cost(inst.X, inst.Y)
    ep = 2
    To, ro, ti, tj, _ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                         step=oracle_mod.DEC, order=oracle_mod.GAP, seed=6, ga_M=1,
                                         max_epochs=ep, trace=True)
    cap = ep * inst.m
    tr = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
    T, res = _solve64(S, h, inst, variant=S.BCFW, step=S.DEC, order=S.GAP_ADAPTIVE, seed=6, ga_M=1,
                      max_epochs=ep, trace=tr, trace_capacity=cap)
    trh = tr.cpu().numpy().reshape(-1, 4)
    np.testing.assert_array_equal(trh[:, 0], ti)
    np.testing.assert_array_equal(trh[:, 1], tj)
    assert np.abs(host(T) - To).max() <= 1e-13
    assert rel(res["objective"], ro["f"]) <= 1e-12


@pytest.mark.parametrize("m,ep", [(64, 5), (9000, 2)])
def test_ga_concentrates_on_large_gaps(S, h, oracle_mod, m, ep):
    """The sampled rows follow the gaps: rows with zero gap are never drawn."""
    inst = W.colour_instance(78, m, 80, rho=10.0)
    a = inst.a.copy()
    a[::2] = 0.0  # zero-weight rows have g_i = 0 at every T
    a /= a.sum()
    cap = ep * inst.m
    tr = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
    T = torch.zeros((inst.m, inst.n), dtype=torch.float64, device="cuda")
    h.solve(dev(a, torch.float64), dev(inst.b, torch.float64), T, X=dev(inst.X, torch.float64),
            Y=dev(inst.Y, torch.float64), precision=S.FP64, rho=inst.rho, variant=S.BCFW, step=S.ELS,
            order=S.GAP_ADAPTIVE, seed=1, max_epochs=ep, trace=tr, trace_capacity=cap)
    rows = tr.cpu().numpy().reshape(-1, 4)[:, 0]
    assert (rows % 2 == 1).all()


@pytest.mark.parametrize("variant,tol", [("BCFW", 1e-4), ("BCPFW", 1e-6)])
@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_ga_converges_to_oracle_optimum(S, h, oracle_mod, variant, tol, prec):
    """Plain BCFW converges sublinearly (the oracle's BCFW-GA is still at a
    relative gap of 8e-6 after 20000 epochs here), so it is run to 1e-4."""
    inst = W.colour_instance(79, 150, 210, rho=10.0, b_dirichlet=True)
    if prec == "FP32":
        inst = inst.rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    _, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCPFW,
                                 step=oracle_mod.ELS, max_epochs=50000, tol_rel_gap=1e-10, gap_every=5)
    dt = torch.float64 if prec == "FP64" else torch.float32
    T = torch.zeros((inst.m, inst.n), dtype=dt, device="cuda")
    res = h.solve(dev(inst.a, dt), dev(inst.b, dt), T, X=dev(inst.X, dt), Y=dev(inst.Y, dt),
                  precision=getattr(S, prec), rho=inst.rho, variant=getattr(S, variant), step=S.ELS,
                  order=S.GAP_ADAPTIVE, seed=3, ga_M=2, max_epochs=20000, tol_rel_gap=tol)
    assert res["status"] == S.OK and res["rel_gap"] <= tol, res
    # f(T) - f* <= g(T) (weak duality), and the GPU's certificate is exact to rounding
    assert ro["f"] - 1e-9 <= res["objective"] <= ro["f"] + 1.2 * tol * ro["f"]
    cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, host(T))
    assert rel(res["objective"], cert["f"]) <= (1e-12 if prec == "FP64" else 2e-7)


def test_fw_fp64_decay_iterates(S, h, oracle_mod):
    inst = W.colour_instance(80, 70, 90, rho=10.0, b_dirichlet=True)
    C = oracle_mod.cost(inst.X, inst.Y)
    it = 40
    To, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.FW,
                                  step=oracle_mod.DEC, max_epochs=it)
    T, res = _solve64(S, h, inst, variant=S.FW, step=S.DEC, max_epochs=it)
    assert res["epochs"] == ro["epochs"] == it
    assert np.abs(host(T) - To).max() <= 1e-12
    assert rel(res["objective"], ro["f"]) <= 1e-12
    assert abs(res["gap"] - ro["g"]) <= 1e-11 * ro["f"]


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_fw_line_search(S, h, oracle_mod, prec):
    inst = W.colour_instance(81, 300, 520, rho=10.0, b_dirichlet=True)
    if prec == "FP32":
        inst = inst.rounded()
    C = oracle_mod.cost(inst.X, inst.Y)
    it = 60
    To, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.FW,
                                  step=oracle_mod.ELS, max_epochs=it)
    dt = torch.float64 if prec == "FP64" else torch.float32
    T = torch.zeros((inst.m, inst.n), dtype=dt, device="cuda")
    res = h.solve(dev(inst.a, dt), dev(inst.b, dt), T, X=dev(inst.X, dt), Y=dev(inst.Y, dt),
                  precision=getattr(S, prec), rho=inst.rho, variant=S.FW, step=S.ELS, max_epochs=it)
    if prec == "FP64":
        assert np.abs(host(T) - To).max() <= 1e-10
        assert rel(res["objective"], ro["f"]) <= 1e-10
    else:
        assert rel(res["objective"], ro["f"]) <= 1e-5
        Tc = host(T)
        assert Tc.min() >= 0.0 and np.allclose(Tc.sum(1), inst.a, rtol=1e-5, atol=0)


def test_fw_reaches_gap_and_stops(S, h, oracle_mod):
    inst = W.colour_instance(82, 40, 60, rho=10.0)
    C = oracle_mod.cost(inst.X, inst.Y)
    _, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.FW,
                                 step=oracle_mod.ELS, max_epochs=100000, tol_rel_gap=1e-4)
    T, res = _solve64(S, h, inst, variant=S.FW, step=S.ELS, max_epochs=100000, tol_rel_gap=1e-4)
    assert res["status"] == S.OK and res["rel_gap"] <= 1e-4
    assert abs(res["epochs"] - ro["epochs"]) <= 2
