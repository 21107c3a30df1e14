"""BF16 tensor-core cost matrix (sr_ot_cost_bf16) and the solver on it.

Reference: the oracle's FP64 squared-Euclidean cost of the BF16-rounded
points (the rounding is the stated input precision of this path). The GPU
accumulates the inner products and the norms in FP32, so the bound per
entry is (d + 4) FP32 roundings of |x~|^2 + |y~|^2.
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


def _gpu_cost(S, h, X, Y):
    m, d = X.shape
    n = Y.shape[0]
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    Xd, Yd = dev(X, torch.float32), dev(Y, torch.float32)  # alive until the call returns
    st = S.lib.sr_ot_cost_bf16(h._h, m, n, d, S._ptr(Xd), S._ptr(Yd), S._ptr(C))
    return st, C


def _check(oracle_mod, X, Y, Cg, rows=None):
    Xr, Yr = W.bf16_round(X), W.bf16_round(Y)
    if rows is not None:
        Xr = Xr[rows]
    Cref = oracle_mod.cost(Xr, Yr)
    nx = (Xr * Xr).sum(1)
    ny = (Yr * Yr).sum(1)
    d = X.shape[1]
    bound = (d + 4) * 2.0 ** -24 * (nx[:, None] + ny[None, :])
    err = np.abs(Cg - Cref)
    assert (err <= bound).all(), (err / bound).max()
    return err.max()


@pytest.mark.parametrize("m,n,d", [(300, 520, 128), (128, 128, 64), (129, 260, 192), (77, 1000, 256),
                                   (1, 4, 64)])
def test_cost_bf16_matches_oracle(S, h, oracle_mod, m, n, d):
    inst = W.feature_instance(31 + d, m, n, d)
    st, C = _gpu_cost(S, h, inst.X, inst.Y)
    assert st == S.OK, h.last_error()
    _check(oracle_mod, inst.X, inst.Y, host(C))
    # the binding's method gives the same matrix
    C2 = h.cost_bf16(dev(inst.X, torch.float32), dev(inst.Y, torch.float32))
    assert torch.equal(C, C2)


def test_cost_bf16_unaligned_points(S, h, oracle_mod):
    """Points that start 4 bytes past a 16-byte boundary take the scalar
    rounding path; the cost stays within the same bound of the oracle."""
    m, n, d = 200, 136, 128
    inst = W.feature_instance(7, m, n, d)
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    bx = torch.zeros(m * d + 1, dtype=torch.float32, device="cuda")
    by = torch.zeros(n * d + 1, dtype=torch.float32, device="cuda")
    bx[1:] = dev(inst.X, torch.float32).reshape(-1)
    by[1:] = dev(inst.Y, torch.float32).reshape(-1)
    Xd, Yd = bx[1:], by[1:]
    assert Xd.data_ptr() % 16 == 4 and Yd.data_ptr() % 16 == 4
    st = S.lib.sr_ot_cost_bf16(h._h, m, n, d, S._ptr(Xd), S._ptr(Yd), S._ptr(C))
    assert st == S.OK, h.last_error()
    _check(oracle_mod, inst.X, inst.Y, host(C))


def test_cost_bf16_full_size_sampled(S, h, oracle_mod):
    """8192 x 8192, d = 128 (the feature-space workload): 48 sampled rows
    against the oracle over all 8192 columns."""
    inst = W.workload("feature8192_d128")
    st, C = _gpu_cost(S, h, inst.X, inst.Y)
    assert st == S.OK, h.last_error()
    rows = np.random.default_rng(2).choice(inst.m, 48, replace=False)
    _check(oracle_mod, inst.X, inst.Y, host(C[torch.as_tensor(rows, device="cuda")]), rows=rows)


def test_cost_bf16_rejects(S, h):
    X = np.zeros((16, 100))
    Y = np.zeros((16, 100))
    st, _ = _gpu_cost(S, h, X, Y)
    assert st == S.EUNSUPPORTED
    st, _ = _gpu_cost(S, h, np.zeros((16, 64)), np.zeros((18, 64)))  # n not a multiple of 4
    assert st == S.EUNSUPPORTED
    st, _ = _gpu_cost(S, h, np.zeros((16, 64)), np.zeros((16, 64)))
    assert st == S.OK


def test_solve_on_bf16_cost(S, h, oracle_mod):
    """SR_OT_FP32_BF16COST: the solver runs on the tensor-core cost; its
    optimum matches the oracle's on the FP64 cost of the rounded points."""
    inst = W.feature_instance(5, 200, 240, 64, rho=2500.0)
    Xr, Yr = W.bf16_round(inst.X), W.bf16_round(inst.Y)
    C = oracle_mod.cost(Xr, Yr)
    a32, b32 = (np.asarray(v, np.float32).astype(np.float64) for v in (inst.a, inst.b))
    _, ro, *_ = oracle_mod.solve(C, a32, b32, rho=inst.rho, variant=oracle_mod.BCPFW, step=oracle_mod.ELS,
                                 max_epochs=50000, tol_rel_gap=1e-10, gap_every=5)
    T = torch.zeros((200, 240), dtype=torch.float32, device="cuda")
    res = h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
                  Y=dev(inst.Y, torch.float32), precision=S.FP32_BF16COST, variant=S.BCPFW, step=S.ELS,
                  rho=inst.rho, max_epochs=20000, tol_rel_gap=1e-6)
    assert res["status"] == S.OK
    # the FP32 cost differs from the FP64 one by ~1e-6 relative per entry
    assert rel(res["objective"], ro["f"]) <= 1e-5
