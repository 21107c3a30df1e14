"""Colour-transfer tail (sr_ot_transfer) against the FP64 oracle.

The oracle's barycentric projection (Sec. 5.1) and the marginal-error and
sparsity metrics (Sec. 5, (iii) and (iv)) are pinned on the CPU; here the GPU
pass is compared with them on the same plans, element by element at sizes that
span several column tiles and row bands with ragged tails, for the FP32 d = 3
path and the generic one, in FP64, on rows that carry no mass, on a solved
plan, and on sampled rows of a 2048 x 2048 plan.
"""
import numpy as np
import pytest
import torch

from paper_2103_05857_gb300 import workloads as W

from .gpu_util import dev, host

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


def _plan(seed, m, n, support=6):
    a = W.dirichlet_weights(seed, m)
    rows, cols, vals = W.feasible_plan(seed, a, n, support)
    T = np.zeros((m, n))
    T[rows, cols] = vals
    b = W.dirichlet_weights(seed + 1, n)
    Y = W.colour_cloud(seed + 2, n)
    return a, b, T, Y


def _check(oracle_mod, Y, a, b, T, Xh, st, fp64):
    ref = oracle_mod.barycentric(Y, T)
    rs = oracle_mod.transfer_stats(a, b, T)
    scale = np.abs(ref).max() + 1e-300
    err = np.abs(Xh - ref).max() / scale
    assert err <= (1e-13 if fp64 else 2e-6), err
    # FP32 row and column sums carry about one rounding of their terms each;
    # their errors add up to ~1e-7 (||a|| + ||b||)
    tol = (1e-13 if fp64 else 2e-6) * (np.linalg.norm(a) + np.linalg.norm(b))
    for k in ("row_err", "col_err", "e_c"):
        assert abs(st[k] - rs[k]) <= tol, (k, st[k], rs[k])
    assert st["sparsity"] == rs["sparsity"]


@pytest.mark.parametrize("m,n,d,fp64", [(300, 700, 3, False), (1025, 130, 3, False), (1, 4, 3, False),
                                        (257, 515, 5, False), (300, 700, 3, True), (70, 1000, 2, True)])
def test_transfer_matches_oracle(S, h, oracle_mod, m, n, d, fp64):
    a, b, T, Y = _plan(40 + m + n, m, n)
    if d != 3:
        Y = np.random.default_rng(m).random((n, d))
    dt = torch.float64 if fp64 else torch.float32
    if not fp64:  # the oracle sees exactly the FP32 values
        a, b, T, Y = (np.asarray(v, dtype=np.float32).astype(np.float64) for v in (a, b, T, Y))
    prec = S.FP64 if fp64 else S.FP32
    Xh, st = h.transfer(dev(T, dt), Y=dev(Y, dt), a=dev(a, dt), b=dev(b, dt), precision=prec)
    _check(oracle_mod, Y, a, b, T, host(Xh), st, fp64)


def test_transfer_rows_without_mass(S, h, oracle_mod):
    m, n = 200, 300
    a, b, T, Y = _plan(9, m, n)
    T[::7] = 0.0
    a[::7] = 0.0
    a, b, T, Y = (np.asarray(v, dtype=np.float32).astype(np.float64) for v in (a, b, T, Y))
    Xh, st = h.transfer(dev(T, torch.float32), Y=dev(Y, torch.float32), a=dev(a, torch.float32),
                        b=dev(b, torch.float32), precision=S.FP32)
    Xh = host(Xh)
    assert np.all(Xh[::7] == 0.0)
    _check(oracle_mod, Y, a, b, T, Xh, st, False)


def test_transfer_on_a_solved_plan(S, h, oracle_mod):
    inst = W.colour_instance(77, 400, 500, rho=10.0, b_dirichlet=True).rounded()
    T = torch.zeros((inst.m, inst.n), dtype=torch.float32, device="cuda")
    h.solve(dev(inst.a, torch.float32), dev(inst.b, torch.float32), T, X=dev(inst.X, torch.float32),
            Y=dev(inst.Y, torch.float32), precision=S.FP32, variant=S.BCPFW, step=S.ELS, rho=inst.rho,
            tol_rel_gap=1e-6, max_epochs=5000)
    Xh, st = h.transfer(T, Y=dev(inst.Y, torch.float32), a=dev(inst.a, torch.float32),
                        b=dev(inst.b, torch.float32), precision=S.FP32)
    _check(oracle_mod, inst.Y, inst.a, inst.b, host(T), host(Xh), st, False)
    assert st["sparsity"] > 0.99  # a converged plan keeps few atoms per row


def test_transfer_projection_or_stats_alone(S, h, oracle_mod):
    a, b, T, Y = _plan(11, 90, 150)
    a, b, T, Y = (np.asarray(v, dtype=np.float32).astype(np.float64) for v in (a, b, T, Y))
    Td = dev(T, torch.float32)
    Xh, st = h.transfer(Td, Y=dev(Y, torch.float32), stats=False, precision=S.FP32)
    assert st is None
    np.testing.assert_allclose(host(Xh), oracle_mod.barycentric(Y, T), rtol=0, atol=2e-6)
    Xh2, st2 = h.transfer(Td, a=dev(a, torch.float32), b=dev(b, torch.float32), projection=False,
                          precision=S.FP32)
    assert Xh2 is None
    assert st2["sparsity"] == oracle_mod.transfer_stats(a, b, T)["sparsity"]


def test_transfer_rejects(S, h):
    T = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    o = S.options(precision=S.FP32)
    stt = S.TransferStats()
    Xh = torch.empty((4, 3), dtype=torch.float32, device="cuda")
    assert S.lib.sr_ot_transfer(h._h, o, 4, 4, 3, None, None, None, S._ptr(T), S._ptr(Xh), None) == S.EINVAL
    assert S.lib.sr_ot_transfer(h._h, o, 4, 4, 3, None, None, None, S._ptr(T), None, stt) == S.EINVAL
    assert S.lib.sr_ot_transfer(h._h, o, 0, 4, 3, None, None, None, S._ptr(T), None, None) == S.EINVAL


def test_transfer_full_size_sampled(S, h, oracle_mod):
    """2048 x 2048 (one instance of the batch workload's size): sampled rows
    of the projection against the oracle row by row, statistics against FP64
    sums of the whole plan."""
    m = n = 2048
    a, b, T, Y = _plan(5, m, n, support=4)
    a, b, T, Y = (np.asarray(v, dtype=np.float32).astype(np.float64) for v in (a, b, T, Y))
    Xh, st = h.transfer(dev(T, torch.float32), Y=dev(Y, torch.float32), a=dev(a, torch.float32),
                        b=dev(b, torch.float32), precision=S.FP32)
    Xh = host(Xh)
    rows = np.random.default_rng(3).choice(m, 24, replace=False)
    ref = oracle_mod.barycentric(Y, T[rows])
    assert np.abs(Xh[rows] - ref).max() <= 2e-6 * np.abs(ref).max()
    rs = oracle_mod.transfer_stats(a, b, T)
    for k in ("row_err", "col_err", "e_c"):
        assert abs(st[k] - rs[k]) <= 2e-6 * (np.linalg.norm(a) + np.linalg.norm(b)), k
    assert st["sparsity"] == rs["sparsity"]


def test_transfer_batched_matches_per_instance(S, h, oracle_mod):
    """One packed pass over uneven instances gives each instance's projection
    and statistics (compared with the oracle instance by instance)."""
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = [W.colour_instance(90 + k, m, n, rho=10.0, b_dirichlet=True).rounded()
             for k, (m, n) in enumerate([(130, 70), (1, 5), (600, 257), (64, 1100)])]
    pb = PackedBatch(insts)
    plans = []
    for k, inst in enumerate(insts):
        a, b, T, _ = _plan(60 + k, inst.m, inst.n, support=3)
        T = np.asarray(T * (inst.a / a)[:, None], dtype=np.float32).astype(np.float64)  # rows sum to inst.a
        pb.plan(k).copy_(dev(T, torch.float32))
        plans.append(T)
    Xh, stats = h.transfer_batched(pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, precision=S.FP32,
                                   xhat_numel=pb.X.numel())
    Xh = host(Xh)
    for k, inst in enumerate(insts):
        ox = pb.offsets[k][0]
        got = Xh[ox:ox + inst.m * 3].reshape(inst.m, 3)
        ref = oracle_mod.barycentric(inst.Y, plans[k])
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), k
        rs = oracle_mod.transfer_stats(inst.a, inst.b, plans[k])
        tol = 2e-6 * (np.linalg.norm(inst.a) + np.linalg.norm(inst.b))
        for key in ("row_err", "col_err", "e_c"):
            assert abs(stats[k][key] - rs[key]) <= tol, (k, key)
        assert stats[k]["sparsity"] == rs["sparsity"], k
