"""Adjoint kernels (sr_ot_grad, sr_ot_grad_batched) and the autograd wrappers
against the FP64 oracle.

The oracle's envelope-theorem gradients are pinned on the CPU (central
finite differences of converged FP64 solves); here the GPU adjoint is compared
with them on the same plans, element by element at sizes that span several
256-column tiles and 64-row chunks with ragged tails, on sampled rows and
columns at the 64 x 2048 x 2048 batch size, and by finite differences of the
optimal value through the FP64 solver.
"""
import numpy as np
import pytest
import torch

from paper_2103_05857_gb300 import workloads as W

from .gpu_util import dev, f32, host

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


def dense_plan(seed, a, n, support):
    r, c, v = W.feasible_plan(seed, a, n, support)
    T = np.zeros((len(a), n))
    T[r, c] = v
    return T


def relnorm(x, ref):
    return np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300)


def points(seed, m, n, d):
    if d == 3:
        inst = W.colour_instance(seed, m, n, rho=10.0, b_dirichlet=True)
        return inst.X, inst.Y, inst.a, inst.b
    X = W.normal(seed, 30, m * d).reshape(m, d)
    Y = W.normal(seed, 31, n * d).reshape(n, d)
    return X, Y, np.full(m, 1.0 / m), W.dirichlet_weights(seed + 1, n)


@pytest.mark.parametrize("m,n,d", [(300, 700, 3), (129, 257, 1), (70, 300, 5), (65, 513, 12), (40, 90, 20)])
def test_grad_fp64_matches_oracle(S, h, oracle_mod, m, n, d):
    X, Y, a, b = points(11 + d, m, n, d)
    T = dense_plan(5, a, n, 6)
    rho = 7.5
    dX0, dY0, db0 = oracle_mod.adjoint(X, Y, b, rho, T)
    out = h.grad(dev(T, torch.float64), X=dev(X, torch.float64), Y=dev(Y, torch.float64),
                 b=dev(b, torch.float64), want=("dC", "dX", "dY", "db"), precision=S.FP64, rho=rho)
    assert np.array_equal(host(out["dC"]), T)  # dC = T exactly
    for got, ref in ((out["dX"], dX0), (out["dY"], dY0), (out["db"], db0)):
        g = host(got)
        assert g.shape == ref.shape
        # FP64 with a different summation order: a few ulps of the largest term
        assert np.abs(g - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1.0)


@pytest.mark.parametrize("m,n,d", [(300, 700, 3), (1000, 1500, 3), (33, 1025, 7)])
def test_grad_fp32_matches_oracle(S, h, oracle_mod, m, n, d):
    X, Y, a, b = (f32(v) for v in points(3 + d, m, n, d))
    T = f32(dense_plan(9, a, n, 8))
    rho = 10.0
    dX0, dY0, db0 = oracle_mod.adjoint(X, Y, b, rho, T)
    out = h.grad(dev(T, torch.float32), X=dev(X, torch.float32), Y=dev(Y, torch.float32),
                 b=dev(b, torch.float32), precision=S.FP32, rho=rho)
    # FP32 partial sums (<= 1024 terms) reduced in FP64: well inside 1e-4
    assert relnorm(host(out["dX"]), dX0) <= 1e-5
    assert relnorm(host(out["dY"]), dY0) <= 1e-5
    assert relnorm(host(out["db"]), db0) <= 1e-5


def test_grad_skips_outputs_and_rejects_bad_args(S, h):
    m, n = 10, 20
    T = torch.full((m, n), 1.0 / (m * n), dtype=torch.float32, device="cuda")
    b = torch.full((n,), 1.0 / n, dtype=torch.float32, device="cuda")
    out = h.grad(T, b=b, want=("db",), precision=S.FP32, rho=2.0)
    assert torch.allclose(out["db"], torch.zeros_like(b), atol=1e-7)
    with pytest.raises(S.SrOtError):
        h.grad(T, want=("dX",), precision=S.FP32, rho=1.0)  # no points
    X = torch.zeros((m, 40), device="cuda")
    Y = torch.zeros((n, 40), device="cuda")
    with pytest.raises(S.SrOtError):
        h.grad(T, X=X, Y=Y, want=("dX",), precision=S.FP32, rho=1.0)  # d > 31


def test_grad_batched_matches_oracle(S, h, oracle_mod):
    from paper_2103_05857_gb300.batch import PackedBatch
    rng = np.random.default_rng(4)
    insts = []
    for k in range(13):
        m, n = (int(v) for v in rng.integers(1, 600, 2))
        insts.append(W.colour_instance(700 + k, m, n, rho=10.0, b_dirichlet=bool(k % 2)).rounded())
    pb = PackedBatch(insts)
    plans = [f32(dense_plan(40 + k, inst.a, inst.n, 5)) for k, inst in enumerate(insts)]
    for k, P in enumerate(plans):
        pb.plan(k).copy_(torch.as_tensor(P, dtype=torch.float32))
    out = h.grad_batched(pb.X, pb.Y, pb.b, pb.T, pb.sizes, pb.offsets, rho=10.0, precision=S.FP32)
    dX, dY, db = host(out["dX"]), host(out["dY"]), host(out["db"])
    for k, inst in enumerate(insts):
        oX, oY, _, ob, _ = pb.offsets[k]
        rX, rY, rb = oracle_mod.adjoint(inst.X, inst.Y, inst.b, 10.0, plans[k])
        assert relnorm(dX[oX:oX + inst.m * 3].reshape(-1, 3), rX) <= 1e-5, k
        assert relnorm(dY[oY:oY + inst.n * 3].reshape(-1, 3), rY) <= 1e-5, k
        assert relnorm(db[ob:ob + inst.n], rb) <= 1e-5, k


def test_grad_batched_full_size_sampled(S, h, oracle_mod):
    """64 instances of 2048 x 2048 (1 GiB of FP32 plans) in the launch
    configuration of the differentiable workload; 16 sampled rows and columns
    per instance are recomputed by the oracle on slices of the plan."""
    insts = [i.rounded() for i in W.workload("colour_batch64_2048")]
    from paper_2103_05857_gb300.batch import PackedBatch
    pb = PackedBatch(insts)
    m = n = 2048
    sparse = []
    for k, inst in enumerate(insts):
        r, c, v = W.feasible_plan(90 + k, inst.a, n, 8)
        v = f32(v)
        sparse.append((r, c, v))
        P = pb.plan(k)
        P.zero_()
        P[torch.as_tensor(r, device="cuda"), torch.as_tensor(c, device="cuda")] = torch.as_tensor(
            v, dtype=torch.float32, device="cuda")
    out = h.grad_batched(pb.X, pb.Y, pb.b, pb.T, pb.sizes, pb.offsets, rho=10.0, precision=S.FP32)
    dX, dY, db = host(out["dX"]), host(out["dY"]), host(out["db"])
    rng = np.random.default_rng(0)
    for k in range(0, 64, 7):
        inst = insts[k]
        r, c, v = sparse[k]
        T = np.zeros((m, n))
        T[r, c] = v
        oX, oY, _, ob, _ = pb.offsets[k]
        for i in rng.choice(m, 16, replace=False):
            rX, _, _ = oracle_mod.adjoint(inst.X[i:i + 1], inst.Y, inst.b, 10.0, T[i:i + 1])
            got = dX[oX + 3 * i:oX + 3 * i + 3]
            assert np.abs(got - rX[0]).max() <= 1e-5 * np.abs(rX).max() + 1e-9, (k, i)
        for j in rng.choice(n, 16, replace=False):
            _, rY, rb = oracle_mod.adjoint(inst.X, inst.Y[j:j + 1], inst.b[j:j + 1], 10.0, T[:, j:j + 1])
            got = dY[oY + 3 * j:oY + 3 * j + 3]
            assert np.abs(got - rY[0]).max() <= 1e-5 * np.abs(rY).max() + 1e-9, (k, j)
            assert abs(db[ob + j] - rb[0]) <= 1e-5 * abs(rb[0]) + 1e-9, (k, j)


def test_grad_matches_finite_differences_of_the_optimal_value(S, h, oracle_mod):
    """Envelope theorem end to end: the adjoint at the GPU's converged FP64
    plan against central differences (h = 1e-4) of the oracle's FP64 optimal
    value, on random coordinates of X, Y and b."""
    inst = W.colour_instance(321, 12, 15, rho=10.0, b_dirichlet=True)
    T = torch.zeros((12, 15), dtype=torch.float64, device="cuda")
    dv = lambda x: dev(x, torch.float64)
    res = h.solve(dv(inst.a), dv(inst.b), T, X=dv(inst.X), Y=dv(inst.Y), precision=S.FP64,
                  variant=S.BCPFW, step=S.ELS, rho=inst.rho, tol_rel_gap=1e-14, max_epochs=200000)
    assert res["rel_gap"] <= 1e-12
    out = h.grad(T, X=dv(inst.X), Y=dv(inst.Y), b=dv(inst.b), precision=S.FP64, rho=inst.rho)

    def value(X, Y, b):
        C = oracle_mod.cost(X, Y)
        _, r, *_ = oracle_mod.solve(C, inst.a, b, rho=inst.rho, variant=oracle_mod.BCPFW,
                                    step=oracle_mod.ELS, max_epochs=200000, tol_rel_gap=1e-14)
        return r["f"]

    hh = 1e-4
    rng = np.random.default_rng(1)
    checked = 0
    for which in ("X", "Y", "b"):
        for _ in range(4):
            X, Y, b = inst.X.copy(), inst.Y.copy(), inst.b.copy()
            arr = {"X": X, "Y": Y, "b": b}[which]
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            arr[idx] += hh
            fp = value(X, Y, b)
            arr[idx] -= 2 * hh
            fm = value(X, Y, b)
            fd = (fp - fm) / (2 * hh)
            g = host(out["d" + which])[idx]
            assert abs(g - fd) <= 1e-4 * max(abs(fd), 1e-3), (which, idx, g, fd)
            checked += 1
    assert checked == 12


def test_autograd_function(S, h):
    from paper_2103_05857_gb300.autograd import semi_relaxed_ot
    inst = W.colour_instance(55, 60, 80, rho=10.0).rounded()
    X = dev(inst.X, torch.float32).requires_grad_(True)
    Y = dev(inst.Y, torch.float32).requires_grad_(True)
    b = dev(inst.b, torch.float32).requires_grad_(True)
    a = dev(inst.a, torch.float32)
    kw = dict(variant=S.BCPFW, step=S.ELS, rho=10.0, tol_rel_gap=1e-7, max_epochs=20000)
    val = semi_relaxed_ot(X, Y, a, b, h, **kw)
    (3.0 * val).backward()
    T = torch.zeros((60, 80), dtype=torch.float32, device="cuda")
    h.solve(a, b.detach(), T, X=X.detach(), Y=Y.detach(), precision=S.FP32, **kw)
    ref = h.grad(T, X=X.detach(), Y=Y.detach(), b=b.detach(), precision=S.FP32, rho=10.0)
    assert torch.allclose(X.grad, 3.0 * ref["dX"], rtol=1e-6, atol=1e-9)
    assert torch.allclose(Y.grad, 3.0 * ref["dY"], rtol=1e-6, atol=1e-9)
    assert torch.allclose(b.grad, 3.0 * ref["db"], rtol=1e-6, atol=1e-9)
    # a few gradient steps on X decrease the optimal value
    Xv = X.detach().clone()
    vals = []
    for _ in range(5):
        Xv.requires_grad_(True)
        v = semi_relaxed_ot(Xv, Y.detach(), a, b.detach(), h, **kw)
        v.backward()
        vals.append(float(v))
        Xv = (Xv - 0.5 * Xv.grad).detach()
    assert vals[-1] < vals[0]


def test_autograd_batched(S, h):
    from paper_2103_05857_gb300.autograd import SemiRelaxedOTBatched
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = [W.colour_instance(900 + k, 50 + 10 * k, 70 - 5 * k, rho=10.0).rounded() for k in range(5)]
    pb = PackedBatch(insts)
    X = pb.X.clone().requires_grad_(True)
    kw = dict(variant=S.BCPFW, step=S.ELS, rho=10.0, tol_rel_gap=1e-7, max_epochs=20000)
    vals = SemiRelaxedOTBatched.apply(X, pb.Y, pb.b, pb.a, pb.sizes, pb.offsets, h, kw)
    w = torch.arange(1, 6, dtype=torch.float32, device="cuda")
    (vals * w).sum().backward()
    T = torch.zeros(pb.total_T, dtype=torch.float32, device="cuda")
    h.solve_batched(pb.X, pb.Y, pb.a, pb.b, T, pb.sizes, pb.offsets, **kw)
    ref = h.grad_batched(pb.X, pb.Y, pb.b, T, pb.sizes, pb.offsets, rho=10.0, precision=S.FP32)
    for k in range(5):
        oX = pb.offsets[k][0]
        sl = slice(oX, oX + 3 * insts[k].m)
        assert torch.allclose(X.grad[sl], (k + 1) * ref["dX"][sl], rtol=1e-6, atol=1e-9)


def test_autograd_uses_the_solves_rho(S, h, oracle_mod):
    """Without an explicit rho the forward solve runs the library default
    (rho = 10); backward must differentiate that same problem, so db equals
    -10 (T^T 1 - b) at the returned plan (the oracle's adjoint at rho = 10),
    and an `opts=` struct carries its rho through as well."""
    from paper_2103_05857_gb300.autograd import semi_relaxed_ot
    inst = W.colour_instance(57, 40, 50, b_dirichlet=True).rounded()
    a = dev(inst.a, torch.float32)
    for kw in (dict(variant=S.BCPFW, step=S.ELS, tol_rel_gap=1e-7, max_epochs=20000),
               dict(opts=S.options(variant=S.BCPFW, step=S.ELS, tol_rel_gap=1e-7, max_epochs=20000,
                                   rho=3.0, precision=S.FP32))):
        rho = 3.0 if "opts" in kw else 10.0
        b = dev(inst.b, torch.float32).requires_grad_(True)
        X = dev(inst.X, torch.float32).requires_grad_(True)
        Y = dev(inst.Y, torch.float32)
        val = semi_relaxed_ot(X, Y, a, b, h, **kw)
        val.backward()
        T = torch.zeros((inst.m, inst.n), dtype=torch.float32, device="cuda")
        h.solve(a, b.detach(), T, X=X.detach(), Y=Y, precision=S.FP32, rho=rho, variant=S.BCPFW, step=S.ELS,
                tol_rel_gap=1e-7, max_epochs=20000)
        dXo, _, dbo = oracle_mod.adjoint(inst.X, inst.Y, inst.b, rho, host(T))
        np.testing.assert_allclose(host(b.grad), dbo, rtol=1e-4, atol=1e-7 * rho)
        np.testing.assert_allclose(host(X.grad), dXo, rtol=1e-4, atol=1e-6)


def test_autograd_refuses_point_gradients_of_the_euclidean_cost(S, h):
    """The adjoint formula for dX, dY is that of the squared cost; a forward
    solve on the Euclidean cost must not be given it: backward carries the
    solve's cost kind to sr_ot_grad, which refuses."""
    from paper_2103_05857_gb300.autograd import semi_relaxed_ot
    inst = W.colour_instance(58, 30, 40).rounded()
    X = dev(inst.X, torch.float32).requires_grad_(True)
    val = semi_relaxed_ot(X, dev(inst.Y, torch.float32), dev(inst.a, torch.float32), dev(inst.b, torch.float32),
                          h, variant=S.BCPFW, step=S.ELS, tol_rel_gap=1e-6, max_epochs=5000,
                          cost_kind=S.COST_EUCLIDEAN)
    with pytest.raises(S.SrOtError) as e:
        val.backward()
    assert e.value.status == S.EUNSUPPORTED
