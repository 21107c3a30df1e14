"""Batched persistent solves (sr_ot_solve_batched) against the FP64 oracle.

Each instance's returned plan is certified independently by the oracle
(Thm 2 in FP64 on the GPU's plan), converged objectives are compared with the
oracle's converged objective (the optimal value is unique), and a decay-rule
batch is compared epoch for epoch with the oracle's trajectory.
"""
import numpy as np
import pytest
import torch

from paper_2103_05857_gb300 import workloads as W

from .gpu_util import host, rel

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


def make_batch(seed, count, lo, hi, rho=10.0):
    rng = np.random.default_rng(seed)
    insts = []
    for k in range(count):
        m, n = (int(v) for v in rng.integers(lo, hi + 1, 2))
        insts.append(W.colour_instance(seed * 1000 + k, m, n, rho=rho, b_dirichlet=bool(k % 2)).rounded())
    return insts


# kernels: AUTO takes the batched speculative form for pairwise steps in
# cyclic or uniform order; TWO_PHASE keeps the persistent two-phase kernel
@pytest.mark.parametrize("variant,order,kernel", [("BCPFW", "CYCLIC", "AUTO"), ("BCPFW", "CYCLIC", "TWO_PHASE"),
                                                  ("BCPFW", "UNIFORM", "AUTO"), ("BCAFW", "UNIFORM", "AUTO"),
                                                  ("BCPFW", "PERMUTE", "AUTO")])
def test_batched_converges_to_oracle_optimum(S, h, oracle_mod, variant, order, kernel):
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = make_batch(7, 9, 20, 300)
    pb = PackedBatch(insts)
    st, res = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets,
                              variant=getattr(S, variant), step=S.ELS, order=getattr(S, order),
                              seed=5, rho=10.0, tol_rel_gap=1e-6, max_epochs=20000,
                              epoch_kernel=getattr(S, "EPOCH_" + kernel))
    assert st == S.OK
    for k, inst in enumerate(insts):
        r = res[k]
        assert r["status"] == S.OK and r["rel_gap"] <= 1e-6, (k, r)
        C = oracle_mod.cost(inst.X, inst.Y)
        Tg = host(pb.plan(k))
        cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, Tg)
        # the in-kernel certificate agrees with the oracle's on the same plan
        assert rel(r["objective"], cert["f"]) <= 2e-7
        assert abs(r["gap"] - cert["g"]) <= 2e-7 * cert["f"]
        assert cert["g"] <= 1.5e-6 * cert["f"]
        assert Tg.min() >= 0.0
        np.testing.assert_allclose(Tg.sum(1), inst.a, rtol=2e-5)
        # the optimum is unique: f(T) - f* <= g(T)
        _, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCPFW,
                                     step=oracle_mod.ELS, max_epochs=40000, tol_rel_gap=1e-10,
                                     gap_every=20)
        assert cert["f"] - ro["f"] <= cert["g"] + 1e-12
        assert rel(cert["f"], ro["f"]) <= 1e-5


def test_batched_decay_rule_trajectory(S, h, oracle_mod):
    """BCFW with the decay rule: each instance's plan after 6 epochs matches the
    oracle's trajectory. Decay-rule supports grow, so some rows outgrow their
    atom records and those instances are finished on the dense path."""
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = make_batch(11, 6, 30, 200)
    pb = PackedBatch(insts)
    st, res = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets,
                              variant=S.BCFW, step=S.DEC, rho=10.0, max_epochs=6)
    assert st == S.OK
    for k, inst in enumerate(insts):
        C = oracle_mod.cost(inst.X, inst.Y)
        To, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCFW,
                                      step=oracle_mod.DEC, max_epochs=6)
        assert rel(res[k]["objective"], ro["f"]) <= 1e-5
        assert np.abs(host(pb.plan(k)) - To).max() <= 1e-6


@pytest.mark.parametrize("kernel", ["AUTO", "TWO_PHASE"])
def test_batched_oversize_and_replay(S, h, oracle_mod, kernel):
    """An instance wider than the batched widths (n = 2600 > 2048 for the
    two-phase kernel, n = 5000 > 4096 for the speculative form) is solved on
    the single-instance path; a second call with the same shapes (replaying
    the captured graph of the two-phase kernel) gives the same results."""
    from paper_2103_05857_gb300.batch import PackedBatch
    wide = 2600 if kernel == "TWO_PHASE" else 5000
    insts = make_batch(3, 4, 50, 150) + [W.colour_instance(99, 40, wide, rho=10.0).rounded()]
    pb = PackedBatch(insts)
    kw = dict(variant=S.BCPFW, step=S.ELS, rho=10.0, max_epochs=25, epoch_kernel=getattr(S, "EPOCH_" + kernel))
    st1, r1 = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, **kw)
    T1 = pb.T.clone()
    st2, r2 = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, **kw)
    assert st1 == st2 == S.OK
    assert torch.equal(T1, pb.T)
    for k, inst in enumerate(insts):
        assert r1[k]["objective"] == r2[k]["objective"]
        C = oracle_mod.cost(inst.X, inst.Y)
        cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, host(pb.plan(k)))
        assert rel(r1[k]["objective"], cert["f"]) <= 2e-7
        assert r1[k]["epochs"] == 25


def test_batched_rejects_bad_input(S, h):
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = make_batch(5, 3, 20, 60)
    insts[1].a[3] = -0.1
    pb = PackedBatch(insts)
    with pytest.raises(S.SrOtError) as ei:
        h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, variant=S.BCPFW,
                        step=S.ELS, max_epochs=2)
    assert ei.value.status == S.EINVAL and "instance 1" in str(ei.value)


def test_batched_instance_turning_non_finite_is_isolated(S, h, oracle_mod):
    """One instance of a batch has a source point so far out (2e19 in each
    coordinate, finite and accepted by the input checks) that its squared
    cost overflows FP32: the first time its last row is updated (mid-way
    through its first epoch) the gradient is not finite. That instance alone
    gets SR_OT_ENUMERIC; every other instance converges and is certified by
    the oracle, and the call returns the worst status."""
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = make_batch(13, 6, 40, 200)
    insts[2].X[-1] = 2e19
    pb = PackedBatch(insts)
    st, res = h.solve_batched_raw(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, variant=S.BCPFW,
                                  step=S.ELS, rho=10.0, tol_rel_gap=1e-6, max_epochs=20000)
    assert st == S.ENUMERIC
    assert res[2]["status"] == S.ENUMERIC
    for k, inst in enumerate(insts):
        if k == 2:
            continue
        r = res[k]
        assert r["status"] == S.OK and r["rel_gap"] <= 1e-6, (k, r)
        C = oracle_mod.cost(inst.X, inst.Y)
        cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, host(pb.plan(k)))
        assert cert["g"] <= 1.5e-6 * cert["f"]
    # the handle stays usable: the same batch without the far point solves
    insts[2].X[-1] = 0.5
    pb2 = PackedBatch(insts)
    st, res = h.solve_batched(pb2.X, pb2.Y, pb2.a, pb2.b, pb2.T, pb2.sizes, pb2.offsets, variant=S.BCPFW,
                              step=S.ELS, rho=10.0, tol_rel_gap=1e-6, max_epochs=20000)
    assert st == S.OK and all(r["status"] == S.OK for r in res)


# every size bucket of the two-phase batched kernel (n <= 256, 512, 1024, 2048;
# the speculative form takes them all in its 2048-column tile), two instances
# each, with m across the whole range of the colour_batch512 workload
FULL_SIZES = [(300, 250), (1900, 256), (700, 500), (2048, 511), (1500, 1000), (400, 1024),
              (2048, 2048), (1200, 1900)]


@pytest.mark.parametrize("kernel", ["AUTO", "TWO_PHASE"])
def test_batched_every_bucket_at_workload_sizes(S, h, oracle_mod, kernel):
    """Instances in every size bucket up to n = 2048 (the sizes of the
    colour_batch512 workload), solved in one batched call to rel. gap 1e-6.
    Each returned plan is certified by the oracle (FP64, Thm 2): its gap is at
    most 1.5e-6 of its objective, so its objective is within that of the
    optimum; for the smaller instances the oracle's own converged optimum is
    compared as well (f* is unique)."""
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = [W.colour_instance(4100 + k, m, n, rho=10.0, b_dirichlet=bool(k % 2)).rounded()
             for k, (m, n) in enumerate(FULL_SIZES)]
    pb = PackedBatch(insts)
    st, res = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, variant=S.BCPFW,
                              step=S.ELS, rho=10.0, tol_rel_gap=1e-6, max_epochs=20000,
                              epoch_kernel=getattr(S, "EPOCH_" + kernel))
    assert st == S.OK
    for k, inst in enumerate(insts):
        r = res[k]
        assert r["status"] == S.OK and r["rel_gap"] <= 1e-6, (k, r)
        C = oracle_mod.cost(inst.X, inst.Y)
        Tg = host(pb.plan(k))
        cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, Tg)
        assert rel(r["objective"], cert["f"]) <= 2e-7
        assert abs(r["gap"] - cert["g"]) <= 2e-7 * cert["f"]
        assert cert["g"] <= 1.5e-6 * cert["f"], (k, cert["g"] / cert["f"])
        assert Tg.min() >= 0.0
        np.testing.assert_allclose(Tg.sum(1), inst.a, rtol=2e-5)
        if inst.m * inst.n <= 600_000:
            _, ro, *_ = oracle_mod.solve(C, inst.a, inst.b, rho=inst.rho, variant=oracle_mod.BCPFW,
                                         step=oracle_mod.ELS, max_epochs=40000, tol_rel_gap=1e-10,
                                         gap_every=20)
            assert cert["f"] - ro["f"] <= cert["g"] + 1e-12
            assert rel(cert["f"], ro["f"]) <= 2e-6


def test_batched_warm_start(S, h, oracle_mod):
    """batch_warm_start: every instance starts from the plan the caller left
    in T. (1) From the converged plans of a cold call the certificate after
    one epoch already meets the tolerance and the objectives agree. (2) After
    the source points move a little (one gradient step on X), the warm solves
    reach the new optima -- certified by the oracle -- in fewer epochs in total
    than cold ones. (3) A plan with a row of 70 atoms (beyond the 63 of a record)
    is finished on the dense path from that plan, and still converges."""
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = make_batch(17, 6, 60, 400)
    pb = PackedBatch(insts)
    kw = dict(variant=S.BCPFW, step=S.ELS, rho=10.0, tol_rel_gap=1e-6, max_epochs=20000)
    st, cold = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, **kw)
    assert st == S.OK
    st, warm = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, batch_warm_start=1, **kw)
    assert st == S.OK
    for c, w in zip(cold, warm):
        assert w["epochs"] <= 10 and w["status"] == S.OK
        assert rel(w["objective"], c["objective"]) <= 2e-6
    # a gradient step on X (towards the barycentric projection), then warm
    g = h.grad_batched(pb.X, pb.Y, pb.b, pb.T, pb.sizes, pb.offsets, rho=10.0, precision=S.FP32, want=("dX",))
    X2 = pb.X - 2.0 * g["dX"]  # x_i moves 4 a_i (<= 7 %) of the way to its barycentric projection
    T_warm = pb.T.clone()
    st, w2 = h.solve_batched(X2, pb.Y, pb.a, pb.b, T_warm, pb.sizes, pb.offsets, batch_warm_start=1, **kw)
    T_cold = torch.zeros_like(pb.T)
    st2, c2 = h.solve_batched(X2, pb.Y, pb.a, pb.b, T_cold, pb.sizes, pb.offsets, **kw)
    assert st == S.OK and st2 == S.OK
    X2h = X2.cpu().double().numpy()
    for k, inst in enumerate(insts):
        oX = pb.offsets[k][0]
        Xk = X2h[oX:oX + 3 * inst.m].reshape(inst.m, 3)
        C = oracle_mod.cost(Xk, inst.Y)
        oT = pb.offsets[k][4]
        Tk = T_warm[oT:oT + inst.m * inst.n].view(inst.m, inst.n)
        cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, host(Tk))
        assert cert["g"] <= 1.5e-6 * cert["f"], (k, cert["g"] / cert["f"])
    # fewer epochs in total (a single slowly converging instance may take a
    # few hundred more from a warm plan than from T0)
    we, ce = [r["epochs"] for r in w2], [r["epochs"] for r in c2]
    assert sum(we) < sum(ce), (we, ce)
    # a warm plan whose row 3 holds 70 atoms: the dense path takes that instance
    inst0 = insts[0]
    T3 = pb.T.clone()
    oT = pb.offsets[0][4]
    T0v = T3[oT:oT + inst0.m * inst0.n].view(inst0.m, inst0.n)
    T0v[3] = 0.0
    T0v[3, :70] = float(inst0.a[3]) / 70.0
    st, w3 = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, T3, pb.sizes, pb.offsets, batch_warm_start=1, **kw)
    assert st == S.OK and w3[0]["status"] == S.OK and w3[0]["rel_gap"] <= 1e-6
    C0 = oracle_mod.cost(inst0.X, inst0.Y)
    cert = oracle_mod.certificate(C0, inst0.a, inst0.b, inst0.rho, host(T3[oT:oT + inst0.m * inst0.n].view(inst0.m, inst0.n)))
    assert cert["g"] <= 1.5e-6 * cert["f"]


def test_batched_speculative_both_widths_at_once(S, h, oracle_mod):
    """The speculative form runs n <= 2048 and 2048 < n <= 4096 as two
    concurrent launches (2048- and 4096-column tiles); instances of both,
    in one call, are each certified by the oracle."""
    from paper_2103_05857_gb300.batch import PackedBatch
    sizes = [(500, 3000), (1200, 700), (300, 2100), (90, 4096), (700, 2048), (64, 65)]
    insts = [W.colour_instance(4200 + k, m, n, rho=10.0, b_dirichlet=bool(k % 2)).rounded()
             for k, (m, n) in enumerate(sizes)]
    pb = PackedBatch(insts)
    st, res = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, variant=S.BCPFW,
                              step=S.ELS, rho=10.0, tol_rel_gap=1e-6, max_epochs=20000)
    assert st == S.OK
    for k, inst in enumerate(insts):
        r = res[k]
        assert r["status"] == S.OK and r["rel_gap"] <= 1e-6, (k, r)
        Tg = host(pb.plan(k))
        cert = oracle_mod.certificate(oracle_mod.cost(inst.X, inst.Y), inst.a, inst.b, inst.rho, Tg)
        assert rel(r["objective"], cert["f"]) <= 2e-7
        assert abs(r["gap"] - cert["g"]) <= 2e-7 * cert["f"]
        assert cert["g"] <= 1.5e-6 * cert["f"], (k, cert["g"] / cert["f"])
        assert Tg.min() >= 0.0
        np.testing.assert_allclose(Tg.sum(1), inst.a, rtol=2e-5)


def test_batched_speculative_fixed_epochs_and_zero_epochs(S, h, oracle_mod):
    """Without a tolerance the batched speculative form runs exactly
    max_epochs epochs of every instance (uniform order here), and the
    reported certificate is the oracle's certificate of the returned plan;
    with max_epochs = 0 the plans stay at T0 = (a_i e_0) (Thm 1) and the
    certificate is that of T0."""
    from paper_2103_05857_gb300.batch import PackedBatch
    insts = make_batch(23, 7, 30, 700)
    for epochs in (0, 13):
        pb = PackedBatch(insts)
        st, res = h.solve_batched(pb.X, pb.Y, pb.a, pb.b, pb.T, pb.sizes, pb.offsets, variant=S.BCPFW,
                                  step=S.ELS, order=S.UNIFORM, seed=9, rho=10.0, max_epochs=epochs)
        assert st == S.OK
        for k, inst in enumerate(insts):
            r = res[k]
            assert r["epochs"] == epochs and r["block_updates"] == epochs * inst.m
            Tg = host(pb.plan(k))
            if epochs == 0:
                T0 = np.zeros((inst.m, inst.n))
                T0[:, 0] = inst.a
                assert np.array_equal(Tg, T0)
            C = oracle_mod.cost(inst.X, inst.Y)
            cert = oracle_mod.certificate(C, inst.a, inst.b, inst.rho, Tg)
            assert rel(r["objective"], cert["f"]) <= 2e-7
            assert abs(r["gap"] - cert["g"]) <= 2e-7 * cert["f"]
            assert Tg.min() >= 0.0
            np.testing.assert_allclose(Tg.sum(1), inst.a, rtol=2e-5)
