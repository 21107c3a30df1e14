"""sr_ot_gap_noalloc: the duality-gap certificate for callers that cannot
allocate memory (code inside a CUDA graph capture or under a caller-owned
memory pool, embedded runtimes that own every allocation, real-time loops).

It has no handle and runs on a fixed scratch array compiled into the
library, so these checks call it through the C ABI and compare it with
sr_ot_gap (which uses a handle's workspace) on two calls in a row with
different inputs, then check that a size beyond the scratch is rejected.
The file sorts last so a run that stops at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2103_05857_gb300 import workloads as W

from .gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu


def _plan(seed, a, n):
    rng = np.random.default_rng(seed)
    m = len(a)
    T = rng.random((m, n)) * (rng.random((m, n)) < 0.3)
    T[np.arange(m), rng.integers(0, n, m)] += 0.5
    return T / T.sum(1, keepdims=True) * a[:, None]


def test_noalloc_certificate_matches_handle_path():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_05857_gb300 import sr_ot as S

    h = S.Handle(0)
    stream = torch.cuda.current_stream(0)
    cases = [(1, 300, 517, S.FP32, "pts"), (2, 1000, 777, S.FP32, "C"), (3, 64, 96, S.FP64, "pts")]
    for seed, m, n, prec, mode in cases:
        dt = torch.float64 if prec == S.FP64 else torch.float32
        inst = W.colour_instance(seed, m, n, rho=10.0, b_dirichlet=True).rounded()
        T = dev(_plan(seed, inst.a, n), dt)
        a, b = dev(inst.a, dt), dev(inst.b, dt)
        if mode == "C":
            Xh, Yh = inst.X, inst.Y
            C = dev(((Xh[:, None, :] - Yh[None, :, :]) ** 2).sum(-1), dt)
            kw = dict(C=C)
            ptrs = (C.data_ptr(), None, None, 0)
        else:
            X, Y = dev(inst.X, dt), dev(inst.Y, dt)
            kw = dict(X=X, Y=Y)
            ptrs = (None, X.data_ptr(), Y.data_ptr(), 3)
        g_ref = torch.empty(m, dtype=torch.float64, device="cuda")
        ref = h.gap(a, b, T, g_rows=g_ref, precision=prec, rho=inst.rho, **kw)

        opts = S.options(precision=prec, rho=inst.rho)
        g_rows = torch.empty(m, dtype=torch.float64, device="cuda")
        res = S.Result()
        st = S.lib.sr_ot_gap_noalloc(0, ct.c_void_p(stream.cuda_stream), ct.byref(opts), m, n,
                                     ptrs[3], ptrs[0], ptrs[1], ptrs[2], a.data_ptr(), b.data_ptr(),
                                     T.data_ptr(), g_rows.data_ptr(), ct.byref(res))
        assert st == S.OK, S.lib.sr_ot_last_error(None)
        # same kernels and fixed-order reductions: the certificate tolerances
        # of the other tests (1e-12 relative) are met, in fact exactly
        assert rel(res.objective, ref["objective"]) <= 1e-12
        assert abs(res.gap - ref["gap"]) <= 1e-12 * abs(ref["objective"])
        assert abs(res.dual - ref["dual"]) <= 1e-12 * abs(ref["objective"])
        np.testing.assert_allclose(host(g_rows), host(g_ref), rtol=1e-12, atol=1e-18)

    # beyond the fixed scratch: a clear error, no allocation attempted
    m, n = 2, 250_000
    a = torch.full((m,), 0.5, device="cuda")
    b = torch.full((n,), 1.0 / n, device="cuda")
    C = torch.zeros((m, n), device="cuda")
    T = torch.zeros((m, n), device="cuda")
    res = S.Result()
    opts = S.options(precision=S.FP32)
    st = S.lib.sr_ot_gap_noalloc(0, ct.c_void_p(stream.cuda_stream), ct.byref(opts), m, n, 0,
                                 C.data_ptr(), None, None, a.data_ptr(), b.data_ptr(), T.data_ptr(),
                                 None, ct.byref(res))
    assert st == S.EUNSUPPORTED
    assert b"scratch" in S.lib.sr_ot_last_error(None)

    # the Euclidean cost is not built from points here (it would need a
    # buffer): rejected, not silently replaced by the squared one
    m, n = 8, 12
    X = torch.rand((m, 3), device="cuda")
    Y = torch.rand((n, 3), device="cuda")
    a = torch.full((m,), 1.0 / m, device="cuda")
    b = torch.full((n,), 1.0 / n, device="cuda")
    T = torch.zeros((m, n), device="cuda")
    opts = S.options(precision=S.FP32, cost_kind=S.COST_EUCLIDEAN)
    st = S.lib.sr_ot_gap_noalloc(0, ct.c_void_p(stream.cuda_stream), ct.byref(opts), m, n, 3, None,
                                 X.data_ptr(), Y.data_ptr(), a.data_ptr(), b.data_ptr(), T.data_ptr(),
                                 None, ct.byref(res))
    assert st == S.EUNSUPPORTED
    h.close()
