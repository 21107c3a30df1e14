"""sr_ot_gap_noalloc: the duality-gap certificate for callers that cannot
allocate device memory where they need it (an application whose caching
allocator has reserved the device up front, a plug-in inside a host program
that owns every allocation, a service that must not fail on fragmentation
after start-up).

It has no handle and runs on a fixed scratch array compiled into the
library, so these checks call it through the C ABI and compare it with the
FP64 oracle's certificate and with sr_ot_gap (which uses a handle's
workspace) on two calls in a row with different inputs, check that the
caller's current device is left as it was, that the documented size bound
holds at its edge, and that a size beyond the scratch is rejected. The file
sorts last so a run that stops at the first failure has already run every
other test; it also passes on its own in a fresh process.
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


def _call(S, stream, opts, m, n, d, C, X, Y, a, b, T, g_rows):
    res = S.Result()
    p = lambda t: None if t is None else t.data_ptr()
    st = S.lib.sr_ot_gap_noalloc(0, ct.c_void_p(stream.cuda_stream), ct.byref(opts), m, n, d, p(C), p(X),
                                 p(Y), p(a), p(b), p(T), p(g_rows), ct.byref(res))
    return st, res


def test_noalloc_certificate_matches_oracle_and_handle_path(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_05857_gb300 import sr_ot as S

    h = S.Handle(0)
    stream = torch.cuda.current_stream(0)
    dev0 = torch.cuda.current_device()
    cases = [(1, 300, 517, S.FP32, "pts"), (2, 1000, 777, S.FP32, "C"), (3, 64, 96, S.FP64, "pts")]
    for seed, m, n, prec, mode in cases:
        dt = torch.float64 if prec == S.FP64 else torch.float32
        inst = W.colour_instance(seed, m, n, rho=10.0, b_dirichlet=True).rounded()
        Tn = _plan(seed, inst.a, n)
        if dt == torch.float32:
            Tn = Tn.astype(np.float32).astype(np.float64)
        T = dev(Tn, dt)
        a, b = dev(inst.a, dt), dev(inst.b, dt)
        Co = oracle_mod.cost(inst.X, inst.Y)
        if mode == "C":
            if dt == torch.float32:
                Co = Co.astype(np.float32).astype(np.float64)
            C = dev(Co, dt)
            kw, ptrs = dict(C=C), (C, None, None, 0)
        else:
            X, Y = dev(inst.X, dt), dev(inst.Y, dt)
            kw, ptrs = dict(X=X, Y=Y), (None, X, Y, 3)
        ref = oracle_mod.certificate(Co, inst.a, inst.b, inst.rho, Tn)
        g_ref = torch.empty(m, dtype=torch.float64, device="cuda")
        hres = h.gap(a, b, T, g_rows=g_ref, precision=prec, rho=inst.rho, **kw)

        opts = S.options(precision=prec, rho=inst.rho)
        g_rows = torch.empty(m, dtype=torch.float64, device="cuda")
        st, res = _call(S, stream, opts, m, n, ptrs[3], ptrs[0], ptrs[1], ptrs[2], a, b, T, g_rows)
        assert st == S.OK, S.lib.sr_ot_last_error(None)
        assert torch.cuda.current_device() == dev0
        # against the oracle: the certificate tolerances of sr_ot_gap's own
        # parity tests (FP64 1e-13; FP32 points: one FP32 rounding per cost
        # entry, 2e-7 of f)
        ftol = 1e-13 if prec == S.FP64 else (1e-9 if mode == "C" else 2e-7)
        assert rel(res.objective, ref["f"]) <= ftol
        assert abs(res.gap - ref["g"]) <= max(ftol, 1e-12) * ref["f"]
        assert abs(res.dual - ref["w"]) <= max(ftol, 1e-12) * ref["f"]
        np.testing.assert_allclose(host(g_rows), ref["g_rows"], rtol=1e-4 if prec != S.FP64 else 1e-9,
                                   atol=1e-6 * ref["f"] / m if prec != S.FP64 else 1e-15)
        # against the handle path: same kernels and fixed-order reductions
        assert rel(res.objective, hres["objective"]) <= 1e-12
        assert abs(res.gap - hres["gap"]) <= 1e-12 * abs(hres["objective"])
        np.testing.assert_allclose(host(g_rows), host(g_ref), rtol=1e-12, atol=1e-18)

    # the Euclidean cost is not built from points here (it would need a
    # buffer): rejected, not silently replaced by the squared one
    m, n = 8, 12
    X = torch.rand((m, 3), device="cuda")
    Y = torch.rand((n, 3), device="cuda")
    a = torch.full((m,), 1.0 / m, device="cuda")
    b = torch.full((n,), 1.0 / n, device="cuda")
    T = torch.zeros((m, n), device="cuda")
    opts = S.options(precision=S.FP32, cost_kind=S.COST_EUCLIDEAN)
    st, _ = _call(S, stream, opts, m, n, 3, None, X, Y, a, b, T, None)
    assert st == S.EUNSUPPORTED
    assert torch.cuda.current_device() == dev0
    h.close()


def test_noalloc_size_bound(oracle_mod):
    """Every n <= 207,552 fits the fixed scratch for any m; the bound is
    reached once the row pass uses its largest grid (m >= 9,721). A size that
    needed two row chunks (m = 10,000, n = 150,000) now runs in one chunk and
    agrees with the handle path; n = 207,553 at m = 10,000 is refused."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_05857_gb300 import sr_ot as S

    stream = torch.cuda.current_stream(0)
    opts = S.options(precision=S.FP32, rho=10.0)
    m = 10_000
    rng = np.random.default_rng(5)
    for n, expect in ((150_000, S.OK), (207_552, S.OK), (207_553, S.EUNSUPPORTED)):
        X = torch.as_tensor(rng.random((m, 3)), dtype=torch.float32, device="cuda")
        Y = torch.as_tensor(rng.random((n, 3)), dtype=torch.float32, device="cuda")
        a = torch.full((m,), 1.0 / m, device="cuda")
        b = torch.full((n,), 1.0 / n, device="cuda")
        # one entry per row: T = a_i e_{j(i)}
        T = torch.zeros((m, n), dtype=torch.float32, device="cuda")
        cols = torch.as_tensor(rng.integers(0, n, m), device="cuda")
        T[torch.arange(m, device="cuda"), cols] = a
        st, res = _call(S, stream, opts, m, n, 3, None, X, Y, a, b, T, None)
        assert st == expect, (n, S.lib.sr_ot_last_error(None))
        if expect == S.OK and n == 150_000:
            h = S.Handle(0)
            ref = h.gap(a, b, T, X=X, Y=Y, precision=S.FP32, rho=10.0)
            h.close()
            assert rel(res.objective, ref["objective"]) <= 1e-12
            assert abs(res.gap - ref["gap"]) <= 1e-12 * ref["objective"]
        if expect != S.OK:
            assert b"scratch" in S.lib.sr_ot_last_error(None)
        del T
        torch.cuda.empty_cache()

