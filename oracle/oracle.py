"""Python face of the plain FP64 CPU oracle (``srot_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only importers. The CUDA library never
imports or calls this module, and this module imports nothing from the
library package.

Orientation follows the library (rows are the blocks, ``T @ 1 = a`` exactly,
column sums pulled toward ``b`` with weight ``rho = 1/lambda``); the paper
states the problem transposed (Sec. 3, eq. 5).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srot_oracle.c")
_LIB = os.path.join(_HERE, "libsrot_oracle.so")
_lock = threading.Lock()
_lib = None

BCFW, BCAFW, BCPFW, FW = 0, 1, 2, 3
CYCLIC, PERMUTE, UNIFORM, GAP = 0, 1, 2, 3
DEC, ELS = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Opts(ct.Structure):
    _fields_ = [
        ("variant", ct.c_int), ("order", ct.c_int), ("step", ct.c_int),
        ("gap_every", ct.c_int), ("rho", ct.c_double), ("tol_rel_gap", ct.c_double),
        ("max_epochs", ct.c_longlong), ("ga_M", ct.c_int), ("ga_global_only", ct.c_int),
        ("ga_init_const", ct.c_double), ("seed", ct.c_uint64), ("warm_start", ct.c_int),
    ]


class Result(ct.Structure):
    _fields_ = [
        ("f", ct.c_double), ("g", ct.c_double), ("w", ct.c_double),
        ("epochs", ct.c_longlong), ("updates", ct.c_longlong), ("n_hist", ct.c_longlong),
        ("converged", ct.c_int), ("status", ct.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            dp, ip = ct.POINTER(ct.c_double), ct.POINTER(ct.c_int)
            lib.srot_or_draw.restype = ct.c_uint64
            lib.srot_or_draw.argtypes = [ct.c_uint64, ct.c_uint64, ct.c_uint64]
            lib.srot_or_cost.argtypes = [ct.c_int, ct.c_int, ct.c_int, dp, dp, ct.c_int, dp]
            lib.srot_or_certificate.argtypes = [ct.c_int, ct.c_int, dp, dp, dp, ct.c_double,
                                                dp, dp, dp, dp]
            lib.srot_or_solve.restype = ct.c_int
            lib.srot_or_solve.argtypes = [ct.c_int, ct.c_int, dp, dp, dp, ct.POINTER(Opts), dp,
                                          ip, ip, ct.c_longlong, dp, ct.POINTER(Result)]
            lib.srot_or_solve_ex.restype = ct.c_int
            lib.srot_or_solve_ex.argtypes = [ct.c_int, ct.c_int, dp, dp, dp, ct.POINTER(Opts), dp,
                                             ip, ip, ct.c_longlong, dp, dp, dp, ct.POINTER(Result)]
            lib.srot_or_sample_from.restype = ct.c_int
            lib.srot_or_sample_from.argtypes = [dp, ct.c_int, ct.c_uint64]
            lib.srot_or_uniform_index.restype = ct.c_int
            lib.srot_or_uniform_index.argtypes = [ct.c_uint64, ct.c_int]
            lib.srot_or_apply_step.restype = None
            lib.srot_or_apply_step.argtypes = [ct.c_int, dp, dp, dp, ct.c_int, ct.c_int, ct.c_int,
                                               ct.c_int, ct.c_double]
            lib.srot_or_block_step.restype = ct.c_int
            lib.srot_or_block_step.argtypes = [ct.c_int, ct.c_int, dp, dp, dp, dp, ct.c_int,
                                               ct.c_longlong, ct.POINTER(Opts), ip, ip, ip, dp]
            lib.srot_or_permutation.argtypes = [ct.c_uint64, ct.c_longlong, ct.c_int, ip]
            lib.srot_or_adjoint.argtypes = [ct.c_int, ct.c_int, ct.c_int, dp, dp, dp, ct.c_double,
                                            dp, dp, dp, dp]
            _lib = lib
    return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _dp(x):
    return None if x is None else x.ctypes.data_as(ct.POINTER(ct.c_double))


def _ip(x):
    return None if x is None else x.ctypes.data_as(ct.POINTER(ct.c_int))


def make_opts(variant=BCFW, order=CYCLIC, step=DEC, rho=10.0, tol_rel_gap=0.0,
              max_epochs=1, gap_every=1, ga_M=1, ga_global_only=0, ga_init_const=0.0,
              seed=0, warm_start=0) -> Opts:
    return Opts(variant, order, step, gap_every, float(rho), float(tol_rel_gap),
                int(max_epochs), ga_M, ga_global_only, float(ga_init_const),
                int(seed) & (2**64 - 1), warm_start)


def draw(seed: int, stream: int, counter: int) -> int:
    """splitmix64 output number counter+1 of the generator seeded with seed ^ (stream << 56)."""
    return int(_load().srot_or_draw(seed & (2**64 - 1), stream, counter))


def permutation(seed: int, epoch: int, m: int) -> np.ndarray:
    out = np.empty(m, dtype=np.int32)
    _load().srot_or_permutation(seed & (2**64 - 1), epoch, m, _ip(out))
    return out


def cost(X, Y, squared: bool = True) -> np.ndarray:
    """C_ij = ||x_i - y_j||^2 (squared) or ||x_i - y_j|| (Sec. 5.1)."""
    X, Y = _f64(X), _f64(Y)
    m, d = X.shape
    n = Y.shape[0]
    C = np.empty((m, n), dtype=np.float64)
    _load().srot_or_cost(m, n, d, _dp(X), _dp(Y), int(bool(squared)), _dp(C))
    return C


def certificate(C, a, b, rho, T):
    """Objective, linearisation gap and Lagrangian dual at T (Thm 2).

    Returns dict(f, g, w, lin, pen, g_rows, s)."""
    C, a, b, T = _f64(C), _f64(a), _f64(b), _f64(T)
    m, n = C.shape
    out = np.zeros(5)
    g_rows = np.empty(m)
    s = np.empty(n)
    _load().srot_or_certificate(m, n, _dp(C), _dp(a), _dp(b), float(rho), _dp(T), _dp(out),
                                _dp(g_rows), _dp(s))
    return dict(f=out[0], g=out[1], w=out[2], lin=out[3], pen=out[4], g_rows=g_rows, s=s)


def solve(C, a, b, T0=None, trace: bool = False, epoch_state: bool = False, **kw):
    """Run the block-coordinate solver (Alg. 1, A.2, A.3, A.4) or full FW (Alg. A.1).

    Returns (T, result_dict, trace_i, trace_j, history) where history rows are
    (epoch, f, g) for every certificate taken. With epoch_state=True the
    result dict also holds "ga_hist" (epochs x m: the gap-adaptive sampling
    gaps at the end of each epoch, after its global update if one was due)
    and "T_hist" (epochs x m x n: the plan at the end of each epoch)."""
    C, a, b = _f64(C), _f64(a), _f64(b)
    m, n = C.shape
    o = make_opts(warm_start=int(T0 is not None), **kw)
    T = _f64(T0).copy() if T0 is not None else np.zeros((m, n))
    cap = int(o.max_epochs) * m if trace else 0
    ti = np.empty(max(cap, 1), dtype=np.int32)
    tj = np.empty(max(cap, 1), dtype=np.int32)
    hist = np.zeros(3 * max(int(o.max_epochs), 1) + 3)
    ga_hist = T_hist = None
    if epoch_state:
        ga_hist = np.full((max(int(o.max_epochs), 1), m), np.nan)
        T_hist = np.full((max(int(o.max_epochs), 1), m, n), np.nan)
    res = Result()
    _load().srot_or_solve_ex(m, n, _dp(C), _dp(a), _dp(b), ct.byref(o), _dp(T),
                             _ip(ti) if trace else None, _ip(tj) if trace else None, cap,
                             _dp(hist), _dp(ga_hist), _dp(T_hist), ct.byref(res))
    if res.status != 0:
        raise ValueError(f"oracle solve rejected the options (status {res.status})")
    rd = dict(f=res.f, g=res.g, w=res.w, epochs=res.epochs, updates=res.updates,
              converged=bool(res.converged))
    if epoch_state:
        rd["ga_hist"] = ga_hist[: int(res.epochs)]
        rd["T_hist"] = T_hist[: int(res.epochs)]
    h = hist.reshape(-1, 3)[: int(res.n_hist)]
    k = int(res.updates)
    return T, rd, (ti[:k] if trace else None), (tj[:k] if trace else None), h


def block_step(C, a, T, r, i, k, **kw):
    """One block update of row i in place on (T, r); returns (jstar, v, dir, gamma)."""
    C, a = _f64(C), _f64(a)
    assert T.dtype == np.float64 and T.flags.c_contiguous
    assert r.dtype == np.float64 and r.flags.c_contiguous
    m, n = C.shape
    o = make_opts(**kw)
    js, v, dr = ct.c_int(), ct.c_int(), ct.c_int()
    gam = ct.c_double()
    st = _load().srot_or_block_step(m, n, _dp(C), _dp(a), _dp(T), _dp(r), int(i), int(k),
                                    ct.byref(o), ct.byref(js), ct.byref(v), ct.byref(dr),
                                    ct.byref(gam))
    if st != 0:
        raise ValueError("oracle block step rejected the options")
    return js.value, v.value, dr.value, gam.value


def apply_step(a, T, r, i, direction, jstar, v, gamma):
    """Apply a given decision (direction 0 FW, 1 away, 2 pairwise, -1 none;
    LMO vertex jstar, away atom v, step gamma) to row i of (T, r) in place,
    with the same update arithmetic as a block step."""
    a = _f64(a)
    assert T.dtype == np.float64 and T.flags.c_contiguous
    assert r.dtype == np.float64 and r.flags.c_contiguous
    n = T.shape[1]
    _load().srot_or_apply_step(n, _dp(a), _dp(T), _dp(r), int(i), int(direction), int(jstar), int(v),
                               float(gamma))


def sample_from(g, u64: int) -> int:
    """The gap-adaptive sampling step (Alg. A.4) for one 64-bit uniform draw:
    an index with probability proportional to max(g_i, 0)."""
    g = _f64(g)
    return int(_load().srot_or_sample_from(_dp(g), len(g), int(u64) & (2**64 - 1)))


def uniform_index(u64: int, m: int) -> int:
    """The uniform block order's index floor(u * m) for one 64-bit draw."""
    return int(_load().srot_or_uniform_index(int(u64) & (2**64 - 1), int(m)))


def adjoint(X, Y, b, rho, T):
    """Envelope-theorem gradients (dX, dY, db) at plan T for the squared cost."""
    X, Y, b, T = _f64(X), _f64(Y), _f64(b), _f64(T)
    m, d = X.shape
    n = Y.shape[0]
    dX = np.empty((m, d))
    dY = np.empty((n, d))
    db = np.empty(n)
    _load().srot_or_adjoint(m, n, d, _dp(X), _dp(Y), _dp(b), float(rho), _dp(T), _dp(dX),
                            _dp(dY), _dp(db))
    return dX, dY, db


def barycentric(Y, T):
    """Colour-transfer projection (Sec. 5.1): the new centroid of source row i
    is the T-weighted mean of the target points, x_hat_i = sum_j T_ij y_j /
    sum_j T_ij (the minimiser of sum_j T_ij ||x - y_j||^2). A row that carries
    no mass has no projection; it is returned as zeros."""
    Y, T = _f64(Y), _f64(T)
    mass = T.sum(axis=1)
    out = np.zeros((T.shape[0], Y.shape[1]))
    for i in range(T.shape[0]):
        if mass[i] > 0.0:
            out[i] = (T[i] @ Y) / mass[i]
    return out


def transfer_stats(a, b, T):
    """Evaluation metrics of Sec. 5: the marginal constraint error
    e_c = ||T 1 - a||_2 + ||T^T 1 - b||_2 (metric iii) with its two terms, and
    the sparsity, the fraction of entries of T that are zero (metric iv)."""
    a, b, T = _f64(a), _f64(b), _f64(T)
    row_err = float(np.linalg.norm(T.sum(axis=1) - a))
    col_err = float(np.linalg.norm(T.sum(axis=0) - b))
    sparsity = float(np.count_nonzero(T == 0.0)) / T.size
    return {"e_c": row_err + col_err, "row_err": row_err, "col_err": col_err, "sparsity": sparsity}


def transport_lp(C, a, b):
    """The optimal plan T*_LP of the unrelaxed, unregularised transport
    problem (Sec. 2: min <C, T> over T >= 0, T 1 = a, T^T 1 = b), the
    reference plan of the evaluation metrics (v) and (vi) of Sec. 5. The
    linear program is solved by a library LP solver (scipy's HiGHS) as one
    step. Both marginals must carry the same total mass; b is rescaled to
    a's total first (float32-rounded weights differ in the last bits)."""
    import scipy.optimize as so
    import scipy.sparse as sp
    C, a, b = _f64(C), _f64(a), _f64(b)
    m, n = C.shape
    b = b * (a.sum() / b.sum())
    rows = sp.kron(sp.eye(m), np.ones((1, n)))
    cols = sp.kron(np.ones((1, m)), sp.eye(n))
    A = sp.vstack([rows, cols]).tocsr()
    res = so.linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([a, b]), bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(f"transport LP failed: {res.message}")
    return np.maximum(res.x.reshape(m, n), 0.0)


def lp_metrics(C, T, T_lp):
    """Evaluation metrics (v) and (vi) of Sec. 5 against the LP plan T*_LP:
    the transport matrix error e_m = ||T - T*_LP|| / ||T*_LP|| (Frobenius
    norm; the paper does not name the norm) and the value error
    e_v = |<T, C> - <T*_LP, C>| / |<T*_LP, C>|."""
    C, T, L = _f64(C), _f64(T), _f64(T_lp)
    diff = float(np.sqrt(((T - L) ** 2).sum()))
    lnorm = float(np.sqrt((L ** 2).sum()))
    value, lp_value = float((T * C).sum()), float((L * C).sum())
    return {"e_m": diff / lnorm, "e_v": abs(value - lp_value) / abs(lp_value), "diff_norm": diff,
            "lp_norm": lnorm, "value": value, "lp_value": lp_value}

