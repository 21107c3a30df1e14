"""ctypes binding of libsr_ot.so (include/sr_ot.h): argument marshalling only.

Every computation runs in the CUDA library; this module only turns torch
tensors into device pointers and host structs. Importing it loads the
library and raises if it has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as ct
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsr_ot.so")

OK, NOT_CONVERGED = 0, 1
EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENUMERIC, EUNSUPPORTED = -1, -2, -3, -4, -5, -6
BCFW, BCAFW, BCPFW, FW = 0, 1, 2, 3
CYCLIC, PERMUTE, UNIFORM, GAP_ADAPTIVE = 0, 1, 2, 3
DEC, ELS = 0, 1
FP64, FP32, FP32_BF16COST = 0, 1, 2
EPOCH_AUTO, EPOCH_TWO_PHASE, EPOCH_PIPELINED, EPOCH_SPECULATIVE, EPOCH_SPECULATIVE_ONE_CHAIN = 0, 1, 2, 3, 4
EPOCH_SPECULATIVE_SPLIT = 5
COST_SQUARED, COST_EUCLIDEAN = 0, 1

EXPORTS = ["sr_ot_default_options", "sr_ot_create", "sr_ot_set_stream", "sr_ot_destroy",
           "sr_ot_last_error", "sr_ot_solve", "sr_ot_solve_batched", "sr_ot_grad",
           "sr_ot_grad_batched", "sr_ot_transfer", "sr_ot_transfer_batched", "sr_ot_gap", "sr_ot_cost_bf16", "sr_ot_launch_count",
           "sr_ot_profile_enable", "sr_ot_profile_read", "sr_ot_gap_noalloc", "sr_ot_lp_metrics",
           "sr_ot_profile_chain_floor"]
PROF_EPOCH, PROF_CERT, PROF_BATCH, PROF_GRAD, PROF_COST, PROF_METRICS = 0, 1, 2, 3, 4, 5


class Options(ct.Structure):
    _fields_ = [
        ("variant", ct.c_int), ("order", ct.c_int), ("step", ct.c_int), ("precision", ct.c_int),
        ("rho", ct.c_double), ("tol_rel_gap", ct.c_double), ("max_epochs", ct.c_longlong),
        ("gap_every", ct.c_int), ("refresh_every", ct.c_int), ("ga_M", ct.c_int),
        ("ga_global_only", ct.c_int), ("seed", ct.c_ulonglong), ("trace", ct.c_void_p),
        ("trace_capacity", ct.c_longlong), ("dense_only", ct.c_int), ("epoch_kernel", ct.c_int), ("cost_kind", ct.c_int),
        ("spin_limit", ct.c_longlong), ("batch_warm_start", ct.c_int), ("start_gate", ct.c_void_p),
        ("cert_schedule", ct.c_int),
    ]


class TransferStats(ct.Structure):
    _fields_ = [("e_c", ct.c_double), ("row_err", ct.c_double), ("col_err", ct.c_double),
                ("sparsity", ct.c_double)]


class LpMetrics(ct.Structure):
    _fields_ = [("e_m", ct.c_double), ("e_v", ct.c_double), ("diff_norm", ct.c_double),
                ("lp_norm", ct.c_double), ("value", ct.c_double), ("lp_value", ct.c_double)]


class Result(ct.Structure):
    _fields_ = [
        ("objective", ct.c_double), ("gap", ct.c_double), ("rel_gap", ct.c_double),
        ("dual", ct.c_double), ("row_err", ct.c_double), ("epochs", ct.c_longlong),
        ("block_updates", ct.c_longlong),
        ("status", ct.c_int), ("reserved", ct.c_int),
    ]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class SrOtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sr_ot status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2103_05857_gb300.build` (no CPU fallback exists)")
    lib = ct.CDLL(LIB_PATH)
    vp, i, ll, d = ct.c_void_p, ct.c_int, ct.c_longlong, ct.c_double
    llp, ip = ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_int)
    lib.sr_ot_default_options.argtypes = [ct.POINTER(Options)]
    lib.sr_ot_default_options.restype = None
    lib.sr_ot_create.argtypes = [ct.POINTER(vp), i, vp]
    lib.sr_ot_set_stream.argtypes = [vp, vp]
    lib.sr_ot_destroy.argtypes = [vp]
    lib.sr_ot_last_error.argtypes = [vp]
    lib.sr_ot_last_error.restype = ct.c_char_p
    lib.sr_ot_solve.argtypes = [vp, ct.POINTER(Options), i, i, i, vp, vp, vp, vp, vp, vp, i,
                                ct.POINTER(Result)]
    lib.sr_ot_solve_batched.argtypes = [vp, ct.POINTER(Options), i, ip, ip, i, llp, llp, llp, llp,
                                        llp, vp, vp, vp, vp, vp, ct.POINTER(Result)]
    lib.sr_ot_grad.argtypes = [vp, ct.POINTER(Options), i, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.sr_ot_transfer.argtypes = [vp, ct.POINTER(Options), i, i, i, vp, vp, vp, vp, vp,
                                   ct.POINTER(TransferStats)]
    lib.sr_ot_transfer_batched.argtypes = [vp, ct.POINTER(Options), i, ip, ip, i, llp, llp, llp, llp, llp,
                                           vp, vp, vp, vp, vp, ct.POINTER(TransferStats)]
    lib.sr_ot_grad_batched.argtypes = [vp, ct.POINTER(Options), i, ip, ip, i, llp, llp, llp, llp,
                                       vp, vp, vp, vp, vp, vp, vp]
    lib.sr_ot_gap.argtypes = [vp, ct.POINTER(Options), i, i, i, vp, vp, vp, vp, vp, vp, vp,
                              ct.POINTER(Result)]
    lib.sr_ot_cost_bf16.argtypes = [vp, i, i, i, vp, vp, vp]
    lib.sr_ot_gap_noalloc.argtypes = [i, vp, ct.POINTER(Options), i, i, i, vp, vp, vp, vp, vp, vp,
                                      vp, ct.POINTER(Result)]
    lib.sr_ot_lp_metrics.argtypes = [vp, ct.POINTER(Options), i, i, i, vp, vp, vp, vp, vp, ct.POINTER(LpMetrics)]
    lib.sr_ot_profile_chain_floor.argtypes = [vp, i, i, ct.POINTER(d)]
    lib.sr_ot_profile_enable.argtypes = [vp, i]
    lib.sr_ot_profile_read.argtypes = [vp, i, ct.POINTER(d), ct.POINTER(ll)]
    for name in EXPORTS:
        fn = getattr(lib, name)
        if name not in ("sr_ot_default_options", "sr_ot_last_error", "sr_ot_launch_count"):
            fn.restype = ct.c_int
    lib.sr_ot_launch_count.argtypes = [vp]
    lib.sr_ot_launch_count.restype = ll
    return lib


lib = _load()


def options(**kw) -> Options:
    o = Options()
    lib.sr_ot_default_options(ct.byref(o))
    for k, v in kw.items():
        if k in ("trace", "start_gate"):
            setattr(o, k, None if v is None else v.data_ptr())
            continue
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ct.c_void_p(t.data_ptr())


def _dtype_of(prec):
    return torch.float64 if prec == FP64 else torch.float32


class Handle:
    """One library handle bound to a device and (by default) torch's current stream."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ct.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream(device)
        st = lib.sr_ot_create(ct.byref(self._h), int(device), ct.c_void_p(s.cuda_stream))
        if st != OK:
            raise SrOtError(st, lib.sr_ot_last_error(None).decode())
        self.device = device

    def close(self):
        if self._h:
            lib.sr_ot_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=(OK, NOT_CONVERGED)):
        if st not in allow:
            raise SrOtError(st, lib.sr_ot_last_error(self._h).decode())
        return st

    def set_stream(self, stream):
        self._check(lib.sr_ot_set_stream(self._h, ct.c_void_p(stream.cuda_stream)))

    def last_error(self) -> str:
        return lib.sr_ot_last_error(self._h).decode()

    def launch_count(self) -> int:
        return int(lib.sr_ot_launch_count(self._h))

    def profile(self, enable: bool = True):
        self._check(lib.sr_ot_profile_enable(self._h, int(bool(enable))), allow=(OK,))

    def chain_floor(self, chain_warps: int = 3, updates: int = 1 << 16) -> float:
        """sr_ot_profile_chain_floor: ns per update of the speculative kernel's
        update chain alone."""
        ns = ct.c_double()
        self._check(lib.sr_ot_profile_chain_floor(self._h, int(chain_warps), int(updates), ct.byref(ns)), allow=(OK,))
        return ns.value

    def profile_read(self, kind: int):
        ms, groups = ct.c_double(), ct.c_longlong()
        self._check(lib.sr_ot_profile_read(self._h, kind, ct.byref(ms), ct.byref(groups)), allow=(OK,))
        return ms.value, groups.value

    # -------------------------------------------------------------------
    def solve(self, a, b, T, C=None, X=None, Y=None, warm_start=False, opts=None, **kw):
        """sr_ot_solve. Returns the result dict; T is updated in place."""
        o = opts if opts is not None else options(**kw)
        m, n = T.shape
        d = 0 if X is None else X.shape[1]
        res = Result()
        st = lib.sr_ot_solve(self._h, ct.byref(o), m, n, d, _ptr(C), _ptr(X), _ptr(Y), _ptr(a),
                             _ptr(b), _ptr(T), int(bool(warm_start)), ct.byref(res))
        self._check(st)
        return res.asdict()

    def solve_raw(self, a, b, T, C=None, X=None, Y=None, warm_start=False, opts=None, **kw):
        """sr_ot_solve returning (status, result dict) without raising."""
        o = opts if opts is not None else options(**kw)
        m, n = T.shape
        d = 0 if X is None else X.shape[1]
        res = Result()
        st = lib.sr_ot_solve(self._h, ct.byref(o), m, n, d, _ptr(C), _ptr(X), _ptr(Y), _ptr(a),
                             _ptr(b), _ptr(T), int(bool(warm_start)), ct.byref(res))
        return st, res.asdict()

    def solve_batched(self, X, Y, a, b, T, sizes, offsets, opts=None, **kw):
        """sr_ot_solve_batched over packed device buffers.

        sizes: list of (m, n); offsets: list of (off_X, off_Y, off_a, off_b, off_T)
        element offsets. Returns (status, list of result dicts)."""
        o = opts if opts is not None else options(**kw)
        B = len(sizes)
        mm = (ct.c_int * B)(*[int(s[0]) for s in sizes])
        nn = (ct.c_int * B)(*[int(s[1]) for s in sizes])
        cols = list(zip(*offsets))
        arrs = [(ct.c_longlong * B)(*[int(v) for v in c]) for c in cols]
        res = (Result * B)()
        st = lib.sr_ot_solve_batched(self._h, ct.byref(o), B, mm, nn, 3, arrs[0], arrs[1], arrs[2],
                                     arrs[3], arrs[4], _ptr(X), _ptr(Y), _ptr(a), _ptr(b), _ptr(T),
                                     res)
        self._check(st)
        return st, [r.asdict() for r in res]

    def solve_batched_raw(self, X, Y, a, b, T, sizes, offsets, opts=None, **kw):
        """sr_ot_solve_batched returning (status, list of result dicts) without
        raising: each instance's own status is in its dict, the call returns
        the worst of them."""
        o = opts if opts is not None else options(**kw)
        B = len(sizes)
        mm = (ct.c_int * B)(*[int(s[0]) for s in sizes])
        nn = (ct.c_int * B)(*[int(s[1]) for s in sizes])
        cols = list(zip(*offsets))
        arrs = [(ct.c_longlong * B)(*[int(v) for v in c]) for c in cols]
        res = (Result * B)()
        st = lib.sr_ot_solve_batched(self._h, ct.byref(o), B, mm, nn, 3, arrs[0], arrs[1], arrs[2],
                                     arrs[3], arrs[4], _ptr(X), _ptr(Y), _ptr(a), _ptr(b), _ptr(T),
                                     res)
        return st, [r.asdict() for r in res]

    def gap(self, a, b, T, C=None, X=None, Y=None, g_rows=None, opts=None, **kw):
        """sr_ot_gap: certificate (f, g, w) of plan T."""
        o = opts if opts is not None else options(**kw)
        m, n = T.shape
        d = 0 if X is None else X.shape[1]
        res = Result()
        st = lib.sr_ot_gap(self._h, ct.byref(o), m, n, d, _ptr(C), _ptr(X), _ptr(Y), _ptr(a),
                           _ptr(b), _ptr(T), _ptr(g_rows), ct.byref(res))
        self._check(st, allow=(OK,))
        return res.asdict()

    def grad(self, T, X=None, Y=None, b=None, want=("dX", "dY", "db"), opts=None, **kw):
        """sr_ot_grad: envelope-theorem gradients at plan T. Returns a dict with
        the requested entries of dC, dX, dY, db (new tensors, T's dtype)."""
        o = opts if opts is not None else options(**kw)
        m, n = T.shape
        d = 3 if X is None else X.shape[1]  # without points the library rejects dX / dY
        out = {}
        shapes = {"dC": (m, n), "dX": (m, d), "dY": (n, d), "db": (n,)}
        for k in want:
            out[k] = torch.empty(shapes[k], dtype=T.dtype, device=T.device)
        st = lib.sr_ot_grad(self._h, ct.byref(o), m, n, 0 if X is None else d, _ptr(X), _ptr(Y), None,
                            _ptr(b), _ptr(T),
                            _ptr(out.get("dC")), _ptr(out.get("dX")), _ptr(out.get("dY")),
                            _ptr(out.get("db")))
        self._check(st, allow=(OK,))
        return out

    def transfer(self, T, Y=None, a=None, b=None, projection=True, stats=True, opts=None, **kw):
        """sr_ot_transfer: barycentric projection Xhat (m x d, a new tensor of
        T's dtype, or None) and the statistics dict {e_c, row_err, col_err,
        sparsity} (or None)."""
        o = opts if opts is not None else options(**kw)
        m, n = T.shape
        d = 3 if Y is None else Y.shape[1]
        Xh = torch.empty((m, d), dtype=T.dtype, device=T.device) if projection else None
        ts = TransferStats()
        st = lib.sr_ot_transfer(self._h, ct.byref(o), m, n, d, _ptr(Y), _ptr(a), _ptr(b), _ptr(T), _ptr(Xh),
                                ct.byref(ts) if stats else None)
        self._check(st, allow=(OK,))
        out = {f: getattr(ts, f) for f, _ in TransferStats._fields_} if stats else None
        return Xh, out

    def transfer_batched(self, Y, a, b, T, sizes, offsets, d=3, projection=True, stats=True, xhat_numel=None,
                         opts=None, **kw):
        """sr_ot_transfer_batched over packed buffers (offsets as in
        solve_batched). Returns (packed Xhat laid out like X, or None; list of
        statistics dicts, or None)."""
        o = opts if opts is not None else options(**kw)
        B = len(sizes)
        mm = (ct.c_int * B)(*[int(s[0]) for s in sizes])
        nn = (ct.c_int * B)(*[int(s[1]) for s in sizes])
        cols = list(zip(*offsets))
        arrs = [(ct.c_longlong * B)(*[int(v) for v in c]) for c in cols]
        Xh = None
        if projection:
            numel = xhat_numel if xhat_numel is not None else max(int(v[0]) + int(s[0]) * d
                                                                  for v, s in zip(offsets, sizes))
            Xh = torch.zeros(numel, dtype=T.dtype, device=T.device)
        ts = (TransferStats * B)()
        st = lib.sr_ot_transfer_batched(self._h, ct.byref(o), B, mm, nn, d, arrs[0], arrs[1], arrs[2], arrs[3],
                                        arrs[4], _ptr(Y), _ptr(a), _ptr(b), _ptr(T), _ptr(Xh),
                                        ts if stats else None)
        self._check(st, allow=(OK,))
        out = [{f: getattr(t, f) for f, _ in TransferStats._fields_} for t in ts] if stats else None
        return Xh, out

    def grad_batched(self, X, Y, b, T, sizes, offsets, want=("dX", "dY", "db"), d=3, opts=None, **kw):
        """sr_ot_grad_batched over packed buffers (offsets as in solve_batched:
        (off_X, off_Y, off_a, off_b, off_T) per instance). Returns packed dX,
        dY, db laid out like X, Y, b."""
        o = opts if opts is not None else options(**kw)
        B = len(sizes)
        mm = (ct.c_int * B)(*[int(s[0]) for s in sizes])
        nn = (ct.c_int * B)(*[int(s[1]) for s in sizes])
        oX = (ct.c_longlong * B)(*[int(v[0]) for v in offsets])
        oY = (ct.c_longlong * B)(*[int(v[1]) for v in offsets])
        ob = (ct.c_longlong * B)(*[int(v[3]) for v in offsets])
        oT = (ct.c_longlong * B)(*[int(v[4]) for v in offsets])
        out = {}
        if "dX" in want:
            out["dX"] = torch.zeros_like(X)
        if "dY" in want:
            out["dY"] = torch.zeros_like(Y)
        if "db" in want:
            out["db"] = torch.zeros_like(b)
        st = lib.sr_ot_grad_batched(self._h, ct.byref(o), B, mm, nn, int(d), oX, oY, ob, oT, _ptr(X),
                                    _ptr(Y), _ptr(b), _ptr(T), _ptr(out.get("dX")),
                                    _ptr(out.get("dY")), _ptr(out.get("db")))
        self._check(st, allow=(OK,))
        return out

    def lp_metrics(self, T, T_lp, C=None, X=None, Y=None, opts=None, **kw):
        """sr_ot_lp_metrics: e_m, e_v (Sec. 5, metrics v and vi) of plan T
        against the reference plan T_lp. Returns a dict."""
        o = opts if opts is not None else options(**kw)
        m, n = T.shape
        d = 0 if X is None else X.shape[1]
        r = LpMetrics()
        st = lib.sr_ot_lp_metrics(self._h, ct.byref(o), m, n, d, _ptr(C), _ptr(X), _ptr(Y), _ptr(T), _ptr(T_lp),
                                  ct.byref(r))
        self._check(st, allow=(OK,))
        return {f: getattr(r, f) for f, _ in LpMetrics._fields_}

    def cost_bf16(self, X, Y, C=None):
        """sr_ot_cost_bf16: C = |x~|^2 + |y~|^2 - 2 X~ Y~^T on the tensor cores
        (float32 X, Y; BF16-rounded inside). Returns C (m x n float32)."""
        m, d = X.shape
        n = Y.shape[0]
        if C is None:
            C = torch.empty((m, n), dtype=torch.float32, device=X.device)
        st = lib.sr_ot_cost_bf16(self._h, m, n, d, _ptr(X), _ptr(Y), _ptr(C))
        self._check(st, allow=(OK,))
        return C
