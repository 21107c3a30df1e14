"""torch.autograd wrappers: the optimal value of the semi-relaxed problem as a
differentiable function of the point clouds X, Y and the target marginal b.

Forward solves through the C ABI (sr_ot_solve / sr_ot_solve_batched); backward
runs the adjoint kernels (sr_ot_grad / sr_ot_grad_batched), which evaluate the
envelope-theorem gradient at the returned plan:
    dX = 2 (diag(T 1) X - T Y),  dY = 2 (diag(T^T 1) Y - T^T X),  db = -rho (T^T 1 - b).
The gradient with respect to the row marginal a is not provided (None).
Only the multiplication by the incoming scalar gradient happens in torch.

Backward reuses the very options struct the forward solve ran with (rho,
precision, cost kind), so the adjoint is always taken for the problem that
was solved: a library default for rho applies to both, and a cost the point
gradients do not cover (the Euclidean cost) is refused by the library's own
check in sr_ot_grad rather than given the squared-cost formula.
"""
from __future__ import annotations

import torch

from . import sr_ot as S


def _solve_options(solve_kw, dtype):
    """The sr_ot_options of a solve: `opts=` as given, else built from the
    keyword arguments (precision defaulting to the tensors' dtype)."""
    kw = dict(solve_kw)
    o = kw.pop("opts", None)
    if o is None:
        kw.setdefault("precision", S.FP32 if dtype == torch.float32 else S.FP64)
        o = S.options(**kw)
    elif kw:
        raise TypeError("pass either opts= or keyword options, not both")
    return o


class SemiRelaxedOT(torch.autograd.Function):
    """value = min_T <C(X, Y), T> + (rho/2) ||T^T 1 - b||^2, T >= 0, T 1 = a."""

    @staticmethod
    def forward(ctx, X, Y, b, a, handle, solve_kw):
        o = _solve_options(solve_kw, X.dtype)
        m, n = X.shape[0], Y.shape[0]
        T = torch.zeros((m, n), dtype=X.dtype, device=X.device)
        res = handle.solve(a, b, T, X=X.contiguous(), Y=Y.contiguous(), opts=o)
        ctx.handle = handle
        ctx.opts = o
        ctx.save_for_backward(X, Y, b, T)
        ctx.result = res
        return torch.tensor(res["objective"], dtype=X.dtype, device=X.device)

    @staticmethod
    def backward(ctx, g):
        X, Y, b, T = ctx.saved_tensors
        want = []
        if ctx.needs_input_grad[0]:
            want.append("dX")
        if ctx.needs_input_grad[1]:
            want.append("dY")
        if ctx.needs_input_grad[2]:
            want.append("db")
        out = ctx.handle.grad(T, X=X.contiguous(), Y=Y.contiguous(), b=b, want=tuple(want), opts=ctx.opts)
        gX = out["dX"] * g if "dX" in out else None
        gY = out["dY"] * g if "dY" in out else None
        gb = out["db"] * g if "db" in out else None
        return gX, gY, gb, None, None, None


def semi_relaxed_ot(X, Y, a, b, handle, **solve_kw):
    """Differentiable optimal value (0-dim tensor) of one instance. Options as
    keyword arguments of sr_ot.options, or one `opts=` struct."""
    return SemiRelaxedOT.apply(X, Y, b, a, handle, solve_kw)


class SemiRelaxedOTBatched(torch.autograd.Function):
    """Optimal values of packed instances (one persistent launch forward, one
    adjoint launch backward). X, Y, a, b are packed 1-D buffers as built by
    PackedBatch; returns a vector of per-instance values."""

    @staticmethod
    def forward(ctx, X, Y, b, a, sizes, offsets, handle, solve_kw):
        o = _solve_options(solve_kw, X.dtype)
        total_T = sum(int(m) * int(n) for m, n in sizes)
        T = torch.zeros(total_T, dtype=X.dtype, device=X.device)
        st, res = handle.solve_batched(X, Y, a, b, T, sizes, offsets, opts=o)
        ctx.handle = handle
        ctx.sizes, ctx.offsets = sizes, offsets
        ctx.opts = o
        ctx.save_for_backward(X, Y, b, T)
        ctx.results = res
        vals = torch.tensor([r["objective"] for r in res], dtype=torch.float64)
        return vals.to(device=X.device, dtype=X.dtype)

    @staticmethod
    def backward(ctx, g):
        X, Y, b, T = ctx.saved_tensors
        out = ctx.handle.grad_batched(X, Y, b, T, ctx.sizes, ctx.offsets, opts=ctx.opts)
        ms = torch.tensor([int(s[0]) for s in ctx.sizes], device=g.device)
        ns = torch.tensor([int(s[1]) for s in ctx.sizes], device=g.device)
        # packed layouts follow the instance order with offsets as built by PackedBatch
        gX = out["dX"] * torch.repeat_interleave(g, ms * 3) if ctx.needs_input_grad[0] else None
        gY = out["dY"] * torch.repeat_interleave(g, ns * 3) if ctx.needs_input_grad[1] else None
        gb = out["db"] * torch.repeat_interleave(g, ns) if ctx.needs_input_grad[2] else None
        return gX, gY, gb, None, None, None, None, None
