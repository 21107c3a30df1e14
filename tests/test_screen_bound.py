"""The FP32 argmin screen of the FP64 single-warp epoch kernel
(solve_f64w.cu), checked on the host.

The kernel takes the exact FP64 gradient grad = C + rho r (Sec. 3.1) only
for the columns whose FP32 interval [g - e, g + e] reaches below the
smallest upper end U of the row, where c = fl32(C), p = fl32(rho r),
g = fl32(c + p) and e = 4 u (|c| + |p|) + 2^-120 (u = 2^-24). That is
exact only if every interval contains the FP64 gradient; these checks
evaluate the kernel's FP32 arithmetic with numpy's IEEE binary32 operations
(the scale of e with and without a fused multiply-add) on random rows, on
rows built to cancel, over a wide range of magnitudes and near subnormals,
and confirm that the screened argmin equals the exact one, ties included.
The constant is read from the kernel source.
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2103_05857_gb300",
                   "csrc", "solve_f64w.cu")


def _kernel_screen():
    with open(SRC) as fh:
        src = fh.read()
    k = float(re.search(r"constexpr float kScreen = ([\d.]+)f \* 0x1\.0p-24f;", src).group(1)) * 2.0 ** -24
    floor = 2.0 ** -int(re.search(r"\+ 0x1\.0p-(\d+)f;", src).group(1))
    return np.float32(k), np.float32(floor)


def _bounds(C, rr):
    k, floor = _kernel_screen()
    c = C.astype(np.float32)
    p = rr.astype(np.float32)
    g = (c + p).astype(np.float32)
    s = (np.abs(c) + np.abs(p)).astype(np.float32)
    e_plain = (k * s + floor).astype(np.float32)
    e_fused = (np.float64(k) * s.astype(np.float64) + np.float64(floor)).astype(np.float32)
    e = np.minimum(e_plain, e_fused)
    lo = (g - e).astype(np.float32)
    hi = (g + e).astype(np.float32)
    return lo, hi


def _check_rows(C, rr):
    g64 = C + rr
    lo, hi = _bounds(C, rr)
    assert np.all(lo.astype(np.float64) <= g64) and np.all(g64 <= hi.astype(np.float64))
    # the screened argmin equals the exact one (smallest index among ties)
    U = hi.min(axis=-1, keepdims=True)
    cand = ~(lo > U)
    masked = np.where(cand, g64, np.inf)
    assert np.array_equal(np.argmin(masked, axis=-1), np.argmin(g64, axis=-1))


def test_screen_contains_the_fp64_gradient():
    rng = np.random.default_rng(0)
    for scale in (1e-30, 1e-6, 1.0, 3.0, 1e6, 1e30):
        C = rng.random((200, 257)) * 3.0 * scale
        rr = (rng.random((200, 257)) - 0.5) * 2.0 * scale
        _check_rows(C, rr)


def test_screen_under_cancellation_and_ties():
    rng = np.random.default_rng(1)
    C = rng.random((300, 129)) * 3.0
    rr = -C + rng.normal(0.0, 1e-9, C.shape)      # C + rho r near zero: heavy cancellation
    _check_rows(C, rr)
    C2 = np.round(rng.random((300, 129)) * 8) / 8  # exact ties in FP64
    rr2 = np.round((rng.random((300, 129)) - 0.5) * 8) / 8
    _check_rows(C2, rr2)
    C3 = np.full((5, 64), 0.1)                      # every entry equal
    _check_rows(C3, np.zeros((5, 64)))


def test_screen_near_subnormal_magnitudes():
    rng = np.random.default_rng(2)
    C = rng.random((100, 64)) * 1e-40
    rr = (rng.random((100, 64)) - 0.5) * 1e-40
    _check_rows(C, rr)
