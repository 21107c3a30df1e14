"""Helpers shared by the GPU tests (input marshalling only)."""
import numpy as np
import torch


def dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    return t.detach().to("cpu", torch.float64).numpy()


def f32(x):
    """Round to float32 and return as float64 (the exact values an FP32 run sees)."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)
