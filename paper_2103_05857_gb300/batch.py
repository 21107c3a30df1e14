"""Packing of instance lists into the flat buffers sr_ot_solve_batched takes
(argument marshalling only)."""
from __future__ import annotations

import numpy as np
import torch


class PackedBatch:
    """Instances (X_k, Y_k, a_k, b_k) packed into float32 device buffers with
    per-instance element offsets; T is one flat buffer of all plans."""

    def __init__(self, instances, device="cuda", pin=False):
        self.sizes = [(inst.m, inst.n) for inst in instances]
        offs, ox, oy, oa, ob, ot = [], 0, 0, 0, 0, 0
        for inst in instances:
            offs.append((ox, oy, oa, ob, ot))
            ox += inst.m * 3
            oy += inst.n * 3
            oa += inst.m
            ob += inst.n
            ot += inst.m * inst.n
        self.offsets = offs
        cat = lambda xs: np.ascontiguousarray(np.concatenate([np.ravel(x) for x in xs]), dtype=np.float32)
        self.hX = torch.from_numpy(cat([i.X for i in instances]))
        self.hY = torch.from_numpy(cat([i.Y for i in instances]))
        self.ha = torch.from_numpy(cat([i.a for i in instances]))
        self.hb = torch.from_numpy(cat([i.b for i in instances]))
        if pin:
            self.hX, self.hY, self.ha, self.hb = (t.pin_memory() for t in (self.hX, self.hY, self.ha, self.hb))
        self.X, self.Y, self.a, self.b = (t.to(device) for t in (self.hX, self.hY, self.ha, self.hb))
        self.T = torch.zeros(ot, dtype=torch.float32, device=device)
        self.total_T = ot

    def plan(self, k):
        m, n = self.sizes[k]
        o = self.offsets[k][4]
        return self.T[o:o + m * n].view(m, n)
