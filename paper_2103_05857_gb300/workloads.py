"""Seeded synthetic inputs shaped like the paper's colour-transfer workloads.

The paper's inputs are k-means colour centroids of two public photographs with
histogram weights (Sec. 5.1); the photographs are not available, so these
generators stand in for them: RGB-like point clouds in [0,1]^3 drawn from
seeded Gaussian mixtures (source and reference palettes use different
mixtures), uniform or Dirichlet(1) weights, and a clustered feature-space
cloud for the d = 128 tensor-core cost workload.

This module holds none of the method's arithmetic (no cost, gradient, gap or
step): it only draws X, Y, a, b and instance sizes. Both the CUDA library's
tests and the CPU oracle consume its arrays.

Randomness: splitmix64 (Steele, Lea & Flood 2014) counter streams, uniform
doubles from the top 53 bits, normals by Box-Muller. Every array is a
deterministic function of its seed on every platform.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _u64(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` splitmix64 outputs of the generator seeded with seed ^ (stream << 56)."""
    z0 = np.uint64((int(seed) ^ (int(stream) << 56)) & (2**64 - 1))
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z0 + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1)."""
    return (_u64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform."""
    half = (count + 1) // 2
    u = uniform(seed, stream, 2 * half)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)])
    return z[:count]


def colour_cloud(seed: int, npts: int, components: int = 8) -> np.ndarray:
    """npts RGB-like points in [0,1]^3 from a seeded `components`-Gaussian mixture.

    Means ~ U[0.15, 0.85]^3, isotropic sigma ~ U[0.03, 0.12], component weights
    Dirichlet(1) (normalised Exp(1)); points are clipped to [0, 1]."""
    K = components
    means = 0.15 + 0.70 * uniform(seed, 1, 3 * K).reshape(K, 3)
    sigma = 0.03 + 0.09 * uniform(seed, 2, K)
    w = -np.log(1.0 - uniform(seed, 3, K))
    cdf = np.cumsum(w / w.sum())
    lab = np.searchsorted(cdf, uniform(seed, 4, npts), side="right").clip(0, K - 1)
    z = normal(seed, 5, 3 * npts).reshape(npts, 3)
    return np.clip(means[lab] + sigma[lab, None] * z, 0.0, 1.0)


def dirichlet_weights(seed: int, n: int) -> np.ndarray:
    """A point of the simplex drawn from Dirichlet(1, ..., 1) (normalised Exp(1))."""
    e = -np.log(1.0 - uniform(seed, 6, n))
    return e / e.sum()


def feature_cloud(seed: int, npts: int, d: int, clusters: int = 16,
                  centre_seed: int | None = None) -> np.ndarray:
    """Clustered features: centre mu_c ~ N(0, I_d), point = mu_c + N(0, I_d),
    cluster labels uniform. Source and target share centres (centre_seed)."""
    cs = seed if centre_seed is None else centre_seed
    mu = normal(cs, 7, clusters * d).reshape(clusters, d)
    lab = np.minimum((uniform(seed, 8, npts) * clusters).astype(np.int64), clusters - 1)
    return mu[lab] + normal(seed, 9, npts * d).reshape(npts, d)


@dataclass
class Instance:
    """One semi-relaxed OT instance: points X (m x d), Y (n x d), weights a, b."""
    X: np.ndarray
    Y: np.ndarray
    a: np.ndarray
    b: np.ndarray
    rho: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.X.shape[0]

    @property
    def n(self) -> int:
        return self.Y.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    def rounded(self, dtype=np.float32) -> "Instance":
        """The same instance with every array rounded to `dtype` and returned as
        float64 again: the exact inputs a reduced-precision run sees."""
        cv = lambda v: np.asarray(v, dtype=dtype).astype(np.float64)
        return Instance(cv(self.X), cv(self.Y), cv(self.a), cv(self.b), self.rho, self.name,
                        dict(self.meta))


def colour_instance(seed: int, m: int, n: int, rho: float = 10.0,
                    b_dirichlet: bool = False, name: str = "") -> Instance:
    """Colour-transfer shaped instance: X, Y in [0,1]^3, a = 1/m, b = 1/n or Dirichlet(1)."""
    X = colour_cloud(seed * 4 + 0, m)
    Y = colour_cloud(seed * 4 + 1, n)
    a = np.full(m, 1.0 / m)
    b = dirichlet_weights(seed * 4 + 2, n) if b_dirichlet else np.full(n, 1.0 / n)
    return Instance(X, Y, a, b, float(rho), name or f"colour{m}x{n}")


def feature_instance(seed: int, m: int, n: int, d: int = 128, clusters: int = 16,
                     rho: float = 5000.0, name: str = "") -> Instance:
    """Feature-space instance (d >= 64), uniform weights."""
    X = feature_cloud(seed * 4 + 0, m, d, clusters, centre_seed=seed * 4 + 3)
    Y = feature_cloud(seed * 4 + 1, n, d, clusters, centre_seed=seed * 4 + 3)
    return Instance(X, Y, np.full(m, 1.0 / m), np.full(n, 1.0 / n), float(rho),
                    name or f"feature{m}x{n}d{d}")


def batch_sizes(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """`count` (m, n) pairs, each uniform on the integers lo..hi."""
    u = uniform(seed, 10, 2 * count)
    v = lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)
    return v.reshape(count, 2)


def colour_batch(seed: int, count: int, lo: int, hi: int, rho: float = 10.0):
    """`count` independent colour instances of uneven sizes m, n ~ U{lo..hi}."""
    sz = batch_sizes(seed, count, lo, hi)
    return [colour_instance(seed * 100003 + 17 * k + 1, int(mm), int(nn), rho)
            for k, (mm, nn) in enumerate(sz)]


# The five workloads the library is measured on (sizes and weights as stated
# for them; seeds fixed here).
WORKLOADS = {
    "colour256_fp64": dict(kind="colour", seed=1000, m=256, n=256, rho=10.0),
    "colour4096_fp32": dict(kind="colour", seed=2000, m=4096, n=4096, rho=10.0, b_dirichlet=True),
    "colour_batch512": dict(kind="batch", seed=3000, count=512, lo=64, hi=2048, rho=10.0),
    "feature8192_d128": dict(kind="feature", seed=4000, m=8192, n=8192, d=128, rho=5000.0),
    "colour_batch64_2048": dict(kind="batch_fixed", seed=5000, count=64, m=2048, n=2048, rho=10.0),
}


def workload(name: str, **override):
    """Build a named workload; keyword overrides replace its parameters."""
    p = dict(WORKLOADS[name])
    p.update(override)
    kind = p.pop("kind")
    if kind == "colour":
        return colour_instance(p["seed"], p["m"], p["n"], p["rho"], p.get("b_dirichlet", False),
                               name=name)
    if kind == "feature":
        return feature_instance(p["seed"], p["m"], p["n"], p["d"], rho=p["rho"], name=name)
    if kind == "batch":
        return colour_batch(p["seed"], p["count"], p["lo"], p["hi"], p["rho"])
    if kind == "batch_fixed":
        return [colour_instance(p["seed"] * 100003 + 17 * k + 1, p["m"], p["n"], p["rho"])
                for k in range(p["count"])]
    raise KeyError(name)


def feasible_plan(seed: int, a: np.ndarray, n: int, support: int = 8) -> tuple:
    """A sparse feasible plan for a: row i has `support` distinct random
    columns with uniform positive weights scaled to sum to a_i (the shape of a
    converged plan, whose rows carry few atoms). Returns (rows, cols, vals)
    in row-major order."""
    m = len(a)
    support = min(support, n)
    u = uniform(seed, 20, m * support).reshape(m, support)
    # distinct columns per row: sorted draws of a stride pattern
    base = (uniform(seed, 21, m) * n).astype(np.int64)
    step = 1 + (uniform(seed, 22, m) * max(n // support - 1, 1)).astype(np.int64)
    cols = (base[:, None] + step[:, None] * np.arange(support)[None, :]) % n
    w = 0.05 + u
    w = w / w.sum(1, keepdims=True) * np.asarray(a, dtype=np.float64)[:, None]
    rows = np.repeat(np.arange(m), support)
    return rows, cols.ravel(), w.ravel()


def bf16_round(x) -> np.ndarray:
    """Values rounded to bfloat16 (round to nearest, ties to even) from their
    float32 images, returned as float64: the exact inputs a BF16 tensor-core
    cost sees. Finite inputs only."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)
