"""Seeded request streams for the serving workload: mixed 2D triangle meshes (1e3 to 2e5
elements) and 3D tetrahedral meshes (1e3 to 1e5 elements), log-uniform sizes, horizon
delta uniform in [2h, 6h], eps = delta/10, constant or truncated-Gaussian kernel (coin flip),
Poisson arrivals.  Plain data; no arithmetic of the method."""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class RequestSpec:
    dim: int
    n: int          # Omega cells per axis, h = 1/n
    layer: int
    delta: float
    eps: float
    kernel: int
    L_max: int
    n_elem: int
    arrival_s: float


def serving_stream(n_requests: int = 512, seed: int = 0, rate_per_s: float = 10.0):
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for _ in range(n_requests):
        dim = 2 if rng.random() < 0.5 else 3
        lo, hi = (1e3, 2e5) if dim == 2 else (1e3, 1e5)
        target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        per_cell = 2 if dim == 2 else 6
        n = max(2, int(round((target / per_cell) ** (1.0 / dim))))
        h = 1.0 / n
        delta = rng.uniform(2.0, 6.0) * h
        eps = delta / 10.0
        layer = int(math.ceil((delta + eps) / h - 1e-9))
        kernel = int(rng.random() < 0.5)
        L_max = 3 if dim == 2 else 2
        n_elem = per_cell * (n + 2 * layer) ** dim
        t += rng.exponential(1.0 / rate_per_s)
        out.append(RequestSpec(dim, n, layer, delta, eps, kernel, L_max, n_elem, t))
    return out
