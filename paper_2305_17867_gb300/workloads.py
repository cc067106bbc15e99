"""Seeded synthetic inputs for the compressed-Taylor FMM.

This module holds random-number recipes and workload shapes only -- none of
the method's arithmetic -- so that the CUDA path, the tests and the CPU
oracle can be fed identical inputs without sharing any method code.

The paper (arXiv 2305.17867) uses no public dataset; its FMM workloads are
particle sets in the unit square/cube.  The five workloads below are the
particle configurations the build is measured on.  Workload ``i`` draws its
positions first and its weights second from ``numpy.random.Generator(PCG64(i))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    kernel: str           # "laplace" | "yukawa" | "biharmonic"
    d: int
    p: int
    levels: int           # leaf depth of the uniform tree; -1 = adaptive
    n_src: int
    n_tgt: int            # 0 => targets are the sources
    src_dist: str         # "uniform" | "plummer"
    w_dist: str           # "uniform" | "normal"
    seed: int
    lam: float = 0.0
    max_leaf: int = 0
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "laplace2d_p8_L4_n2k": Workload("laplace2d_p8_L4_n2k", "laplace", 2, 8, 4, 2000, 0,
                                    "uniform", "uniform", 1),
    "laplace3d_p10_L5_n1m": Workload("laplace3d_p10_L5_n1m", "laplace", 3, 10, 5, 1_000_000, 0,
                                     "uniform", "uniform", 2),
    "yukawa3d_p12_adaptive_n2m": Workload("yukawa3d_p12_adaptive_n2m", "yukawa", 3, 12, -1,
                                          2_000_000, 2_000_000, "plummer", "normal", 3,
                                          lam=1.0, max_leaf=64),
    "laplace3d_p8_L5_bwd_n1m": Workload("laplace3d_p8_L5_bwd_n1m", "laplace", 3, 8, 5, 1_000_000,
                                        1_000_000, "uniform", "uniform", 4),
    "biharmonic3d_p8_L6_n4m": Workload("biharmonic3d_p8_L6_n4m", "biharmonic", 3, 8, 6, 4_000_000,
                                       0, "uniform", "uniform", 5),
}


def uniform_points(rng: np.random.Generator, n: int, d: int) -> np.ndarray:
    """n points uniform in [0, 1)^d, row-major (n, d) float64."""
    return rng.random((n, d))


def plummer_points(rng: np.random.Generator, n: int, d: int = 3, a: float = 0.1,
                   center: float = 0.5) -> np.ndarray:
    """Plummer sphere of scale ``a`` about (center,)*d, restricted to [0,1)^d.

    Radius from the inverse cumulative mass r = a / sqrt(u^(-2/3) - 1),
    direction uniform on the sphere; samples outside the unit cube are
    rejected and redrawn (the distribution's tail is cut at the box).
    """
    out = np.empty((0, d))
    while out.shape[0] < n:
        m = int((n - out.shape[0]) * 1.2) + 16
        u = rng.random(m)
        u = np.clip(u, 1e-12, 1.0 - 1e-12)
        r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        v = rng.normal(size=(m, d))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        x = center + r[:, None] * v
        keep = np.all((x >= 0.0) & (x < 1.0), axis=1)
        out = np.concatenate([out, x[keep]], axis=0)
    return np.ascontiguousarray(out[:n])


def weights(rng: np.random.Generator, n: int, dist: str) -> np.ndarray:
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, n)
    if dist == "normal":
        return rng.normal(size=n)
    raise ValueError(dist)


def make_inputs(wl: Workload, n_src: int | None = None, n_tgt: int | None = None,
                seed: int | None = None):
    """(src, w, tgt) float64 arrays; tgt is src itself when the workload says so."""
    rng = np.random.Generator(np.random.PCG64(wl.seed if seed is None else seed))
    ns = wl.n_src if n_src is None else n_src
    if wl.src_dist == "uniform":
        src = uniform_points(rng, ns, wl.d)
    else:
        src = plummer_points(rng, ns, wl.d)
    w = weights(rng, ns, wl.w_dist)
    nt = wl.n_tgt if n_tgt is None else n_tgt
    if wl.n_tgt == 0:
        tgt = src
    else:
        tgt = uniform_points(rng, nt, wl.d)
    return src, w, tgt


def cotangent(n: int, seed: int) -> np.ndarray:
    """u ~ N(0, 1) for loss = sum(u * phi) in the backward workload."""
    rng = np.random.Generator(np.random.PCG64(10_000 + seed))
    return rng.normal(size=n)
