"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds no arithmetic of the method: only parameter sets (the
lattice, model constants, scheme and step of each workload) and seeded
numpy draws of initial fields, so that the CUDA library and the oracle are
fed identical inputs without either importing the other.

Workloads (the paper's simulation set-ups of Sec. V, at stated sizes):
  model_a_64      Model A, d=2, 64^2, dx=1, Gamma=1, r=-0.5, u=1, T=0.5, SETD1,
                  h=0.01, phi0 ~ N(0, 0.1^2)
  model_b_1024    Model B, d=2, 1024^2, dx=1, Gamma=1, r=-1, u=1, T=0.1,
                  h in {0.1, 0.05, 0.025}, all three schemes, phi0 ~ N(0, 0.01^2)
  kpz_1d / kpz_2d KPZ nu=1, lambda=2, noise sqrt(D) xi with D=1 (the paper's
                  sqrt(2D) eta with D=1/2), h=0.01, flat start
  cgl_2048        CGL d=2, 2048^2, dx=0.5, alpha=2, beta=-0.5, eps=1e-4, SETD2,
                  h=0.05, A0 = 0.01 (N(0,1) + i N(0,1))
  model_a_128_3d  Model A d=3, 128^3, Gamma=1, r=0.2, u=1, T=1, SETD1, h=0.01
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

MODEL_A, MODEL_B, KPZ, CGL, CUSTOM = 0, 1, 2, 3, 4
EM, SETD1, SETD2 = 0, 1, 2


@dataclasses.dataclass
class Workload:
    name: str
    d: int
    n: Sequence[int]          # x first
    dx: Sequence[float]
    model: int
    p: Sequence[float]
    scheme: int
    h: float
    seed: int
    replicas: int = 1
    sigma0: float = 0.0       # std of the iid initial field
    dealias: int = 1

    @property
    def shape(self):
        return tuple(reversed(list(self.n)[: self.d]))

    @property
    def sites(self):
        return int(np.prod(list(self.n)[: self.d]))

    @property
    def complex_field(self):
        return self.model == CGL

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def model_a_64(**kw) -> Workload:
    w = Workload("model_a_64", 2, [64, 64], [1.0, 1.0], MODEL_A, [1.0, -0.5, 1.0, 0.5], SETD1, 0.01,
                 seed=1001, sigma0=0.1)
    return w.with_(**kw)


def model_b_1024(**kw) -> Workload:
    w = Workload("model_b_1024", 2, [1024, 1024], [1.0, 1.0], MODEL_B, [1.0, -1.0, 1.0, 0.1], SETD1, 0.05,
                 seed=2001, sigma0=0.01)
    return w.with_(**kw)


def kpz_1d(L: int, **kw) -> Workload:
    w = Workload("kpz_1d_%d" % L, 1, [L], [1.0], KPZ, [1.0, 2.0, 0.5], SETD1, 0.01, seed=3001)
    return w.with_(**kw)


def kpz_2d(**kw) -> Workload:
    w = Workload("kpz_2d_256", 2, [256, 256], [1.0, 1.0], KPZ, [1.0, 2.0, 0.5], SETD1, 0.01, seed=3101)
    return w.with_(**kw)


def cgl_2048(**kw) -> Workload:
    w = Workload("cgl_2048", 2, [2048, 2048], [0.5, 0.5], CGL, [2.0, -0.5, 1e-4], SETD2, 0.05, seed=4001,
                 sigma0=0.01)
    return w.with_(**kw)


def model_a_128_3d(**kw) -> Workload:
    w = Workload("model_a_128_3d", 3, [128, 128, 128], [1.0, 1.0, 1.0], MODEL_A, [1.0, 0.2, 1.0, 1.0], SETD1,
                 0.01, seed=5001)
    return w.with_(**kw)


def kpz_ensemble_lengths(count: int = 512, seed: int = 3000, lo_log2: int = 10, hi_log2: int = 16):
    """Lattice lengths of the uneven 1-D KPZ ensemble: powers of two drawn
    uniformly from 2^lo .. 2^hi with a fixed numpy seed."""
    rng = np.random.default_rng(seed)
    return [int(2 ** k) for k in rng.integers(lo_log2, hi_log2 + 1, size=count)]


def initial_fields(w: Workload, replicas: Optional[int] = None, seed_offset: int = 0) -> np.ndarray:
    """Seeded iid N(0, sigma0^2) initial fields, shape (R,) + shape; complex
    fields get sigma0 (N(0,1) + i N(0,1))."""
    R = w.replicas if replicas is None else replicas
    rng = np.random.default_rng(w.seed * 7919 + seed_offset)
    shape = (R,) + w.shape
    if w.complex_field:
        return w.sigma0 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return w.sigma0 * rng.standard_normal(shape)


def smooth_field(w: Workload, amplitude: float = 0.3, modes: int = 3, seed: int = 7, replicas: int = 1):
    """A band-limited random field (a few low Fourier modes, all within the
    dealiasing band), for deterministic convergence studies."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.arange(n) / n for n in w.shape], indexing="ij")
    out = np.zeros((replicas,) + w.shape, dtype=np.complex128 if w.complex_field else np.float64)
    for r in range(replicas):
        f = np.zeros(w.shape, dtype=out.dtype)
        for _ in range(modes):
            ks = rng.integers(-2, 3, size=len(w.shape))
            ph = rng.uniform(0, 2 * np.pi)
            arg = 2 * np.pi * sum(k * g for k, g in zip(ks, grids)) + ph
            amp = amplitude * rng.uniform(0.3, 1.0)
            f = f + amp * (np.exp(1j * arg) if w.complex_field else np.cos(arg))
        out[r] = f
    return out
