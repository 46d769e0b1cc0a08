"""Seeded synthetic inputs for the Kryging hot path.

This module is shared by the GPU path's callers (tests, bench) and by the FP64
oracle's tests.  It draws random numbers and lays out grids, masks and
covariates; it holds none of the method's arithmetic (no covariance function,
no FFT, no Krylov step).  Random numbers that the method itself consumes (the
white noise of a circulant-embedding sample) are drawn here and passed in.

Workload shapes follow the paper's simulation studies (Sec. 4: Gaussian
processes on regular unit-square grids, a share of cells held out) and its
MODIS application (Sec. 5: cloud-like clustered gaps).  No dataset is read.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Cov:
    """Matern covariance parameters (Sec. 2): sigma2 * rho_nu(d / range) + tau2 * I.

    Geometric anisotropy (Sec. 2, last sentence of the model paragraph): the
    lag is rotated by ``angle`` (radians, counter-clockwise from +x) and the
    minor axis is shortened by ``ratio`` (1 = isotropic)."""

    sigma2: float = 1.0
    range: float = 0.1
    nu: float = 0.5
    tau2: float = 0.1
    angle: float = 0.0
    ratio: float = 1.0


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: a grid, a mask recipe, covariance and Krylov settings."""

    name: str
    n1: int
    n2: int
    cov: Cov
    mask: str                    # "full" | "uniform" | "circles" | "mixed"
    frac_missing: float
    mask_seed: int
    data_seed: int
    beta: tuple = (1.0, 0.5, -0.5)
    nprobe: int = 20
    nsteps: int = 50
    probe_seed: int = 0
    cg_tol: float = 1e-8
    reorth: int = 0              # Lanczos basis: 0 plain recurrence, 1 partial reorthogonalisation
    extra: dict = field(default_factory=dict)


# The five workloads of the hot path: sizes, mask recipes and seeds.
WORKLOADS = {
    "tiny32": Workload("tiny32", 32, 32, Cov(1.0, 0.1, 0.5, 0.1), "full", 0.0, 0, 0,
                       nprobe=20, nsteps=50, probe_seed=0, cg_tol=1e-8,
                       extra={"n_sites": 100, "site_seed": 1}),
    "grid1024": Workload("grid1024", 1024, 1024, Cov(1.0, 0.05, 1.5, 0.05), "uniform", 0.5, 2, 20,
                         nprobe=64, nsteps=60, probe_seed=2, cg_tol=1e-6, reorth=1),
    "search512": Workload("search512", 512, 512, Cov(1.0, 0.08, 1.0, 0.1), "uniform", 0.3, 3, 30,
                          nprobe=32, nsteps=50, probe_seed=3, cg_tol=1e-6, reorth=1,
                          extra={"ranges": [0.02 * (k + 1) for k in range(8)],
                                 "nus": [0.5, 1.0, 1.5, 2.5]}),
    "serve": Workload("serve", 0, 0, Cov(), "mixed", 0.0, 4, 40,
                      nprobe=16, nsteps=50, probe_seed=4, cg_tol=1e-6, reorth=1,
                      extra={"n_requests": 2000, "side_min": 128, "side_max": 2048}),
    "large4096": Workload("large4096", 4096, 4096,
                          Cov(1.0, 0.05, 0.5, 0.05, angle=math.radians(30.0), ratio=3.0),
                          "circles", 0.3, 5, 50, nprobe=32, nsteps=80, probe_seed=5, cg_tol=1e-6, reorth=1,
                          extra={"n_var_cells": 10000, "var_seed": 6}),
}


def cell_centres(n1: int, n2: int):
    """Cell-centre coordinates ((i + 1/2)/n1, (j + 1/2)/n2) of an n1 x n2 grid on
    the unit square, as two (n1, n2) arrays (row index i -> first coordinate)."""
    s1 = (np.arange(n1, dtype=np.float64) + 0.5) / n1
    s2 = (np.arange(n2, dtype=np.float64) + 0.5) / n2
    return np.meshgrid(s1, s2, indexing="ij")


def covariates(s1, s2):
    """Design matrix X = [1, s1, s2] (one row per site)."""
    s1 = np.asarray(s1, dtype=np.float64).ravel()
    s2 = np.asarray(s2, dtype=np.float64).ravel()
    return np.stack([np.ones_like(s1), s1, s2], axis=1)


def mask_full(n1: int, n2: int):
    return np.ones((n1, n2), dtype=bool)


def mask_uniform(n1: int, n2: int, frac_missing: float, seed: int):
    """Exactly round(frac_missing * N) cells missing, chosen by a seeded shuffle."""
    N = n1 * n2
    n_miss = int(round(frac_missing * N))
    perm = np.random.default_rng(seed).permutation(N)
    m = np.ones(N, dtype=bool)
    m[perm[:n_miss]] = False
    return m.reshape(n1, n2)


def mask_circles(n1: int, n2: int, frac_missing: float, seed: int,
                 rmin: float = 0.02, rmax: float = 0.15, base=None):
    """Cloud-cover-like gaps: circular holes with centres U(0,1)^2 and radii
    U[rmin, rmax] are added until at least ``frac_missing`` of the cells are
    missing (the last circle may overshoot).  ``base`` is an existing mask to
    punch holes into."""
    rng = np.random.default_rng(seed)
    s1, s2 = cell_centres(n1, n2)
    m = mask_full(n1, n2) if base is None else base.copy()
    N = n1 * n2
    target = int(math.ceil(frac_missing * N))
    while (N - int(m.sum())) < target:
        c1, c2 = rng.random(2)
        r = rng.uniform(rmin, rmax)
        m &= ~(((s1 - c1) ** 2 + (s2 - c2) ** 2) <= r * r)
    return m


def mask_mixed(n1: int, n2: int, frac_missing: float, seed: int):
    """Half of the missing share as clustered circles, half as uniform holes."""
    rng = np.random.default_rng(seed)
    m = mask_circles(n1, n2, 0.5 * frac_missing, int(rng.integers(1 << 31)))
    N = n1 * n2
    need = int(round(frac_missing * N)) - (N - int(m.sum()))
    if need > 0:
        obs = np.flatnonzero(m.ravel())
        drop = np.random.default_rng(int(rng.integers(1 << 31))).choice(obs, size=min(need, obs.size - 1),
                                                                          replace=False)
        mr = m.ravel().copy()
        mr[drop] = False
        m = mr.reshape(n1, n2)
    return m


def variance_cells(w: Workload, mask):
    """The workload's kriging-variance targets: n_var_cells of the unobserved cells, a seeded
    choice (var_seed), as sorted flat row-major indices."""
    miss = np.flatnonzero(~np.asarray(mask, bool).ravel())
    k = min(int(w.extra["n_var_cells"]), miss.size)
    return np.sort(np.random.default_rng(w.extra["var_seed"]).choice(miss, k, replace=False)).astype(np.int64)


def make_mask(w: Workload):
    if w.mask == "full":
        return mask_full(w.n1, w.n2)
    if w.mask == "uniform":
        return mask_uniform(w.n1, w.n2, w.frac_missing, w.mask_seed)
    if w.mask == "circles":
        return mask_circles(w.n1, w.n2, w.frac_missing, w.mask_seed)
    if w.mask == "mixed":
        return mask_mixed(w.n1, w.n2, w.frac_missing, w.mask_seed)
    raise ValueError(w.mask)


def normals(shape, seed: int):
    """Standard normal draws (NumPy PCG64 stream ``seed``)."""
    return np.random.default_rng(seed).standard_normal(shape)


def uniform_sites(m: int, seed: int):
    """m sites uniform on the unit square, shape (m, 2)."""
    return np.random.default_rng(seed).random((m, 2))


def field_noise(M1: int, M2: int, seed: int):
    """Complex white noise for a circulant-embedding sample on an M1 x M2 torus,
    as a (2, M1, M2) float64 array (real part, imaginary part)."""
    return normals((2, M1, M2), seed)


def serve_requests(n_requests: int, seed: int, side_min: int = 128, side_max: int = 2048,
                   rate: float = 1.0):
    """Poisson-arrival request stream: side n = round(exp(U[ln side_min, ln side_max])),
    missing share U[0.1, 0.9], nu in {1/2, 3/2}, range U[0.02, 0.2], tau2 U[0.01, 0.3],
    kind 'loglik' or 'krige' with equal odds; arrival gaps Exp(rate)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(side_min), math.log(side_max)))))
        out.append(dict(id=k, arrival=t, n=n,
                        frac_missing=float(rng.uniform(0.1, 0.9)),
                        nu=float(rng.choice([0.5, 1.5])),
                        range=float(rng.uniform(0.02, 0.2)),
                        tau2=float(rng.uniform(0.01, 0.3)),
                        kind=("loglik" if rng.random() < 0.5 else "krige"),
                        mask_seed=int(rng.integers(1 << 31)),
                        data_seed=int(rng.integers(1 << 31))))
    return out


def data_noise(M1: int, M2: int, p: int, seed: int):
    """White noise for one synthetic data set: (xi, eps) with xi the (2, M1, M2)
    complex field noise of a circulant-embedding sample and eps the (p,) nugget
    noise.  Both are fixed by ``seed``."""
    return normals((2, M1, M2), seed), normals(p, seed + 7919)
