"""Seeded synthetic inputs for the fractional-Laplacian workloads.

This module holds no arithmetic of the discretization: it only draws grids,
random smooth fields, problem mixes and arrival times.  Both the FP64 oracle
side (tests, CPU baseline) and the GPU side (tests, bench) take their inputs
from here, so the two never share anything else.

Layout: a field on the interior grid of (-1, 1)^d with n points per axis is a
C-ordered float64 array of shape (n,) * d; the last axis is x^{(1)} (fastest).
Base seed 2103.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 2103


def interior_grid(n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """x_i = lo + i h, i = 1..n, h = (hi - lo) / (n + 1)."""
    h = (hi - lo) / (n + 1)
    return lo + h * np.arange(1, n + 1)


def radius2(d: int, n: int) -> np.ndarray:
    x = interior_grid(n)
    grids = np.meshgrid(*([x] * d), indexing="ij")
    return sum(g * g for g in grids)


def ball_power(d: int, n: int, s: float) -> np.ndarray:
    """u = (1 - |x|^2)_+^s on the interior grid."""
    return np.clip(1.0 - radius2(d, n), 0.0, None) ** s


def ball_power_rhs(d: int, n: int, alpha: float) -> np.ndarray:
    """Right-hand side f whose exact solution is u = (1 - |x|^2)_+^{1+alpha/2}
    (g = 0): 2^alpha Gamma(2+alpha/2) Gamma((d+alpha)/2) / Gamma(d/2)
    * (1 - (1 + alpha/d) |x|^2), the s = 1 + alpha/2 case of Eq. (fun0)."""
    pref = 2.0 ** alpha * math.gamma(2 + alpha / 2) * math.gamma((d + alpha) / 2) / math.gamma(d / 2)
    return pref * (1.0 - (1.0 + alpha / d) * radius2(d, n))


def smooth_field(d: int, n: int, seed: int, modes: int = 32, kmax: int = 16) -> np.ndarray:
    """u = sum_{j<modes} c_j cos(pi k_j . x + phi_j), k_j uniform on
    {-kmax..kmax}^d minus 0, c_j ~ N(0,1) / (1 + |k_j|^2), phi_j ~ U(0, 2 pi).

    Evaluated separably: cos(a_1 + ... + a_d) is expanded into products of
    cos(a_i) and sin(a_i) along each axis (axis 0 carries phi_j)."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < modes:
        k = rng.integers(-kmax, kmax + 1, size=d)
        if np.any(k):
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    cs = rng.standard_normal(modes) / (1.0 + np.sum(ks * ks, axis=1))
    phis = rng.uniform(0.0, 2.0 * math.pi, size=modes)
    x = interior_grid(n)
    ang = [math.pi * ks[:, i:i + 1] * x[None, :] for i in range(d)]      # (modes, n) per axis
    ang[0] = ang[0] + phis[:, None]
    C = [np.cos(a) for a in ang]
    S = [np.sin(a) for a in ang]
    if d == 1:
        return cs @ C[0]
    if d == 2:
        # cos(a+b) = cos a cos b - sin a sin b
        return (C[0].T * cs) @ C[1] - (S[0].T * cs) @ S[1]
    # cos(a+b+c) = cos a cos b cos c - cos a sin b sin c - sin a cos b sin c - sin a sin b cos c
    u = np.zeros((n, n, n))
    for sa, sb, sc, sg in ((C, C, C, 1.0), (C, S, S, -1.0), (S, C, S, -1.0), (S, S, C, -1.0)):
        ab = np.einsum("ji,jk->jik", sa[0] * cs[:, None], sb[1])          # (modes, n, n)
        u += sg * np.einsum("jik,jl->ikl", ab, sc[2])
    return u


def smooth_fields(d: int, n: int, count: int, seed0: int = BASE_SEED) -> np.ndarray:
    """``count`` fields, field j seeded with seed0 + j; shape (count,) + (n,) * d."""
    return np.stack([smooth_field(d, n, seed0 + j) for j in range(count)])


@dataclass
class Problem:
    d: int
    n: int
    alpha: float
    degree: int
    lam: float
    seed: int


def batch_problems(count: int = 256, seed: int = BASE_SEED) -> list[Problem]:
    """Mixed problems: d in {1, 2} with equal odds; 1D n log-uniform in
    [63, 4095], 2D side log-uniform in [63, 511]; alpha ~ U(0.1, 1.9); degree
    uniform in {0, 1, 2} (n made odd when degree = 2, so N = n + 1 is even);
    lambda ~ U(0, 2)."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        d = 1 if rng.random() < 0.5 else 2
        hi = 4095 if d == 1 else 511
        n = int(round(math.exp(rng.uniform(math.log(63), math.log(hi)))))
        alpha = float(rng.uniform(0.1, 1.9))
        degree = int(rng.integers(0, 3))
        lam = float(rng.uniform(0.0, 2.0))
        if degree == 2 and n % 2 == 0:
            n += 1
        out.append(Problem(d, n, alpha, degree, lam, seed * 1000 + j))
    return out


def arrival_times(rate: float = 200.0, duration: float = 60.0, seed: int = BASE_SEED) -> np.ndarray:
    """Poisson arrivals: exponential gaps with mean 1/rate, up to ``duration`` s."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.array(out)
        out.append(t)


def served_problems(count: int, seed: int = BASE_SEED, sides3d=(63, 127, 255)) -> list[Problem]:
    """Request mix: d in {1, 2, 3} with weights 0.4/0.4/0.2; 1D/2D sizes as in
    ``batch_problems``; 3D side uniform over ``sides3d``."""
    rng = np.random.default_rng(seed + 1)
    out = []
    for j in range(count):
        r = rng.random()
        d = 1 if r < 0.4 else (2 if r < 0.8 else 3)
        if d == 3:
            n = int(sides3d[rng.integers(0, len(sides3d))])
        else:
            hi = 4095 if d == 1 else 511
            n = int(round(math.exp(rng.uniform(math.log(63), math.log(hi)))))
        alpha = float(rng.uniform(0.1, 1.9))
        degree = int(rng.integers(0, 3))
        lam = float(rng.uniform(0.0, 2.0))
        if degree == 2 and n % 2 == 0:
            n += 1
        out.append(Problem(d, n, alpha, degree, lam, seed * 7919 + j))
    return out
