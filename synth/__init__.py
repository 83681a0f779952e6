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


def extended_points(d: int, n, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """The grid points lo + e h, e in [1-N, n_i+N] on array axis i (n an int: n_i = n on
    every axis, else one extent per array axis; N = max n_i + 1, h = (hi - lo) / N): the
    interior grid and the exterior points within N h of it, where nonhomogeneous exterior
    data g is sampled.  Shape (n_i + 2N)_i + (d,), indexing "ij"."""
    shape = (int(n),) * d if np.isscalar(n) else tuple(int(v) for v in n)
    N = max(shape) + 1
    h = (hi - lo) / N
    axes = [lo + h * np.arange(1 - N, m + N + 1) for m in shape]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)


def radius2(d: int, n: int) -> np.ndarray:
    x = interior_grid(n)
    grids = np.meshgrid(*([x] * d), indexing="ij")
    return sum(g * g for g in grids)


def ball_power(d: int, n: int, s: float) -> np.ndarray:
    """u = (1 - |x|^2)_+^s on the interior grid."""
    return np.clip(1.0 - radius2(d, n), 0.0, None) ** s


def ball_power_rhs(d: int, n: int, alpha: float) -> np.ndarray:
    """Right-hand side f = (-Delta)^{alpha/2} u of u = (1 - |x|^2)_+^{1+alpha/2}
    on the interior grid of (-1, 1)^d (data of the continuous problem, g = 0).

    Inside the unit ball: 2^alpha Gamma(2+alpha/2) Gamma((d+alpha)/2) / Gamma(d/2)
    * (1 - (1 + alpha/d) |x|^2), the s = 1 + alpha/2 case of Eq. (fun0).
    At the corners of the cube (|x| > 1, d >= 2), where u = 0, the definition
    Eq. (fL-nD) gives f(x) = -c_{d,alpha} int_{|y|<1} u(y) |x - y|^{-d-alpha} dy;
    it is radial, reduced to a 1D integral over rho = |y| (closed-form angular
    integral) and tabulated in r = |x| (see ``_outside_ball``)."""
    pref = 2.0 ** alpha * math.gamma(2 + alpha / 2) * math.gamma((d + alpha) / 2) / math.gamma(d / 2)
    r2 = radius2(d, n)
    f = pref * (1.0 - (1.0 + alpha / d) * r2)
    if d >= 2:
        out = r2 > 1.0
        if np.any(out):
            f[out] = _outside_ball(d, alpha, 1.0 + alpha / 2)(np.sqrt(r2[out]))
    return f


_OUT_CACHE: dict = {}


def _outside_ball(d: int, alpha: float, s: float):
    """r -> -c_{d,alpha} int_{|y|<1} (1-|y|^2)^s |x-y|^{-d-alpha} dy for |x| = r in (1, sqrt(d)].

    Angular integrals in closed form: d = 3, int_{S^2} |x - rho w|^{-3-alpha} dw
    = 2 pi ((r - rho)^{-1-alpha} - (r + rho)^{-1-alpha}) / ((1 + alpha) r rho);
    d = 2, int_0^{2 pi} (a - b cos phi)^{-nu} dphi = 2 pi a^{-nu} 2F1(nu/2, (nu+1)/2; 1; (b/a)^2)
    with a = r^2 + rho^2, b = 2 r rho, nu = 1 + alpha/2.  The rho-integral is
    done by adaptive quadrature on 500 points t = sqrt(r - 1) and interpolated
    by a cubic spline in t."""
    key = (d, round(alpha, 15), round(s, 15))
    if key in _OUT_CACHE:
        return _OUT_CACHE[key]
    from scipy import integrate, interpolate, special
    c = 2.0 ** (alpha - 1) * alpha * math.gamma((d + alpha) / 2) / (math.pi ** (d / 2) * math.gamma(1 - alpha / 2))

    def value(r: float) -> float:
        if d == 3:
            g = lambda rho: rho * (1 - rho * rho) ** s * ((r - rho) ** (-1 - alpha) - (r + rho) ** (-1 - alpha))  # noqa: E731
            v = integrate.quad(g, 0.0, 1.0, epsabs=0.0, epsrel=1e-11, limit=400)[0]
            return -c * 2.0 * math.pi / (r * (1.0 + alpha)) * v
        nu = 1.0 + alpha / 2.0

        def g(rho):
            a = r * r + rho * rho
            return rho * (1 - rho * rho) ** s * 2.0 * math.pi * a ** (-nu) * special.hyp2f1(
                nu / 2, (nu + 1) / 2, 1.0, (2.0 * r * rho / a) ** 2)
        v = integrate.quad(g, 0.0, 1.0, epsabs=0.0, epsrel=1e-11, limit=400)[0]
        return -c * v

    import warnings
    t = np.linspace(1e-3, math.sqrt(math.sqrt(d) - 1.0) + 1e-3, 500)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        vals = np.array([value(1.0 + ti * ti) for ti in t])
    spline = interpolate.CubicSpline(t, vals)
    fn = lambda r: spline(np.sqrt(np.maximum(np.asarray(r) - 1.0, 0.0)))  # noqa: E731
    fn.value = value
    _OUT_CACHE[key] = fn
    return fn


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


def served_problems_repeat(count: int, seed: int = BASE_SEED, fixed: int = 16, share: float = 0.8,
                           sides3d=(63, 127, 255)) -> list[Problem]:
    """The served mix with repeats: a share ``share`` of the requests are drawn
    from ``fixed`` fixed problems (d, n, alpha, degree, lambda), the rest fresh."""
    base = served_problems(fixed, seed=seed + 17, sides3d=sides3d)
    fresh = served_problems(count, seed=seed, sides3d=sides3d)
    rng = np.random.default_rng(seed + 23)
    out = []
    for j in range(count):
        if rng.random() < share:
            b = base[int(rng.integers(0, fixed))]
            out.append(Problem(b.d, b.n, b.alpha, b.degree, b.lam, seed * 104729 + j))
        else:
            out.append(fresh[j])
    return out
