"""FP64 CPU oracle: operator-factorization scheme for (-Delta)^{alpha/2} and its
tempered form on uniform grids of (-1, 1)^d, d = 1, 2, 3.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product never
imports this module.

Notation follows Section 2 of the paper.  The splitting parameter gamma in
(alpha, 2] defaults to 2 (used in all of Section 3), zeta = floor(gamma / 2):
1 at gamma = 2, 0 below (Eq. (gamma2)).  N intervals per
axis, h = L / N, n = N - 1 interior points per axis; arrays of grid values
have shape (n,) * d.  The operator is symmetric under permutations of the
axes (the weights are, and so is every rule below), so the axis order of an
array does not matter.

Readings of the paper that this oracle takes (each pinned by a test):
  * Appendix, p = 2: the even-k and k = N weight formulas carry index typos;
    the oracle does not use the appendix for its weights at all (it
    integrates Eq. (wi-1D) numerically); ``weights_1d_appendix`` restates
    the appendix with xi_{k-3/2}, xi_{k+3/2} and xi_{N-3/2} in place of the
    printed xi_{k-1/2}, xi_{k+1/2}, xi_{N-3/4}, and a test checks the two agree.
  * Origin value Phi(x, xi_0) (Eq. (gamma1) and its 2D analogue): replaced by
    (1/d) sum_i sum_j e_j Phi(x, j h e_i) with e = (1,) for p in {0, 1} and
    e = (4/3, -1/3) for p = 2.  In 1D this is Eq. (gamma1) for p <= 1 and the
    fourth-order difference for p = 2; in 2D with p = 1 it is the a_10 of
    Eq. (2D-scheme) together with a_11 = omega_11 / |xi_11|^2 (no zeta term).
    These reproduce Tables 3-2-1, 3-1-2, 3-1-3 and 3-2-2.
  * 3D scheme (omitted by the paper, Sec. 2): the same rules with d = 3.
  * Tempered kernel (Remark 2.2): mu -> |xi|^{2-d-alpha} exp(-lambda |xi|),
    with the normalisation c_bar_{d,alpha} := c_{d,alpha} so that lambda = 0
    is the fractional Laplacian (Example 3.2.2).
  * Degrees p = 3, 4 (the paper only says higher degrees raise the accuracy):
    Lagrange bases on elements of p intervals, origin rules of order 6 and 8.
  * Boundary vector (Eq. (L2)): g on every exterior grid point within the
    generator's reach N (per axis, also on rectangles, where the generator's
    cube spans the longest axis), the far field integrated along rays.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy import integrate, linalg, special

def zeta(gamma: float) -> int:
    """zeta = floor(gamma / 2) (after Eq. (L1h)): 1 for gamma = 2, 0 for gamma in (alpha, 2)."""
    return int(math.floor(gamma / 2.0))


# ---------------------------------------------------------------------------
# Constants
# ---------------------------------------------------------------------------

def c_dalpha(d: int, alpha: float) -> float:
    """c_{d,alpha} = 2^{alpha-1} alpha Gamma((d+alpha)/2) / (pi^{d/2} Gamma(1-alpha/2)),
    the normalisation defined after Eq. (fL-nD)."""
    return (2.0 ** (alpha - 1.0) * alpha * math.gamma((d + alpha) / 2.0)
            / (math.pi ** (d / 2.0) * math.gamma(1.0 - alpha / 2.0)))


def _radial_moment(a: float, lam_c, H: float):
    """int_0^H r^{a-1} exp(-lam_c r) dr (a > 0), exactly, via the regularised
    lower incomplete gamma function of scipy."""
    lam_c = np.asarray(lam_c, dtype=np.float64)
    if np.all(lam_c == 0.0):
        return np.full(lam_c.shape, H ** a / a)
    out = np.empty_like(lam_c)
    zero = lam_c == 0.0
    out[zero] = H ** a / a
    lc = lam_c[~zero]
    out[~zero] = special.gamma(a) * special.gammainc(a, lc * H) / lc ** a
    return out


def far_field(d: int, alpha: float, L: float, lam: float = 0.0) -> float:
    """F_d = int over R_+^d minus [0, L]^d of |xi|^{-d-alpha} exp(-lambda |xi|) dxi,
    the u(x) part of Eq. (L2) (1D: Eq. (L2h), 1/(alpha L^alpha) when lambda = 0).

    The region is split by the coordinate that is largest: xi = rho (1, s),
    rho > L, s in [0, 1]^{d-1}, Jacobian rho^{d-1}; the d pieces are equal.
    """
    def radial(cs: float) -> float:
        # int_L^inf r^{-1-alpha} e^{-lambda c r} dr
        if lam == 0.0:
            return L ** (-alpha) / alpha
        val, _ = integrate.quad(lambda r: r ** (-1.0 - alpha) * math.exp(-lam * cs * r),
                                L, np.inf, epsabs=0.0, epsrel=1e-13, limit=200)
        return val

    if d == 1:
        return radial(1.0)
    xs, ws = special.roots_legendre(48)
    s, w = 0.5 * (xs + 1.0), 0.5 * ws
    total = 0.0
    if d == 2:
        for si, wi in zip(s, w):
            cs = math.sqrt(1.0 + si * si)
            total += wi * cs ** (-d - alpha) * radial(cs)
    elif d == 3:
        for si, wi in zip(s, w):
            for sj, wj in zip(s, w):
                cs = math.sqrt(1.0 + si * si + sj * sj)
                total += wi * wj * cs ** (-d - alpha) * radial(cs)
    else:
        raise ValueError("d must be 1, 2 or 3")
    return d * total


# ---------------------------------------------------------------------------
# Weight integrals omega_k^p  (Eq. (wi-1D), Eq. (2D-scheme0) and its 3D analogue)
# ---------------------------------------------------------------------------

def axis_elements(N: int, h: float, p: int):
    """Elements of the 1D Lagrange basis of degree p on the nodes xi_k = k h,
    k = 0..N, as used in Eq. (interpolation).

    Returns a list of (lo, hi, [(node, roots, scale), ...]); on [lo, hi] the
    basis function of ``node`` is scale * prod(xi - root for root in roots).
      p = 0: indicator of [xi_{k-1/2}, xi_{k+1/2}] cut to [0, L];
      p = 1: hat functions on the cells [j h, (j+1) h];
      p = 2: quadratic Lagrange polynomials on [2m h, (2m+2) h] (N even);
      p = 3, 4: Lagrange polynomials of degree p on [p m h, (p m + p) h] (N a
             multiple of p; the higher degrees the paper says raise the accuracy further).
    """
    L = N * h
    els = []
    if p == 0:
        for k in range(N + 1):
            els.append((max(0.0, (k - 0.5) * h), min(L, (k + 0.5) * h), [(k, (), 1.0)]))
    elif p in (1, 2, 3, 4):
        if N % p:
            raise ValueError(f"p = {p} needs a number of intervals N divisible by {p}")
        for m in range(N // p):
            pts = [(p * m + t) * h for t in range(p + 1)]
            loc = []
            for t in range(p + 1):
                others = tuple(pts[s] for s in range(p + 1) if s != t)
                scale = 1.0 / np.prod([pts[t] - o for o in others])
                loc.append((p * m + t, others, scale))
            els.append((pts[0], pts[-1], loc))
    else:
        raise ValueError("p must be 0, 1, 2, 3 or 4")
    return els


def _eval_local(loc, x):
    """Values of the local basis functions ``loc`` at points x: shape (nloc,) + x.shape."""
    out = []
    for _, roots, scale in loc:
        v = np.full(np.shape(x), scale)
        for r in roots:
            v = v * (x - r)
        out.append(v)
    return np.array(out)


def _origin_block(d, alpha, lam, H, loc, qs=24, gamma=2.0):
    """int over [0, H]^d of prod_i phi_{l_i}(xi_i) |xi|^{gamma-d-alpha} exp(-lambda |xi|),
    for every choice (l_1..l_d) of local basis functions on the origin element.

    For degrees p <= 2 (and in 1D) by ``_origin_duffy`` on the whole element.  For p >= 3
    in d >= 2 the element [0, p h]^d is cut into its p^d cells of side h: the cell at the
    origin by ``_origin_duffy`` on [0, h]^d, every other cell (the integrand is smooth
    there) by a 24-point tensor Gauss-Legendre rule with the basis functions evaluated in
    product form.  (The monomial expansion over the whole element multiplies the degree-p d
    products by up to (H / h)^{p d}, 4^12 for p = 4 in 3D, and cancels to 1e-11 relative;
    on [0, h]^d it does not.)
    """
    p = len(loc) - 1
    if d == 1 or p <= 2:
        return _origin_duffy(d, alpha, lam, H, loc, qs, gamma)
    h = H / p
    out = _origin_duffy(d, alpha, lam, h, loc, qs, gamma)
    xs, ws = special.roots_legendre(24)
    for cell in itertools.product(range(p), repeat=d):
        if not any(cell):
            continue
        X, WB = [], []
        for c in cell:
            x = (c + 0.5 * (xs + 1.0)) * h
            X.append(x)
            WB.append(0.5 * h * ws * _eval_local(loc, x))          # (nloc, q)
        grids = np.meshgrid(*X, indexing="ij")
        r = np.sqrt(sum(g * g for g in grids))
        mu = r ** (gamma - d - alpha) * np.exp(-lam * r)           # (q,)*d
        letters = "abc"[:d]                                        # quadrature axes
        spec = ",".join(f"{'lmn'[i]}{letters[i]}" for i in range(d)) + "," + letters + "->" + "lmn"[:d]
        out += np.einsum(spec, *WB, mu, optimize=True)
    return out


def _origin_duffy(d, alpha, lam, H, loc, qs=24, gamma=2.0):
    """int over [0, H]^d of prod_i phi_{l_i}(xi_i) |xi|^{gamma-d-alpha} exp(-lambda |xi|)
    for every choice (l_1..l_d) of local basis functions given on an element that
    contains [0, H]^d.

    Duffy split into the d pyramids {xi_i = max_j xi_j}: xi = r (s with s_i = 1),
    Jacobian r^{d-1}, |xi| = r c(s), c = sqrt(1 + |s|^2); the radial factor is
    r^{gamma-1-alpha} times a polynomial in r times exp(-lambda c r), integrated
    exactly (incomplete gamma); the s-integral uses Gauss-Legendre.
    """
    nloc = len(loc)
    polys = [scale * np.poly(np.array(roots, dtype=np.float64))[::-1] if roots else np.array([scale])
             for _, roots, scale in loc]  # ascending monomial coefficients in xi
    beta = d + alpha - gamma
    out = np.zeros((nloc,) * d)
    if d == 1:
        for l in range(nloc):
            for m, cm in enumerate(polys[l]):
                out[l] += cm * _radial_moment(gamma - alpha + m, np.array([lam]), H)[0]
        return out
    xs, ws = special.roots_legendre(qs)
    s1, w1 = 0.5 * (xs + 1.0), 0.5 * ws
    grids = np.meshgrid(*([s1] * (d - 1)), indexing="ij")
    S = np.stack([g.reshape(-1) for g in grids], axis=1)            # (Q, d-1)
    Wq = np.prod(np.meshgrid(*([w1] * (d - 1)), indexing="ij"), axis=0).reshape(-1)
    cs = np.sqrt(1.0 + np.sum(S * S, axis=1))
    maxdeg = sum(len(pl) - 1 for pl in polys[:1]) * d
    R = np.stack([_radial_moment(gamma - alpha + m, lam * cs, H) for m in range(maxdeg + 1)], axis=1)
    base = Wq * cs ** (-beta)                                          # (Q,)
    for i in range(d):                                                 # pyramid: axis i is the largest
        coords = []
        col = 0
        for j in range(d):
            if j == i:
                coords.append(np.ones_like(cs))
            else:
                coords.append(S[:, col])
                col += 1
        for ls in itertools.product(range(nloc), repeat=d):
            # polynomial in r: prod_j phi_{l_j}(r s_j) = prod_j sum_m c_m s_j^m r^m
            P = np.ones((len(cs), 1))
            for j, l in enumerate(ls):
                pj = polys[l][None, :] * coords[j][:, None] ** np.arange(len(polys[l]))[None, :]
                prod = np.zeros((len(cs), P.shape[1] + pj.shape[1] - 1))
                for m1 in range(P.shape[1]):
                    for m2 in range(pj.shape[1]):
                        prod[:, m1 + m2] += P[:, m1] * pj[:, m2]
                P = prod
            out[ls] += np.sum(base * np.sum(P * R[:, :P.shape[1]], axis=1))
    return out


def _gauss_points(lo, hi, q):
    xs, ws = special.roots_legendre(q)
    return 0.5 * (hi - lo) * xs + 0.5 * (hi + lo), 0.5 * (hi - lo) * ws


def weights(d: int, N: int, h: float, alpha: float, p: int, lam: float = 0.0, q: int = 20,
            gamma: float = 2.0, first=None) -> np.ndarray:
    """omega_k^p for every k in {0..N}^d (Eq. (wi-1D); Eq. (2D-scheme0); Remark 2.2 for lambda > 0).

    omega_k = int over [0, L]^d of prod_i phi_{k_i}(xi_i) mu(xi) dxi with
    mu(xi) = |xi|^{gamma-d-alpha} exp(-lambda |xi|) (mu_gamma of Eq. (eq0)), summed element by element:
    the origin element by ``_origin_block``; every other element, where the
    integrand is smooth, by a q^d-point tensor Gauss-Legendre rule.

    ``first`` (d >= 2): a range of element indices along the first array axis;
    only the elements in that range are summed (the sum over all ranges of a
    partition is the whole array; a test driver uses this to spread the 3D
    generator of the largest grids over processes).
    """
    els = axis_elements(N, h, p)
    ne = len(els)
    nloc = len(els[0][2])
    H0 = els[0][1]
    X = np.empty((ne, q))
    W = np.empty((ne, q))
    B = np.empty((ne, nloc, q))
    nodes = np.empty((ne, nloc), dtype=np.int64)
    for e, (lo, hi, loc) in enumerate(els):
        X[e], W[e] = _gauss_points(lo, hi, q)
        B[e] = _eval_local(loc, X[e])
        nodes[e] = [nd for nd, _, _ in loc]
    WB = W[:, None, :] * B                                          # (ne, nloc, q)
    omega = np.zeros((N + 1,) * d)
    letters = "abc"[: d - 1]
    qlet = "pqr"[: d - 1]
    spec = ",".join(f"{letters[i]}{qlet[i]}" for i in range(d - 1))
    spec = (spec + "," if spec else "") + "elz," + "e" + "".join(qlet) + "z->e" + letters + "l"
    ranges = [range(ne)] * (d - 1)
    if first is not None and d > 1:
        ranges[0] = first
    for outer in itertools.product(*ranges):
        r2 = np.zeros((ne,) + (q,) * d)
        for i, e in enumerate(outer):
            shape = [1] * (d + 1)
            shape[1 + i] = q
            r2 = r2 + (X[e] ** 2).reshape(shape)
        shape = [ne] + [1] * (d - 1) + [q]
        r2 = r2 + (X ** 2).reshape(shape)
        r = np.sqrt(r2)
        Mu = r ** (gamma - d - alpha)
        if lam != 0.0:
            Mu = Mu * np.exp(-lam * r)
        ops = [WB[e] for e in outer] + [WB, Mu]
        C = np.einsum(spec, *ops, optimize=True)                      # (ne, nloc.., nloc)
        if all(e == 0 for e in outer):
            C[0] = _origin_block(d, alpha, lam, H0, els[0][2], gamma=gamma)
        idx = []
        for i, e in enumerate(outer):
            shape = [1] * (d + 1)
            shape[1 + i] = nloc
            idx.append(nodes[e].reshape(shape))
        shape = [ne] + [1] * (d - 1) + [nloc]
        idx.append(nodes.reshape(shape))
        idx = np.broadcast_arrays(*idx)
        np.add.at(omega, tuple(idx), C)
    return omega


def weights_at(d: int, N: int, h: float, alpha: float, p: int, lam: float, nodes, q: int = 20,
               gamma: float = 2.0) -> np.ndarray:
    """omega_k^p for the multi-indices in ``nodes`` only (same integrals as
    ``weights``: origin element by ``_origin_block``, the others by tensor
    Gauss-Legendre), for sizes where the whole generator is out of reach."""
    els = axis_elements(N, h, p)
    owner = [[] for _ in range(N + 1)]
    for e, (_, _, loc) in enumerate(els):
        for l, (nd, _, _) in enumerate(loc):
            owner[nd].append((e, l))
    origin = _origin_block(d, alpha, lam, els[0][1], els[0][2], gamma=gamma)
    xs, ws = special.roots_legendre(q)
    out = np.empty(len(nodes))
    for t, k in enumerate(nodes):
        tot = 0.0
        for combo in itertools.product(*[owner[int(ki)] for ki in k]):
            es = [e for e, _ in combo]
            ls = [l for _, l in combo]
            if all(e == 0 for e in es):
                tot += origin[tuple(ls)]
                continue
            r2 = np.zeros((q,) * d)
            wb = np.ones((q,) * d)
            for i, (e, l) in enumerate(combo):
                lo, hi, loc = els[e]
                x = 0.5 * (hi - lo) * xs + 0.5 * (hi + lo)
                w = 0.5 * (hi - lo) * ws * _eval_local([loc[l]], x)[0]
                shape = [1] * d
                shape[i] = q
                r2 = r2 + (x * x).reshape(shape)
                wb = wb * w.reshape(shape)
            r = np.sqrt(r2)
            tot += float(np.sum(wb * r ** (gamma - d - alpha) * np.exp(-lam * r)))
        out[t] = tot
    return out


def weights_1d_appendix(N: int, h: float, alpha: float, p: int, gamma: float = 2.0) -> np.ndarray:
    """Closed forms of the Appendix for omega_k^p, 1D, lambda = 0, sigma_0 = gamma - alpha.

    p = 2, even 0 < k < N and k = N: uses xi_{k-3/2}, xi_{k+3/2} and
    xi_{N-3/2} where the paper prints xi_{k-1/2}, xi_{k+1/2}, xi_{N-3/4}
    (the printed forms disagree with Eq. (wi-1D); the corrected ones agree).
    """
    s0 = gamma - alpha
    s1, s2 = s0 + 1.0, s0 + 2.0
    xi = lambda t: t * h  # noqa: E731
    w = np.zeros(N + 1)
    if p == 0:
        w[0] = xi(0.5) ** s0
        w[N] = xi(N) ** s0 - xi(N - 0.5) ** s0
        for k in range(1, N):
            w[k] = xi(k + 0.5) ** s0 - xi(k - 0.5) ** s0
        return w / s0
    if p == 1:
        w[0] = h ** s1
        w[N] = xi(N - 1) ** s1 - xi(N) ** s1 + s1 * h * xi(N) ** s0
        for k in range(1, N):
            w[k] = xi(k + 1) ** s1 + xi(k - 1) ** s1 - 2.0 * xi(k) ** s1
        return w / (h * s1 * s0)
    if p == 2:
        if N % 2:
            raise ValueError("p = 2 needs even N")
        w[0] = xi(2) ** s2 / s2 - xi(3) * xi(2) ** s1 / s1 + 2 * h * h * xi(2) ** s0 / s0
        w[N] = ((xi(N) ** s2 - xi(N - 2) ** s2) / s2
                - 2 * xi(N - 1.5) * (xi(N) ** s1 - xi(N - 2) ** s1) / s1
                + xi(N - 1) * xi(N - 2) * (xi(N) ** s0 - xi(N - 2) ** s0) / s0)
        for k in range(1, N):
            if k % 2:
                w[k] = (-2 * (xi(k + 1) ** s2 - xi(k - 1) ** s2) / s2
                        + 4 * xi(k) * (xi(k + 1) ** s1 - xi(k - 1) ** s1) / s1
                        - 2 * xi(k + 1) * xi(k - 1) * (xi(k + 1) ** s0 - xi(k - 1) ** s0) / s0)
            else:
                w[k] = ((xi(k + 2) ** s2 - xi(k - 2) ** s2) / s2
                        - 2.0 / s1 * (xi(k - 1.5) * (xi(k) ** s1 - xi(k - 2) ** s1)
                                      + xi(k + 1.5) * (xi(k + 2) ** s1 - xi(k) ** s1))
                        + 1.0 / s0 * (xi(k - 2) * xi(k - 1) * (xi(k) ** s0 - xi(k - 2) ** s0)
                                      + xi(k + 2) * xi(k + 1) * (xi(k + 2) ** s0 - xi(k) ** s0)))
        return w / (2 * h * h)
    raise ValueError("p must be 0, 1 or 2")


# ---------------------------------------------------------------------------
# Stencil a_k and the multilevel Toeplitz operator  (Eq. (1D-scheme), Eq. (2D-scheme))
# ---------------------------------------------------------------------------

# Weights e_j of the origin rule Phi(x, xi_0) ~ sum_j e_j Phi(x, j h) (per axis): the
# second difference (p <= 1), the fourth-order combination (p = 2: sum e_j = 1,
# sum e_j j^2 = 0) and, for p = 3, the sixth-order one (also sum e_j j^4 = 0), so that
# the origin value is no less accurate than the cubic interpolation around it; p = 4 the
# eighth-order one (sum e_j j^6 = 0 as well).
ORIGIN_RULE = {0: (1.0,), 1: (1.0,), 2: (4.0 / 3.0, -1.0 / 3.0), 3: (1.5, -0.6, 0.1),
               4: (1.6, -0.8, 8.0 / 35.0, -1.0 / 35.0)}


def stencil(d: int, N: int, h: float, alpha: float, p: int, lam: float = 0.0,
            omega: np.ndarray | None = None, q: int = 20, gamma: float = 2.0) -> np.ndarray:
    """Generator a_k, k in {0..N}^d, of the scheme; a[(0,)*d] holds a_0.

    * k != 0: a_k = 2^{z(k)} omega_k / |xi_k|^gamma, z(k) = number of zero entries
      of k (each distinct neighbour x + s o xi_k appears 2^{z(k)} times in the
      sum over m in varkappa_1 of Eq. (eq0)).
    * origin term: zeta omega_0 Phi(x, xi_0) ~ zeta omega_0 (1/d) sum_i sum_j
      e_j Phi(x, j h e_i), which adds 2^{d-1} zeta e_j omega_0 / (d (j h)^2)
      to a_{j e_i} (gamma = 2 only: zeta = 0 below, Eq. (gamma2)).
    * a_0 = -sum_{k != 0} 2^{d-z(k)} a_k - 2^d F_d  (Eq. (1D-scheme): a_0;
      Eq. (2D-scheme): a_00).
    """
    if omega is None:
        omega = weights(d, N, h, alpha, p, lam, q=q, gamma=gamma)
    K = np.indices((N + 1,) * d)
    k2 = np.sum(K * K, axis=0)
    z = np.sum(K == 0, axis=0)
    nz = k2 > 0
    a = np.zeros_like(omega)
    if gamma == 2.0:
        a[nz] = 2.0 ** z[nz] * omega[nz] / (h * h * k2[nz])
    else:
        a[nz] = 2.0 ** z[nz] * omega[nz] / (h * np.sqrt(k2[nz])) ** gamma
    o0 = omega[(0,) * d]
    for i in range(d):
        for j, ej in enumerate(ORIGIN_RULE[p], start=1):
            idx = [0] * d
            idx[i] = j
            a[tuple(idx)] += 2.0 ** (d - 1) * zeta(gamma) * ej * o0 / (d * (j * h) ** 2)
    mult = 2.0 ** (d - z)
    a[(0,) * d] = -math.fsum((mult * a)[nz].ravel()) - 2.0 ** d * far_field(d, alpha, N * h, lam)
    return a


def grid_shape(a: np.ndarray, n) -> tuple:
    """The grid's array shape: (n,)*d for an int n, else the given shape (one extent per
    array axis, C order; a rectangular grid of Sec. 2.2 with N_2 < N_1)."""
    return (int(n),) * a.ndim if np.isscalar(n) else tuple(int(v) for v in n)


def toeplitz_matrix(a: np.ndarray, n) -> np.ndarray:
    """Dense symmetric multilevel Toeplitz matrix T with T[i, j] = a[|i - j|]
    (componentwise), rows/columns in C order of the grid of shape grid_shape(a, n)
    (A^{(1)} after Eq. (1D-scheme); A^{(2)} after Eq. (2D-scheme), block Toeplitz with
    Toeplitz blocks also when N_2 < N_1)."""
    d = a.ndim
    I = np.indices(grid_shape(a, n)).reshape(d, -1)
    D = tuple(np.abs(I[i][:, None] - I[i][None, :]) for i in range(d))
    return a[D]


def operator_matrix(a: np.ndarray, c: float, n) -> np.ndarray:
    """A = -c_{d,alpha} T(a)."""
    return -c * toeplitz_matrix(a, n)


def apply_dense(a: np.ndarray, c: float, u: np.ndarray) -> np.ndarray:
    """y = A u with A = -c T(a), by the dense sum of the scheme (all rows)."""
    return (operator_matrix(a, c, u.shape) @ u.reshape(-1)).reshape(u.shape)


def apply_rows(a: np.ndarray, c: float, u: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """(A u)_i = -c sum_j a[|i - j|] u_j for the multi-indices i in ``rows`` (R, d)."""
    d = u.ndim
    J = np.indices(u.shape).reshape(d, -1)
    uf = u.reshape(-1)
    out = np.empty(len(rows))
    for t, r in enumerate(np.asarray(rows)):
        D = tuple(np.abs(J[i] - r[i]) for i in range(d))
        out[t] = -c * math.fsum(a[D] * uf)
    return out


def spectral_bound(a: np.ndarray, c: float, n) -> float:
    """max |eigenvalue| of the circulant of side 2 n_i per axis whose leading block is
    A = -c T(a) on the grid of shape grid_shape(a, n) (first column a_{min(j, M_i - j)}
    for min(j, M_i - j) < n_i, zero elsewhere).  A is a principal submatrix of that
    symmetric circulant, so this bounds ||A||_2 from above, and it is the largest
    |Lambda| of an embedding of A; the eigenvalues are the DFT of the first column
    (numpy's FFT as the library primitive).  Used to scale apply errors."""
    shp = grid_shape(a, n)
    C = np.zeros(tuple(2 * v for v in shp))
    idx = []
    for v in shp:
        j = np.arange(2 * v)
        m = np.minimum(j, 2 * v - j)
        idx.append(np.where(m < v, m, -1))
    grids = np.meshgrid(*idx, indexing="ij")
    live = np.all([g >= 0 for g in grids], axis=0)
    C[live] = a[tuple(g[live] for g in grids)]
    lam = -c * np.real(np.fft.fftn(C))
    return float(np.max(np.abs(lam)))


def norm_bound(a: np.ndarray, c: float, n) -> float:
    """c * sum over the offsets o in (-(n_i-1)..n_i-1) per axis of |a_{|o|}|: the largest
    absolute row sum bound, hence an upper bound of ||A||_2 for the grid of shape
    grid_shape(a, n); used to normalise apply errors."""
    sub = a[tuple(slice(0, v) for v in grid_shape(a, n))]
    K = np.indices(sub.shape)
    mult = 2.0 ** np.sum(K > 0, axis=0)
    return c * float(np.sum(mult * np.abs(sub)))


# ---------------------------------------------------------------------------
# Boundary vector b  (Eq. (1D-scheme): b_i; Eq. (2D-scheme): b_ij)
# ---------------------------------------------------------------------------

def extended_samples(d: int, N: int, h: float, g, lo: float = -1.0, shape=None) -> np.ndarray:
    """g at the extended grid points lo + e h, e in [1-N, n_i+N] on array axis i (axis i
    of the array = coordinate i; n_i = shape[i], default N - 1 on every axis: the square
    grid), zero at the interior points e in [1, n_i] (there the unknown u, not g,
    enters the scheme).  The generator reaches N points on every axis (its cube has
    side L = N h, Sec. 2.2 for N_2 < N_1).  Shape (n_i + 2N)_i."""
    shape = (N - 1,) * d if shape is None else tuple(int(v) for v in shape)
    exts = [np.arange(1 - N, m + N + 1) for m in shape]
    grids = np.meshgrid(*[lo + e * h for e in exts], indexing="ij")
    G = g(np.stack(grids, axis=-1))
    inside = np.ones(G.shape, dtype=bool)
    for i, (e, m) in enumerate(zip(exts, shape)):
        sh = [1] * d
        sh[i] = len(e)
        inside = inside & ((e >= 1) & (e <= m)).reshape(sh)
    return np.where(inside, 0.0, G)


def boundary_near(a: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Near-field part of Eq. (L2) at every interior point: sum over o in [-N, N]^d
    of a_{|o|} G[x_i + o h], G the extended samples (``extended_samples``; zero
    inside, so only exterior points count), N + 1 = the generator's extent and
    n_i = G.shape[i] - 2N.  Shape (n_i)_i."""
    d = G.ndim
    N = a.shape[0] - 1
    shape = tuple(m - 2 * N for m in G.shape)
    near = np.zeros(shape)
    for o in itertools.product(range(-N, N + 1), repeat=d):
        coef = a[tuple(abs(t) for t in o)]
        sl = tuple(slice(N + t, N + t + m) for t, m in zip(o, shape))  # interior index i+1 -> ext offset (i+1)-(1-N)
        near += coef * G[sl]
    return near


def boundary_far(d: int, N: int, h: float, alpha: float, g, lam: float = 0.0, lo: float = -1.0,
                 nq: int = 96, shape=None) -> np.ndarray:
    """Far-field part of Eq. (L2) at every interior point:
    sum_{m in varkappa_1} int over Upsilon_+^c of g(x_i + (-1)^m o xi)
    |xi|^{-d-alpha} exp(-lambda |xi|) dxi.  xi = rho (1, s) with rho = L / t:
    rho^{-1-alpha} d rho = L^{-alpha} t^{alpha-1} dt, integrated by Gauss-Jacobi
    in t and Gauss-Legendre in s; L = N h, the side of the generator's cube.
    Shape ``shape`` (default (N-1,)*d)."""
    shape = (N - 1,) * d if shape is None else tuple(int(v) for v in shape)
    L = N * h
    xt, wt = special.roots_jacobi(nq, 0.0, alpha - 1.0)     # weight (1+x)^{alpha-1} on [-1, 1]
    t = 0.5 * (xt + 1.0)
    wt = wt * 0.5 ** alpha                                   # int_0^1 t^{alpha-1} f(t) dt
    rho = L / t
    X = np.stack(np.meshgrid(*[lo + (np.arange(m) + 1) * h for m in shape], indexing="ij"), axis=-1)
    far = np.zeros(shape)
    if d == 1:
        for sgn in (-1.0, 1.0):
            vals = g(X[..., None, :] + sgn * rho[:, None])          # (n, nq)
            far += L ** (-alpha) * np.sum(wt * np.exp(-lam * rho) * vals, axis=-1)
    else:
        xs, ws = special.roots_legendre(nq // 2)
        s1, w1 = 0.5 * (xs + 1.0), 0.5 * ws
        S = np.stack([g_.reshape(-1) for g_ in np.meshgrid(*([s1] * (d - 1)), indexing="ij")], axis=1)
        WS = np.prod(np.meshgrid(*([w1] * (d - 1)), indexing="ij"), axis=0).reshape(-1)
        cs = np.sqrt(1.0 + np.sum(S * S, axis=1))
        for i in range(d):
            dirs = np.ones((len(cs), d))
            dirs[:, [j for j in range(d) if j != i]] = S
            for m in itertools.product((-1.0, 1.0), repeat=d):
                sd = dirs * np.array(m)                              # (Q, d)
                for ti in range(nq):
                    pts = X[..., None, :] + rho[ti] * sd            # (n..,Q,d)
                    wq = WS * cs ** (-d - alpha) * np.exp(-lam * rho[ti] * cs)
                    far += L ** (-alpha) * wt[ti] * np.sum(wq * g(pts), axis=-1)
    return far


def boundary_vector(d: int, N: int, h: float, alpha: float, a: np.ndarray, c: float, g,
                    lam: float = 0.0, lo: float = -1.0, nq: int = 96, shape=None) -> np.ndarray:
    """-c b_i for every interior point: b_i is the near-field sum of a_{|o|} g
    over the exterior grid points x_i + o h (o in [-N, N]^d, ``boundary_near``)
    plus the far field (``boundary_far``), Eq. (L2).  ``g`` maps an array
    (..., d) of points to values."""
    near = boundary_near(a, extended_samples(d, N, h, g, lo, shape))
    far = boundary_far(d, N, h, alpha, g, lam, lo, nq, shape)
    return -c * (near + far)


# ---------------------------------------------------------------------------
# Solves
# ---------------------------------------------------------------------------

def solve_dense(a: np.ndarray, c: float, rhs: np.ndarray) -> np.ndarray:
    """Solve A u = rhs by dense Cholesky (A is symmetric positive definite)."""
    A = operator_matrix(a, c, rhs.shape)
    cf = linalg.cho_factor(A, lower=True)
    return linalg.cho_solve(cf, rhs.reshape(-1)).reshape(rhs.shape)


def solve_cg(a: np.ndarray, c: float, rhs: np.ndarray, rtol: float = 1e-12, maxiter: int = 100000):
    """Plain conjugate gradients with the dense apply; returns (u, iterations)."""
    A = operator_matrix(a, c, rhs.shape)
    b = rhs.reshape(-1)
    x = np.zeros_like(b)
    r = b.copy()
    pvec = r.copy()
    rr = r @ r
    bn = math.sqrt(b @ b)
    it = 0
    while math.sqrt(rr) > rtol * bn and it < maxiter:
        q = A @ pvec
        alpha_k = rr / (pvec @ q)
        x += alpha_k * pvec
        r -= alpha_k * q
        rr_new = r @ r
        pvec = r + (rr_new / rr) * pvec
        rr = rr_new
        it += 1
    return x.reshape(rhs.shape), it


# ---------------------------------------------------------------------------
# tau preconditioner (the paper names no solver; this is the preconditioned CG
# the library offers).  The tau matrix of a symmetric Toeplitz matrix T_m with
# first column t_0..t_{m-1} is tau(T_m) = T_m - H_m, H_m the Hankel matrix with
# H_ij = t_{i+j+2} (i + j <= m - 3) and t_{2m-i-j} (i + j >= m + 1), 0-based;
# it is diagonalised by the sine transform S_jk = sqrt(2/(m+1)) sin(pi j k/(m+1)),
# j, k = 1..m, with eigenvalues the symbol t_0 + 2 sum_j t_j cos(pi j k/(m+1)).
# Multilevel: tensor products over the axes.  For n interior points the
# preconditioner is the tau matrix of size m = M/2 - 1 >= n (M the FFT length
# of the apply) of the Toeplitz matrix whose generator is a zero beyond n - 1,
# restricted to the leading n^d block: P = R tau(T_m)^{-1} R^T.  PARITY
# UNPINNED against the paper (it has no solver); pinned to the definition of
# the tau algebra by the Hankel identity in tests.
# ---------------------------------------------------------------------------

def fft_len(n: int) -> int:
    """FFT length of the circulant embedding: max(2, 2^ceil(log2(2n - 1)))."""
    M = 2
    while M < 2 * n - 1:
        M *= 2
    return M


def sine_matrix(m: int) -> np.ndarray:
    """Orthogonal, symmetric DST-I matrix of size m."""
    j = np.arange(1, m + 1)
    return math.sqrt(2.0 / (m + 1)) * np.sin(np.pi * np.outer(j, j) / (m + 1))


def tau_hankel_1d(t: np.ndarray) -> np.ndarray:
    """H_m of tau(T_m) = T_m - H_m for the symmetric Toeplitz column t (length m)."""
    m = len(t)
    H = np.zeros((m, m))
    for i in range(m):
        for j in range(m):
            s = i + j
            if s <= m - 3:
                H[i, j] = t[s + 2]
            elif s >= m + 1:
                H[i, j] = t[2 * m - s]
    return H


def tau_symbol(a: np.ndarray, c: float, n, m) -> np.ndarray:
    """Eigenvalues of -c tau(T_m) on k in [1..m_i] per axis: the symbol of the generator
    a (entries |j| <= n_i - 1 along axis i, zero beyond) at theta_k = pi k / (m_i + 1).
    n, m: ints (every axis) or one extent per array axis."""
    d = a.ndim
    ns = grid_shape(a, n)
    ms = grid_shape(a, m)
    out = a[tuple(slice(0, v) for v in ns)].copy()
    for ax in range(d):
        k = np.arange(1, ms[ax] + 1)
        j = np.arange(0, ns[ax])
        Cm = np.cos(np.pi * np.outer(k, j) / (ms[ax] + 1))   # (m_i, n_i)
        Cm[:, 1:] *= 2.0                                       # +-j folded
        out = np.moveaxis(np.tensordot(Cm, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return -c * out


def tau_precond(a: np.ndarray, c: float, v: np.ndarray, m=None) -> np.ndarray:
    """P v = R tau(T_m)^{-1} R^T v with m_i = M_i/2 - 1 per axis (default), v of the grid's shape."""
    d = v.ndim
    ns = v.shape
    ms = tuple(fft_len(x) // 2 - 1 for x in ns) if m is None else grid_shape(a, m)
    if any(mi < ni for mi, ni in zip(ms, ns)):
        raise ValueError("tau system smaller than the problem (an n_i is a power of two)")
    w = np.zeros(ms)
    w[tuple(slice(0, x) for x in ns)] = v
    for ax in range(d):
        S = sine_matrix(ms[ax])
        w = np.moveaxis(np.tensordot(S, np.moveaxis(w, ax, 0), axes=(1, 0)), 0, ax)
    w = w / tau_symbol(a, c, ns, ms)
    for ax in range(d):
        S = sine_matrix(ms[ax])
        w = np.moveaxis(np.tensordot(S, np.moveaxis(w, ax, 0), axes=(1, 0)), 0, ax)
    return w[tuple(slice(0, x) for x in ns)]


def solve_pcg(a: np.ndarray, c: float, rhs: np.ndarray, rtol: float = 1e-12, maxiter: int = 100000):
    """Conjugate gradients preconditioned by tau_precond; stops on the true
    residual ||r|| <= rtol ||rhs||; returns (u, iterations)."""
    A = operator_matrix(a, c, rhs.shape)
    b = rhs.reshape(-1)
    x = np.zeros_like(b)
    r = b.copy()
    z = tau_precond(a, c, r.reshape(rhs.shape)).reshape(-1)
    pvec = z.copy()
    rz = r @ z
    bn = math.sqrt(b @ b)
    it = 0
    while math.sqrt(r @ r) > rtol * bn and it < maxiter:
        q = A @ pvec
        alpha_k = rz / (pvec @ q)
        x += alpha_k * pvec
        r -= alpha_k * q
        z = tau_precond(a, c, r.reshape(rhs.shape)).reshape(-1)
        rz_new = r @ z
        pvec = z + (rz_new / rz) * pvec
        rz = rz_new
        it += 1
    return x.reshape(rhs.shape), it


# ---------------------------------------------------------------------------
# Grids and closed-form references
# ---------------------------------------------------------------------------

def interior_points(N: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """x_i = a + i h, i = 1..N-1 (Sec. 2.1)."""
    h = (hi - lo) / N
    return lo + h * np.arange(1, N)


def radius2(N: int, d: int) -> np.ndarray:
    """|x|^2 on the interior grid of (-1, 1)^d, shape (N-1,)*d."""
    x = interior_points(N)
    grids = np.meshgrid(*([x] * d), indexing="ij")
    return sum(g * g for g in grids)


def fl_ball_power(d: int, alpha: float, s: float, r2) -> np.ndarray:
    """(-Delta)^{alpha/2} (1 - |x|^2)_+^s for |x| < 1:
    2^alpha Gamma(1+s) Gamma((d+alpha)/2) / (Gamma(d/2) Gamma(1+s-alpha/2))
    * 2F1((d+alpha)/2, alpha/2 - s; d/2; |x|^2)  (Eq. (fun0) for d = 1)."""
    pref = (2.0 ** alpha * math.gamma(1 + s) * math.gamma((d + alpha) / 2)
            / (math.gamma(d / 2) * math.gamma(1 + s - alpha / 2)))
    return pref * special.hyp2f1((d + alpha) / 2, alpha / 2 - s, d / 2, np.asarray(r2))


def fl_lorentzian_1d(alpha: float, x) -> np.ndarray:
    """(-Delta)^{alpha/2} 1/(1+x^2) = Gamma(1+alpha) cos((1+alpha) arctan x) / (1+x^2)^{(1+alpha)/2},
    from the pseudo-differential definition Eq. (pseudo) (Fourier transform pi e^{-|k|})."""
    x = np.asarray(x)
    return math.gamma(1 + alpha) * np.cos((1 + alpha) * np.arctan(x)) / (1 + x * x) ** ((1 + alpha) / 2)


def fl_gaussian(d: int, alpha: float, r2) -> np.ndarray:
    """(-Delta)^{alpha/2} exp(-|x|^2) = 2^alpha Gamma((d+alpha)/2)/Gamma(d/2) 1F1((d+alpha)/2; d/2; -|x|^2)
    (Example 3.2.3 states the d = 2 case)."""
    return (2.0 ** alpha * math.gamma((d + alpha) / 2) / math.gamma(d / 2)
            * special.hyp1f1((d + alpha) / 2, d / 2, -np.asarray(r2)))


def build_operator(d: int, N: int, alpha: float, p: int, lam: float = 0.0, L: float = 2.0, q: int = 20):
    """Convenience: (a, c, h) for the scheme on (-1, 1)^d with N intervals."""
    h = L / N
    return stencil(d, N, h, alpha, p, lam, q=q), c_dalpha(d, alpha), h
