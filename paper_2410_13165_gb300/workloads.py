"""Seeded synthetic inputs shared by the CUDA path's tests and benchmark and by the oracle's tests.

This module holds none of the method's arithmetic: it draws workload parameters from a
counter-based generator and evaluates smooth input fields (initial data, their gradients, target
and source fields) on the lattice nodes. Numbers come from splitmix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), so they are identical on every
machine.

Workload recipe (the paper's data are analytic, Example 2/3): phi0(x) = sum_m a_m sin(kappa_m .
(x - lo) + theta_m) with kappa_m = 2 pi k_m / L, k_m in {1..kmax}^d (independent uniform integer
components), a_m ~ U(-1, 1), theta_m ~ U(0, 2 pi). The exact solution of the L-HE with constant
R is phi0(x - u t) + R t.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + self.next_u64() % (hi - lo + 1)


SEED_BASE = 2410131650


class FourierField:
    """phi(x) = sum_m a_m sin(kappa_m . (x - lo) + theta_m) on a box with lower corner lo."""

    def __init__(self, a, k, theta, L, lo):
        self.a = np.asarray(a, dtype=np.float64)
        self.k = np.asarray(k, dtype=np.int64)
        self.theta = np.asarray(theta, dtype=np.float64)
        self.L = np.asarray(L, dtype=np.float64)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.kappa = 2.0 * np.pi * self.k / self.L[None, :]

    @property
    def d(self):
        return self.k.shape[1]

    def value(self, X: np.ndarray, shift=None) -> np.ndarray:
        """X: (d, S) coordinates; shift: optional displacement subtracted from X (e.g. u t)."""
        Y = X - self.lo[:, None] - (0.0 if shift is None else np.asarray(shift, dtype=np.float64)[:, None])
        return np.sum(self.a[:, None] * np.sin(self.kappa @ Y + self.theta[:, None]), axis=0)

    def grad(self, X: np.ndarray, shift=None) -> np.ndarray:
        Y = X - self.lo[:, None] - (0.0 if shift is None else np.asarray(shift, dtype=np.float64)[:, None])
        c = self.a[:, None] * np.cos(self.kappa @ Y + self.theta[:, None])  # (M, S)
        return self.kappa.T @ c                                             # (d, S)

    def wave_params(self):
        """The same field written as sum_m a_m sin(kappa_m . x + theta'_m) (absolute coordinates)."""
        theta_abs = self.theta - self.kappa @ self.lo
        return list(self.a), [list(r) for r in self.kappa], list(theta_abs)


def fourier_field(d: int, nmodes: int, seed: int, lo=0.0, hi=1.0, kmax: int = 3) -> FourierField:
    rng = SplitMix64(SEED_BASE + seed)
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (d,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (d,))
    a, k, th = [], [], []
    for _ in range(nmodes):
        a.append(rng.uniform(-1.0, 1.0))
        k.append([rng.integer(1, kmax) for _ in range(d)])
        th.append(rng.uniform(0.0, 2.0 * math.pi))
    return FourierField(a, k, th, hi - lo, lo)


def node_coords(d: int, n, lo, dx: float, halfway: bool = False) -> np.ndarray:
    """(d, S) node coordinates, x_1 fastest: lo + i dx (periodic, full-way) or lo + (i + 1/2) dx."""
    n = list(n) if hasattr(n, "__len__") else [n] * d
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (d,))
    axes = [lo[i] + dx * (np.arange(n[i]) + (0.5 if halfway else 0.0)) for i in range(d)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    return np.stack([g.ravel() for g in grids])


def lattice_spacing(n: int, lo: float, hi: float, bc: str) -> float:
    return (hi - lo) / ((n - 1) if bc == "fullway" else n)


def periodic_problem(d: int, n: int, nmodes: int, seed: int, lo=0.0, hi=1.0):
    """phi0, grad phi0 (numpy) and the field of a periodic Fourier workload on n^d nodes."""
    dx = (hi - lo) / n
    X = node_coords(d, n, lo, dx)
    F = fourier_field(d, nmodes, seed, lo, hi)
    return F.value(X), F.grad(X), F, X


def wave_solution(X: np.ndarray, t: float, u, R: float, a, kappa, theta, b: float = 0.0, g=None):
    """Value and gradient of h = b + R t + g.(x - u t) + sum_m a_m sin(kappa_m.(x - u t) + theta_m) at the
    (d, S) coordinates X: an exact solution of d_t h + u.grad h = R (the Dirichlet data family of the
    library); used to build initial data and to measure errors."""
    d = X.shape[0]
    Y = X - np.asarray(u, dtype=np.float64)[:, None] * t
    gv = np.zeros(d) if g is None else np.asarray(g, dtype=np.float64)
    val = b + R * t + gv @ Y
    grad = np.repeat(gv[:, None], X.shape[1], axis=1)
    for am, km, tm in zip(a, kappa, theta):
        km = np.asarray(km, dtype=np.float64)
        arg = km @ Y + tm
        val = val + am * np.sin(arg)
        grad = grad + am * km[:, None] * np.cos(arg)[None, :]
    return val, grad


def tanh_bubble(X: np.ndarray, t: float, u, lo, hi):
    """Example 2's field phi = 1/2 - 1/2 tanh((r0 - |x - u t|) / (2 W)) on the periodic box [lo, hi]^d,
    r0 = 1/(5(d-1)), W = (5-d)/75, with the distance taken to the nearest periodic image of the
    moving centre; returns the value and its gradient at the (d, S) coordinates X."""
    d = X.shape[0]
    L = np.asarray(hi, dtype=np.float64) - np.asarray(lo, dtype=np.float64)
    L = np.broadcast_to(L, (d,))
    r0, W = 1.0 / (5.0 * (d - 1)), (5.0 - d) / 75.0
    Y = X - np.asarray(u, dtype=np.float64)[:, None] * t
    Y = Y - L[:, None] * np.round(Y / L[:, None])
    r = np.sqrt(np.sum(Y * Y, axis=0))
    z = (r0 - r) / (2.0 * W)
    val = 0.5 - 0.5 * np.tanh(z)
    dval_dr = 0.25 / W / np.cosh(z) ** 2
    with np.errstate(invalid="ignore", divide="ignore"):
        grad = np.where(r > 0, dval_dr * Y / np.where(r > 0, r, 1.0), 0.0)
    return val, grad


# ---- boundary data as jets (every derivative of order 0..3 in (t, x_1..x_d) at given points) ----

def _jet_tuples(d: int):
    """Variable tuples of a jet (0: t, i: x_i): lengths 0..3, non-decreasing, lexicographic."""
    import itertools

    return [tup for q in range(4) for tup in itertools.combinations_with_replacement(range(d + 1), q)]


def wave_jets(points: np.ndarray, t: float, u, R: float, a, kappa, theta, b: float = 0.0, g=None) -> np.ndarray:
    """Jets of h = b + R t + g.(x - u t) + sum_m a_m sin(kappa_m.(x - u t) + theta_m) at points (P, d):
    a derivative over x_i contributes kappa_mi, one over t contributes -kappa_m.u, to the m-th mode."""
    P, d = points.shape
    u = np.asarray(u, dtype=np.float64)
    g = np.zeros(d) if g is None else np.asarray(g, dtype=np.float64)
    tuples = _jet_tuples(d)
    out = np.zeros((P, len(tuples)))
    Y = points - u[None, :] * t
    for col, tup in enumerate(tuples):
        if len(tup) == 0:
            out[:, col] = b + R * t + Y @ g
        elif len(tup) == 1:
            out[:, col] = (R - g @ u) if tup[0] == 0 else g[tup[0] - 1]
        for m in range(len(a)):
            km = np.asarray(kappa[m], dtype=np.float64)
            fac = a[m]
            for v in tup:
                fac *= -(km @ u) if v == 0 else km[v - 1]
            xi = Y @ km + theta[m]
            out[:, col] += fac * [np.sin, np.cos, lambda z: -np.sin(z), lambda z: -np.cos(z)][len(tup) % 4](xi)
    return out


def gaussian_jets(points: np.ndarray, t: float, u, R: float, A: float, xc, sigma: float) -> np.ndarray:
    """Jets of phi = A exp(-|x - u t - xc|^2 / (2 sigma^2)) + R t, an exact solution of
    phi_t + u.grad phi = R that the sine family does not contain. A derivative over t acts on the pulse
    as -u.grad."""
    import itertools

    P, d = points.shape
    u = np.asarray(u, dtype=np.float64)
    Y = points - u[None, :] * t - np.asarray(xc, dtype=np.float64)[None, :]
    s2 = sigma * sigma
    G = A * np.exp(-np.sum(Y * Y, axis=1) / (2.0 * s2))

    def spatial(idx):  # derivative of the pulse over the spatial indices idx (0-based), order <= 3
        if len(idx) == 0:
            return G
        if len(idx) == 1:
            i, = idx
            return -Y[:, i] / s2 * G
        if len(idx) == 2:
            i, j = idx
            return (Y[:, i] * Y[:, j] / s2 ** 2 - (1.0 if i == j else 0.0) / s2) * G
        i, j, k = idx
        return (-Y[:, i] * Y[:, j] * Y[:, k] / s2 ** 3
                + ((i == j) * Y[:, k] + (i == k) * Y[:, j] + (j == k) * Y[:, i]) / s2 ** 2) * G

    tuples = _jet_tuples(d)
    out = np.zeros((P, len(tuples)))
    for col, tup in enumerate(tuples):
        nt = sum(1 for v in tup if v == 0)
        sp = [v - 1 for v in tup if v != 0]
        acc = np.zeros(P)
        for ls in itertools.product(range(d), repeat=nt):  # (-u.grad)^nt
            w = 1.0
            for l in ls:
                w *= -u[l]
            acc += w * spatial(sp + list(ls))
        out[:, col] = acc
        if len(tup) == 0:
            out[:, col] += R * t
        elif tup == (0,):
            out[:, col] += R
    return out


def gaussian_value(X: np.ndarray, t: float, u, R: float, A: float, xc, sigma: float) -> np.ndarray:
    """The pulse solution at nodes X (d, S)."""
    Y = X - np.asarray(u, dtype=np.float64)[:, None] * t - np.asarray(xc, dtype=np.float64)[:, None]
    return A * np.exp(-np.sum(Y * Y, axis=0) / (2.0 * sigma * sigma)) + R * t


def gaussian_grad(X: np.ndarray, t: float, u, A: float, xc, sigma: float) -> np.ndarray:
    Y = X - np.asarray(u, dtype=np.float64)[:, None] * t - np.asarray(xc, dtype=np.float64)[:, None]
    G = A * np.exp(-np.sum(Y * Y, axis=0) / (2.0 * sigma * sigma))
    return -Y / (sigma * sigma) * G[None, :]


# ---- manufactured solution with a source: phi = A exp(-lam t) prod_i sin(kappa_i x_i + theta_i),
#      R = phi_t + u.grad phi (defaults: A = lam = 1, kappa_i = pi, theta_i = 0) ----

def _sp_params(d, kappa, theta):
    k = np.full(d, np.pi) if kappa is None else np.asarray(kappa, dtype=np.float64)[:d]
    th = np.zeros(d) if theta is None else np.asarray(theta, dtype=np.float64)[:d]
    return k, th


def sine_product_value(X: np.ndarray, t: float, A=1.0, lam=1.0, kappa=None, theta=None) -> np.ndarray:
    k, th = _sp_params(X.shape[0], kappa, theta)
    return A * np.prod(np.sin(k[:, None] * X + th[:, None]), axis=0) * math.exp(-lam * t)


def sine_product_grad(X: np.ndarray, t: float, A=1.0, lam=1.0, kappa=None, theta=None) -> np.ndarray:
    d = X.shape[0]
    k, th = _sp_params(d, kappa, theta)
    z = k[:, None] * X + th[:, None]
    s, c = np.sin(z), np.cos(z)
    out = np.empty_like(X)
    for i in range(d):
        out[i] = A * k[i] * c[i] * np.prod(np.delete(s, i, axis=0), axis=0) * math.exp(-lam * t)
    return out


def sine_product_source(X: np.ndarray, t: float, u, A=1.0, lam=1.0, kappa=None, theta=None) -> np.ndarray:
    """R(x, t) = phi_t + u.grad phi of the manufactured solution (varies in x and t)."""
    return -lam * sine_product_value(X, t, A, lam, kappa, theta) \
        + np.asarray(u, dtype=np.float64) @ sine_product_grad(X, t, A, lam, kappa, theta)


def sine_product_jets(points: np.ndarray, t: float, A=1.0, lam=1.0, kappa=None, theta=None) -> np.ndarray:
    """Jets of the manufactured solution at points (P, d): a t-derivative gives -lam, an x_i-derivative
    one more derivative of sin(kappa_i x_i + theta_i) (a factor kappa_i)."""
    P, d = points.shape
    k, th = _sp_params(d, kappa, theta)
    tuples = _jet_tuples(d)
    out = np.zeros((P, len(tuples)))
    derivs = [np.sin, np.cos, lambda z: -np.sin(z), lambda z: -np.cos(z)]
    for col, tup in enumerate(tuples):
        val = np.full(P, A * math.exp(-lam * t) * (-lam) ** sum(1 for v in tup if v == 0))
        for i in range(d):
            q = sum(1 for v in tup if v == i + 1)
            val = val * k[i] ** q * derivs[q % 4](k[i] * points[:, i] + th[i])
        out[:, col] = val
    return out
