"""Closed-form discrete solution of the schemes for a periodic plane wave.

TEST INFRASTRUCTURE ONLY (see the package docstring).

On a periodic grid every stencil sum of Eq. notations2 maps a Fourier mode
onto itself.  With theta = (k1 h, k2 h) the delta sums have the symbols
    delta(1,0) -> 2 cos th1 + 2 cos th2 - 4
    delta(1,1) -> 4 cos th1 cos th2 - 4
    delta(2,0) -> 2 cos 2th1 + 2 cos 2th2 - 4
(evaluated below in the equivalent half-angle forms, free of cancellation
for long waves),
so Lambda_a = a10 delta(1,0) + a11 delta(1,1) + a20 delta(2,0) has the symbol
S_a (likewise S_b with the b coefficients of the first step).  Writing
u^n = A_n cos(k.x) + B_n sin(k.x):
* the first step (Eq. A1 in the forms comp5.1 / 9.1 / 13.1) gives
  (A_1, B_1) = (1 + S_a/2)(A_0, B_0) + tau (1 + S_b)(C_0, D_0) for
  v^0 = C_0 cos + D_0 sin;
* the two-step (Eq. A2) gives X_{n+1} = (2 + S_a) X_n - X_{n-1}, whose
  solution with cos(phi) = 1 + S_a/2, i.e. sin(phi/2) = sqrt(-S_a/4), is
  X_n = X_0 cos(n phi) + (X_1 - X_0 cos phi) sin(n phi) / sin(phi).
The coefficients are the printed Section 6 ones, written here independently
of the C oracle.  The result is exact up to rounding at any grid size, which
makes it the reference for large grids and long runs.
"""
from __future__ import annotations

import math

import numpy as np


def section6_coeffs(scheme: int, lam: float, conventional: bool = False):
    """(a10, a11, a20), (b10, b11, b20) of Section 6."""
    l2 = lam * lam
    if scheme == 5:
        return (l2, 0.0, 0.0), ((0.0 if conventional else l2 / 6.0), 0.0, 0.0)
    if scheme == 9:
        if conventional:
            return (2.0 * l2 / 3.0, l2 / 6.0, 0.0), (0.0, 0.0, 0.0)
        return (l2 * (1 - l2 / 3), l2 * l2 / 6, 0.0), (l2 / 6 * (1 - l2 / 5), l2 * l2 / 60, 0.0)
    if scheme == 13:
        a = (l2 * (4 - 2 * l2) / 3, l2 * l2 / 6, l2 * (l2 - 1) / 12)
        if conventional:
            return a, (0.0, 0.0, 0.0)
        return a, (l2 / 6 * (4 / 3 - 2 * l2 / 5), l2 * l2 / 60, l2 / 6 * (l2 / 20 - 1 / 12))
    raise ValueError(f"unknown scheme {scheme}")


def symbol(coef, th1: float, th2: float) -> float:
    """Symbol of a10 delta(1,0) + a11 delta(1,1) + a20 delta(2,0), written with
    2 cos(x) - 2 = -4 sin^2(x/2) so that long waves (theta -> 0) lose no
    digits to cancellation:
        delta(1,0) -> -4 (sin^2(th1/2) + sin^2(th2/2))
        delta(1,1) -> -4 (sin^2((th1+th2)/2) + sin^2((th1-th2)/2))
        delta(2,0) -> -4 (sin^2(th1) + sin^2(th2))."""
    s2 = lambda x: math.sin(x) ** 2
    d10 = -4.0 * (s2(th1 / 2) + s2(th2 / 2))
    d11 = -4.0 * (s2((th1 + th2) / 2) + s2((th1 - th2) / 2))
    d20 = -4.0 * (s2(th1) + s2(th2))
    return coef[0] * d10 + coef[1] * d11 + coef[2] * d20


def class_symbol(classes, coef, th1: float, th2: float) -> float:
    """Symbol of sum_c coef_c delta_c for a scheme in class form (a class
    (q1, q2) being all nodes (+-q1, +-q2), (+-q2, +-q1)): each node q adds
    cos(q . theta) - 1 = -2 sin^2(q . theta / 2)."""
    total = 0.0
    for cls, a in zip(classes, coef):
        q1, q2 = cls
        nodes = {(s1 * u, s2 * v) for u, v in ((q1, q2), (q2, q1)) for s1 in (1, -1) for s2 in (1, -1)}
        total += a * sum(-2.0 * math.sin((n1 * th1 + n2 * th2) / 2) ** 2 for n1, n2 in nodes)
    return total


def _chebyshev_ratio(n: int, phi: float, cphi: float) -> float:
    """sin(n phi) / sin(phi), continuous at sin(phi) = 0."""
    s = math.sin(phi)
    if s == 0.0:
        # U_{n-1}(+-1)
        return float(n) if cphi > 0 else (-1.0) ** (n - 1) * n
    return math.sin(n * phi) / s


def amplitudes(scheme, lam, tau, k1, k2, h, n, a0=1.0, b0=0.0, c0=0.0, d0=None, c=1.0,
               conventional=False):
    """(A_n, B_n) of u^n = A_n cos(k.x) + B_n sin(k.x).

    Defaults are the plane wave cos(k.x - c|k|t): u^0 = cos(k.x),
    v^0 = c|k| sin(k.x)."""
    if d0 is None:
        d0 = c * math.hypot(k1, k2)
    a, b = section6_coeffs(scheme, lam, conventional)
    th1, th2 = k1 * h, k2 * h
    return _amplitudes(symbol(a, th1, th2), symbol(b, th1, th2), tau, n, a0, b0, c0, d0)


def class_amplitudes(classes, a, b, tau, k1, k2, h, n, a0=1.0, b0=0.0, c0=0.0, d0=None, c=1.0):
    """(A_n, B_n) for a scheme in class form with coefficient values a, b
    (evaluated at the Courant number); defaults as in ``amplitudes``."""
    if d0 is None:
        d0 = c * math.hypot(k1, k2)
    th1, th2 = k1 * h, k2 * h
    return _amplitudes(class_symbol(classes, a, th1, th2), class_symbol(classes, b, th1, th2), tau, n,
                       a0, b0, c0, d0)


def _amplitudes(sa, sb, tau, n, a0, b0, c0, d0):
    A1 = (1 + sa / 2) * a0 + tau * (1 + sb) * c0
    B1 = (1 + sa / 2) * b0 + tau * (1 + sb) * d0
    if n == 0:
        return a0, b0
    if n == 1:
        return A1, B1
    cphi = 1 + sa / 2
    if sa > 0 or sa < -4:
        raise ValueError("mode is outside the stability region")
    # cos(phi) = 1 + S/2 = 1 - 2 sin^2(phi/2): take phi from sin(phi/2), which
    # stays well conditioned when phi is small
    phi = 2.0 * math.asin(math.sqrt(-sa / 4.0))
    r = _chebyshev_ratio(n, phi, cphi)
    cn = math.cos(n * phi)
    return a0 * cn + (A1 - a0 * cphi) * r, b0 * cn + (B1 - b0 * cphi) * r


def stability_limit(classes, a_of_lam, n_theta: int = 257, lam_hi: float = 2.0) -> float:
    """Largest Courant number lam such that every lam' <= lam keeps the
    symbol of the two-step in [-4, 0] on an n_theta x n_theta grid of
    [0, pi]^2 (von Neumann: the roots of g^2 - (2 + S) g + 1 stay on the
    unit circle).  a_of_lam(lam) returns the class coefficients."""
    th = np.linspace(0.0, math.pi, n_theta)
    T1, T2 = np.meshgrid(th, th, indexing="ij")
    sig = []
    for q1, q2 in classes:
        nodes = {(s1 * u, s2 * v) for u, v in ((q1, q2), (q2, q1)) for s1 in (1, -1) for s2 in (1, -1)}
        sig.append(sum(-2.0 * np.sin((n1 * T1 + n2 * T2) / 2) ** 2 for n1, n2 in nodes))

    def stable(lam):
        S = sum(ac * sg for ac, sg in zip(a_of_lam(lam), sig))
        return bool(np.all(S >= -4.0 - 1e-13) and np.all(S <= 1e-13))

    step, lam = 1.0 / 512, 0.0
    while lam + step <= lam_hi and stable(lam + step):
        lam += step
    lo, hi = lam, lam + step
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if stable(mid) else (lo, mid)
    return lo


def field(scheme, lam, tau, k1, k2, h, nx, ny, n, x_off=0.0, **kw) -> np.ndarray:
    """u^n on the (ny, nx) node set x = (i + x_off) h."""
    an, bn = amplitudes(scheme, lam, tau, k1, k2, h, n, **kw)
    x1 = (np.arange(nx) + x_off) * h
    x2 = (np.arange(ny) + x_off) * h
    ph = k1 * x1[None, :] + k2 * x2[:, None]
    return an * np.cos(ph) + bn * np.sin(ph)


def sample(scheme, lam, tau, k1, k2, h, n, ii, jj, x_off=0.0, **kw) -> np.ndarray:
    """u^n at the nodes (ii[m], jj[m])."""
    an, bn = amplitudes(scheme, lam, tau, k1, k2, h, n, **kw)
    ph = k1 * (np.asarray(ii) + x_off) * h + k2 * (np.asarray(jj) + x_off) * h
    return an * np.cos(ph) + bn * np.sin(ph)
