"""Pin P5: polynomial exactness (Sections 4-5: the interpolation is exact on
P_m and so is the integration), and pin P9 (Section 6.1: comp5.1 and
comp5.1a agree for linear v0).

Exact solutions of the wave equation whose time slices lie in the scheme's
polynomial space are built with sympy from the series
    u = sum_k c^{2k} [ t^{2k}/(2k)! Lap^k u0 + t^{2k+1}/(2k+1)! Lap^k v0 ],
checked to satisfy u_tt = c^2 Lap u, and compared with the oracle at nodes
whose domain of dependence (radius R per step) stays inside the grid.
"""
import math

import numpy as np
import pytest

from initial_data import BC_ZERO, mesh

sp = pytest.importorskip("sympy")
X1, X2, T, C = sp.symbols("x1 x2 t c")

RADIUS = {5: 1, 9: 1, 13: 2}


def series_solution(u0, v0, terms=4):
    lap = lambda f: sp.diff(f, X1, 2) + sp.diff(f, X2, 2)
    u = 0
    fu, fv = u0, v0
    for k in range(terms):
        u += C ** (2 * k) * (T ** (2 * k) / sp.factorial(2 * k) * fu
                             + T ** (2 * k + 1) / sp.factorial(2 * k + 1) * fv)
        fu, fv = lap(fu), lap(fv)
    assert sp.simplify(fu) == 0 and sp.simplify(fv) == 0, "series must terminate"
    u = sp.expand(u)
    assert sp.simplify(sp.diff(u, T, 2) - C ** 2 * lap(u)) == 0
    return u


CASES = {
    # all schemes: slices in P_6 = span{1, x1, x2, x1 x2, x1^2, x2^2}
    "x1^2+c^2t^2": (5, X1 ** 2, 0),
    "x2^2": (5, X2 ** 2, 0),
    "x1x2": (5, X1 * X2, 0),
    "linear": (5, 3 * X1 - 2 * X2 + 1, X1 + 0.5 * X2 - 2),
    "t x1^2 + c^2 t^3/3": (5, 0, X1 ** 2),
    "t x1 x2": (5, 0, X1 * X2),
    # 9- and 13-point: P_11 adds x1^2 x2, x1 x2^2, x1^3, x2^3, x1^2 x2^2
    "x1^3/3 + c^2 x1 t^2": (9, X1 ** 3 / 3, 0),
    "x1^2 x2^2": (9, X1 ** 2 * X2 ** 2, 0),
    "t x1^2 x2^2": (9, 0, X1 ** 2 * X2 ** 2),
    "x1^2 x2 + t x2^3": (9, X1 ** 2 * X2, X2 ** 3),
    "t x1 x2^2": (9, 0, X1 * X2 ** 2),
    # 13-point: P_15 = all of degree <= 4
    "x1^4 + 6c^2x1^2t^2 + c^4t^4": (13, X1 ** 4, 0),
    "t x1^3 x2": (13, 0, X1 ** 3 * X2),
    "x2^4 + t x1 x2^3": (13, X2 ** 4, X1 * X2 ** 3),
}


def _np(expr):
    return sp.lambdify((X1, X2, T, C), expr, "numpy")


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("name", list(CASES))
def test_polynomial_solutions_are_reproduced(orc, scheme, name):
    min_scheme, u0s, v0s = CASES[name]
    if scheme < min_scheme:
        pytest.skip("polynomial outside this scheme's space")
    u = series_solution(sp.sympify(u0s), sp.sympify(v0s))
    f = _np(u)
    nx, ny, h, c, lam = 41, 37, 0.05, 1.3, 0.55
    tau = lam * h / c
    XX, YY = mesh(nx, ny, h, BC_ZERO)
    full = lambda t: np.broadcast_to(f(XX, YY, t, c), (ny, nx)).astype(np.float64)
    u0 = full(0.0)
    v0 = np.broadcast_to(_np(sp.diff(u, T))(XX, YY, 0.0, c), (ny, nx)).astype(np.float64)
    R = RADIUS[scheme]
    scale = np.max(np.abs(u0)) + np.max(np.abs(v0)) + 1.0
    for n_t in (1, 2, 5, 8):
        _, un, _ = orc.run(scheme, u0, v0, lam, tau, n_t, bc=orc.BC_ZERO)
        m = R * n_t
        inner = (slice(m, ny - m), slice(m, nx - m))
        ue = full(n_t * tau)
        err = np.max(np.abs(un[inner] - ue[inner]))
        assert err < 1e-12 * scale, (name, scheme, n_t, err)


def test_conventional_first_step_misses_the_b_term(orc):
    """For u = t x1^2 + c^2 t^3/3 the epsilon term supplies c^2 tau^3/3;
    the conventional comp5.1a lacks it (Section 6.1)."""
    nx = ny = 21
    h, lam, c = 0.1, 0.6, 1.0
    tau = lam * h / c
    XX, YY = mesh(nx, ny, h, BC_ZERO)
    u0 = np.zeros((ny, nx))
    v0 = XX ** 2
    u1n = orc.first_step(5, u0, v0, lam, tau)
    u1c = orc.first_step(5, u0, v0, lam, tau, conventional=True)
    inner = (slice(1, -1), slice(1, -1))
    exact = tau * XX ** 2 + c * c * tau ** 3 / 3
    assert np.max(np.abs(u1n - exact)[inner]) < 1e-15
    assert np.allclose((exact - u1c)[inner], c * c * tau ** 3 / 3, rtol=1e-9, atol=0)


def test_first_steps_agree_for_linear_v0(orc):
    """Pin P9: for v0 linear in x the epsilon sums vanish, so comp5.1 and
    comp5.1a coincide (Section 6.1)."""
    rng = np.random.default_rng(7)
    nx, ny, h = 30, 26, 0.02
    XX, YY = mesh(nx, ny, h, orc.BC_PERIODIC)
    u0 = rng.standard_normal((ny, nx))
    v0 = 0.7 * XX - 1.9 * YY + 0.25
    for scheme in (5, 9, 13):
        a = orc.first_step(scheme, u0, v0, 0.5, 0.5 * h)
        b = orc.first_step(scheme, u0, v0, 0.5, 0.5 * h, conventional=(scheme == 5))
        R = RADIUS[scheme]
        inner = (slice(R, -R), slice(R, -R))
        if scheme == 5:
            assert np.max(np.abs(a - b)[inner]) < 1e-15
    # and a non-linear v0 makes them differ
    v0q = XX ** 2
    a = orc.first_step(5, u0, v0q, 0.5, 0.5 * h)
    b = orc.first_step(5, u0, v0q, 0.5, 0.5 * h, conventional=True)
    assert np.max(np.abs(a - b)[1:-1, 1:-1]) > 1e-9
