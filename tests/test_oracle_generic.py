"""Pins of the oracle for derived schemes beyond Section 6 (larger segments
M*_{<=m} of the derivation of Sections 4-5).

* The node-weight form of the algorithm (``oracle.run_nodes``: Eq. A1 and
  Eq. A2 with the weights A phi_q, B phi_q / tau) equals the printed Section 6
  forms of ``oracle.run`` for the 5-, 9- and 13-point segments: two
  independently written evaluations of the same operator.
* The weights satisfy their defining moment conditions exactly: for every
  monomial mu of the segment, sum_q w_q mu(q) equals the exact integral
  A(mu) of Eq. exact1 (resp. B(mu) / tau of Eq. exact2).
* Polynomial exactness: solutions whose time slices lie in the span of the
  segment are reproduced to round-off, and the previous symmetric segment,
  which lacks the top monomials, is not exact on them.
* The class-form symbol equals the Section 6 symbol on the old segments, the
  closed-form plane wave equals stepping, and the von Neumann limit found by
  the symbol scan reproduces the printed limits and separates bounded from
  growing runs.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from initial_data import BC_PERIODIC, BC_ZERO, mesh
from oracle import derive, plane_wave

DERIVED = (24, 28, 37, 41, 45)


@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC])
@pytest.mark.parametrize("scheme", [5, 9, 13])
def test_node_form_equals_printed_form(orc, scheme, bc):
    rng = np.random.default_rng(scheme + 10 * bc)
    ny, nx = 13, 17
    u0 = rng.standard_normal((ny, nx))
    v0 = rng.standard_normal((ny, nx))
    lam, h = 0.6, 0.1
    tau = lam * h
    nodes, wa, wb = derive.node_weights(derive.SEGMENT[scheme], lam)
    for n_t in (1, 2, 9):
        _, got = orc.run_nodes(nodes, wa, wb, u0, v0, tau, n_t, bc=bc)
        _, ref, _ = orc.run(scheme, u0, v0, lam, tau, n_t, bc=bc)
        assert np.max(np.abs(got - ref)) < 1e-12 * (1 + np.max(np.abs(ref)))


@pytest.mark.parametrize("m", DERIVED)
def test_weights_satisfy_the_moment_conditions(m):
    nodes, wa, wb, _ = derive.stencil_weights(m)
    for mono in derive.monomial_segment(m):
        ea, eb = derive.a_of_monomial(mono), derive.b_of_monomial(mono)
        sa, sb = {}, {}
        for q in nodes:
            mv = Fraction(q[0]) ** mono[0] * Fraction(q[1]) ** mono[1]
            for k, v in wa[q].items():
                sa[k] = sa.get(k, Fraction(0)) + v * mv
            for k, v in wb[q].items():
                sb[k] = sb.get(k, Fraction(0)) + v * mv
        assert {k: v for k, v in sa.items() if v} == ea, (m, mono)
        assert {k: v for k, v in sb.items() if v} == eb, (m, mono)


@pytest.mark.parametrize("m", DERIVED)
def test_derived_schemes_have_symmetric_classes(m):
    classes, a, b = derive.class_scheme(m)
    nodes, wa, _, _ = derive.stencil_weights(m)
    # the weights of A sum to 1 (A applied to a constant), so the centre
    # weight is 1 - sum of the others and the two-step reads 2u - u + Lambda u
    total = {}
    for q in nodes:
        for k, v in wa[q].items():
            total[k] = total.get(k, Fraction(0)) + v
    assert {k: v for k, v in total.items() if v} == {0: Fraction(1)}
    n_points = 1 + sum(len(derive.class_nodes(c)) for c in classes)
    assert n_points == sum(1 for q in nodes if wa[q] or q == (0, 0))
    assert all(p for p in a)


def test_asymmetric_segments_are_rejected():
    for m in (5, 14, 23, 27, 40, 44):
        with pytest.raises(ValueError):
            derive.class_scheme(m)


sp = pytest.importorskip("sympy")
X1, X2, T, C = sp.symbols("x1 x2 t c")


def _series_solution(u0, v0, terms=6):
    lap = lambda f: sp.diff(f, X1, 2) + sp.diff(f, X2, 2)
    u, fu, fv = 0, u0, v0
    for k in range(terms):
        u += C ** (2 * k) * (T ** (2 * k) / sp.factorial(2 * k) * fu
                             + T ** (2 * k + 1) / sp.factorial(2 * k + 1) * fv)
        fu, fv = lap(fu), lap(fv)
    assert sp.simplify(fu) == 0 and sp.simplify(fv) == 0
    u = sp.expand(u)
    assert sp.simplify(sp.diff(u, T, 2) - C ** 2 * lap(u)) == 0
    return u


# (segment, previous symmetric segment, u0, v0): the monomials of the highest
# degree are the ones the segment adds over the previous one (the order g of
# Eq. g brings in x1^3 x2^3, x1^4 x2^2, x1^2 x2^4 at m = 22-24, x1^5 x2, x1 x2^5,
# x1^6, x2^6 by m = 28, x1^4 x2^4 at m = 37, x1^5 x2^3 .. x1^2 x2^6 by m = 41
# and x1^8, x2^8 by m = 45), so the previous segment must fail the case.
POLY_CASES = {
    "m24": (24, 15, X1 ** 4 * X2 ** 2 - X1 ** 3 * X2 ** 3, X1 ** 2 * X2 ** 4),
    "m28": (28, 24, X1 ** 6 - 2 * X1 * X2 ** 5, X2 ** 6 + X1 ** 5 * X2),
    "m37": (37, 28, X1 ** 4 * X2 ** 4 + X1 ** 7, X1 ** 4 * X2 ** 4),
    "m41": (41, 37, X1 ** 6 * X2 ** 2 - 3 * X1 ** 3 * X2 ** 5, X1 ** 2 * X2 ** 6),
    "m45": (45, 41, X1 ** 8 - X1 ** 5 * X2 ** 3, X2 ** 8),
}


def _max_error(orc, m, f, ft, n_t):
    n = 45
    h, c, lam = 0.1, 1.1, 0.5
    tau = lam * h / c
    x = (np.arange(n) - (n - 1) / 2) * h  # centred, |x| <= 2.2
    XX, YY = np.meshgrid(x, x)
    u0 = np.broadcast_to(f(XX, YY, 0.0, c), (n, n)).astype(np.float64)
    v0 = np.broadcast_to(ft(XX, YY, 0.0, c), (n, n)).astype(np.float64)
    nodes, wa, wb = derive.node_weights(m, lam)
    _, un = orc.run_nodes(nodes, wa, wb, u0, v0, tau, n_t, bc=BC_ZERO)
    ue = np.broadcast_to(f(XX, YY, n_t * tau, c), (n, n))
    k = 4 * n_t  # nodes whose domain of dependence stays inside the grid
    inner = (slice(k, n - k), slice(k, n - k))
    return np.max(np.abs(un[inner] - ue[inner])) / np.max(np.abs(ue[inner]))


@pytest.mark.parametrize("name", list(POLY_CASES))
def test_polynomial_solutions_are_reproduced(orc, name):
    m, prev, u0s, v0s = POLY_CASES[name]
    u = _series_solution(sp.sympify(u0s), sp.sympify(v0s))
    f = sp.lambdify((X1, X2, T, C), u, "numpy")
    ft = sp.lambdify((X1, X2, T, C), sp.diff(u, T), "numpy")
    for n_t in (1, 2, 5):
        assert _max_error(orc, m, f, ft, n_t) < 1e-13, (name, n_t)
    # the previous segment lacks the top monomials and is not exact
    assert _max_error(orc, prev, f, ft, 2) > 1e-12, name


@pytest.mark.parametrize("scheme", [5, 9, 13])
def test_class_symbol_equals_section6_symbol(scheme):
    lam = 0.55
    classes, a, b = derive.class_scheme(derive.SEGMENT[scheme])
    av = [derive.evaluate(p, lam) for p in a]
    bv = [derive.evaluate(p, lam) for p in b]
    sa6, sb6 = plane_wave.section6_coeffs(scheme, lam)
    rng = np.random.default_rng(1)
    for th1, th2 in rng.uniform(-math.pi, math.pi, (20, 2)):
        assert abs(plane_wave.class_symbol(classes, av, th1, th2) - plane_wave.symbol(sa6, th1, th2)) < 1e-14
        assert abs(plane_wave.class_symbol(classes, bv, th1, th2) - plane_wave.symbol(sb6, th1, th2)) < 1e-14


@pytest.mark.parametrize("m", DERIVED)
def test_class_plane_wave_matches_stepping(orc, m):
    n = 24
    h = 1.0 / n
    classes, a, b = derive.class_scheme(m)
    lam = 0.9 * plane_wave.stability_limit(classes, lambda l: [derive.evaluate(p, l) for p in a])
    tau = lam * h
    av = [derive.evaluate(p, lam) for p in a]
    bv = [derive.evaluate(p, lam) for p in b]
    k1, k2 = 2 * math.pi * 3, 2 * math.pi * 2
    XX, YY = mesh(n, n, h, BC_PERIODIC)
    u0 = np.cos(k1 * XX + k2 * YY)
    v0 = math.hypot(k1, k2) * np.sin(k1 * XX + k2 * YY)
    nodes, wa, wb = derive.node_weights(m, lam)
    for n_t in (1, 2, 40):
        _, got = orc.run_nodes(nodes, wa, wb, u0, v0, tau, n_t, bc=BC_PERIODIC)
        an, bn = plane_wave.class_amplitudes(classes, av, bv, tau, k1, k2, h, n_t)
        ref = an * np.cos(k1 * XX + k2 * YY) + bn * np.sin(k1 * XX + k2 * YY)
        assert np.max(np.abs(got - ref)) < 1e-11


@pytest.mark.parametrize("scheme,limit", [(5, 1 / math.sqrt(2)), (9, math.sqrt((3 - math.sqrt(3)) / 2)),
                                          (13, 1 / math.sqrt(2))])
def test_stability_scan_reproduces_printed_limits(scheme, limit):
    classes, a, _ = derive.class_scheme(derive.SEGMENT[scheme])
    got = plane_wave.stability_limit(classes, lambda l: [derive.evaluate(p, l) for p in a])
    assert abs(got - limit) < 1e-9


@pytest.mark.parametrize("m", [24, 37, 41])
def test_stability_limit_separates_bounded_and_growing_runs(orc, m):
    classes, a, _ = derive.class_scheme(m)
    lmax = plane_wave.stability_limit(classes, lambda l: [derive.evaluate(p, l) for p in a])
    n = 16
    rng = np.random.default_rng(m)
    u0 = rng.standard_normal((n, n))
    v0 = np.zeros((n, n))
    peaks = []
    for lam in (0.999 * lmax, 1.02 * lmax):
        nodes, wa, wb = derive.node_weights(m, lam)
        _, un = orc.run_nodes(nodes, wa, wb, u0, v0, lam / n, 600, bc=BC_PERIODIC)
        peaks.append(np.max(np.abs(un)))
    assert peaks[0] < 50 * np.max(np.abs(u0)) and peaks[1] > 1e3 * np.max(np.abs(u0))
