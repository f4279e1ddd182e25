"""Pin P4: the Section 6 coefficients used by the oracle equal those obtained
by carrying out Sections 4-5 (ordered monomials, McKinney nodes, D^{-1},
exact integrals) in exact rational arithmetic."""
import math
from fractions import Fraction

import pytest

from oracle import derive

LAMS = [0.1, 0.3, 0.5, 0.6, 0.707, 0.75, 0.79]


def test_order_function_matches_printed_sequences():
    """Eq. g reproduces the printed monomial sequences M*_{<=6}, M*_{<=11}
    and M*_{<=15} (Eq. mono6, monomials11, monomials15)."""
    assert derive.monomial_segment(6) == [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2)]
    assert derive.monomial_segment(11) == [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2),
                                           (2, 1), (1, 2), (3, 0), (0, 3), (2, 2)]
    assert derive.monomial_segment(15)[11:] == [(3, 1), (1, 3), (4, 0), (0, 4)]
    # g is a bijection onto 1, 2, 3, ... (Section 4)
    vals = sorted(derive.g(a, d - a) for d in range(8) for a in range(d + 1))
    assert vals == list(range(1, len(vals) + 1))


def test_mckinney_map_is_inverse():
    for q in range(-6, 7):
        assert derive.q_of_alpha(derive.alpha(q)) == q
    # printed node sequence for the five-point case (Section 6.1)
    assert derive.nodes_of(derive.monomial_segment(6)) == [(0, 0), (-1, 0), (0, -1), (-1, -1), (1, 0), (0, 1)]


def test_determinant_five_point():
    """det D = 4 h^8 (Section 6.1); in the scaled variables det D = 4."""
    _, _, _, det = derive.stencil_weights(6)
    assert det == 4


def test_five_point_lagrange_weights_match_printed():
    """Eq. A6 and Eq. B6."""
    nodes, wa, wb, _ = derive.stencil_weights(6)
    assert wa[(0, 0)] == {0: Fraction(1), 2: Fraction(-2)}
    assert wb[(0, 0)] == {0: Fraction(1), 2: Fraction(-2, 3)}
    assert wa[(-1, -1)] == {} and wb[(-1, -1)] == {}
    for q in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
        assert wa[q] == {2: Fraction(1, 2)}
        assert wb[q] == {2: Fraction(1, 6)}


def test_nine_point_weights_match_printed():
    """Eq. A11 and Eq. B11; the nodes (-2,0) and (0,-2) drop out."""
    _, wa, wb, _ = derive.stencil_weights(11)
    assert wa[(0, 0)] == {0: 1, 2: -2, 4: Fraction(1, 3)}
    assert wb[(0, 0)] == {0: 1, 2: Fraction(-2, 3), 4: Fraction(1, 15)}
    for q in [(1, 1), (1, -1), (-1, 1), (-1, -1)]:
        assert wa[q] == {4: Fraction(1, 12)} and wb[q] == {4: Fraction(1, 60)}
    for q in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
        assert wa[q] == {2: Fraction(1, 2), 4: Fraction(-1, 6)}
        assert wb[q] == {2: Fraction(1, 6), 4: Fraction(-1, 30)}
    assert wa[(-2, 0)] == {} and wa[(0, -2)] == {} and wb[(-2, 0)] == {} and wb[(0, -2)] == {}


def test_thirteen_point_dropped_nodes():
    """(-2,-1) and (-1,-2) drop out of the 15-node interpolation (Section 6.3)."""
    _, wa, wb, _ = derive.stencil_weights(15)
    assert wa[(-2, -1)] == {} and wa[(-1, -2)] == {}
    assert wb[(-2, -1)] == {} and wb[(-1, -2)] == {}


@pytest.mark.parametrize("m", [6, 11, 15])
def test_weights_are_consistent_and_d4_symmetric(m):
    nodes, wa, wb, _ = derive.stencil_weights(m)
    # A 1 = 1 and B 1 = tau: the weights sum to one
    sa, sb = {}, {}
    for q in nodes:
        for k, v in wa[q].items():
            sa[k] = sa.get(k, 0) + v
        for k, v in wb[q].items():
            sb[k] = sb.get(k, 0) + v
    assert {k: v for k, v in sa.items() if v} == {0: 1}
    assert {k: v for k, v in sb.items() if v} == {0: 1}
    # every surviving node's weight equals that of its 90-degree rotations
    live = {q for q in nodes if wa[q] or wb[q]}
    for (q1, q2) in live:
        for r in [(-q2, q1), (-q1, -q2), (q2, -q1), (q2, q1)]:
            assert r in live
            assert wa[r] == wa[(q1, q2)] and wb[r] == wb[(q1, q2)]


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("lam", LAMS)
def test_oracle_coefficients_equal_derivation(orc, scheme, lam):
    a_poly, b_poly = derive.delta_coefficients(scheme)
    a, b = orc.coeffs(scheme, lam)
    for i in range(3):
        assert abs(a[i] - derive.evaluate(a_poly[i], lam)) < 1e-15
        assert abs(b[i] - derive.evaluate(b_poly[i], lam)) < 1e-15


def test_conventional_coefficients(orc):
    """Conventional schemes: no epsilon term; isotropic 9-point Laplacian
    weights 2/3, 1/6 (Eq. comp9.2b)."""
    for lam in LAMS:
        a, b = orc.coeffs(9, lam, conventional=True)
        assert list(b) == [0, 0, 0]
        assert abs(a[0] - 2 * lam * lam / 3) < 1e-16 and abs(a[1] - lam * lam / 6) < 1e-16
        a5, b5 = orc.coeffs(5, lam, conventional=True)
        assert list(b5) == [0, 0, 0] and a5[0] == lam * lam
        a13, b13 = orc.coeffs(13, lam, conventional=True)
        a13n, _ = orc.coeffs(13, lam)
        assert list(b13) == [0, 0, 0] and list(a13) == list(a13n)


def test_exact_integrals_of_monomials():
    """Eq. exact1 / exact2 against a direct evaluation of the operator A on a
    monomial: (1/2pi) int_{|z|<1} (f + lam z.grad f)/sqrt(1-|z|^2), done in
    polar coordinates with a Gauss-Jacobi-like substitution r = sin(s)."""
    np = pytest.importorskip("numpy")
    lam = 0.6
    s, ws = np.polynomial.legendre.leggauss(80)
    s = (s + 1) * (math.pi / 4)      # s in (0, pi/2): r = sin s, dr/sqrt(1-r^2) = ds
    ws = ws * (math.pi / 4)
    th, wt = np.polynomial.legendre.leggauss(96)
    th = (th + 1) * math.pi
    wt = wt * math.pi
    r = np.sin(s)[:, None]
    z1, z2 = r * np.cos(th)[None, :], r * np.sin(th)[None, :]
    for a1 in range(0, 5):
        for a2 in range(0, 5 - a1):
            f = (lam * z1) ** a1 * (lam * z2) ** a2
            # z . grad f in scaled variables = (a1 + a2) f
            integrand = (1 + a1 + a2) * f * r  # r from the polar Jacobian
            val = float(np.sum(ws[:, None] * wt[None, :] * integrand)) / (2 * math.pi)
            expect = derive.evaluate(derive.a_of_monomial((a1, a2)), lam)
            assert abs(val - expect) < 1e-12, (a1, a2, val, expect)
            vb = float(np.sum(ws[:, None] * wt[None, :] * f * r)) / (2 * math.pi)
            eb = derive.evaluate(derive.b_of_monomial((a1, a2)), lam)
            assert abs(vb - eb) < 1e-12, (a1, a2, vb, eb)
