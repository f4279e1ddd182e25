"""Derivation of the stencil weights from Sections 4-5 of arXiv:1904.04048.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Exact rational arithmetic (``fractions.Fraction``); polynomials in the
Courant number lambda are dicts {power: Fraction}.  The steps follow the
paper's order:

1. the ordinal function g(alpha1, alpha2) of Eq. g defines the ordered
   monomial set M* and its initial segments M*_{<=m} (Section 4);
2. the McKinney map, Eq. alpha and its inverse Eq. invMcKinney, assigns to
   each monomial x1^a1 x2^a2 the stencil node (q(a1), q(a2));
3. the matrix D = [mu_s(x_(r))] of Eq. matrix1 is built in the scaled
   variables x/h (so node coordinates are the integers q) and inverted
   exactly, giving the Lagrange basis of Eq. Lagrange;
4. the operators A and B of Eq. Op1 / Op2 act on scaled monomials by the
   closed forms Eq. exact1 / exact2 (Section 5);
5. the weight of node q in the first step u^1 = A u^0 + B v^0 (Eq. A1) is
   A phi_q resp. B phi_q, and 2 A phi_q in the two-step (Eq. A2).
"""
from __future__ import annotations

from fractions import Fraction
from typing import Dict, List, Tuple

Poly = Dict[int, Fraction]


def g(a1: int, a2: int) -> int:
    """Ordinal number of x1^a1 x2^a2, Eq. g."""
    s = (a1 + a2) * (a1 + a2 + 1) // 2
    if a2 < a1:
        return s + (a1 - a2)
    return s + (a2 - a1 + 1)


def monomial_segment(m: int) -> List[Tuple[int, int]]:
    """The initial segment M*_{<=m}: the m monomials with the smallest g."""
    deg = 0
    while (deg + 1) * (deg + 2) // 2 < m:
        deg += 1
    cands = [(a1, d - a1) for d in range(deg + 1) for a1 in range(d + 1)]
    cands.sort(key=lambda a: g(*a))
    return cands[:m]


def alpha(q: int) -> int:
    """McKinney exponent of a stencil index, Eq. alpha."""
    return 2 * abs(q) - 1 if q < 0 else 2 * q


def q_of_alpha(a: int) -> int:
    """Inverse map, Eq. invMcKinney: (-1)^a * floor((a + 1) / 2)."""
    return (-1) ** a * ((a + 1) // 2)


def nodes_of(monos: List[Tuple[int, int]]) -> List[Tuple[int, int]]:
    return [(q_of_alpha(a1), q_of_alpha(a2)) for a1, a2 in monos]


def _mono_at(mono: Tuple[int, int], node: Tuple[int, int]) -> Fraction:
    (a1, a2), (q1, q2) = mono, node
    return Fraction(q1) ** a1 * Fraction(q2) ** a2  # 0**0 == 1


def matrix_d(monos, nodes) -> List[List[Fraction]]:
    """D[r][s] = mu_s evaluated at node r (scaled coordinates), Eq. matrix1."""
    return [[_mono_at(mu, x) for mu in monos] for x in nodes]


def _solve_inverse(m: List[List[Fraction]]):
    """Exact Gauss-Jordan inverse and determinant."""
    n = len(m)
    a = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(m)]
    det = Fraction(1)
    for col in range(n):
        piv = next((r for r in range(col, n) if a[r][col] != 0), None)
        if piv is None:
            raise ValueError("D is singular: interpolation problem not unisolvent")
        if piv != col:
            a[col], a[piv] = a[piv], a[col]
            det = -det
        p = a[col][col]
        det *= p
        a[col] = [x / p for x in a[col]]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col]
                a[r] = [x - f * y for x, y in zip(a[r], a[col])]
    return [row[n:] for row in a], det


def _double_factorial(k: int) -> int:
    if k <= 0:
        return 1  # (-1)!! = 0!! = 1
    out = 1
    while k > 0:
        out *= k
        k -= 2
    return out


def a_of_monomial(mono: Tuple[int, int]) -> Poly:
    """A(x_ij, tau) applied to (y1/h)^a1 (y2/h)^a2, Eq. exact1 / exact2."""
    a1, a2 = mono
    if a1 % 2 or a2 % 2:
        return {}
    c = Fraction(_double_factorial(a1 - 1) * _double_factorial(a2 - 1),
                 _double_factorial(a1 + a2 - 1))
    return {a1 + a2: c}


def b_of_monomial(mono: Tuple[int, int]) -> Poly:
    """B(x_ij, tau) applied to the scaled monomial, divided by tau (Eq. exact2)."""
    a1, a2 = mono
    return {p: c / (a1 + a2 + 1) for p, c in a_of_monomial(mono).items()}


def _padd(p: Poly, q: Poly, scale: Fraction = Fraction(1)) -> Poly:
    out = dict(p)
    for k, v in q.items():
        out[k] = out.get(k, Fraction(0)) + scale * v
        if out[k] == 0:
            del out[k]
    return out


def stencil_weights(m: int):
    """Weights of every interpolation node for the segment M*_{<=m}.

    Returns (nodes, wA, wB, det): wA[q] = A phi_q and wB[q] = B phi_q / tau as
    polynomials in lambda, and det(D) in the scaled variables."""
    monos = monomial_segment(m)
    nodes = nodes_of(monos)
    if len(set(nodes)) != m:
        raise ValueError("McKinney map is not one-to-one on this segment")
    d = matrix_d(monos, nodes)
    w, det = _solve_inverse(d)  # L_t = sum_s w[s][t] mu_s
    wa, wb = {}, {}
    for t, node in enumerate(nodes):
        pa: Poly = {}
        pb: Poly = {}
        for s, mu in enumerate(monos):
            if w[s][t] != 0:
                pa = _padd(pa, a_of_monomial(mu), w[s][t])
                pb = _padd(pb, b_of_monomial(mu), w[s][t])
        wa[node] = pa
        wb[node] = pb
    return nodes, wa, wb, det


def evaluate(p: Poly, lam: float) -> float:
    return float(sum(float(c) * lam ** k for k, c in p.items()))


SEGMENT = {5: 6, 9: 11, 13: 15}


def delta_coefficients(scheme: int):
    """(a10, a11, a20), (b10, b11, b20) of the delta / epsilon form as
    polynomials in lambda: the two-step adds a . delta(u^k) (a = 2 A phi on
    the shells (1,0), (1,1), (2,0)), the first step a/2 . delta(u^0) +
    tau * b . epsilon(v^0)."""
    nodes, wa, wb, _ = stencil_weights(SEGMENT[scheme])
    shells = [(1, 0), (1, 1), (2, 0)]
    a, b = [], []
    for s in shells:
        pa = wa.get(s, {})
        a.append({k: 2 * v for k, v in pa.items()})
        b.append(wb.get(s, {}))
    return a, b


# ---------------------------------------------------------------------------
# Derived schemes beyond Section 6.  Larger segments M*_{<=m} give further
# stencils; where the weights are symmetric under the eight symmetries of the
# square they group into classes, a class being every node (+-q1, +-q2),
# (+-q2, +-q1) with q1 > 0, 0 <= q2 <= q1 (4 nodes if q2 == 0 or q2 == q1,
# else 8).  A class is named by (q1, q2).
# ---------------------------------------------------------------------------
def class_of(node: Tuple[int, int]) -> Tuple[int, int]:
    a, b = abs(node[0]), abs(node[1])
    return (max(a, b), min(a, b))


def class_nodes(cls: Tuple[int, int]) -> List[Tuple[int, int]]:
    q1, q2 = cls
    out = set()
    for a, b in ((q1, q2), (q2, q1)):
        for s1 in (1, -1):
            for s2 in (1, -1):
                out.add((s1 * a, s2 * b))
    return sorted(out)


def node_weights(m: int, lam: float):
    """(nodes, wa, wb) at Courant number lam for the segment M*_{<=m}, nodes
    with a non-zero weight polynomial only: wa = A phi_q, wb = B phi_q / tau."""
    nodes, wa, wb, _ = stencil_weights(m)
    keep = [q for q in nodes if wa[q] or wb[q]]
    return keep, [evaluate(wa[q], lam) for q in keep], [evaluate(wb[q], lam) for q in keep]


def class_scheme(m: int):
    """The stencil of the segment M*_{<=m} in class form.

    Returns (classes, a, b): the two-step adds sum_c a_c delta_c(u^k) and the
    first step a_c / 2 delta_c(u^0) + tau b_c delta_c(v^0), where delta_c is
    the sum of a level over the class's nodes minus (number of nodes) times
    the centre value; a_c = 2 A phi_q, b_c = B phi_q / tau (any q in c), as
    polynomials in lambda.  Classes are sorted by (radius, q2).  Raises
    ValueError if the weights are not symmetric."""
    nodes, wa, wb, _ = stencil_weights(m)
    groups: Dict[Tuple[int, int], List[Tuple[int, int]]] = {}
    for q in nodes:
        if q != (0, 0) and (wa[q] or wb[q]):
            groups.setdefault(class_of(q), []).append(q)
    classes = sorted(groups, key=lambda c: (c[0], c[1]))
    a, b = [], []
    for cls in classes:
        members = class_nodes(cls)
        pa, pb = wa.get(members[0], {}), wb.get(members[0], {})
        for q in members:
            if wa.get(q, {}) != pa or wb.get(q, {}) != pb:
                raise ValueError(f"segment {m}: weights are not symmetric on class {cls}")
        a.append({k: 2 * v for k, v in pa.items()})
        b.append(dict(pb))
    return classes, a, b
