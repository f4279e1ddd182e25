"""Host side of the derived schemes through the C ABI (no GPU needed):
wave2d_derive_scheme against the oracle's exact-rational derivation, and
wave2d_scheme_lambda_max against the oracle's symbol scan and the printed
Section 6 limits."""
import math

import pytest

from oracle import derive, plane_wave


@pytest.fixture(scope="module")
def w():
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def _oracle_polys(m):
    """Oracle class form mapped onto chain positions: {chain index: (a, b)}."""
    from paper_1904_04048_gb300.wave2d import CLASS_CHAIN
    classes, a, b = derive.class_scheme(m)
    out = {}
    for cls, pa, pb in zip(classes, a, b):
        c = CLASS_CHAIN.index(cls)
        out[c] = ([float(pa.get(p, 0)) for p in range(9)], [float(pb.get(p, 0)) for p in range(9)])
    return out


@pytest.mark.parametrize("m", [6, 11, 15, 24, 28, 37, 41, 45])
def test_derivation_matches_exact_rationals(w, m):
    s = w.derive_scheme(m)
    ref = _oracle_polys(m)
    assert s.segment == m
    assert s.n_classes == max(ref) + 1
    assert s.radius == max(w.CLASS_CHAIN[c][0] for c in ref)
    classes, _, _ = derive.class_scheme(m)
    assert s.n_points == 1 + sum(len(derive.class_nodes(c)) for c in classes)
    for c in range(8):
        ra, rb = ref.get(c, ([0.0] * 9, [0.0] * 9))
        for p in range(9):
            assert abs(s.a[c][p] - ra[p]) <= 1e-14 * max(1.0, abs(ra[p])), (m, c, p)
            assert abs(s.b[c][p] - rb[p]) <= 1e-14 * max(1.0, abs(rb[p])), (m, c, p)


def test_section6_segments_give_the_printed_coefficients(w):
    lam = 0.6
    for scheme, m in derive.SEGMENT.items():
        s = w.derive_scheme(m)
        a6, b6 = plane_wave.section6_coeffs(scheme, lam)
        for c in range(3):
            a = sum(s.a[c][p] * lam ** p for p in range(9))
            b = sum(s.b[c][p] * lam ** p for p in range(9))
            assert abs(a - a6[c]) < 1e-15 and abs(b - b6[c]) < 1e-15


@pytest.mark.parametrize("m", [0, 5, 14, 23, 27, 40, 44, 50, 1, 4])
def test_rejected_segments(w, m):
    with pytest.raises(w.Wave2DError) as e:
        w.derive_scheme(m)
    assert e.value.code == w.ERR_ARG


@pytest.mark.parametrize("m,limit", [(6, 1 / math.sqrt(2)), (11, math.sqrt((3 - math.sqrt(3)) / 2)),
                                     (15, 1 / math.sqrt(2))])
def test_lambda_max_of_section6_segments(w, m, limit):
    assert abs(w.scheme_lambda_max(w.derive_scheme(m)) - limit) < 1e-12


@pytest.mark.parametrize("m", [24, 28, 37, 41, 45])
def test_lambda_max_matches_oracle_scan(w, m):
    classes, a, _ = derive.class_scheme(m)
    ref = plane_wave.stability_limit(classes, lambda l: [derive.evaluate(p, l) for p in a])
    assert abs(w.scheme_lambda_max(w.derive_scheme(m)) - ref) < 1e-9


def test_invalid_scheme_structs_are_rejected(w):
    s = w.derive_scheme(24)
    for mutate in (lambda t: setattr(t, "n_classes", 0), lambda t: setattr(t, "n_classes", 9)):
        t = w.wave2d_scheme.from_buffer_copy(s)
        mutate(t)
        with pytest.raises(w.Wave2DError):
            w.scheme_lambda_max(t)
    t = w.wave2d_scheme.from_buffer_copy(s)
    t.a[6][2] = 1.0  # beyond n_classes = 4
    with pytest.raises(w.Wave2DError):
        w.scheme_lambda_max(t)
    t = w.wave2d_scheme.from_buffer_copy(s)
    t.b[0][0] = float("nan")
    with pytest.raises(w.Wave2DError):
        w.scheme_lambda_max(t)
