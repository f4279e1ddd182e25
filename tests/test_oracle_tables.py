"""Pins P1-P3: the oracle reproduces the accuracy tables printed in the paper.

Table 1 (Section 6.1.2) pins the 5-point first steps (new and conventional),
the 5-point two-step, the zero boundary and the error norm E(n, n_t).  Table 2
(Section 6.2.2) pins the conventional 9-point scheme, including the diagonal
sums delta(1,1).  Table 3 (Section 6.3) pins the 13-point first steps, the
13-point two-step and the periodic boundary.
"""
import math

import numpy as np
import pytest

from conftest import load_golden
from initial_data import BC_PERIODIC, BC_ZERO, standing_wave_ic


def spacetime_error(orc, scheme, n, n_t, lam, bc, conventional):
    h = 1.0 / n
    tau = lam * h  # c = 1
    nn = n - 1 if bc == BC_ZERO else n
    u0, v0 = standing_wave_ic(nn, nn, h, bc)
    _, _, err = orc.run(scheme, u0, v0, lam, tau, n_t, bc=bc, conventional=conventional,
                        exact=orc.EXACT_STANDING, exact_params=(1.0, 1.0), h=h,
                        x_off=1.0 if bc == BC_ZERO else 0.0)
    return orc.relative_spacetime_error(err)


def close_digits(ours, printed, digits=5):
    """Equal when rounded to the printed number of significant digits."""
    return float(f"{ours:.{digits - 1}e}") == printed


@pytest.mark.parametrize("row", load_golden("table1.txt"), ids=lambda r: f"n{int(r[0])}_nt{int(r[1])}")
def test_table1_five_point(orc, row):
    n, n_t, e_p5, e_c5 = int(row[0]), int(row[1]), row[2], row[3]
    ours_c = spacetime_error(orc, 5, n, n_t, 0.707, BC_ZERO, True)
    ours_p = spacetime_error(orc, 5, n, n_t, 0.707, BC_ZERO, False)
    assert close_digits(ours_c, e_c5), (ours_c, e_c5)
    # E_P5 reproduces to all printed digits for 6 of 12 rows and within 0.2 %
    # for the rest (largest gap at n = 80).
    assert abs(ours_p - e_p5) / e_p5 < 3e-3, (ours_p, e_p5)


def test_table1_five_point_exact_rows(orc):
    exact_rows = [r for r in load_golden("table1.txt") if int(r[0]) == 10 or (int(r[0]) == 20 and int(r[1]) < 40)]
    assert len(exact_rows) == 5
    for r in exact_rows:
        ours = spacetime_error(orc, 5, int(r[0]), int(r[1]), 0.707, BC_ZERO, False)
        assert close_digits(ours, r[2]), (r, ours)


@pytest.mark.parametrize("row", load_golden("table2.txt"), ids=lambda r: f"n{int(r[0])}_lam{r[2]}")
def test_table2_nine_point_conventional(orc, row):
    n, n_t, lam, _e_p9, e_c9 = int(row[0]), int(row[1]), row[2], row[3], row[4]
    ours = spacetime_error(orc, 9, n, n_t, lam, BC_ZERO, True)
    assert close_digits(ours, e_c9), (ours, e_c9)


def test_table2_nine_point_new_scheme_is_more_accurate(orc):
    """The printed E_P9 values do not reproduce; the qualitative claim of
    Section 6.2.2 (new scheme more accurate than the isotropic one at both
    Courant numbers) does."""
    for row in load_golden("table2.txt"):
        n, lam = int(row[0]), row[2]
        e_new = spacetime_error(orc, 9, n, n, lam, BC_ZERO, False)
        e_conv = spacetime_error(orc, 9, n, n, lam, BC_ZERO, True)
        assert e_new < e_conv


@pytest.mark.parametrize("row", load_golden("table3.txt"), ids=lambda r: f"n{int(r[0])}")
def test_table3_thirteen_point_periodic(orc, row):
    n, n_t, e_p13, e_c13 = int(row[0]), int(row[1]), row[2], row[3]
    assert close_digits(spacetime_error(orc, 13, n, n_t, 0.707, BC_PERIODIC, False), e_p13)
    assert close_digits(spacetime_error(orc, 13, n, n_t, 0.707, BC_PERIODIC, True), e_c13)


@pytest.mark.parametrize("n,lam", [(10, 0.707), (20, 0.707), (40, 0.5), (16, 0.3)])
def test_conventional_first_step_error_closed_form(orc, n, lam):
    """With u0 = 0 the conventional first step gives u^1 = tau v0 while the
    exact solution is sin(w tau)/w * v0, so E_C5(n, 1) = |w tau - sin w tau| /
    |sin w tau| with w = 2 sqrt2 pi (this is 6.8938e-2 at n = 10, Table 1)."""
    w = 2.0 * math.sqrt(2.0) * math.pi
    tau = lam / n
    expect = abs(w * tau - math.sin(w * tau)) / abs(math.sin(w * tau))
    ours = spacetime_error(orc, 5, n, 1, lam, BC_ZERO, True)
    assert abs(ours - expect) < 1e-12 * expect + 1e-15
