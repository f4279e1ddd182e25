"""Pins of the oracle's odd-reflection boundary (the Dirichlet condition of
Section 6.1.2 with the field continued as an odd function beyond the boundary
nodes, a reading for stencils wider than one node):

* radius-1 stencils (5 and 9 points) read only the boundary nodes, so the
  odd continuation gives exactly the zero boundary;
* on any initial data the odd-boundary run equals the periodic run on the
  odd extension of the data (period 2(n + 1)), restricted to the interior —
  the periodic boundary is separate oracle code, so this pins the reflection
  rule, its signs and the corner (double) reflections;
* the 13-point standing wave of Table 3 (periodic in the paper) is odd about
  the boundary lines, so the odd boundary on the Dirichlet node set reproduces
  the printed E_P13 and E_C13 values.
"""
import numpy as np
import pytest

from conftest import load_golden
from initial_data import BC_ODD, BC_PERIODIC, BC_ZERO, standing_wave_ic
from oracle import derive


def _smooth(nx, ny, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((ny, nx))
    v = rng.standard_normal((ny, nx))
    return u, v


@pytest.mark.parametrize("scheme", [5, 9])
def test_radius_one_equals_zero_boundary(orc, scheme):
    u0, v0 = _smooth(11, 7, scheme)
    a = orc.run(scheme, u0, v0, 0.6, 0.06, 12, bc=BC_ODD)
    b = orc.run(scheme, u0, v0, 0.6, 0.06, 12, bc=BC_ZERO)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _odd_extension(u):
    """Periodic array of shape (2(ny+1), 2(nx+1)) holding u, its odd mirror
    images about the boundary nodes, and zeros on the boundary nodes."""
    ny, nx = u.shape

    def line(n):
        # extended index e -> (interior index, sign); boundary -> (-1, 0)
        idx, sgn = [], []
        for e in range(2 * (n + 1)):
            if e < n:
                idx.append(e); sgn.append(1.0)
            elif e == n or e == 2 * n + 1:
                idx.append(0); sgn.append(0.0)
            else:
                idx.append(2 * n - e); sgn.append(-1.0)
        return np.array(idx), np.array(sgn)

    ix, sx = line(nx)
    iy, sy = line(ny)
    return u[np.ix_(iy, ix)] * sy[:, None] * sx[None, :]


@pytest.mark.parametrize("scheme", [13])
@pytest.mark.parametrize("shape", [(9, 6), (14, 11)])
def test_equals_periodic_run_on_odd_extension(orc, scheme, shape):
    nx, ny = shape
    u0, v0 = _smooth(nx, ny, nx)
    lam, h = 0.6, 0.1
    up, uc, _ = orc.run(scheme, u0, v0, lam, lam * h, 15, bc=BC_ODD)
    ep, ec, _ = orc.run(scheme, _odd_extension(u0), _odd_extension(v0), lam, lam * h, 15, bc=BC_PERIODIC)
    # equal up to rounding: the printed forms sum the four rotations in
    # sequence, so on the extension the boundary nodes keep residues of
    # order 1e-18 instead of exact zeros
    scale = 1 + np.max(np.abs(ec))
    assert np.max(np.abs(uc - ec[:ny, :nx])) < 1e-13 * scale
    assert np.max(np.abs(up - ep[:ny, :nx])) < 1e-13 * scale


@pytest.mark.parametrize("m", [28, 45])
def test_node_form_equals_periodic_run_on_odd_extension(orc, m):
    nx, ny = 12, 10  # radius 3 and 4 reach the second mirror image
    u0, v0 = _smooth(nx, ny, m)
    lam, h = 0.5, 0.1
    nodes, wa, wb = derive.node_weights(m, lam)
    _, uc = orc.run_nodes(nodes, wa, wb, u0, v0, lam * h, 12, bc=BC_ODD)
    _, ec = orc.run_nodes(nodes, wa, wb, _odd_extension(u0), _odd_extension(v0), lam * h, 12, bc=BC_PERIODIC)
    assert np.max(np.abs(uc - ec[:ny, :nx])) < 1e-13 * (1 + np.max(np.abs(ec)))


@pytest.mark.parametrize("row", load_golden("table3.txt"), ids=lambda r: f"n{int(r[0])}")
def test_table3_on_the_dirichlet_node_set(orc, row):
    n, n_t, e_p13, e_c13 = int(row[0]), int(row[1]), row[2], row[3]
    h = 1.0 / n
    u0, v0 = standing_wave_ic(n - 1, n - 1, h, BC_ODD)
    for conventional, printed in ((False, e_p13), (True, e_c13)):
        _, _, err = orc.run(13, u0, v0, 0.707, 0.707 * h, n_t, bc=BC_ODD, conventional=conventional,
                            exact=orc.EXACT_STANDING, exact_params=(1.0, 1.0), h=h, x_off=1.0)
        ours = orc.relative_spacetime_error(err)
        assert float(f"{ours:.4e}") == printed, (conventional, ours, printed)
