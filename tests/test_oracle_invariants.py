"""Pins P6-P8 and P10 of the oracle, plus the stability limits.

P6  closed-form discrete plane wave (discrete dispersion relation) vs stepping;
P7  the discrete energy ||u^{k+1}-u^k||^2 - <u^{k+1}, Lambda u^k> is conserved
    inside the stability region (Lambda is symmetric) and the solution grows
    just outside it;
P8  D4 symmetry: delta sums over all four 90-degree rotations (Eq.
    notations2), so rotating or reflecting the data rotates or reflects u;
P10 brute force: a dense N^2 x N^2 update matrix assembled from the weights of
    the Section 4-5 derivation, applied by mat-vec, equals the stencil oracle.
"""
import math

import numpy as np
import pytest

from initial_data import BC_PERIODIC, BC_ZERO, LAMBDA_MAX, plane_wave_ic
from oracle import derive, plane_wave

SCHEMES = [5, 9, 13]


# ---------------------------------------------------------------- stability

def min_symbol(scheme, lam, conventional=False, n=721):
    a, _ = plane_wave.section6_coeffs(scheme, lam, conventional)
    th = np.linspace(0, 2 * math.pi, n)
    T1, T2 = np.meshgrid(th, th)
    c1, c2 = np.cos(T1), np.cos(T2)
    s = a[0] * (2 * c1 + 2 * c2 - 4) + a[1] * (4 * c1 * c2 - 4) + a[2] * (2 * np.cos(2 * T1) + 2 * np.cos(2 * T2) - 4)
    return float(s.min())


@pytest.mark.parametrize("scheme,lmax", [(5, 1 / math.sqrt(2)), (9, math.sqrt((3 - math.sqrt(3)) / 2)),
                                          (13, 1 / math.sqrt(2))])
def test_von_neumann_limits(scheme, lmax):
    """Two-step amplification g solves g^2 - (2 + S) g + 1 = 0; |g| <= 1 iff
    -4 <= S <= 0.  The limit of Eq. stability9 is read as sqrt((3-sqrt3)/2)."""
    assert abs(LAMBDA_MAX[scheme] - lmax) < 1e-15
    assert min_symbol(scheme, 0.999 * lmax) >= -4.0
    assert min_symbol(scheme, 1.01 * lmax) < -4.0
    a, _ = plane_wave.section6_coeffs(scheme, 0.5)
    assert max(0.0, -min_symbol(scheme, 0.5)) > 0  # S <= 0 everywhere, nonzero somewhere


def test_conventional_nine_point_limit():
    """The isotropic scheme is stable up to sqrt(3)/2 (Section 6.2)."""
    lmax = math.sqrt(3) / 2
    assert min_symbol(9, 0.999 * lmax, conventional=True) >= -4.0
    assert min_symbol(9, 1.01 * lmax, conventional=True) < -4.0


# ------------------------------------------------------------ plane wave (P6)

@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("m", [(1, 0), (3, 4), (2, 5)])
@pytest.mark.parametrize("conventional", [False, True])
def test_discrete_plane_wave_closed_form(orc, scheme, m, conventional):
    n = 32
    h = 1.0 / n
    lam = 0.9 * LAMBDA_MAX[scheme]
    tau = lam * h
    k1, k2 = 2 * math.pi * m[0], 2 * math.pi * m[1]
    u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
    for n_t in (1, 2, 7, 60):
        _, un, _ = orc.run(scheme, u0, v0, lam, tau, n_t, bc=BC_PERIODIC, conventional=conventional)
        cf = plane_wave.field(scheme, lam, tau, k1, k2, h, n, n, n_t, conventional=conventional)
        assert np.max(np.abs(un - cf)) < 1e-12, (n_t, np.max(np.abs(un - cf)))


def test_discrete_plane_wave_long_run(orc):
    n = 24
    h = 1.0 / n
    lam = 0.9 / math.sqrt(2)
    k1, k2 = 2 * math.pi * 3, 2 * math.pi * 1
    u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
    _, un, _ = orc.run(13, u0, v0, lam, lam * h, 500, bc=BC_PERIODIC)
    cf = plane_wave.field(13, lam, lam * h, k1, k2, h, n, n, 500)
    assert np.max(np.abs(un - cf)) < 5e-12


# ---------------------------------------------------------- energy (P7)

def lambda_op(scheme, lam, u, bc):
    """Lambda_a applied with the weights of the Section 4-5 derivation
    (independent of the oracle's printed expressions)."""
    a_poly, _ = derive.delta_coefficients(scheme)
    a = [derive.evaluate(p, lam) for p in a_poly]
    if bc == BC_PERIODIC:
        sh = lambda di, dj: np.roll(np.roll(u, -dj, axis=0), -di, axis=1)
    else:
        pad = np.pad(u, 2)
        ny, nx = u.shape
        sh = lambda di, dj: pad[2 + dj:2 + dj + ny, 2 + di:2 + di + nx]
    out = np.zeros_like(u)
    for coef, (q1, q2) in zip(a, [(1, 0), (1, 1), (2, 0)]):
        if coef == 0:
            continue
        s = sh(q1, q2) + sh(-q2, q1) + sh(-q1, -q2) + sh(q2, -q1) - 4 * u
        out += coef * s
    return out


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC])
def test_energy_is_conserved_inside_stability_region(orc, scheme, bc):
    rng = np.random.default_rng(11)
    n = 20
    lam = 0.97 * LAMBDA_MAX[scheme]
    u0 = rng.standard_normal((n, n))
    v0 = rng.standard_normal((n, n))
    up, uc, _ = orc.run(scheme, u0, v0, lam, 0.01, 2, bc=bc)
    energies = []
    for _ in range(200):
        e = np.sum((uc - up) ** 2) - np.sum(uc * lambda_op(scheme, lam, up, bc))
        energies.append(e)
        up, uc = orc.continue_run(scheme, up, uc, lam, 1, bc=bc)
    energies = np.array(energies)
    assert energies.min() > 0
    assert np.max(np.abs(energies - energies[0])) < 1e-11 * energies[0]
    assert np.max(np.abs(uc)) < 1e3


@pytest.mark.parametrize("scheme", SCHEMES)
def test_solution_grows_just_outside_stability_region(orc, scheme):
    rng = np.random.default_rng(12)
    n = 32  # even: the unstable checkerboard mode (pi, pi) lives on the grid
    lam = 1.01 * LAMBDA_MAX[scheme]
    u0 = rng.standard_normal((n, n))
    v0 = rng.standard_normal((n, n))
    _, un, _ = orc.run(scheme, u0, v0, lam, 0.01, 400, bc=BC_PERIODIC)
    assert np.max(np.abs(un)) > 1e6
    _, us, _ = orc.run(scheme, u0, v0, 0.99 * LAMBDA_MAX[scheme], 0.01, 400, bc=BC_PERIODIC)
    assert np.max(np.abs(us)) < 1e3


# ---------------------------------------------------------- symmetry (P8)

@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC])
def test_d4_symmetry(orc, scheme, bc):
    rng = np.random.default_rng(13)
    n = 17
    u0 = rng.standard_normal((n, n))
    v0 = rng.standard_normal((n, n))
    lam = 0.6
    _, ref, _ = orc.run(scheme, u0, v0, lam, 0.05, 25, bc=bc)
    scale = np.max(np.abs(ref))
    for op in (lambda a: np.rot90(a, 1), lambda a: np.rot90(a, 2), lambda a: np.rot90(a, 3),
               lambda a: a.T.copy(), lambda a: a[::-1].copy(), lambda a: a[:, ::-1].copy()):
        _, got, _ = orc.run(scheme, op(u0), op(v0), lam, 0.05, 25, bc=bc)
        assert np.max(np.abs(got - op(ref))) < 1e-12 * scale


# -------------------------------------------------------- brute force (P10)

def dense_operators(scheme, lam, nx, ny, bc):
    """Dense matrices W_A, W_B with u^1 = W_A u^0 + tau W_B v^0 and
    u^{k+1} = 2 W_A u^k - u^{k-1}, from the derived node weights."""
    nodes, wa, wb, _ = derive.stencil_weights(derive.SEGMENT[scheme])
    N = nx * ny
    WA = np.zeros((N, N))
    WB = np.zeros((N, N))
    for j in range(ny):
        for i in range(nx):
            row = j * nx + i
            for (q1, q2) in nodes:
                ii, jj = i + q1, j + q2
                if bc == BC_PERIODIC:
                    ii, jj = ii % nx, jj % ny
                elif not (0 <= ii < nx and 0 <= jj < ny):
                    continue
                WA[row, jj * nx + ii] += derive.evaluate(wa[(q1, q2)], lam)
                WB[row, jj * nx + ii] += derive.evaluate(wb[(q1, q2)], lam)
    return WA, WB


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("shape", [(8, 8), (5, 7), (13, 13)])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC])
def test_brute_force_dense_evaluation(orc, scheme, shape, bc):
    ny, nx = shape
    rng = np.random.default_rng(17)
    u0 = rng.standard_normal((ny, nx))
    v0 = rng.standard_normal((ny, nx))
    lam, tau = 0.65, 0.03
    WA, WB = dense_operators(scheme, lam, nx, ny, bc)
    prev = u0.ravel()
    cur = WA @ prev + tau * (WB @ v0.ravel())
    for n_t in range(1, 21):
        if n_t > 1:
            prev, cur = cur, 2 * (WA @ cur) - prev
        _, un, _ = orc.run(scheme, u0, v0, lam, tau, n_t, bc=bc)
        assert np.max(np.abs(un.ravel() - cur)) < 1e-12 * max(1.0, np.max(np.abs(cur))), n_t
