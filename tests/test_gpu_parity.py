"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every scheme x storage type x boundary x kernel on small and ragged grids
that span several tiles, element by element, within the per-dtype tolerances
of gpu_util.TOL; bitwise agreement between kernels that share the per-node
arithmetic; the paper's space-time error E(n, n_t) from the fused reduction.
"""
import math

import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, LAMBDA_MAX, standing_wave_ic

pytestmark = pytest.mark.gpu

SIZES = [(8, 8), (13, 31), (64, 64), (257, 130), (300, 97)]


@pytest.fixture(scope="module")
def w():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def run_gpu(w, scheme, u0, v0, h, lam, steps, bc, dtype, kernel, flags=0):
    ny, nx = u0.shape
    with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=dtype, flags=flags) as sim:
        sim.set_tuning(kernel=kernel, use_graph=0)
        sim.first_step(u0, v0)
        if steps > 1:
            sim.step_n(steps - 1)
        up, uc, k = sim.get_state()
    assert k == steps
    return up, uc


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("dtype", [0, 1, 2], ids=["f64", "f32", "f32x2"])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("shape", SIZES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_parity_simple_kernel(orc, w, scheme, dtype, bc, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, bc, seed=nx * 7 + ny)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 40
    up, uc = run_gpu(w, scheme, u0, v0, h, lam, steps, bc, dtype, w.KERNEL_SIMPLE)
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, steps, bc=bc)
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < TOL[dtype] and linf < TOL[dtype], (l2, linf)


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("dtype", [0, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("shape", SIZES + [(520, 75)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_parity_tma_kernel(orc, w, scheme, dtype, bc, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, bc, seed=nx + 3 * ny)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 40
    up, uc = run_gpu(w, scheme, u0, v0, h, lam, steps, bc, dtype, w.KERNEL_TMA)
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, steps, bc=bc)
    l2, linf = rel_errors(uc, rc)
    assert l2 < TOL[dtype] and linf < TOL[dtype], (l2, linf)
    # same per-node arithmetic as the one-node-per-thread kernel: bitwise equal
    sp, sc = run_gpu(w, scheme, u0, v0, h, lam, steps, bc, dtype, w.KERNEL_SIMPLE)
    assert np.array_equal(uc, sc) and np.array_equal(up, sp)


@pytest.mark.parametrize("scheme", [5, 9, 13])
def test_conventional_schemes(orc, w, scheme):
    nx, ny = 70, 45
    u0, v0, h = smooth_ic(nx, ny, BC_ZERO, seed=3)
    lam = 0.6
    up, uc = run_gpu(w, scheme, u0, v0, h, lam, 30, BC_ZERO, 0, w.KERNEL_SIMPLE, flags=w.CONVENTIONAL)
    _, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, 30, bc=BC_ZERO, conventional=True)
    l2, linf = rel_errors(uc, rc)
    assert l2 < 1e-12 and linf < 1e-12


@pytest.mark.parametrize("kernel", ["simple", "tma"])
def test_fp32_thousand_steps_tolerance(orc, w, kernel):
    """The stated FP32 bound at its stated length: 1000 steps, 13 points."""
    n = 256
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=5)
    lam = 0.9 * LAMBDA_MAX[13]
    kern = w.KERNEL_SIMPLE if kernel == "simple" else w.KERNEL_TMA
    _, uc = run_gpu(w, 13, u0, v0, h, lam, 1000, BC_PERIODIC, 1, kern)
    _, rc, _ = orc.run(13, u0, v0, lam, lam * h, 1000, bc=BC_PERIODIC)
    l2, linf = rel_errors(uc, rc)
    assert l2 < 1e-5 and linf < 1e-5, (l2, linf)


# ----------------------------------------------------------- paper tables

@pytest.mark.parametrize("scheme,n,n_t,conv,bc", [
    (5, 20, 40, False, BC_ZERO), (5, 40, 40, True, BC_ZERO), (9, 20, 20, True, BC_ZERO),
    (9, 40, 40, False, BC_ZERO), (13, 40, 40, False, BC_PERIODIC), (13, 20, 20, True, BC_PERIODIC)])
@pytest.mark.parametrize("dtype", [0, 2], ids=["f64", "f32x2"])
def test_spacetime_error_matches_oracle(orc, w, scheme, n, n_t, conv, bc, dtype):
    """E(n, n_t) of Eq. error from the fused per-step reduction (Tables 1-3)."""
    h = 1.0 / n
    lam = 0.707
    nn = n - 1 if bc == BC_ZERO else n
    x_off = 1.0 if bc == BC_ZERO else 0.0
    u0, v0 = standing_wave_ic(nn, nn, h, bc)
    ex = w.exact(w.EXACT_STANDING, amp=1.0, m=1.0, x_off=x_off)
    with w.Wave2D(nn, nn, h, lam * h, scheme=scheme, bc=bc, dtype=dtype,
                  flags=w.CONVENTIONAL if conv else 0) as sim:
        sim.track_error(ex)
        sim.first_step(u0, v0)
        sim.step_n(n_t - 1)
        l2, linf, E = sim.error_vs_exact(ex)
        _, uc, _ = sim.get_state()
    _, rc, err = orc.run(scheme, u0, v0, lam, lam * h, n_t, bc=bc, conventional=conv,
                         exact=orc.EXACT_STANDING, exact_params=(1.0, 1.0), h=h, x_off=x_off)
    E_ref = orc.relative_spacetime_error(err)
    # E is a relative error of the field, so rounding differences of the
    # field (bounded by the dtype tolerance relative to ||u||) bound |dE|.
    assert abs(E - E_ref) <= TOL[dtype] + 1e-9 * E_ref, (E, E_ref)
    s = orc.error_sums(uc, h, x_off, orc.EXACT_STANDING, (1.0, 1.0), 1.0, n_t * lam * h)
    assert abs(l2 - math.sqrt(s[0] / s[1])) <= 1e-9 * l2  # same field: reduction order only


def test_plane_wave_error_norms(orc, w):
    n = 64
    h = 1.0 / n
    lam = 0.5
    k1, k2 = 2 * math.pi * 3, 2 * math.pi * 2
    from initial_data import plane_wave_ic
    u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
    ex = w.exact(w.EXACT_PLANE, amp=1.0, k1=k1, k2=k2, x_off=0.0)
    with w.Wave2D(n, n, h, lam * h, scheme=13, bc=BC_PERIODIC, dtype=0) as sim:
        sim.first_step(u0, v0)
        sim.step_n(99)
        l2, linf, E = sim.error_vs_exact(ex)
        _, uc, _ = sim.get_state()
    assert math.isnan(E)
    s = orc.error_sums(uc, h, 0.0, orc.EXACT_PLANE, (1.0, k1, k2), 1.0, 100 * lam * h)
    assert abs(l2 - math.sqrt(s[0] / s[1])) <= 1e-9 * l2
    X = np.arange(n) * h
    ue = np.cos(k1 * X[None, :] + k2 * X[:, None] - math.hypot(k1, k2) * 100 * lam * h)
    assert abs(linf - np.max(np.abs(uc - ue)) / np.max(np.abs(ue))) <= 1e-9 * linf
