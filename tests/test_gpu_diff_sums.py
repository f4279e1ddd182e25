"""GPU tests of WAVE2D_DIFF_SUMS (stencil sums formed from differences to
the centre): parity against the FP64 oracle for the Section 6 and derived
schemes, bitwise agreement of its kernels and bitwise D4 symmetry, the
refusals, and the accuracy gain for a long wave in FP32."""
import math

import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, LAMBDA_MAX, plane_wave_ic
from oracle import derive, plane_wave

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def _run(w, scheme, u0, v0, h, lam, steps, bc, dtype, kernel, flags):
    ny, nx = u0.shape
    with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=dtype, flags=flags) as sim:
        sim.set_tuning(kernel=kernel, use_graph=0)
        sim.first_step(u0, v0)
        sim.step_n(steps - 1)
        return sim.get_state()


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("dtype,kernel", [(0, 1), (0, 2), (1, 1), (1, 2)])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("shape", [(13, 31), (300, 97)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_parity_section6(orc, w, scheme, dtype, kernel, bc, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, bc, seed=nx + scheme)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 40
    up, uc, k = _run(w, scheme, u0, v0, h, lam, steps, bc, dtype, kernel, w.DIFF_SUMS)
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, steps, bc=bc)
    assert k == steps
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < TOL[dtype] and linf < TOL[dtype], (l2, linf)


@pytest.mark.parametrize("m", [28, 45])
@pytest.mark.parametrize("dtype,kernel", [(0, 2), (1, 1), (1, 2)])
def test_parity_derived(orc, w, m, dtype, kernel):
    n = 150
    u0, v0, h = smooth_ic(n, 77, BC_PERIODIC, seed=m)
    s = w.derive_scheme(m)
    lam = 0.9 * w.scheme_lambda_max(s)
    steps = 30
    _, uc, _ = _run(w, s, u0, v0, h, lam, steps, BC_PERIODIC, dtype, kernel, w.DIFF_SUMS)
    nodes, wa, wb = derive.node_weights(m, lam)
    _, rc = orc.run_nodes(nodes, wa, wb, u0, v0, lam * h, steps, bc=BC_PERIODIC)
    l2, linf = rel_errors(uc, rc)
    assert l2 < TOL[dtype] and linf < TOL[dtype], (l2, linf)


@pytest.mark.parametrize("scheme", [9, 13])
@pytest.mark.parametrize("dtype", [0, 1])
def test_tma_equals_simple_bitwise(w, scheme, dtype):
    n = 260
    u0, v0, h = smooth_ic(n, 150, BC_PERIODIC, seed=scheme)
    lam = 0.9 * LAMBDA_MAX[scheme]
    a = _run(w, scheme, u0, v0, h, lam, 60, BC_PERIODIC, dtype, w.KERNEL_SIMPLE, w.DIFF_SUMS)
    b = _run(w, scheme, u0, v0, h, lam, 60, BC_PERIODIC, dtype, w.KERNEL_TMA, w.DIFF_SUMS)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("kernel", [1, 2])
def test_d4_symmetry_is_bitwise(w, kernel):
    n = 133
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=5)
    lam = 0.9 * LAMBDA_MAX[13]

    def run(a, b):
        return _run(w, 13, a, b, h, lam, 40, BC_PERIODIC, 1, kernel, w.DIFF_SUMS)[1]

    ref = run(u0, v0)
    for op in (lambda a: np.rot90(a).copy(), lambda a: a.T.copy(), lambda a: a[::-1].copy()):
        assert np.array_equal(run(op(u0), op(v0)), op(ref))


def test_refusals(w):
    n = 32
    with pytest.raises(w.Wave2DError) as e:
        w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=13, dtype=w.F32X2, flags=w.DIFF_SUMS)
    assert e.value.code == w.ERR_ARG
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=13, dtype=w.F32, flags=w.DIFF_SUMS) as sim:
        with pytest.raises(w.Wave2DError) as e:
            sim.set_tuning(kernel=w.KERNEL_TEMPORAL)
        assert e.value.code == w.ERR_ARG
        assert sim.info().scheme == 13 and sim.info().n_classes == 3
        with pytest.raises(w.Wave2DError) as e:
            w.Batch([sim])
        assert e.value.code == w.ERR_ARG


def test_conventional_with_difference_sums(orc, w):
    n = 96
    u0, v0, h = smooth_ic(n, n, BC_ZERO, seed=2)
    lam = 0.7
    _, uc, _ = _run(w, 9, u0, v0, h, lam, 50, BC_ZERO, 1, w.KERNEL_TMA, w.DIFF_SUMS | w.CONVENTIONAL)
    _, rc, _ = orc.run(9, u0, v0, lam, lam * h, 50, bc=BC_ZERO, conventional=True)
    l2, linf = rel_errors(uc, rc)
    assert l2 < TOL[1] and linf < TOL[1]


def test_long_wave_is_more_accurate_in_fp32(w):
    """Mode (1, 0) on a 1024^2 periodic grid, 13 points, 3000 steps, FP32:
    against the closed-form discrete solution the difference sums keep the
    error several times lower than the plain sums (the class sums of a long
    wave cancel to (omega tau)^2 of the field)."""
    n, steps = 1024, 3000
    h = 1.0 / n
    lam = 0.9 * LAMBDA_MAX[13]
    tau = lam * h
    k1, k2 = 2 * math.pi, 0.0
    u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
    an, bn = plane_wave.amplitudes(13, lam, tau, k1, k2, h, steps)
    x = np.arange(n) * h
    ref = an * np.cos(k1 * x) + bn * np.sin(k1 * x)
    errs = []
    for flags in (0, w.DIFF_SUMS):
        _, uc, _ = _run(w, 13, u0, v0, h, lam, steps, BC_PERIODIC, w.F32, w.KERNEL_TMA, flags)
        errs.append(float(np.sqrt(np.mean((uc - ref[None, :]) ** 2)) / np.sqrt(np.mean(ref ** 2))))
    assert errs[1] < errs[0] / 3, errs


# ---------------------------------------------------------------- difference form
@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC], ids=["zero", "periodic"])
@pytest.mark.parametrize("shape", [(13, 31), (300, 97)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_diff_form_parity(orc, w, scheme, kernel, bc, shape):
    nx, ny = shape
    u0, v0, h = smooth_ic(nx, ny, bc, seed=3 * nx + scheme)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 40
    up, uc, k = _run(w, scheme, u0, v0, h, lam, steps, bc, w.F32, kernel, w.DIFF_FORM)
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, steps, bc=bc)
    assert k == steps
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < TOL[1] and linf < TOL[1], (l2, linf)


@pytest.mark.parametrize("m", [28, 45])
@pytest.mark.parametrize("kernel", [1, 2])
def test_diff_form_parity_derived(orc, w, m, kernel):
    n = 150
    u0, v0, h = smooth_ic(n, 77, BC_PERIODIC, seed=m + 1)
    s = w.derive_scheme(m)
    lam = 0.9 * w.scheme_lambda_max(s)
    steps = 30
    _, uc, _ = _run(w, s, u0, v0, h, lam, steps, BC_PERIODIC, w.F32, kernel, w.DIFF_FORM)
    nodes, wa, wb = derive.node_weights(m, lam)
    _, rc = orc.run_nodes(nodes, wa, wb, u0, v0, lam * h, steps, bc=BC_PERIODIC)
    l2, linf = rel_errors(uc, rc)
    assert l2 < TOL[1] and linf < TOL[1], (l2, linf)


def test_diff_form_kernels_agree_and_symmetry(w):
    n = 132
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=7)
    lam = 0.9 * LAMBDA_MAX[13]
    a = _run(w, 13, u0, v0, h, lam, 50, BC_PERIODIC, w.F32, w.KERNEL_SIMPLE, w.DIFF_FORM)
    b = _run(w, 13, u0, v0, h, lam, 50, BC_PERIODIC, w.F32, w.KERNEL_TMA, w.DIFF_FORM)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    r = _run(w, 13, np.rot90(u0).copy(), np.rot90(v0).copy(), h, lam, 50, BC_PERIODIC, w.F32, w.KERNEL_TMA,
             w.DIFF_FORM)
    assert np.array_equal(r[1], np.rot90(b[1]))


def test_diff_form_state_raw_and_autotune(orc, w):
    n = 96
    u0, v0, h = smooth_ic(n, n, BC_ZERO, seed=9)
    lam = 0.6
    with w.Wave2D(n, n, h, lam * h, scheme=9, bc=BC_ZERO, dtype=w.F32, flags=w.DIFF_FORM) as sim:
        sim.first_step(u0, v0)
        sim.step_n(20)
        raw, k = sim.get_raw()
        best = sim.autotune(steps=8)  # state restored exactly
        assert best.kernel in (w.KERNEL_SIMPLE, w.KERNEL_TMA, w.KERNEL_STREAM)
        assert sim.info().k == 21 and np.array_equal(sim.get_raw()[0], raw)
        sim.step_n(30)
        _, ref, _ = sim.get_state()
    with w.Wave2D(n, n, h, lam * h, scheme=9, bc=BC_ZERO, dtype=w.F32, flags=w.DIFF_FORM) as sim:
        sim.set_raw(raw, k)
        sim.step_n(30)
        _, got, kk = sim.get_state()
    assert kk == 51 and np.array_equal(got, ref)
    # set_state from the oracle's levels, then continue against the oracle
    rp, rc, _ = orc.run(9, u0, v0, lam, lam * h, 10, bc=BC_ZERO)
    with w.Wave2D(n, n, h, lam * h, scheme=9, bc=BC_ZERO, dtype=w.F32, flags=w.DIFF_FORM) as sim:
        sim.set_state(rp, rc, 10)
        p2, c2, _ = sim.get_state()
        assert rel_errors(p2, rp)[1] < 1e-6 and rel_errors(c2, rc)[1] < 1e-6
        sim.step_n(25)
        _, got, _ = sim.get_state()
    _, ref = orc.continue_run(9, rp, rc, lam, 25, bc=BC_ZERO)
    l2, linf = rel_errors(got, ref)
    assert l2 < TOL[1] and linf < TOL[1]


def test_diff_form_refusals(w):
    n = 32
    for dtype in (w.F64, w.F32X2):
        with pytest.raises(w.Wave2DError) as e:
            w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=13, dtype=dtype, flags=w.DIFF_FORM)
        assert e.value.code == w.ERR_ARG
    with w.Wave2D(n, n, 1.0 / n, 0.5 / n, scheme=13, dtype=w.F32, flags=w.DIFF_FORM) as sim:
        with pytest.raises(w.Wave2DError):
            sim.set_tuning(kernel=w.KERNEL_TEMPORAL)


@pytest.mark.parametrize("scheme", [9, 13])
def test_diff_form_long_wave_accuracy(w, scheme):
    """Mode (1, 0), 1024^2 periodic, 3000 steps, FP32: the difference form
    keeps the error against the closed-form discrete solution at least 20x
    below the plain two-step (exact FP32 emulation: 48x for 9 points, 74x for
    13 points)."""
    n, steps = 1024, 3000
    h = 1.0 / n
    lam = 0.9 * LAMBDA_MAX[scheme]
    tau = lam * h
    k1 = 2 * math.pi
    u0, v0 = plane_wave_ic(n, n, h, k1, 0.0, BC_PERIODIC)
    an, bn = plane_wave.amplitudes(scheme, lam, tau, k1, 0.0, h, steps)
    x = np.arange(n) * h
    ref = an * np.cos(k1 * x) + bn * np.sin(k1 * x)
    errs = []
    for flags in (0, w.DIFF_FORM):
        _, uc, _ = _run(w, scheme, u0, v0, h, lam, steps, BC_PERIODIC, w.F32, w.KERNEL_TMA, flags)
        errs.append(float(np.sqrt(np.mean((uc - ref[None, :]) ** 2)) / np.sqrt(np.mean(ref ** 2))))
    assert errs[1] < errs[0] / 20, errs
